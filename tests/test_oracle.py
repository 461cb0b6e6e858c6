"""Pins for the CPU oracle, checked against things other than itself.

Each test fixes the oracle to a value the paper prints, a closed form, an
invariant of C = P^T A P, a textbook routine (dense products), or brute force
on tiny inputs.  Random matrices are non-symmetric and P is rectangular, so a
transposed operand, a dropped term or a wrong index fails at least one test.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1905_08423_gb300 import problems as pb

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TAU64 = 1e-12


def _read_eq5():
    mats = {}
    cur = None
    with open(os.path.join(GOLDEN, "eq5_rowwise_pattern.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] in ("A", "P", "C"):
                cur = parts[0]
                mats[cur] = (int(parts[1]), int(parts[2]), [])
            else:
                mats[cur][2].append([int(x) - 1 for x in parts])
    out = {}
    for k, (r, c, rows) in mats.items():
        lens = [len(x) for x in rows]
        rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
        ci = np.array([x for row in rows for x in row], dtype=np.int32)
        out[k] = pb.CSR(r, c, rp, ci, np.ones(ci.size))
    return out


def test_eq5_rowwise_pattern():
    """Section 2, Eq. 5: the pattern of A P printed in the paper."""
    m = _read_eq5()
    C = oracle.spgemm(m["A"], m["P"])
    np.testing.assert_array_equal(C.row_ptr, m["C"].row_ptr)
    np.testing.assert_array_equal(C.col_idx, m["C"].col_idx)
    # Row 1 of C combines rows 1, 2 and 5 of P (0-based 0, 1, 4).
    A = m["A"]
    assert list(A.col_idx[A.row_ptr[0]:A.row_ptr[1]]) == [0, 1, 4]
    # Rows 1-2 belong to the first process; their off-process columns are 3 and 5.
    cols = set(A.col_idx[A.row_ptr[0]:A.row_ptr[2]].tolist())
    assert sorted(c for c in cols if c not in (0, 1)) == [2, 4]


def _dense_ptap(A, P):
    Ad, Pd = A.to_dense(), P.to_dense()
    return Pd.T @ Ad @ Pd


def _pattern_ptap(A, P):
    a = A.pattern_dense().astype(np.int64)
    p = P.pattern_dense().astype(np.int64)
    return (p.T @ a @ p) > 0


@pytest.mark.parametrize("seed", range(12))
def test_brute_force_tiny(seed):
    """Dense brute force: exact values (small integers) and the boolean pattern."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 41))
    m = int(rng.integers(1, 13))
    A = pb.random_csr(n, n, rng.uniform(0.05, 0.4), rng)
    P = pb.random_csr(n, m, rng.uniform(0.05, 0.5), rng)
    C = oracle.ptap(A, P)
    assert C.nrows == m and C.ncols == m
    np.testing.assert_array_equal(C.to_dense(), _dense_ptap(A, P))
    pat = np.zeros((m, m), dtype=bool)
    rows = np.repeat(np.arange(m), np.diff(C.row_ptr))
    pat[rows, C.col_idx] = True
    np.testing.assert_array_equal(pat, _pattern_ptap(A, P))
    # columns sorted and unique per row
    for i in range(m):
        c = C.col_idx[C.row_ptr[i]:C.row_ptr[i + 1]]
        assert (np.diff(c) > 0).all()


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_real_values(seed):
    rng = np.random.default_rng(100 + seed)
    n, m = 30, 9
    A = pb.random_csr(n, n, 0.2, rng, int_values=False)
    P = pb.random_csr(n, m, 0.3, rng, int_values=False)
    C = oracle.ptap(A, P)
    B = oracle.ptap_bound(A, P)
    np.testing.assert_array_equal(C.row_ptr, B.row_ptr)
    err = np.abs(C.to_dense() - _dense_ptap(A, P))
    assert (err <= TAU64 * B.to_dense() + 1e-300).all()


def test_identity():
    """P = I gives C = A exactly, pattern included."""
    rng = np.random.default_rng(7)
    A = pb.random_csr(25, 25, 0.2, rng, int_values=False)
    C = oracle.ptap(A, pb.identity_csr(25))
    np.testing.assert_array_equal(C.row_ptr, A.row_ptr)
    np.testing.assert_array_equal(C.col_idx, A.col_idx)
    np.testing.assert_array_equal(C.val, A.val)


def _tridiag(n, a, b):
    return np.diag(np.full(n, a)) + np.diag(np.full(n - 1, b), 1) + np.diag(np.full(n - 1, b), -1)


def _csr_from_dense(d):
    n, m = d.shape
    rows, cols = np.nonzero(d)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rp[1:])
    return pb.CSR(n, m, rp.astype(np.int32), cols.astype(np.int32), d[rows, cols])


def test_1d_closed_form():
    """tridiag(-1,2,-1) with linear interpolation (1/2, 1, 1/2) gives 1/2 tridiag(-1,2,-1)."""
    n = 15
    A = _csr_from_dense(_tridiag(n, 2.0, -1.0))
    P = pb.trilinear_P((1, 1, n))   # 1D: only x varies
    assert P.ncols == n // 2
    C = oracle.ptap(A, P)
    np.testing.assert_array_equal(C.to_dense(), 0.5 * _tridiag(n // 2, 2.0, -1.0))
    np.testing.assert_array_equal(np.diff(C.row_ptr), [2] + [3] * (n // 2 - 2) + [2])


def test_3d_closed_form_15():
    """15^3 7-point Laplacian, trilinear P: C = 1/2 T(x)M(x)M + M(x)1/2 T(x)M + M(x)M(x)1/2 T."""
    n = 15
    A, P = pb.model_problem(n)
    C = oracle.ptap(A, P)
    md = n // 2
    T = _tridiag(md, 2.0, -1.0)
    M = _tridiag(md, 1.5, 0.25)
    expect = (np.kron(np.kron(M, M), 0.5 * T) + np.kron(np.kron(M, 0.5 * T), M)
              + np.kron(np.kron(0.5 * T, M), M))
    np.testing.assert_array_equal(C.to_dense(), expect)
    # structural pattern = 27-point coupling truncated at the boundary
    assert C.nnz == (3 * md - 2) ** 3 == 6859
    d = C.to_dense()
    assert set(np.unique(np.round(d[d != 0], 12))) == {6.75, -0.375, -0.3125, -0.09375}


def _closed_form_row_lengths(md):
    k = np.full(md, 3)
    k[0] = k[-1] = 2
    if md == 1:
        k[:] = 1
    return (k[None, None, :] * k[None, :, None] * k[:, None, None]).reshape(-1)


def test_model_row_lengths_closed_form():
    """Row lengths of C for the model problem: product over axes of coarse neighbours."""
    for n in (9, 15, 17):
        A, P = pb.model_problem(n)
        C = oracle.ptap(A, P)
        np.testing.assert_array_equal(np.diff(C.row_ptr), _closed_form_row_lengths(n // 2))


def test_symmetry_algebraic():
    """C is symmetric when A is (27-point lognormal, smoothed aggregation)."""
    A, P = pb.algebraic_problem(11, seed=3)
    C = oracle.ptap(A, P)
    B = oracle.ptap_bound(A, P)
    d, b = C.to_dense(), B.to_dense()
    np.testing.assert_array_equal(d != 0, (d != 0).T)
    assert (np.abs(d - d.T) <= TAU64 * b).all()


def test_zero_row_sums_neumann():
    """Constant-preserving P on a zero-row-sum A gives C 1 = 0."""
    A, P = pb.algebraic_problem(10, seed=5, neumann=True)
    assert np.abs(A.to_dense().sum(axis=1)).max() < 1e-12 * np.abs(A.val).max()
    P1 = P.to_dense().sum(axis=1)
    np.testing.assert_allclose(P1, 1.0, rtol=0, atol=1e-14)
    C = oracle.ptap(A, P)
    B = oracle.ptap_bound(A, P)
    rs = np.abs(C.to_dense().sum(axis=1))
    assert (rs <= 1e-12 * B.to_dense().sum(axis=1)).all()


def test_scaling_exact():
    """C(2^k A) = 2^k C(A) and C(2P) = 4 C(P), exactly."""
    A, P = pb.algebraic_problem(8, seed=11)
    C = oracle.ptap(A, P)
    C8 = oracle.ptap(A.with_values(A.val * 8.0), P)
    np.testing.assert_array_equal(C8.val, 8.0 * C.val)
    C2 = oracle.ptap(A, P.with_values(P.val * 2.0))
    np.testing.assert_array_equal(C2.val, 4.0 * C.val)


def test_permutation_invariance():
    """A symmetric permutation of the fine index (P's rows permuted alike) leaves C unchanged."""
    A, P = pb.algebraic_problem(7, seed=2)
    perm = np.random.default_rng(0).permutation(A.nrows)
    Ap, Pp = pb.permute_fine(A, P, perm)
    C = oracle.ptap(A, P)
    Cp = oracle.ptap(Ap, Pp)
    B = oracle.ptap_bound(A, P)
    np.testing.assert_array_equal(C.row_ptr, Cp.row_ptr)
    np.testing.assert_array_equal(C.col_idx, Cp.col_idx)
    assert (np.abs(C.val - Cp.val) <= TAU64 * B.val).all()


def test_vs_scipy():
    """Dense values agree with scipy's P.T @ A @ P (patterns differ: scipy drops zeros)."""
    sp = pytest.importorskip("scipy.sparse")
    A, P = pb.algebraic_problem(9, seed=4)
    As = sp.csr_matrix((A.val, A.col_idx, A.row_ptr), shape=(A.nrows, A.ncols))
    Ps = sp.csr_matrix((P.val, P.col_idx, P.row_ptr), shape=(P.nrows, P.ncols))
    ref = (Ps.T @ As @ Ps).toarray()
    C = oracle.ptap(A, P)
    B = oracle.ptap_bound(A, P)
    assert (np.abs(C.to_dense() - ref) <= TAU64 * B.to_dense() + 1e-300).all()


def test_rows_form_matches_two_step():
    """The row form (Eq. 8) and the two-step form (Eq. 6) agree."""
    A, P = pb.algebraic_problem(9, seed=8)
    C = oracle.ptap(A, P)
    B = oracle.ptap_bound(A, P)
    rows = np.arange(P.ncols, dtype=np.int32)
    R = oracle.ptap_rows(A, P, rows)
    np.testing.assert_array_equal(R.row_ptr, C.row_ptr)
    np.testing.assert_array_equal(R.col_idx, C.col_idx)
    assert (np.abs(R.val - C.val) <= TAU64 * B.val).all()
    rng = np.random.default_rng(1)
    for _ in range(3):
        n, m = 20, 7
        A = pb.random_csr(n, n, 0.25, rng)
        P = pb.random_csr(n, m, 0.3, rng)
        C = oracle.ptap(A, P)
        R = oracle.ptap_rows(A, P, np.arange(m, dtype=np.int32))
        np.testing.assert_array_equal(R.row_ptr, C.row_ptr)
        np.testing.assert_array_equal(R.col_idx, C.col_idx)
        np.testing.assert_array_equal(R.val, C.val)


def test_row_block_partition_sums_to_C():
    """Summing the contributions of a block-row partition of the fine rows gives C."""
    rng = np.random.default_rng(3)
    n, m = 37, 10
    A = pb.random_csr(n, n, 0.2, rng)
    P = pb.random_csr(n, m, 0.3, rng)
    C = oracle.ptap(A, P).to_dense()
    cuts = [0, 9, 20, 21, 37]
    acc = np.zeros_like(C)
    for r0, r1 in zip(cuts[:-1], cuts[1:]):
        acc += oracle.ptap_row_block(A, P, r0, r1).to_dense()
    np.testing.assert_array_equal(acc, C)


def test_empty_and_degenerate():
    """Empty P rows and columns, empty A rows, 1x1 problems."""
    rng = np.random.default_rng(5)
    A = pb.random_csr(12, 12, 0.3, rng)
    P = pb.random_csr(12, 5, 0.3, rng, empty_row_frac=0.5)
    P.val[:] = 0.0   # all stored P values zero: pattern stays structural
    C = oracle.ptap(A, P)
    np.testing.assert_array_equal(C.val, 0.0)
    np.testing.assert_array_equal(C.to_dense() != 0, np.zeros((5, 5), bool))
    assert C.nnz == int(_pattern_ptap(A, P).sum())
    one = pb.CSR(1, 1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([3.0]))
    C1 = oracle.ptap(one, pb.CSR(1, 1, np.array([0, 1], np.int32), np.array([0], np.int32),
                                  np.array([2.0])))
    assert C1.nnz == 1 and C1.val[0] == 12.0
    Z = pb.CSR(4, 4, np.zeros(5, np.int32), np.zeros(0, np.int32), np.zeros(0))
    C0 = oracle.ptap(Z, pb.identity_csr(4))
    assert C0.nnz == 0 and C0.nrows == 4


def _loss_and_grads(A, P, Ct):
    C = oracle.ptap(A, P)
    assert np.array_equal(C.col_idx, Ct.col_idx)
    R = C.val - Ct.val
    G = pb.CSR(C.nrows, C.ncols, C.row_ptr, C.col_idx, 2.0 * R)
    dA, dP = oracle.ptap_backward(A, P, G)
    return float((R * R).sum()), dA, dP


def test_backward_finite_differences():
    """Central differences of L = ||P^T A P - C_t||_F^2 along random directions (FP64)."""
    A, P = pb.poisson2d_problem(16)
    Pt = pb.perturb_values(P, seed=5)
    Ct = oracle.ptap(A, Pt)
    L0, dA, dP = _loss_and_grads(A, P, Ct)
    rng = np.random.default_rng(0)
    for _ in range(3):
        vA = rng.standard_normal(A.nnz)
        vP = rng.standard_normal(P.nnz)
        hA = 1e-6 * np.abs(A.val).max()
        hP = 1e-6 * np.abs(P.val).max()
        Lp = _loss_and_grads(A.with_values(A.val + hA * vA), P, Ct)[0]
        Lm = _loss_and_grads(A.with_values(A.val - hA * vA), P, Ct)[0]
        fd = (Lp - Lm) / (2 * hA)
        an = float(dA @ vA)
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-30)
        Lp = _loss_and_grads(A, P.with_values(P.val + hP * vP), Ct)[0]
        Lm = _loss_and_grads(A, P.with_values(P.val - hP * vP), Ct)[0]
        fd = (Lp - Lm) / (2 * hP)
        an = float(dP @ vP)
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-30)
    # individual entries of dP
    for e in rng.choice(P.nnz, 8, replace=False):
        h = 1e-6 * max(abs(P.val[e]), 1.0)
        vp = P.val.copy(); vp[e] += h
        vm = P.val.copy(); vm[e] -= h
        fd = (_loss_and_grads(A, P.with_values(vp), Ct)[0]
              - _loss_and_grads(A, P.with_values(vm), Ct)[0]) / (2 * h)
        assert abs(fd - dP[e]) <= 1e-6 * max(abs(dP).max(), 1e-30)


def test_backward_dense_reference():
    """dA = (P G P^T) on pat(A), dP = (A P G^T + A^T P G) on pat(P), against dense FP64."""
    rng = np.random.default_rng(9)
    n, m = 30, 8
    A = pb.random_csr(n, n, 0.2, rng, int_values=False)
    P = pb.random_csr(n, m, 0.3, rng, int_values=False)
    C = oracle.ptap(A, P)
    G = pb.CSR(m, m, C.row_ptr, C.col_idx, rng.standard_normal(C.nnz))
    dA, dP = oracle.ptap_backward(A, P, G)
    Ad, Pd, Gd = A.to_dense(), P.to_dense(), G.to_dense()
    rA = np.repeat(np.arange(n), A.row_lengths())
    rP = np.repeat(np.arange(n), P.row_lengths())
    eA = (Pd @ Gd @ Pd.T)[rA, A.col_idx]
    eP = (Ad @ Pd @ Gd.T + Ad.T @ Pd @ Gd)[rP, P.col_idx]
    np.testing.assert_allclose(dA, eA, rtol=1e-10, atol=1e-12 * np.abs(eA).max())
    np.testing.assert_allclose(dP, eP, rtol=1e-10, atol=1e-12 * np.abs(eP).max())


def test_generators_invariants():
    """Input generators: CSR invariants and the sizes of the named workloads."""
    A, P = pb.model_problem(15)
    A.check(); P.check()
    assert (A.nrows, A.nnz, P.ncols, P.nnz) == (3375, 22275, 343, 9261)
    A3, P3 = pb.algebraic_problem(12, seed=3)
    A3.check(); P3.check()
    assert P3.ncols == 4 ** 3
    assert P3.row_lengths().max() <= 8 and P3.row_lengths().min() >= 1
    A5, P5 = pb.poisson2d_problem(64)
    A5.check(); P5.check()
    assert (A5.nrows, A5.nnz, P5.ncols, P5.nnz) == (4096, 20224, 1024, 12032)
    d = A3.to_dense()
    np.testing.assert_array_equal(d, d.T)


@pytest.mark.parametrize("seed", range(3))
def test_bound_is_abs_triple_product(seed):
    """The tolerance bound B = |P|^T |A| |P|: equal to a dense brute force of that product,
    never below |C| entrywise (triangle inequality), and equal to C when A, P >= 0."""
    rng = np.random.default_rng(700 + seed)
    A = pb.random_csr(25, 25, 0.25, rng, int_values=False)
    P = pb.random_csr(25, 7, 0.3, rng, int_values=False)
    B = oracle.ptap_bound(A, P).to_dense()
    Ad, Pd = np.abs(A.to_dense()), np.abs(P.to_dense())
    np.testing.assert_allclose(B, Pd.T @ Ad @ Pd, rtol=1e-13, atol=0)
    C = oracle.ptap(A, P).to_dense()
    assert (np.abs(C) <= B * (1 + 1e-13)).all()
    Ap, Pp = A.with_values(np.abs(A.val)), P.with_values(np.abs(P.val))
    np.testing.assert_array_equal(oracle.ptap(Ap, Pp).val, oracle.ptap_bound(A, P).val)
