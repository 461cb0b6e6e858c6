"""Pins of the hierarchy oracle (oracle/amg.py): aggregation and the smoothed
prolongator (Section 4.2.2's multilevel setup, read as smoothed aggregation).

* One pass run to convergence equals sequential greedy matching over the
  edges in decreasing key order, an independent formulation of the matching.
* A converged pass is maximal: no two unmatched nodes are adjacent.
* Every row gets one aggregate, and aggregates are connected in A's graph;
  one pass gives greedy pairs plus the unmatched rows that joined them.
* omega = 0 gives P = T exactly; P agrees with the dense (I - omega D^-1 A) T;
  P's row sums are 1 - omega (D^-1 A 1)(i), so a zero-row-sum A gives P 1 = 1.
"""
import numpy as np
import pytest

import oracle
from oracle import amg as oamg
from paper_1905_08423_gb300 import problems as pb


def _random_sym(n, density, seed):
    rng = np.random.default_rng(seed)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(i + 1, n):
            if rng.random() < density:
                D[i, j] = D[j, i] = -rng.lognormal()
    np.fill_diagonal(D, -D.sum(axis=1) + 1.0)
    rows, cols = np.nonzero(D)
    rp = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=n))]).astype(np.int32)
    return pb.CSR(n, n, rp, cols.astype(np.int32), D[rows, cols]), D


def _dense(M):
    D = np.zeros((M.nrows, M.ncols))
    for i in range(M.nrows):
        for e in range(M.row_ptr[i], M.row_ptr[i + 1]):
            D[i, M.col_idx[e]] = M.val[e]
    return D


@pytest.mark.parametrize("seed", range(6))
def test_one_pass_equals_greedy_matching(seed):
    A, _ = _random_sym(40, 0.12, seed)
    agg, n_agg = oamg.aggregate(A, passes=1, rounds=200)
    partner = oamg.greedy_matching(A)
    single = {i for i in range(A.nrows) if partner[i] < 0}
    # converged: the unmatched rows are an independent set (a maximal matching)
    for i in single:
        for e in range(A.row_ptr[i], A.row_ptr[i + 1]):
            j = A.col_idx[e]
            assert j == i or j not in single
    # every aggregate is one greedy pair with the unmatched rows that joined it, or
    # an unmatched row with no matched neighbour
    for a in range(n_agg):
        mem = np.nonzero(agg == a)[0].tolist()
        paired = [i for i in mem if partner[i] >= 0]
        if paired:
            assert len(paired) == 2 and partner[paired[0]] == paired[1]
            for i in mem:
                if i in single:
                    nb = set(A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]].tolist())
                    assert nb & set(paired)
        else:
            (i,) = mem
            nb = set(A.col_idx[A.row_ptr[i]:A.row_ptr[i + 1]].tolist()) - {i}
            assert all(partner[j] < 0 for j in nb)


@pytest.mark.parametrize("passes", [1, 2, 3])
def test_aggregates_cover_and_are_connected(passes):
    A, _ = pb.algebraic_problem(6, seed=2)
    agg, n_agg = oamg.aggregate(A, passes=passes)
    assert agg.min() == 0 and agg.max() == n_agg - 1 and len(np.unique(agg)) == n_agg
    assert n_agg < A.nrows
    for a in range(n_agg):
        mem = set(np.nonzero(agg == a)[0].tolist())
        seen, stack = set(), [min(mem)]
        while stack:
            i = stack.pop()
            if i in seen:
                continue
            seen.add(i)
            for e in range(A.row_ptr[i], A.row_ptr[i + 1]):
                j = int(A.col_idx[e])
                if j in mem and j not in seen:
                    stack.append(j)
        assert seen == mem, a


def test_prolongator_closed_forms():
    A, D = _random_sym(30, 0.2, 7)
    agg, n_agg = oamg.aggregate(A, passes=2)
    T = np.zeros((A.nrows, n_agg))
    T[np.arange(A.nrows), agg] = 1.0
    # omega = 0: P = T exactly, on the pattern of A T
    rp, ci, v = oamg.prolongator(A, agg, n_agg, omega=0.0)
    P0 = np.zeros_like(T)
    for i in range(A.nrows):
        P0[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
    assert np.array_equal(P0, T)
    pat = (np.abs(D) > 0).astype(float) @ T > 0
    for i in range(A.nrows):
        assert sorted(ci[rp[i]:rp[i + 1]]) == list(np.nonzero(pat[i])[0])
    # omega = 2/3 against the dense definition, and its row sums
    om = 2.0 / 3.0
    rp, ci, v = oamg.prolongator(A, agg, n_agg, omega=om)
    P = np.zeros_like(T)
    for i in range(A.nrows):
        P[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
    want = (np.eye(A.nrows) - om * np.diag(1.0 / np.diag(D)) @ D) @ T
    np.testing.assert_allclose(P, want, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(P.sum(axis=1), 1.0 - om * (D.sum(axis=1) / np.diag(D)), rtol=1e-13, atol=1e-14)


def test_zero_row_sum_preserves_constants():
    # the Neumann graph Laplacian: rows sum to zero, so P 1 = 1
    A, _ = pb.algebraic_problem(5, seed=4, neumann=True)
    agg, n_agg = oamg.aggregate(A, passes=2)
    rp, ci, v = oamg.prolongator(A, agg, n_agg)
    sums = np.add.reduceat(v, rp[:-1]) if len(v) else np.zeros(0)
    np.testing.assert_allclose(sums, 1.0, rtol=0, atol=1e-12)


def test_galerkin_level_dense():
    A, D = _random_sym(24, 0.25, 9)
    agg, n_agg = oamg.aggregate(A, passes=2)
    rp, ci, v = oamg.prolongator(A, agg, n_agg)
    P = pb.CSR(A.nrows, n_agg, rp.astype(np.int32), ci.astype(np.int32), v)
    C = oracle.ptap(A, P)
    Pd = _dense(P)
    np.testing.assert_allclose(_dense(C), Pd.T @ D @ Pd, rtol=1e-12, atol=1e-12)


def test_filtered_prolongator_dense():
    """theta > 0: P = (I - omega D^-1 A_F) T with A_F = strong entries + diagonal and
    D = diag(A); row sums 1 - omega (A_F 1)(i) / A(i,i)."""
    A, D = _random_sym(30, 0.3, 12)
    agg, n_agg = oamg.aggregate(A, passes=2)
    T = np.zeros((A.nrows, n_agg))
    T[np.arange(A.nrows), agg] = 1.0
    theta, om = 0.4, 2.0 / 3.0
    off = D - np.diag(np.diag(D))
    strong = np.abs(off) >= theta * np.abs(off).max(axis=1, keepdims=True)
    strong &= off != 0
    AF = np.where(strong, off, 0.0) + np.diag(np.diag(D))
    want = (np.eye(A.nrows) - om * np.diag(1.0 / np.diag(D)) @ AF) @ T
    rp, ci, v = oamg.prolongator(A, agg, n_agg, omega=om, theta=theta)
    P = np.zeros_like(T)
    for i in range(A.nrows):
        P[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
        assert sorted(ci[rp[i]:rp[i + 1]]) == sorted(set(agg[np.nonzero(strong[i])[0]]) | {agg[i]})
    np.testing.assert_allclose(P, want, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(P.sum(axis=1), 1.0 - om * AF.sum(axis=1) / np.diag(D), rtol=1e-13, atol=1e-14)
