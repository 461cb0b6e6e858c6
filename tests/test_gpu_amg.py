"""The multigrid hierarchy on the GPU (Section 4.2.2: a multilevel setup with one
triple product per level) against the oracle, level by level.

ptap_aggregate must equal the oracle's aggregation bit for bit (it takes only
exact decisions: maxima and comparisons of the stored values, ties broken by
an integer hash).  The prolongator's pattern must be equal and its values
within 1e-13 of sum |terms|; each level's C = P^T A P is checked against the
oracle's product of that level's own (downloaded) A and P: pattern exact,
values within tau * (|P|^T|A||P|).  Then the numeric phases alone are re-run
for rescaled fine values -- directly and replayed from a CUDA graph -- and
every level is checked again.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import amg as oamg
from paper_1905_08423_gb300 import amg
from paper_1905_08423_gb300 import problems as pb
from paper_1905_08423_gb300 import ptap
from parity import TAU, to_dev

pytestmark = pytest.mark.gpu


def _host(M: ptap.Csr) -> pb.CSR:
    return pb.CSR(M.nrows, M.ncols, M.row_ptr.cpu().numpy(), M.col_idx.cpu().numpy(),
                  M.val.detach().cpu().numpy().astype(np.float64))


@pytest.mark.parametrize("theta", [0.0, 0.25])
@pytest.mark.parametrize("passes", [1, 2, 3])
@pytest.mark.parametrize("kind", ["algebraic", "poisson2d", "model"])
def test_aggregate_and_prolongator(kind, passes, theta):
    A = {"algebraic": lambda: pb.algebraic_problem(12, seed=5)[0],
         "poisson2d": lambda: pb.poisson2d_problem(40)[0],
         "model": lambda: pb.model_problem(13)[0]}[kind]()
    dA = to_dev(A, torch.float64)
    agg, n_agg = ptap.aggregate(dA, passes=passes, rounds=16)
    want, n_want = oamg.aggregate(A, passes=passes, rounds=16)
    assert n_agg == n_want
    np.testing.assert_array_equal(agg.cpu().numpy(), want)
    prol = ptap.Prolongator(dA, agg, n_agg, theta)
    P = prol.numeric(dA, 2.0 / 3.0)
    torch.cuda.synchronize()
    prol.check()
    rp, ci, v = oamg.prolongator(A, want, n_want, 2.0 / 3.0, theta)
    np.testing.assert_array_equal(prol.row_ptr.cpu().numpy(), rp)
    np.testing.assert_array_equal(prol.col_idx.cpu().numpy(), ci)
    np.testing.assert_allclose(P.cpu().numpy(), v, rtol=1e-13, atol=1e-13)
    prol.destroy()


def _tau(A, P, dtype):
    """Value tolerance of one level.  FP64: tau = 1e-12.  FP32: the product accumulates
    each entry in FP32 over at most k = (longest column of P) + (longest row of A) + 2
    roundings, so |error| <= k * 2^-24 * B; tau = max(1e-5, k * 2^-24)."""
    if dtype == torch.float64:
        return TAU[dtype]
    kcol = int(np.bincount(P.col_idx, minlength=P.ncols).max()) if P.nnz else 0
    krow = int(np.diff(A.row_ptr).max()) if A.nrows else 0
    return max(TAU[dtype], (kcol + krow + 2) * 2.0 ** -24)


def _check_levels(h: amg.Hierarchy, dtype, strength):
    """Every level against the oracle; ``strength`` holds each level's operator as it was
    at setup, whose values decided the strong entries (fixed with the pattern)."""
    torch.cuda.synchronize()
    h.check()
    for k, lv in enumerate(h.levels):
        A, P = _host(lv.A), _host(lv.P)
        rp, ci, v = oamg.prolongator(A, lv.agg.cpu().numpy(), lv.P.ncols, h.omega, h.theta, S=strength[k])
        np.testing.assert_array_equal(lv.P.row_ptr.cpu().numpy(), rp)
        np.testing.assert_array_equal(lv.P.col_idx.cpu().numpy(), ci)
        tol = 1e-13 if dtype == torch.float64 else 1e-5
        np.testing.assert_allclose(P.val, v, rtol=tol, atol=tol)
        ref, bnd = oracle.ptap(A, P), oracle.ptap_bound(A, P)
        crp, cci = lv.plan.pattern()
        np.testing.assert_array_equal(crp.cpu().numpy(), ref.row_ptr)
        np.testing.assert_array_equal(cci.cpu().numpy(), ref.col_idx)
        err = np.abs(lv.C.cpu().numpy().astype(np.float64) - ref.val)
        tau = _tau(A, P, dtype)
        assert np.all(np.where(bnd.val > 0, err <= tau * bnd.val, err == 0)), (k, tau)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_hierarchy_levels(dtype):
    A, _ = pb.algebraic_problem(22, seed=8)
    h = amg.Hierarchy(to_dev(A, dtype), coarse_rows=60)
    assert len(h.levels) >= 4
    # aggregation of every level equals the oracle's on that level's operator (FP64 values)
    if dtype == torch.float64:
        for lv in h.levels:
            want, n_want = oamg.aggregate(_host(lv.A), passes=2, rounds=16)
            assert lv.P.ncols == n_want
            np.testing.assert_array_equal(lv.agg.cpu().numpy(), want)
    strength = [_host(lv.A) for lv in h.levels]
    _check_levels(h, dtype, strength)
    st = h.stats()
    assert st["levels"] == len(h.levels) + 1 and st["products"] == len(h.levels)
    # numeric phases only, for new fine values
    g = torch.Generator(device="cuda").manual_seed(11)
    fine = h.levels[0].A
    fine.val.mul_(0.5 + 1.5 * torch.rand(fine.val.shape, generator=g, device="cuda", dtype=dtype))
    fine.val.copy_(0.5 * (fine.val + _transpose_vals(fine)))     # keep it symmetric
    h.renumeric()
    _check_levels(h, dtype, strength)
    # the same from a CUDA graph after another rescale
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        h.renumeric(stream=s)
        s.synchronize()
        with torch.cuda.graph(graph, stream=s):
            h.renumeric(stream=s)
    torch.cuda.current_stream().wait_stream(s)
    fine.val.mul_(1.25)
    graph.replay()
    _check_levels(h, dtype, strength)
    h.destroy()


def _transpose_vals(M: ptap.Csr) -> torch.Tensor:
    """Values of M^T on M's (symmetric) pattern."""
    n = M.nrows
    rows = torch.repeat_interleave(torch.arange(n, device="cuda"), torch.diff(M.row_ptr.long()))
    key = rows * n + M.col_idx.long()
    tkey = M.col_idx.long() * n + rows
    order = torch.argsort(key)
    pos = torch.searchsorted(key[order], tkey)
    return M.val[order[pos]]
