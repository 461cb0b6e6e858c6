"""Compact owner-mode chunks (regions grown over C's graph) vs the oracle.

With compact chunks a coarse row's chunk and accumulator offset come from a
packed per-row table instead of a row range, and the values go back to C row
by row.  These tests check values against the oracle for the interpreter and
the compiled classes, FP32 and FP64, many small chunks and large ones, the
persistent batch, and every way a plan falls back to row ranges.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1905_08423_gb300 import problems as pb
from paper_1905_08423_gb300 import ptap
from parity import check_values, rounded, run_and_check, to_dev

pytestmark = pytest.mark.gpu

DTYPES = [torch.float64, torch.float32]

CONFIGS = [
    dict(),
    dict(chunk_entries=256),                      # many chunks, most rows visit several
    dict(chunk_entries=1024, specialize=4),       # compiled and interpreted classes mixed
    dict(specialize=8, block_threads=1024, chunk_entries=32768),
    dict(block_threads=1024, chunk_entries=32768),  # interpreter, rows of A P in global scratch
    dict(cache_indices=True, specialize=4, chunk_entries=1024),
    dict(visit_block_log2=6),
    dict(compact_chunks=32),                      # regions grown by runs of 32 rows
    dict(compact_chunks=16, specialize=8, block_threads=1024, chunk_entries=32768),
    dict(compact_chunks=7, chunk_entries=256),    # runs that do not divide the lines
]


@pytest.mark.parametrize("cfg", CONFIGS, ids=[str(c) for c in CONFIGS])
@pytest.mark.parametrize("dtype", DTYPES)
def test_compact_configs(cfg, dtype):
    for k, (A, P) in enumerate((pb.model_problem(17), pb.algebraic_problem(13, seed=7),
                                pb.poisson2d_problem(40))):
        plan, _ = run_and_check(A, P, dtype, ptap.make_config(**dict(dict(compact_chunks=True), **cfg)))
        st = plan.stats()
        assert st["compact_chunks"] == st["fast_path"]   # compact chunks serve class programs only
        if k == 0:
            assert st["compact_chunks"] == 1


@pytest.mark.parametrize("dtype", DTYPES)
def test_compact_exact_and_fewer_visits(dtype):
    """Dyadic model problem: exact values; on a 3D mesh the regions cut the visits."""
    A, P = pb.model_problem(63)
    cfg = dict(specialize=8, block_threads=1024, chunk_entries=16384)
    plan_c, C_c = run_and_check(A, P, dtype, ptap.make_config(compact_chunks=True, **cfg))
    plan_r, C_r = run_and_check(A, P, dtype, ptap.make_config(**cfg))
    ref = oracle.ptap(A, P)
    np.testing.assert_array_equal(C_c.cpu().numpy().astype(np.float64), ref.val)
    sc, sr = plan_c.stats(), plan_r.stats()
    assert sc["compact_chunks"] == 1 and sr["compact_chunks"] == 0
    assert sc["n_chunks"] > 8
    assert sc["chunk_fine_rows"] < 0.9 * sr["chunk_fine_rows"], (sc["chunk_fine_rows"], sr["chunk_fine_rows"])


def test_compact_fallbacks():
    """Requests that cannot use compact chunks keep row ranges and stay correct."""
    A, P = pb.model_problem(15)
    plan, _ = run_and_check(A, P, torch.float64, ptap.make_config(compact_chunks=True, class_programs=False))
    assert plan.stats()["compact_chunks"] == 0
    plan, _ = run_and_check(A, P, torch.float64, ptap.make_config(compact_chunks=True, mode=ptap.MODE_ATOMIC))
    assert plan.stats()["compact_chunks"] == 0
    plan, _ = run_and_check(A, P, torch.float64, ptap.make_config(compact_chunks=True), two_step=True)
    assert plan.stats()["compact_chunks"] == 0
    # rows beyond the class-program limits: the plan ends on the general kernel
    rng = np.random.default_rng(17)
    A2 = pb.random_csr(120, 120, 0.4, rng)
    P2 = pb.random_csr(120, 20, 0.1, rng)
    plan, _ = run_and_check(A2, P2, torch.float64, ptap.make_config(compact_chunks=True))
    st = plan.stats()
    assert st["fast_path"] == 0 and st["compact_chunks"] == 0
    # random patterns, stored zeros, empty rows and columns
    for seed in range(4):
        rng = np.random.default_rng(2000 + seed)
        n, m = int(rng.integers(1, 200)), int(rng.integers(1, 60))
        A3 = pb.random_csr(n, n, rng.uniform(0.01, 0.1), rng)
        P3 = pb.random_csr(n, m, rng.uniform(0.02, 0.06), rng)
        run_and_check(A3, P3, torch.float32, ptap.make_config(compact_chunks=True, chunk_entries=256))


@pytest.mark.parametrize("dtype", DTYPES)
def test_compact_batch(dtype):
    """The batch runs compact plans, also beside a general-kernel plan (each kind on its
    own kernel); the no-allocation entry point refuses them."""
    probs = [pb.model_problem(n) for n in (11, 14, 17)] + [pb.poisson2d_problem(30)]
    devs, plans, Cs = [], [], []
    for A, P in probs:
        dA, dP = to_dev(A, dtype), to_dev(P, dtype)
        plan = ptap.symbolic(dA, dP, ptap.make_config(compact_chunks=True, chunk_entries=512))
        assert plan.stats()["compact_chunks"] == 1
        devs.append((dA, dP))
        plans.append(plan)
        Cs.append(torch.empty(plan.nnz, dtype=dtype, device="cuda"))
    batch = ptap.Batch(plans, [d[0] for d in devs], [d[1] for d in devs], Cs)
    batch.numeric()
    torch.cuda.synchronize()
    for (A, P), C in zip(probs, Cs):
        Ar, Pr = rounded(A, dtype), rounded(P, dtype)
        check_values(C, oracle.ptap(Ar, Pr).val, oracle.ptap_bound(Ar, Pr).val, dtype)
    # a general-kernel plan in the same batch
    A, P = probs[0]
    dA, dP = to_dev(A, dtype), to_dev(P, dtype)
    general = ptap.symbolic(dA, dP, ptap.make_config(class_programs=False, chunk_entries=512))
    Cg = torch.full((general.nnz,), float("nan"), dtype=dtype, device="cuda")
    Cs[0].fill_(float("nan"))
    mixed = ptap.Batch([plans[0], general], [devs[0][0], dA], [devs[0][1], dP], [Cs[0], Cg])
    mixed.numeric()
    torch.cuda.synchronize()
    Ar, Pr = rounded(A, dtype), rounded(P, dtype)
    for C in (Cs[0], Cg):
        check_values(C, oracle.ptap(Ar, Pr).val, oracle.ptap_bound(Ar, Pr).val, dtype)
    mixed.destroy()
    with pytest.raises(ptap.PtapError, match="UNSUPPORTED"):
        ptap.batch_numeric_noalloc(plans[:1], [devs[0][0]], [devs[0][1]], Cs[:1])
