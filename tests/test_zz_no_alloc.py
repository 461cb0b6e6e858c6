"""The no-allocation batched numeric entry point, through the C ABI.

ptap_batch_numeric_noalloc serves callers that cannot allocate device memory
while the products run (a device footprint fixed up front by their own pool,
or no room for an allocation's implicit synchronisation).  Its outputs must
match the existing ptap_numeric entry point within the parity tolerance, on
two calls in a row (the shared device array keeps the previous call's
contents), for plans built with the default configuration and with the large
chunks the autotuner picks for the class-program kernels.  Refusals: too many
problems or chunks, plans whose kernel shapes differ, bad output buffers and
stream capture.
This file is collected last so that a stop at the first failure has run every
other test first.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1905_08423_gb300 import problems as pb
from paper_1905_08423_gb300 import ptap
from parity import TAU, rounded, to_dev

pytestmark = pytest.mark.gpu

CONFIGS = {
    "chunk512": dict(chunk_entries=512),
    "default": dict(),
    # the class-program configurations the autotuner offers at the largest chunks
    "tuned_f32": dict(specialize=32, block_threads=1024, chunk_entries=32768),
    "tuned_f32_max": dict(specialize=32, block_threads=1024, chunk_entries=49152),
    "tuned_f64": dict(specialize=32, block_threads=512, chunk_entries=20480),
}


def _setup(dtype, cfg, count=5, lo=10, hi=26):
    probs = pb.batch_problems(seed=4, count=count, lo=lo, hi=hi)
    plans, devs, refs, bounds = [], [], [], []
    for A, P in probs:
        dA, dP = to_dev(A, dtype), to_dev(P, dtype)
        plan = ptap.symbolic(dA, dP, ptap.make_config(**cfg))
        plans.append(plan)
        devs.append((dA, dP))
        refs.append(ptap.numeric(plan, dA, dP))          # the existing entry point
        Ar, Pr = rounded(A, dtype), rounded(P, dtype)
        bounds.append(oracle.ptap_bound(Ar, Pr).val)
    torch.cuda.synchronize()
    return plans, devs, refs, bounds


def _library_bytes(plans):
    return [(p.stats()["plan_bytes"], p.stats()["peak_bytes"]) for p in plans]


@pytest.mark.parametrize("name", list(CONFIGS))
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_matches_numeric(dtype, name):
    plans, devs, refs, bounds = _setup(dtype, CONFIGS[name])
    Cs = [torch.full_like(r, float("nan")) for r in refs]
    before = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    lib_before = _library_bytes(plans)
    for call in range(2):
        for C in Cs:
            C.fill_(float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        ptap.batch_numeric_noalloc(plans, [d[0] for d in devs], [d[1] for d in devs], Cs)
        torch.cuda.synchronize()
        if call == 1:
            # the first call may load the library's module; the second must not take
            # device memory at all (any device allocation takes at least 2 MiB)
            assert torch.cuda.mem_get_info()[0] > free0 - (2 << 20)
        for C, R, B in zip(Cs, refs, bounds):
            got = C.cpu().numpy().astype(np.float64)
            want = R.cpu().numpy().astype(np.float64)
            err = np.abs(got - want)
            ok = np.where(B > 0, err <= TAU[dtype] * B, err == 0)
            assert ok.all(), f"call {call}: {(~ok).sum()} entries differ"
    # nothing went through the torch allocator or the plans' allocators during the calls
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == before
    assert _library_bytes(plans) == lib_before
    for p in plans:
        p.check()


def _small(dtype=torch.float64, cfg=None):
    A, P = pb.model_problem(7)
    dA, dP = to_dev(A, dtype), to_dev(P, dtype)
    plan = ptap.symbolic(dA, dP, ptap.make_config(**(cfg or {})))
    C = torch.empty(plan.nnz, dtype=dtype, device="cuda")
    return plan, dA, dP, C


def test_noalloc_rejects_oversize():
    plan, dA, dP, C = _small()
    n = 1025   # one more than PTAP_NOALLOC_MAX_PROBLEMS
    with pytest.raises(ptap.PtapError) as e:
        ptap.batch_numeric_noalloc([plan] * n, [dA] * n, [dP] * n, [C] * n)
    assert e.value.code == 3


def test_noalloc_rejects_too_many_chunks():
    # 64-entry chunks of the 31^3 model problem: over a thousand chunks a plan, so 1024
    # copies exceed PTAP_NOALLOC_MAX_ITEMS (1,000,000); refused before anything runs
    A, P = pb.model_problem(31)
    dA, dP = to_dev(A, torch.float64), to_dev(P, torch.float64)
    plan = ptap.symbolic(dA, dP, ptap.make_config(chunk_entries=64, class_programs=False))
    chunks = plan.stats()["n_chunks"]
    n = 1024
    assert chunks * n > 1_000_000
    C = torch.empty(plan.nnz, dtype=torch.float64, device="cuda")
    with pytest.raises(ptap.PtapError) as e:
        ptap.batch_numeric_noalloc([plan] * n, [dA] * n, [dP] * n, [C] * n)
    assert e.value.code == 3


@pytest.mark.parametrize("other", [dict(group_lanes=16), dict(ap_slots=128)])
def test_noalloc_rejects_mixed_kernel_shapes(other):
    # lanes per fine row and hash slots are compiled into the one kernel that serves all plans
    base = dict(chunk_entries=512, class_programs=False)
    p1, dA, dP, C1 = _small(cfg=base)
    p2, _, _, C2 = _small(cfg=dict(base, **other))
    with pytest.raises(ptap.PtapError) as e:
        ptap.batch_numeric_noalloc([p1, p2], [dA, dA], [dP, dP], [C1, C2])
    assert e.value.code == 1


def test_noalloc_mixed_chunk_sizes():
    # plans with different chunk sizes and CTA sizes share one call
    p1, dA, dP, C1 = _small(cfg=dict(chunk_entries=512))
    p2, _, _, C2 = _small(cfg=dict(specialize=32, block_threads=1024, chunk_entries=32768))
    want = ptap.numeric(p1, dA, dP)
    ptap.batch_numeric_noalloc([p1, p2], [dA, dA], [dP, dP], [C1, C2])
    torch.cuda.synchronize()
    for C in (C1, C2):
        np.testing.assert_allclose(C.cpu().numpy(), want.cpu().numpy(), rtol=1e-12, atol=1e-12)


def test_noalloc_rejects_bad_outputs():
    plan, dA, dP, C = _small()
    with pytest.raises(ptap.PtapError):
        ptap.batch_numeric_noalloc([plan], [dA], [dP], [C.float()])      # wrong dtype
    with pytest.raises(ptap.PtapError):
        ptap.batch_numeric_noalloc([plan], [dA], [dP], [C[:-1]])         # too short


def test_noalloc_refused_during_capture():
    plan, dA, dP, C = _small()
    ptap.batch_numeric_noalloc([plan], [dA], [dP], [C])   # first call outside capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    codes = []
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            try:
                ptap.batch_numeric_noalloc([plan], [dA], [dP], [C], stream=s)
            except ptap.PtapError as e:
                codes.append(e.code)
    torch.cuda.synchronize()
    assert codes == [8]
