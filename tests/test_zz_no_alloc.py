"""The no-allocation batched numeric entry point, through the C ABI.

ptap_batch_numeric_noalloc serves callers that cannot allocate device memory
while the products run (a device footprint fixed up front by their own pool,
or no room for an allocation's implicit synchronisation).  Its outputs must
match the existing ptap_numeric entry point within the parity tolerance, on
two calls in a row (the shared device array keeps the previous call's
contents).  This file is collected last so that a stop at the first failure
has run every other test first.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1905_08423_gb300 import problems as pb
from paper_1905_08423_gb300 import ptap
from parity import TAU, rounded, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_matches_numeric(dtype):
    probs = pb.batch_problems(seed=4, count=5, lo=10, hi=26)
    plans, devs, refs, bounds = [], [], [], []
    for A, P in probs:
        dA, dP = to_dev(A, dtype), to_dev(P, dtype)
        plan = ptap.symbolic(dA, dP, ptap.make_config(chunk_entries=512))
        plans.append(plan)
        devs.append((dA, dP))
        refs.append(ptap.numeric(plan, dA, dP))          # the existing entry point
        Ar, Pr = rounded(A, dtype), rounded(P, dtype)
        bounds.append(oracle.ptap_bound(Ar, Pr).val)
    torch.cuda.synchronize()
    Cs = [torch.full_like(r, float("nan")) for r in refs]
    before = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for call in range(2):
        for C in Cs:
            C.fill_(float("nan"))
        ptap.batch_numeric_noalloc(plans, [d[0] for d in devs], [d[1] for d in devs], Cs)
        torch.cuda.synchronize()
        for C, R, B in zip(Cs, refs, bounds):
            got = C.cpu().numpy().astype(np.float64)
            want = R.cpu().numpy().astype(np.float64)
            err = np.abs(got - want)
            ok = np.where(B > 0, err <= TAU[dtype] * B, err == 0)
            assert ok.all(), f"call {call}: {(~ok).sum()} entries differ"
    # nothing went through the torch allocator during the calls
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == before
    for p in plans:
        p.check()


def test_noalloc_rejects_oversize():
    A, P = pb.model_problem(7)
    dA, dP = to_dev(A, torch.float64), to_dev(P, torch.float64)
    plan = ptap.symbolic(dA, dP)
    C = torch.empty(plan.nnz, dtype=torch.float64, device="cuda")
    n = 1025   # one more than PTAP_NOALLOC_MAX_PROBLEMS
    with pytest.raises(ptap.PtapError) as e:
        ptap.batch_numeric_noalloc([plan] * n, [dA] * n, [dP] * n, [C] * n)
    assert e.value.code == 3
