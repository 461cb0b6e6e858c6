"""The 64-problem uneven batch (sides U{16..96}; 7- and 27-point operators;
trilinear and smoothed-aggregation P) in one batched launch, against the oracle.

Every product of the batch is checked on sampled coarse rows (Eq. 8 row form)
within tau * (|P|^T|A||P|)(i,j), in FP32 and FP64, for every configuration
the batch tuner offers (the interpreter, the batch-wide specialised kernel at
each CTA size, with indices cached per visit, and the general kernel).  A
CUDA graph that captured the batched launch is then replayed after every
stored value of every A is rescaled in place by a factor drawn from
U(0.5, 2), and all 64 products are checked again against the oracle on the
rescaled values (Section 4.1: numeric products repeated on one symbolic
result).
"""
import numpy as np
import pytest
import torch

from paper_1905_08423_gb300 import autotune
from paper_1905_08423_gb300 import problems as pb
from paper_1905_08423_gb300 import ptap
from parity import check_sampled, sample_rows, sampled_reference, to_dev

pytestmark = pytest.mark.gpu


def _configs():
    props = torch.cuda.get_device_properties(0)
    optin = int(getattr(props, "shared_memory_per_block_optin", 232448))
    return {name: autotune.batch_candidate_list(vb, optin) for vb, name in ((4, "f32"), (8, "f64"))}


# every candidate of the batch tuner (their number does not depend on the device)
_N_CANDIDATES = len(autotune.batch_candidate_list(4, 232448))


@pytest.fixture(scope="module")
def batch64():
    return pb.batch_problems(seed=4, count=64)


def _run(probs, dtype, cfg):
    devs = [(to_dev(A, dtype), to_dev(P, dtype)) for A, P in probs]
    plans = [ptap.symbolic(a, p, ptap.make_config(**cfg)) for a, p in devs]
    Cs = [torch.full((p.nnz,), float("nan"), dtype=dtype, device="cuda") for p in plans]
    batch = ptap.Batch(plans, [a for a, _ in devs], [p for _, p in devs], Cs)
    return devs, plans, Cs, batch


def _check_all(probs, plans, Cs, dtype, seed):
    for q, ((A, P), plan, C) in enumerate(zip(probs, plans, Cs)):
        rows = sample_rows(P.ncols, 150, seed + q)
        ref, bnd = sampled_reference(A, P, dtype, rows)
        check_sampled(plan, C, ref, bnd, rows, dtype)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("k", range(_N_CANDIDATES))
def test_batch64_every_product(batch64, dtype, k):
    cfg = _configs()["f32" if dtype == torch.float32 else "f64"][k]
    devs, plans, Cs, batch = _run(batch64, dtype, cfg)
    batch.numeric()
    torch.cuda.synchronize()
    for p in plans:
        p.check()
    _check_all(batch64, plans, Cs, dtype, 500)
    batch.destroy()


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_batch64_graph_replay_after_rescale(batch64, dtype):
    cfg = _configs()["f32" if dtype == torch.float32 else "f64"][3]   # specialised, 1024 threads
    devs, plans, Cs, batch = _run(batch64, dtype, cfg)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        batch.numeric(stream=s)
        s.synchronize()
        with torch.cuda.graph(g, stream=s):
            batch.numeric(stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    rng = np.random.default_rng(77)
    scaled = []
    for (A, P), (dA, _) in zip(batch64, devs):
        f = rng.uniform(0.5, 2.0, size=A.nnz)
        vals = A.val * f
        dA.val.copy_(torch.as_tensor(vals, dtype=dtype, device="cuda"))
        scaled.append((A.with_values(vals), P))
    for C in Cs:
        C.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    for p in plans:
        p.check()
    _check_all(scaled, plans, Cs, dtype, 900)
    batch.destroy()
