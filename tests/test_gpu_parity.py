"""CUDA path vs the oracle, element by element, through the C ABI.

Sizes span several chunks and hash tiles and leave ragged tails; configs force
heavy chunks, tiny on-chip tables (spill / overflow paths) and both numeric
schemes.  All inputs are seeded.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1905_08423_gb300 import problems as pb
from paper_1905_08423_gb300 import ptap
from parity import check_pattern, check_values, rounded, run_and_check, to_dev

pytestmark = pytest.mark.gpu

DTYPES = [torch.float64, torch.float32]


@pytest.mark.parametrize("dtype", DTYPES)
def test_model_problem_15(dtype):
    """15^3 7-point Laplacian, trilinear P: pattern exact, values exact (dyadic)."""
    A, P = pb.model_problem(15)
    plan, C = run_and_check(A, P, dtype)
    ref = oracle.ptap(A, P)
    np.testing.assert_array_equal(C.cpu().numpy().astype(np.float64), ref.val)
    assert plan.nnz == 6859


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("dtype", DTYPES)
def test_random_small_int(seed, dtype):
    """Random patterns with stored zeros and empty rows; integer values are exact."""
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(1, 200))
    m = int(rng.integers(1, 60))
    A = pb.random_csr(n, n, rng.uniform(0.01, 0.15), rng)
    P = pb.random_csr(n, m, rng.uniform(0.02, 0.2), rng)
    plan, C = run_and_check(A, P, dtype)
    ref = oracle.ptap(A, P)
    np.testing.assert_array_equal(C.cpu().numpy().astype(np.float64), ref.val)


@pytest.mark.parametrize("dtype", DTYPES)
def test_algebraic_20(dtype):
    """27-point lognormal operator with smoothed aggregation (uneven rows)."""
    A, P = pb.algebraic_problem(20, seed=3)
    run_and_check(A, P, dtype)


CONFIGS = [
    dict(),
    dict(chunk_entries=64),                       # many small chunks
    dict(chunk_entries=16),                       # every C row heavier than a chunk
    dict(group_lanes=4), dict(group_lanes=16), dict(group_lanes=32),
    dict(block_threads=128, group_lanes=8, ap_slots=32),
    dict(force_spill=True),                       # tiny tables: spill + overflow paths
    dict(force_spill=True, chunk_entries=64),
    dict(debug_checks=True),
    dict(mode=ptap.MODE_ATOMIC),
    dict(mode=ptap.MODE_ATOMIC, force_spill=True),
    dict(mode=ptap.MODE_ATOMIC, group_lanes=32),
    dict(class_programs=False),                   # general owner kernel
    dict(chunk_entries=256),                      # class programs, many small chunks
    dict(chunk_entries=600, block_threads=128),
    dict(visit_block_log2=6),                     # class programs in 64-row blocks
    dict(visit_block_log2=8, chunk_entries=2048),
    dict(specialize=4, chunk_entries=1024),       # compiled classes and interpreted ones mixed
    dict(block_threads=1024, chunk_entries=32768),  # interpreter, rows of A P in global scratch
    dict(block_threads=512, class_programs=False),  # general kernel: CTA clamped to 256
    dict(class_programs=False, general_kernel=1),  # general kernel with hash groups
    dict(class_programs=False, chunk_entries=128),  # sort-based general kernel, heavy chunks
    dict(class_programs=False, block_threads=64),  # sort-based general kernel, 2 warps a CTA
    dict(cache_indices=True),                     # cached P row starts, interpreter
    dict(cache_indices=True, specialize=4, chunk_entries=1024),  # ... and compiled classes
    dict(cache_indices="visits"),                 # piece records, interpreter
    dict(cache_indices="visits", specialize=4, chunk_entries=1024),  # ... and compiled classes
    dict(cache_indices="visits", chunk_entries=64),  # records over many small chunks
]


LARGE_CTA = [
    dict(specialize=8, block_threads=512, chunk_entries=16384),
    dict(specialize=4, block_threads=1024, chunk_entries=32768),
    dict(block_threads=1024, chunk_entries=32768),
    dict(block_threads=512, chunk_entries=12288),
    dict(specialize=8, block_threads=1024, chunk_entries=32768, cache_indices=True),
    dict(specialize=8, block_threads=1024, chunk_entries=24576, cache_indices="visits"),
]


@pytest.mark.parametrize("cfg", LARGE_CTA, ids=[str(c) for c in LARGE_CTA])
@pytest.mark.parametrize("dtype", DTYPES)
def test_large_ctas_many_chunks(cfg, dtype):
    """CTAs of 512/1024 threads with large chunks, over many chunks (dynamic schedule)."""
    A, P = pb.model_problem(63)
    plan, _ = run_and_check(A, P, dtype, ptap.make_config(**cfg))
    st = plan.stats()
    assert st["fast_path"] == 1 and st["block_threads"] == cfg["block_threads"]
    assert st["n_chunks"] > 8
    if dtype == torch.float64:
        assert st["chunk_entries"] <= 24576     # the accumulator must fit shared memory
    else:
        assert st["chunk_entries"] == cfg["chunk_entries"]


@pytest.mark.parametrize("cfg", CONFIGS, ids=[str(c) for c in CONFIGS])
@pytest.mark.parametrize("dtype", DTYPES)
def test_configs(cfg, dtype):
    A, P = pb.algebraic_problem(13, seed=7)
    run_and_check(A, P, dtype, ptap.make_config(**cfg))
    A2, P2 = pb.model_problem(17)
    run_and_check(A2, P2, dtype, ptap.make_config(**cfg))


def test_two_step_with_large_cta_config():
    """A configuration tuned for the class-program kernels also drives the two-step path."""
    A, P = pb.algebraic_problem(12, seed=5)
    cfg = ptap.make_config(specialize=8, block_threads=1024, chunk_entries=32768)
    plan, _ = run_and_check(A, P, torch.float32, config=cfg, two_step=True)
    assert plan.stats()["block_threads"] == 256


@pytest.mark.parametrize("dtype", DTYPES)
def test_two_step_comparator(dtype):
    A, P = pb.algebraic_problem(14, seed=5)
    plan, C = run_and_check(A, P, dtype, two_step=True)
    st = plan.stats()
    assert st["kind"] == 1
    plan1, C1 = run_and_check(A, P, dtype)
    # the two-step plan holds A P and P^T: more memory than the all-at-once plan
    assert st["plan_bytes"] > plan1.stats()["plan_bytes"]


def test_edge_cases():
    # identity P gives A back
    rng = np.random.default_rng(4)
    A = pb.random_csr(50, 50, 0.1, rng, int_values=False)
    plan, C = run_and_check(A, pb.identity_csr(50), torch.float64)
    np.testing.assert_array_equal(C.cpu().numpy(), A.val)
    # all P rows empty: C has no entries
    Pz = pb.CSR(50, 7, np.zeros(51, np.int32), np.zeros(0, np.int32), np.zeros(0))
    plan, C = run_and_check(A, Pz, torch.float64)
    assert plan.nnz == 0 and C.numel() == 0
    # A with no entries
    Az = pb.CSR(30, 30, np.zeros(31, np.int32), np.zeros(0, np.int32), np.zeros(0))
    Pr = pb.random_csr(30, 9, 0.3, rng)
    plan, C = run_and_check(Az, Pr, torch.float64)
    assert plan.nnz == 0
    # one-by-one problem
    one = pb.CSR(1, 1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([3.0]))
    plan, C = run_and_check(one, one.with_values(np.array([2.0])), torch.float64)
    assert C.item() == 12.0
    # dense-ish rows: a P with a full row and an A row hitting many P rows
    n, m = 40, 300
    rp = np.arange(n + 1, dtype=np.int32) * 0
    cols, vals, lens = [], [], []
    for i in range(n):
        c = np.arange(m) if i == 3 else np.sort(rng.choice(m, 5, replace=False))
        cols.append(c)
        lens.append(len(c))
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    ci = np.concatenate(cols).astype(np.int32)
    Pd = pb.CSR(n, m, rp, ci, rng.standard_normal(ci.size))
    Ad = pb.random_csr(n, n, 0.5, rng, int_values=False)
    run_and_check(Ad, Pd, torch.float64)
    run_and_check(Ad, Pd, torch.float32)
    run_and_check(Ad, Pd, torch.float64, ptap.make_config(chunk_entries=64))


def test_errors():
    A, P = pb.model_problem(7)
    dA, dP = to_dev(A, torch.float64), to_dev(P, torch.float64)
    with pytest.raises(ptap.PtapError) as e:
        ptap.symbolic(dP, dA)   # P is not square
    assert e.value.code == 1
    plan = ptap.symbolic(dA, dP)
    A2, P2 = pb.model_problem(9)
    with pytest.raises(ptap.PtapError) as e:
        ptap.numeric(plan, to_dev(A2, torch.float64), to_dev(P2, torch.float64),
                     out=torch.empty(plan.nnz, dtype=torch.float64, device="cuda"))
    assert e.value.code == 2
    # unsorted columns are rejected when checks are on
    bad = pb.CSR(A.nrows, A.ncols, A.row_ptr, A.col_idx.copy(), A.val)
    bad.col_idx[1], bad.col_idx[2] = bad.col_idx[2], bad.col_idx[1]
    with pytest.raises(ptap.PtapError) as e:
        ptap.symbolic(to_dev(bad, torch.float64), dP, ptap.make_config(debug_checks=True))
    assert e.value.code == 1


@pytest.mark.parametrize("dtype", DTYPES)
def test_backward_vs_oracle(dtype):
    A, P = pb.poisson2d_problem(64)
    Pt = pb.perturb_values(P, seed=5)
    Ar, Pr = rounded(A, dtype), rounded(P, dtype)
    dA_, dP_ = to_dev(A, dtype), to_dev(P, dtype)
    plan = ptap.symbolic(dA_, dP_)
    C = ptap.numeric(plan, dA_, dP_)
    Ct = ptap.numeric(plan, dA_, to_dev(Pt, dtype))
    G = 2.0 * (C - Ct)
    gA, gP = ptap.backward(plan, dA_, dP_, G)
    torch.cuda.synchronize()
    Cref = oracle.ptap(Ar, Pr)
    Gh = pb.CSR(Cref.nrows, Cref.ncols, Cref.row_ptr, Cref.col_idx,
                G.cpu().numpy().astype(np.float64))
    eA, eP = oracle.ptap_backward(Ar, Pr, Gh)
    # bounds: the same products on absolute values
    absG = Gh.with_values(np.abs(Gh.val))
    bA, bP = oracle.ptap_backward(Ar.abs(), Pr.abs(), absG)
    check_values(gA, eA, bA, dtype)
    check_values(gP, eP, bP, dtype)


def test_autograd_function():
    A, P = pb.poisson2d_problem(32)
    dA_, dP_ = to_dev(A, torch.float64), to_dev(P, torch.float64)
    plan = ptap.symbolic(dA_, dP_)
    Pt = to_dev(pb.perturb_values(P, seed=1), torch.float64)
    Ct = ptap.numeric(plan, dA_, Pt)
    Av = dA_.val.clone().requires_grad_(True)
    Pv = dP_.val.clone().requires_grad_(True)
    C = ptap.PtAP.apply(Av, Pv, plan, dA_, dP_)
    loss = ((C - Ct) ** 2).sum()
    loss.backward()
    # central differences along a random direction
    g = torch.Generator(device="cuda").manual_seed(0)
    v = torch.randn(Pv.shape, generator=g, device="cuda", dtype=torch.float64)
    h = 1e-6
    with torch.no_grad():
        lp = ((ptap.PtAP.apply(Av, Pv + h * v, plan, dA_, dP_) - Ct) ** 2).sum()
        lm = ((ptap.PtAP.apply(Av, Pv - h * v, plan, dA_, dP_) - Ct) ** 2).sum()
    fd = (lp - lm).item() / (2 * h)
    an = (Pv.grad * v).sum().item()
    assert abs(fd - an) <= 1e-6 * abs(an)


def _oracle_gd(A, P, Pt, lr, steps):
    """Gradient descent on P's values with the oracle's product and gradient."""
    Ct = oracle.ptap(A, Pt)
    pv, hist = P.val.copy(), []
    for _ in range(steps):
        Pc = P.with_values(pv)
        C = oracle.ptap(A, Pc)
        d = C.val - Ct.val
        hist.append(float((d * d).sum()))
        _, gP = oracle.ptap_backward(A, Pc, pb.CSR(C.nrows, C.ncols, C.row_ptr, C.col_idx, 2 * d))
        pv = pv - lr * gP
    return hist


@pytest.mark.parametrize("dtype", DTYPES)
def test_gradient_descent_on_P(dtype):
    """Descent on P's values through the coarse operator follows the oracle's descent.

    Loss ||P^T A P - C_target||_F^2, C_target from P's values plus N(0, 0.05)
    noise; fixed step 1/32 (the largest power of two whose first step lowers
    the loss on this case).
    """
    A, P = pb.poisson2d_problem(64)
    Pt = pb.perturb_values(P, seed=5)
    Ar, Pr, Ptr = rounded(A, dtype), rounded(P, dtype), rounded(Pt, dtype)
    dA_, dP_ = to_dev(A, dtype), to_dev(P, dtype)
    plan = ptap.symbolic(dA_, dP_)
    Ct = ptap.numeric(plan, dA_, to_dev(Pt, dtype))
    Pv = dP_.val.clone().requires_grad_(True)
    lr, steps, hist = 1.0 / 32, 10, []
    for _ in range(steps):
        Pv.grad = None
        loss = ((ptap.PtAP.apply(dA_.val, Pv, plan, dA_, dP_) - Ct) ** 2).sum()
        loss.backward()
        hist.append(loss.item())
        with torch.no_grad():
            Pv -= lr * Pv.grad
    ref = _oracle_gd(Ar, Pr, Ptr, lr, steps)
    assert all(y < x for x, y in zip(hist, hist[1:]))
    assert hist[-1] < 0.05 * hist[0]
    tol = 1e-9 if dtype == torch.float64 else 2e-3
    for g, r in zip(hist, ref):
        assert abs(g - r) <= tol * r, (hist, ref)


@pytest.mark.parametrize("dtype", DTYPES)
def test_batch_and_graph(dtype):
    probs = pb.batch_problems(seed=4, count=6, lo=8, hi=20)
    devs, plans, Cs, refs = [], [], [], []
    for A, P in probs:
        dA_, dP_ = to_dev(A, dtype), to_dev(P, dtype)
        plan = ptap.symbolic(dA_, dP_)
        devs.append((dA_, dP_))
        plans.append(plan)
        Cs.append(torch.empty(plan.nnz, dtype=dtype, device="cuda"))
    batch = ptap.Batch(plans, [d[0] for d in devs], [d[1] for d in devs], Cs)
    batch.numeric()
    torch.cuda.synchronize()
    for (A, P), C in zip(probs, Cs):
        Ar, Pr = rounded(A, dtype), rounded(P, dtype)
        check_values(C, oracle.ptap(Ar, Pr).val, oracle.ptap_bound(Ar, Pr).val, dtype)
    # capture once, rescale A's values in place, replay
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        batch.numeric(stream=s)  # warm-up on the capture stream
        s.synchronize()
        with torch.cuda.graph(graph, stream=s):
            batch.numeric(stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for r in range(2):
        scaled = []
        for q, (A, P) in enumerate(probs):
            A2 = pb.rescale_values(A, seed=40 + 10 * r + q)
            devs[q][0].val.copy_(torch.as_tensor(A2.val, dtype=dtype, device="cuda"))
            scaled.append(A2)
        graph.replay()
        torch.cuda.synchronize()
        for (A, P), A2, C in zip(probs, scaled, Cs):
            Ar, Pr = rounded(A2, dtype), rounded(P, dtype)
            check_values(C, oracle.ptap(Ar, Pr).val, oracle.ptap_bound(Ar, Pr).val, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
def test_class_programs_engaged(dtype):
    """Mesh operators run on per-class programs; results match the oracle and the general kernel."""
    for A, P in (pb.model_problem(19), pb.algebraic_problem(16, seed=9), pb.poisson2d_problem(40)):
        plan, C = run_and_check(A, P, dtype)
        st = plan.stats()
        assert st["fast_path"] == 1 and st["n_classes"] > 0 and st["n_segments"] >= st["n_chunks"]
        plan_g, C_g = run_and_check(A, P, dtype, ptap.make_config(class_programs=False))
        assert plan_g.stats()["fast_path"] == 0


def test_class_programs_declined():
    """Rows beyond the fast-path limits (here: 40 entries in a row of A) use the general kernel."""
    rng = np.random.default_rng(17)
    A = pb.random_csr(120, 120, 0.4, rng)
    P = pb.random_csr(120, 20, 0.1, rng)
    plan, C = run_and_check(A, P, torch.float64)
    assert plan.stats()["fast_path"] == 0


@pytest.mark.parametrize("dtype", DTYPES)
def test_specialized_classes(dtype):
    """Plan-time compiled class code matches the oracle and the interpreter."""
    for A, P in (pb.model_problem(21), pb.algebraic_problem(15, seed=12), pb.poisson2d_problem(48)):
        plan, C = run_and_check(A, P, dtype, ptap.make_config(specialize=8))
        st = plan.stats()
        assert st["fast_path"] == 1 and 0 < st["n_specialized"] <= 8
        plan_i, C_i = run_and_check(A, P, dtype, ptap.make_config())
        assert plan_i.stats()["n_specialized"] == 0
        tol = 1e-12 if dtype == torch.float64 else 1e-5
        B = oracle.ptap_bound(rounded(A, dtype), rounded(P, dtype)).val
        err = np.abs(C.cpu().numpy().astype(np.float64) - C_i.cpu().numpy().astype(np.float64))
        assert (err <= 2 * tol * B + 1e-300).all()


_JIT_PROBE = """
import sys
sys.path.insert(0, {root!r})
import torch
from paper_1905_08423_gb300 import problems as pb, ptap
A, P = pb.model_problem(17)
dA = ptap.Csr.from_host(A, "cuda", torch.float32)
dP = ptap.Csr.from_host(P, "cuda", torch.float32)
st = ptap.symbolic(dA, dP, ptap.make_config(specialize=6)).stats()
print(st["n_specialized"], st["specialize_us"])
"""


def test_specialized_disk_cache(tmp_path):
    """A second process with the same classes loads the cubin instead of compiling it."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PTAP_JIT_CACHE=str(tmp_path / "jit"))
    code = _JIT_PROBE.format(root=root)
    runs = []
    for _ in range(2):
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                           timeout=600, cwd=root)
        assert r.returncode == 0, r.stderr[-2000:]
        runs.append([int(x) for x in r.stdout.split()[-2:]])
    assert runs[0][0] > 0 and runs[1][0] == runs[0][0]
    assert len(list((tmp_path / "jit").glob("jit_*_sm103a.cubin"))) == 1
    assert runs[1][1] < runs[0][1] / 3, runs     # load instead of compile


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("pinned", [True, False])
def test_numeric_host(dtype, pinned):
    """ptap_numeric_host: successive products from host values, each checked against the oracle.

    Three calls in a row (A rescaled before each) overlap through the staging
    buffers; every host result must match its own inputs.
    """
    A, P = pb.model_problem(31)
    dA_, dP_ = to_dev(A, dtype), to_dev(P, dtype)
    plan = ptap.symbolic(dA_, dP_)
    ins, outs = [], []
    for k in range(3):
        Ak = pb.rescale_values(A, seed=80 + k)
        hA = torch.as_tensor(rounded(Ak, dtype).val).to(dtype)
        hP = torch.as_tensor(rounded(P, dtype).val).to(dtype)
        hC = torch.full((plan.nnz,), float("nan"), dtype=dtype)
        if pinned:
            hA, hP, hC = hA.pin_memory(), hP.pin_memory(), hC.pin_memory()
        ptap.numeric_host(plan, dA_, dP_, hA, hP, hC)
        ins.append(Ak)
        outs.append(hC)
    torch.cuda.synchronize()
    Pr = rounded(P, dtype)
    for Ak, hC in zip(ins, outs):
        Ar = rounded(Ak, dtype)
        check_values(hC, oracle.ptap(Ar, Pr).val, oracle.ptap_bound(Ar, Pr).val, dtype)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_background_specialisation(dtype):
    """specialize_async: ptap_symbolic returns before NVRTC finishes; numeric products run
    the interpreter until the compiled kernel is loaded, then switch to it; both agree with
    the oracle."""
    import time
    A, P = pb.model_problem(33)
    Ar, Pr = rounded(A, dtype), rounded(P, dtype)
    ref, bound = oracle.ptap(Ar, Pr), oracle.ptap_bound(Ar, Pr)
    dA, dP = to_dev(A, dtype), to_dev(P, dtype)
    # a class count no other test compiles, so the compile is not already cached in the process
    cfg = ptap.make_config(specialize=5, specialize_async=True, block_threads=512, chunk_entries=2048)
    plan = ptap.symbolic(dA, dP, cfg)
    check_pattern(plan, ref)
    C = ptap.numeric(plan, dA, dP)           # interpreter or compiled, whichever is ready
    torch.cuda.synchronize()
    check_values(C, ref.val, bound.val, dtype)
    t0 = time.time()
    while plan.stats()["n_specialized"] == 0 and time.time() - t0 < 120:
        time.sleep(0.05)
    assert plan.stats()["n_specialized"] > 0, "the background compile did not finish"
    C2 = ptap.numeric(plan, dA, dP)
    torch.cuda.synchronize()
    plan.check()
    check_values(C2, ref.val, bound.val, dtype)
    plan.destroy()


def test_background_specialisation_destroy_while_compiling():
    """Destroying a plan whose compile is still running waits for it; nothing leaks or faults."""
    A, P = pb.model_problem(21)
    dA, dP = to_dev(A, torch.float64), to_dev(P, torch.float64)
    plan = ptap.symbolic(dA, dP, ptap.make_config(specialize=6, specialize_async=True, chunk_entries=1024))
    plan.destroy()


@pytest.mark.parametrize("dtype", DTYPES)
def test_piece_records(dtype):
    """Indices cached per visit: the plan holds piece records (one int32 per entry of A(I,:)
    and one uint16 per entry of P(I,:) for every lane of every piece, plus an offset per
    piece), the compiled and interpreted classes both read them, and C matches the oracle;
    compact chunks fall back to the per-entry cache."""
    A, P = pb.model_problem(31)
    cfg = dict(cache_indices="visits", specialize=8, block_threads=1024, chunk_entries=8192)
    plan, _ = run_and_check(A, P, dtype, ptap.make_config(**cfg))
    st = plan.stats()
    assert st["fast_path"] == 1 and st["cache_indices"] == 2 and st["n_specialized"] == 8
    assert 0 < st["specialized_permille"] < 1000            # interpreted classes too
    assert st["cached_index_bytes"] >= 4 * st["n_pieces"] + 2 * 32 * st["n_pieces"]
    plan_c, _ = run_and_check(A, P, dtype, ptap.make_config(**dict(cfg, compact_chunks=1)))
    stc = plan_c.stats()
    assert stc["compact_chunks"] == 1 and stc["cache_indices"] == 1
    assert stc["cached_index_bytes"] == 4 * A.nnz
