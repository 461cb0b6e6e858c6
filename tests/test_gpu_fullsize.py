"""Full-size parity with the default launch configuration (the configurations
the autotuner offers, one of which the benchmark times, are covered at full
size by test_gpu_tuned.py).

At these sizes the oracle computes sampled rows of C one by one (Eq. 8 row
form); properties that hold at any size are checked on the whole output:
the model problem's row lengths have a closed form (product over axes of the
coarse neighbours in range), and nnz(C) = (3 m_d - 2)^3 on cubes.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1905_08423_gb300 import problems as pb
from paper_1905_08423_gb300 import ptap
from parity import TAU, rounded, to_dev

pytestmark = pytest.mark.gpu


def _sample_rows(m, k, seed):
    rng = np.random.default_rng(seed)
    head = np.arange(min(300, m))
    tail = np.arange(max(0, m - 300), m)
    mid = rng.choice(m, size=min(k, m), replace=False)
    return np.unique(np.concatenate([head, tail, mid])).astype(np.int32)


def _check_sampled(plan, C, A, P, dtype, rows):
    Ar, Pr = rounded(A, dtype), rounded(P, dtype)
    PT = oracle.transpose(Pr)
    ref = oracle.ptap_rows(Ar, Pr, rows, PT=PT)
    bnd = oracle.ptap_rows(Ar.abs(), Pr.abs(), rows, PT=oracle.transpose(Pr.abs()))
    rp, ci = plan.pattern()
    rp = rp.cpu().numpy().astype(np.int64)
    ci_t, C_t = ci, C
    idx = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows])
    got_c = ci_t[torch.as_tensor(idx, device=ci_t.device)].cpu().numpy()
    got_v = C_t[torch.as_tensor(idx, device=C_t.device)].cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(np.diff(ref.row_ptr), rp[rows + 1] - rp[rows])
    np.testing.assert_array_equal(got_c, ref.col_idx)
    err = np.abs(got_v - ref.val)
    ok = np.where(bnd.val > 0, err <= TAU[dtype] * bnd.val, err == 0)
    assert ok.all(), f"{(~ok).sum()} sampled entries out of tolerance"


def _closed_form_lengths(md):
    k = np.full(md, 3, dtype=np.int64)
    k[0] = k[-1] = 2
    return (k[None, None, :] * k[None, :, None] * k[:, None, None]).reshape(-1)


@pytest.fixture(scope="module")
def model319():
    return pb.model_problem(319)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_model_problem_319(model319, dtype):
    A, P = model319
    dA, dP = to_dev(A, dtype), to_dev(P, dtype)
    plan = ptap.symbolic(dA, dP)
    assert plan.nnz == 107_171_875 == (3 * 159 - 2) ** 3
    rp, _ = plan.pattern()
    np.testing.assert_array_equal(np.diff(rp.cpu().numpy().astype(np.int64)),
                                  _closed_form_lengths(159))
    C = ptap.numeric(plan, dA, dP)
    torch.cuda.synchronize()
    plan.check()
    _check_sampled(plan, C, A, P, dtype, _sample_rows(P.ncols, 3000, 1))
    # interior rows of the Galerkin operator of a Laplacian with linear P sum to zero
    del dA, dP
    plan.destroy()
    torch.cuda.empty_cache()


def test_model_problem_319_two_step(model319):
    A, P = model319
    dtype = torch.float64
    dA, dP = to_dev(A, dtype), to_dev(P, dtype)
    plan = ptap.two_step_symbolic(dA, dP)
    assert plan.nnz == 107_171_875
    C = ptap.numeric(plan, dA, dP)
    torch.cuda.synchronize()
    plan.check()
    _check_sampled(plan, C, A, P, dtype, _sample_rows(P.ncols, 1000, 2))
    plan.destroy()
    torch.cuda.empty_cache()


def test_algebraic_200():
    A, P = pb.algebraic_problem(200, seed=3)
    dtype = torch.float64
    dA, dP = to_dev(A, dtype), to_dev(P, dtype)
    plan = ptap.symbolic(dA, dP)
    assert plan.nnz == (3 * 67 - 2) ** 3 == 7_880_599
    C = ptap.numeric(plan, dA, dP)
    torch.cuda.synchronize()
    plan.check()
    _check_sampled(plan, C, A, P, dtype, _sample_rows(P.ncols, 2000, 3))
    plan.destroy()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_poisson_512_full(dtype):
    A, P = pb.poisson2d_problem(512)
    Ar, Pr = rounded(A, dtype), rounded(P, dtype)
    dA, dP = to_dev(A, dtype), to_dev(P, dtype)
    plan = ptap.symbolic(dA, dP)
    C = ptap.numeric(plan, dA, dP)
    torch.cuda.synchronize()
    ref = oracle.ptap(Ar, Pr)
    bnd = oracle.ptap_bound(Ar, Pr)
    rp, ci = plan.pattern()
    np.testing.assert_array_equal(rp.cpu().numpy(), ref.row_ptr)
    np.testing.assert_array_equal(ci.cpu().numpy(), ref.col_idx)
    err = np.abs(C.cpu().numpy().astype(np.float64) - ref.val)
    assert (np.where(bnd.val > 0, err <= TAU[dtype] * bnd.val, err == 0)).all()
