"""Shared checks of the CUDA path against the oracle (imported by the tests).

Tolerance (values): |C_gpu(i,j) - C_oracle(i,j)| <= tau * B(i,j) with
B = |P|^T |A| |P|, tau = 1e-12 for float64 and 1e-5 for float32; where
B(i,j) = 0 the values must be equal.  For float32 the oracle runs in float64
on the float32-rounded inputs, so input rounding is not charged to the kernel.
Patterns (row_ptr, col_idx) must match bit for bit.
"""
import numpy as np
import torch

import oracle
from paper_1905_08423_gb300 import ptap
from paper_1905_08423_gb300.problems import CSR

TAU = {torch.float64: 1e-12, torch.float32: 1e-5}


def rounded(M: CSR, dtype) -> CSR:
    """Host copy of M with values rounded to ``dtype`` and held in float64."""
    if dtype == torch.float32:
        return M.with_values(M.val.astype(np.float32).astype(np.float64))
    return M


def to_dev(M: CSR, dtype) -> ptap.Csr:
    return ptap.Csr.from_host(M, device="cuda", dtype=dtype)


def check_pattern(plan: ptap.Plan, ref) -> None:
    rp, ci = plan.pattern()
    np.testing.assert_array_equal(rp.cpu().numpy(), ref.row_ptr)
    np.testing.assert_array_equal(ci.cpu().numpy(), ref.col_idx)


def check_values(vals: torch.Tensor, ref_vals: np.ndarray, bound: np.ndarray, dtype) -> float:
    got = vals.detach().cpu().numpy().astype(np.float64)
    err = np.abs(got - ref_vals)
    tau = TAU[dtype]
    ok = np.where(bound > 0, err <= tau * bound, err == 0)
    if not ok.all():
        bad = np.nonzero(~ok)[0][:5]
        raise AssertionError(f"{(~ok).sum()} entries out of tolerance; first {bad}: "
                             f"got {got[bad]}, want {ref_vals[bad]}, bound {bound[bad]}")
    rel = err / np.where(bound > 0, bound, 1.0)
    return float(rel.max()) if rel.size else 0.0


def run_and_check(A: CSR, P: CSR, dtype=torch.float64, config=None, two_step=False):
    """Symbolic + numeric on the GPU, checked against the oracle.  Returns the plan."""
    Ar, Pr = rounded(A, dtype), rounded(P, dtype)
    ref = oracle.ptap(Ar, Pr)
    bound = oracle.ptap_bound(Ar, Pr)
    dA, dP = to_dev(A, dtype), to_dev(P, dtype)
    plan = (ptap.two_step_symbolic if two_step else ptap.symbolic)(dA, dP, config)
    check_pattern(plan, ref)
    C = ptap.numeric(plan, dA, dP)
    torch.cuda.synchronize()
    plan.check()
    check_values(C, ref.val, bound.val, dtype)
    # a second numeric on the same plan gives the same answer (re-product)
    C2 = ptap.numeric(plan, dA, dP)
    torch.cuda.synchronize()
    check_values(C2, ref.val, bound.val, dtype)
    return plan, C


def sample_rows(m: int, k: int, seed: int) -> np.ndarray:
    """The first and last 300 coarse rows plus k random ones (sorted, unique)."""
    rng = np.random.default_rng(seed)
    head = np.arange(min(300, m))
    tail = np.arange(max(0, m - 300), m)
    mid = rng.choice(m, size=min(k, m), replace=False)
    return np.unique(np.concatenate([head, tail, mid])).astype(np.int32)


def sampled_reference(A: CSR, P: CSR, dtype, rows: np.ndarray):
    """Oracle rows of C and of the bound B = |P|^T|A||P| for the coarse rows ``rows`` (Eq. 8)."""
    Ar, Pr = rounded(A, dtype), rounded(P, dtype)
    ref = oracle.ptap_rows(Ar, Pr, rows, PT=oracle.transpose(Pr))
    Aa, Pa = Ar.abs(), Pr.abs()
    bnd = oracle.ptap_rows(Aa, Pa, rows, PT=oracle.transpose(Pa))
    return ref, bnd


def check_sampled(plan: ptap.Plan, C: torch.Tensor, ref, bnd, rows: np.ndarray, dtype) -> float:
    """Row lengths, columns and values of the sampled rows of C against the oracle's."""
    rp, ci = plan.pattern()
    rp = rp.cpu().numpy().astype(np.int64)
    idx = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows])
    it = torch.as_tensor(idx, device=ci.device)
    got_c = ci[it].cpu().numpy()
    got_v = C[it].cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(np.diff(ref.row_ptr), rp[rows + 1] - rp[rows])
    np.testing.assert_array_equal(got_c, ref.col_idx)
    return check_values_np(got_v, ref.val, bnd.val, dtype)


def check_values_np(got: np.ndarray, want: np.ndarray, bound: np.ndarray, dtype) -> float:
    err = np.abs(got - want)
    ok = np.where(bound > 0, err <= TAU[dtype] * bound, err == 0)
    if not ok.all():
        bad = np.nonzero(~ok)[0][:5]
        raise AssertionError(f"{(~ok).sum()} sampled entries out of tolerance; first {bad}: "
                             f"got {got[bad]}, want {want[bad]}, bound {bound[bad]}")
    rel = err / np.where(bound > 0, bound, 1.0)
    return float(rel.max()) if rel.size else 0.0
