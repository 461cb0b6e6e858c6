"""Full-size parity of every launch configuration the autotuner may choose.

The benchmark times the configuration ``autotune.tune`` picks on its own
workload.  The tuner picks among ``autotune.candidates_all(A, P)`` (its first round and
the second-round refinements of each), so checking every one of those at full
size covers whichever wins, on the same
inputs the benchmark uses: the 319^3 model problem (FP32 and FP64) and the
200^3 algebraic case (FP64).  For each candidate the whole pattern is checked
by its closed form and ~3,600 sampled coarse rows against the oracle's rows of
Eq. 8, within tau * (|P|^T|A||P|)(i,j).  Each plan runs two numeric products
(the second on a re-product with the pattern resident).
"""
import json

import numpy as np
import pytest
import torch

from paper_1905_08423_gb300 import autotune
from paper_1905_08423_gb300 import problems as pb
from paper_1905_08423_gb300 import ptap
from parity import check_sampled, sample_rows, sampled_reference, to_dev

pytestmark = pytest.mark.gpu


def _closed_form_lengths(md):
    k = np.full(md, 3, dtype=np.int64)
    k[0] = k[-1] = 2
    return (k[None, None, :] * k[None, :, None] * k[:, None, None]).reshape(-1)


@pytest.fixture(scope="module")
def model319():
    return pb.model_problem(319)


def _every_candidate(A, P, dtype, rows, lengths=None, nnz=None):
    dA, dP = to_dev(A, dtype), to_dev(P, dtype)
    ref, bnd = sampled_reference(A, P, dtype, rows)
    cands = autotune.candidates_all(dA, dP)
    assert cands, "the tuner offered no candidate"
    checked = []
    for cand in cands:
        plan = ptap.symbolic(dA, dP, ptap.make_config(**cand))
        if nnz is not None:
            assert plan.nnz == nnz, cand
        if lengths is not None:
            rp, _ = plan.pattern()
            np.testing.assert_array_equal(np.diff(rp.cpu().numpy().astype(np.int64)), lengths)
        C = torch.full((plan.nnz,), float("nan"), dtype=dtype, device="cuda")
        for _ in range(2):
            ptap.numeric(plan, dA, dP, C)
            torch.cuda.synchronize()
            plan.check()
            try:
                check_sampled(plan, C, ref, bnd, rows, dtype)
            except AssertionError as e:
                raise AssertionError(f"candidate {json.dumps(cand)}: {e}") from None
        checked.append((cand, plan.stats()["fast_path"], plan.stats()["n_specialized"]))
        plan.destroy()
        del C
    torch.cuda.empty_cache()
    return checked


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_model319_every_candidate(model319, dtype):
    A, P = model319
    rows = sample_rows(P.ncols, 3000, 11)
    checked = _every_candidate(A, P, dtype, rows, _closed_form_lengths(159), 107_171_875)
    # the class-program kernels with compiled classes are among those checked
    assert any(fast and spec > 0 for _, fast, spec in checked)


def test_algebraic200_every_candidate():
    A, P = pb.algebraic_problem(200, seed=3)
    rows = sample_rows(P.ncols, 2000, 12)
    _every_candidate(A, P, torch.float64, rows, nnz=7_880_599)
