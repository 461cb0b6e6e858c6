"""Autotuner: signature and cache logic on the CPU; tuning on the GPU."""
import json

import numpy as np
import pytest

from paper_1905_08423_gb300 import autotune
from paper_1905_08423_gb300 import problems as pb


def test_signature_and_cache(tmp_path):
    A, P = pb.model_problem(9)
    A2, P2 = pb.algebraic_problem(9, seed=1)
    s1, s2 = autotune.signature(A, P), autotune.signature(A2, P2)
    assert s1 == autotune.signature(A, P) and s1 != s2
    # same sizes, different pattern -> different signature
    B = pb.CSR(A.nrows, A.ncols, A.row_ptr.copy(), A.col_idx, A.val)
    B.row_ptr[1] += 0  # unchanged pattern
    assert autotune.signature(B, P) == s1
    path = str(tmp_path / "cache.json")
    assert autotune.load_cache(path) == {}
    key = autotune.cache_key("GPU", "f32", s1)
    autotune.save_cache({key: {"config": {"chunk_entries": 4096}, "ms": 1.5}}, path)
    c = autotune.load_cache(path)
    assert c[key]["config"] == {"chunk_entries": 4096} and c[key]["ms"] == 1.5
    open(path, "w").write("not json")
    assert autotune.load_cache(path) == {}


@pytest.mark.gpu
def test_tune_and_parity(tmp_path):
    import torch
    from paper_1905_08423_gb300 import ptap
    from parity import run_and_check, to_dev
    A, P = pb.algebraic_problem(14, seed=21)
    dA, dP = to_dev(A, torch.float64), to_dev(P, torch.float64)
    path = str(tmp_path / "tune.json")
    cands = [dict(specialize=False), dict(class_programs=False), dict(mode=ptap.MODE_ATOMIC),
             dict(chunk_entries=1024, specialize=False)]
    r = autotune.tune(dA, dP, candidates=cands, reps=2, warmup=1, cache_path=path)
    assert r.config in cands and r.ms > 0 and len(r.trials) == len(cands) and not r.cached
    again = autotune.tune(dA, dP, candidates=cands, cache_path=path)
    assert again.cached and again.config == r.config
    run_and_check(A, P, torch.float64, ptap.make_config(**r.config))


def test_candidate_rounds():
    """First round: every class-program launch with 16 compiled classes, with and without
    cached indices (per entry of A; per visit at the resident CTA size); second round: the
    same launch with 32 and 64 classes, never fewer than the first, none for the interpreter."""
    optin = 232448
    for vb, bt in ((4, 1024), (8, 512)):
        first = autotune.candidate_list(True, 439, vb, optin)
        spec = {c["specialize"] for c in first if "specialize" in c}
        assert spec == {16}
        assert any(c.get("cache_indices") is True for c in first)
        visits = [c for c in first if c.get("cache_indices") == "visits"]
        assert visits and all(c["block_threads"] == bt for c in visits)
        assert len({json.dumps(c, sort_keys=True) for c in first}) == len(first)
        for c in first:
            r = autotune.refinements(c, 439)
            if "specialize" in c:
                assert r == [dict(c, specialize=32), dict(c, specialize=64)]
            else:
                assert r == []
    # few classes: the counts stop at the class count
    few = autotune.candidate_list(True, 20, 4, optin)
    assert {c["specialize"] for c in few if "specialize" in c} == {16}
    assert all(autotune.refinements(c, 20) == ([dict(c, specialize=20)] if "specialize" in c else [])
               for c in few)
    assert autotune.refinements(dict(specialize=16), 12) == []
    assert autotune.refinements(dict(specialize=32), 40) == [dict(specialize=40)]
    # outside the class programs: general kernels and the atomic scheme only
    gen = autotune.candidate_list(False, 0, 8, optin)
    assert all("specialize" not in c for c in gen) and dict(mode=2, group_lanes=8, ap_slots=64) in gen
