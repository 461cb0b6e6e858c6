"""Autotuner for the triple product's launch parameters.

The numeric product is repeated many times on one symbolic result (Section
4.1: one symbolic and eleven numeric products per setup), so a few trial
products to pick the launch parameters pay for themselves.  ``tune`` builds a
plan per candidate configuration (chunk size of the on-chip accumulator, CTA
size, lanes per fine row and hash slots of the general kernel, visit order,
plan-time specialisation and chunk shape (row ranges or compact regions of C's
graph) of the class-program kernel, owner or atomic scheme),
times repeated numeric products with CUDA events, and returns the fastest.
Choices are cached in a JSON file keyed by (GPU name, dtype, problem
signature); the signature is the shapes, the nonzero counts and a hash of the
row-length sequences of A and P.
"""
from __future__ import annotations

import hashlib
import json
import os
from dataclasses import dataclass, field

import numpy as np

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "ptap_autotune.json")

# Candidate configurations (keyword arguments of ptap.make_config).
CANDIDATES = [
    dict(),
    dict(specialize=8),
    dict(specialize=8, block_threads=512, chunk_entries=16384),
    dict(specialize=8, block_threads=1024, chunk_entries=32768),
    dict(specialize=16, block_threads=1024, chunk_entries=32768),
    dict(specialize=32, block_threads=1024, chunk_entries=32768),
    dict(specialize=32, block_threads=1024, chunk_entries=32768, compact_chunks=32),
    dict(specialize=4, block_threads=1024, chunk_entries=32768),
    dict(block_threads=512, chunk_entries=16384),
    dict(chunk_entries=4096),
    dict(class_programs=False),
    dict(mode=2, group_lanes=8, ap_slots=32),
]


def signature(A, P) -> str:
    """Shape, nonzero counts and a hash of the row-length sequences of A and P."""
    h = hashlib.sha1()
    for M in (A, P):
        rp = np.asarray(M.row_ptr.cpu() if hasattr(M.row_ptr, "cpu") else M.row_ptr, dtype=np.int64)
        h.update(np.diff(rp).astype(np.int32).tobytes())
    return f"{A.nrows}x{A.ncols}:{A.nnz}|{P.nrows}x{P.ncols}:{P.nnz}|{h.hexdigest()[:16]}"


def cache_key(gpu: str, dtype: str, sig: str) -> str:
    return f"{gpu}|{dtype}|{sig}"


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str = DEFAULT_CACHE) -> None:
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


@dataclass
class TuneResult:
    config: dict
    ms: float
    trials: list = field(default_factory=list)  # (config, ms or error string)
    cached: bool = False
    symbolic_ms: list = field(default_factory=list)  # (config, symbolic ms incl. any code generation)


def _time_numeric(ptap, plan, A, P, C, reps: int, warmup: int) -> float:
    import torch
    for _ in range(warmup):
        ptap.numeric(plan, A, P, C)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        ptap.numeric(plan, A, P, C)
    e1.record()
    torch.cuda.synchronize()
    plan.check()
    return e0.elapsed_time(e1) / reps


def tune(A, P, candidates=None, reps: int = 5, warmup: int = 2, cache_path: str | None = DEFAULT_CACHE,
         use_cache: bool = True) -> TuneResult:
    """Times each candidate configuration on the device matrices A, P (ptap.Csr).

    Returns the fastest configuration (keyword arguments of ptap.make_config).
    Candidates that fail (for example by exceeding shared memory) are skipped.
    """
    import torch

    from . import ptap
    gpu = torch.cuda.get_device_name()
    dtype = "f64" if A.dtype_code == ptap.F64 else "f32"
    key = cache_key(gpu, dtype, signature(A, P))
    cache = load_cache(cache_path) if (cache_path and use_cache) else {}
    if use_cache and key in cache:
        e = cache[key]
        return TuneResult(dict(e["config"]), float(e["ms"]), [], cached=True)
    best, best_ms, trials, sym = None, float("inf"), [], []
    for cand in (candidates or CANDIDATES):
        try:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            plan = ptap.symbolic(A, P, ptap.make_config(**cand))
            e1.record()
            torch.cuda.synchronize()
            sym.append((cand, e0.elapsed_time(e1)))
            C = torch.empty(plan.nnz, dtype=plan.torch_dtype, device=A.row_ptr.device)
            ms = _time_numeric(ptap, plan, A, P, C, reps, warmup)
            plan.destroy()
            del C
        except ptap.PtapError as e:
            trials.append((cand, str(e)))
            continue
        trials.append((cand, ms))
        if ms < best_ms:
            best, best_ms = dict(cand), ms
    if best is None:
        raise RuntimeError("no candidate configuration ran")
    if cache_path:
        cache = load_cache(cache_path)
        cache[key] = {"config": best, "ms": best_ms}
        save_cache(cache, cache_path)
    return TuneResult(best, best_ms, trials, symbolic_ms=sym)
