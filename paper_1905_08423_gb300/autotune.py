"""Autotuner for the triple product's launch parameters.

The numeric product is repeated many times on one symbolic result (Section
4.1: one symbolic and eleven numeric products per setup), so a few trial
products to pick the launch parameters pay for themselves.

``candidates`` derives the configurations to try from the problem itself:
one default symbolic pass tells whether the fine rows fall into structure
classes (the class-program kernels) and how many classes carry the visits;
the device's opt-in shared memory and the value size bound the on-chip
accumulator (chunk entries) for each CTA size; the general kernels get their
lanes per fine row, hash slots and chunk sizes, and the atomic scheme (Alg. 8
taken literally) is always among them.  ``tune`` builds a plan per candidate,
times repeated numeric products with CUDA events, tries more compiled classes
for the two fastest, and returns the fastest.
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

# Shared memory a class-program CTA keeps beside its accumulator (row offsets,
# per-warp program buffers); the library sizes its largest chunk the same way.
_FAST_RESERVE = 32 * 1024
_MAX_CHUNK = 65536
_GENERAL_MAX_CHUNK = 16384


def chunk_limit(value_bytes: int, smem_optin: int) -> int:
    """Largest class-program chunk (entries) whose accumulator fits the opt-in shared memory."""
    n = (smem_optin - _FAST_RESERVE) // value_bytes
    return max(1024, min(_MAX_CHUNK, n & ~1023))


def _spec_counts(n_classes: int) -> list:
    """Compiled-class counts the tuner tries: 16 in the first round, 32 and 64 in the second
    (fewer if the problem has fewer).  More classes compiled means fewer interpreted visits
    but more code competing for the instruction cache, and which wins depends on the problem:
    64 on the 319^3 model problem (57 compiled, the 99% rule), 16 on the 200^3 algebraic one,
    whose 27-entry rows of A make each class's code long."""
    return sorted({min(16, n_classes), min(32, n_classes), min(64, n_classes)} - {0})


def candidate_list(fast_path: bool, n_classes: int, value_bytes: int, smem_optin: int) -> list:
    """First-round candidate configurations (ptap.make_config keywords) for one problem.

    fast_path / n_classes come from a default symbolic pass.  For class-program
    plans: CTAs of the size the compiled code keeps resident (1024 threads for
    4-byte values, 512 for 8-byte ones), with the largest chunk the
    accumulator allows and smaller ones (fewer entries per CTA: more CTAs for
    the same C, more fine rows visiting two chunks), without cached indices,
    with the cached P row start per entry of A, and with the indices cached
    per visit (piece records, which also let a chunk between the middle size
    and the largest pay off), each with plan-time specialisation of the 16
    most visited classes (fewer if the problem has fewer), plus the
    interpreter alone.  ``refinements`` gives the second round (more compiled
    classes for the best of these).  For plans outside the class programs:
    the sort-based and the hash-group general kernels over lanes per fine
    row, hash slots and chunk sizes (class-program plans try the default
    general kernel only).  The atomic scheme closes both lists.
    """
    out = []
    if fast_path:
        lim = chunk_limit(value_bytes, smem_optin)
        k = _spec_counts(n_classes)[0]
        mid = 32768 if lim > 32768 else max(1024, (lim * 5 // 6) & ~4095)
        # compiled classes: the CTA size their code is built to keep resident, one CTA per SM
        # (1024 threads for 4-byte values; 512 for 8-byte ones, whose code holds twice the
        # registers).  The other size measured 1.5-3x slower on every problem tried, from
        # spills or half the threads per SM.
        bt = 1024 if value_bytes <= 4 else 512
        chunks = sorted({lim, mid, max(1024, lim // 2)}, reverse=True)
        for ch in chunks:
            out.append(dict(specialize=k, block_threads=bt, chunk_entries=ch))
        # the plan's cached indices (Section 4.2's memory-for-time trade), every chunk size:
        # per entry of A, and per visit
        for ch in chunks:
            out.append(dict(specialize=k, block_threads=bt, chunk_entries=ch, cache_indices=True))
        rec_chunks = sorted(set(chunks) | ({(mid + lim) // 2 & ~4095} if lim > mid + 4096 else set()),
                            reverse=True)
        for ch in rec_chunks:
            out.append(dict(specialize=k, block_threads=bt, chunk_entries=ch, cache_indices="visits"))
        out.append(dict())                                    # interpreter, 256 threads
        out.append(dict(block_threads=1024, chunk_entries=lim))  # interpreter, large CTAs
    out.append(dict(class_programs=False))                   # sort-based general kernel
    if not fast_path:
        out.append(dict(class_programs=False, chunk_entries=_GENERAL_MAX_CHUNK // 2))
        for ch in (4096, _GENERAL_MAX_CHUNK // 2):
            for g, slots in ((8, 64), (16, 128)):
                out.append(dict(class_programs=False, general_kernel=1, chunk_entries=ch,
                                group_lanes=g, ap_slots=slots))
    out.append(dict(mode=2, group_lanes=8, ap_slots=64))     # atomic scatter (Alg. 8)
    return _unique(out)


def refinements(cfg: dict, n_classes: int) -> list:
    """Second-round candidates from a first-round one: the same launch with more
    classes compiled (each costs compile time and instruction-cache room, so
    whether it pays depends on the problem)."""
    k = cfg.get("specialize")
    if not k or k is True:
        return []
    return [dict(cfg, specialize=c) for c in _spec_counts(n_classes) if c > k]


def _unique(cands: list) -> list:
    """Drops duplicates, keeps order."""
    seen, uniq = set(), []
    for c in cands:
        key = json.dumps(c, sort_keys=True)
        if key not in seen:
            seen.add(key)
            uniq.append(c)
    return uniq


def _problem(A, P):
    """(fast_path, n_classes, value bytes, opt-in shared memory) from one default symbolic pass."""
    import torch

    from . import ptap
    plan = ptap.symbolic(A, P)
    st = plan.stats()
    plan.destroy()
    props = torch.cuda.get_device_properties(A.row_ptr.device)
    optin = int(getattr(props, "shared_memory_per_block_optin", 232448))
    vb = 8 if A.dtype_code == ptap.F64 else 4
    return bool(st["fast_path"]), int(st["n_classes"]), vb, optin


def candidates(A, P) -> list:
    """First-round candidates for device matrices A, P (ptap.Csr)."""
    return candidate_list(*_problem(A, P))


def candidates_all(A, P) -> list:
    """Every configuration ``tune`` may choose for A, P: the first round and the
    refinements of each of its candidates."""
    fast, n_classes, vb, optin = _problem(A, P)
    first = candidate_list(fast, n_classes, vb, optin)
    return _unique(first + [r for c in first for r in refinements(c, n_classes)])


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
         use_cache: bool = True, slow_factor: float = 3.0) -> TuneResult:
    """Times each candidate configuration on the device matrices A, P (ptap.Csr).

    ``candidates`` defaults to ``candidates(A, P)``, followed by a second round:
    the ``refinements`` (more compiled classes) of the two fastest.  Returns
    the fastest configuration (keyword arguments of ptap.make_config).  A candidate whose
    first product takes more than ``slow_factor`` times the best so far is
    recorded with that one time and not repeated.  Candidates that fail (for
    example by exceeding shared memory) are skipped.
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
    n_classes = None
    if candidates is None:
        fast, n_classes, vb, optin = _problem(A, P)
        candidates = candidate_list(fast, n_classes, vb, optin)
    best, best_ms, trials, sym = None, float("inf"), [], []

    def run(cand):
        nonlocal best, best_ms
        try:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            plan = ptap.symbolic(A, P, ptap.make_config(**cand))
            e1.record()
            torch.cuda.synchronize()
            sym.append((cand, e0.elapsed_time(e1)))
            C = torch.empty(plan.nnz, dtype=plan.torch_dtype, device=A.row_ptr.device)
            first = _time_numeric(ptap, plan, A, P, C, 1, 1)
            ms = first if first > slow_factor * best_ms else _time_numeric(ptap, plan, A, P, C, reps, warmup)
            plan.destroy()
            del C
        except ptap.PtapError as e:
            trials.append((cand, str(e)))
            return
        trials.append((cand, ms))
        if ms < best_ms:
            best, best_ms = dict(cand), ms

    for cand in candidates:
        run(cand)
    # second round (default candidates only): more compiled classes for the two fastest
    if n_classes is not None:
        timed = sorted((t for t in trials if isinstance(t[1], float)), key=lambda t: t[1])
        seen = {json.dumps(c, sort_keys=True) for c, _ in trials}
        for cand, _ in timed[:2]:
            for r in refinements(cand, n_classes):
                if json.dumps(r, sort_keys=True) not in seen:
                    seen.add(json.dumps(r, sort_keys=True))
                    run(r)
    if best is None:
        raise RuntimeError("no candidate configuration ran")
    if cache_path:
        cache = load_cache(cache_path)
        cache[key] = {"config": best, "ms": best_ms}
        save_cache(cache, cache_path)
    return TuneResult(best, best_ms, trials, symbolic_ms=sym)


def batch_candidate_list(value_bytes: int, smem_optin: int) -> list:
    """Candidates for a batch of products (ptap.make_config keywords, one config for all plans).

    The interpreter at 256 threads; batch-wide specialisation of the 32 or 64
    most visited class programs over the whole batch (compiled once, when the
    batch is created) at 256, 512 and 1024 threads with the chunks each allows,
    and with the indices cached per visit; and the general kernel.
    """
    lim = chunk_limit(value_bytes, smem_optin)
    out = [dict()]
    for k in (32, 64):
        out.append(dict(specialize=k, specialize_in_batch=True))
        out.append(dict(specialize=k, specialize_in_batch=True, block_threads=512,
                        chunk_entries=max(1024, lim // 2)))
        out.append(dict(specialize=k, specialize_in_batch=True, block_threads=1024, chunk_entries=lim))
    # indices cached per visit (piece records)
    out.append(dict(specialize=64, specialize_in_batch=True, cache_indices="visits"))
    out.append(dict(specialize=64, specialize_in_batch=True, block_threads=1024, chunk_entries=lim,
                    cache_indices="visits"))
    out.append(dict(class_programs=False))
    return out


def tune_batch(problems, candidates=None, reps: int = 5, warmup: int = 2):
    """Times one persistent batched launch per candidate over ``problems`` (a list of
    device (A, P) pairs of one dtype) and returns the fastest configuration."""
    import torch

    from . import ptap
    A0 = problems[0][0]
    if candidates is None:
        props = torch.cuda.get_device_properties(A0.row_ptr.device)
        optin = int(getattr(props, "shared_memory_per_block_optin", 232448))
        candidates = batch_candidate_list(8 if A0.dtype_code == ptap.F64 else 4, optin)
    best, best_ms, trials = None, float("inf"), []
    for cand in candidates:
        plans, batch = [], None
        try:
            cfg = ptap.make_config(**cand)
            plans = [ptap.symbolic(A, P, cfg) for A, P in problems]
            Cs = [torch.empty(p.nnz, dtype=p.torch_dtype, device=A0.row_ptr.device) for p in plans]
            batch = ptap.Batch(plans, [a for a, _ in problems], [p for _, p in problems], Cs)
            for _ in range(warmup):
                batch.numeric()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                batch.numeric()
            e1.record()
            torch.cuda.synchronize()
            for p in plans:
                p.check()
            ms = e0.elapsed_time(e1) / reps
        except ptap.PtapError as e:
            trials.append((cand, str(e)))
            continue
        finally:
            if batch is not None:
                batch.destroy()
            for p in plans:
                p.destroy()
        trials.append((cand, ms))
        if ms < best_ms:
            best, best_ms = dict(cand), ms
    if best is None:
        raise RuntimeError("no candidate configuration ran")
    return TuneResult(best, best_ms, trials)
