"""Python binding of the C ABI in include/ptap.h (argument marshalling only).

Every step of the triple product runs in the CUDA library ``libptap.so``;
this module passes device pointers and sizes across the ABI with ctypes.
PyTorch supplies device memory (its caching allocator is handed to the library
as a ``ptap_allocator``) and streams.  There is no CPU fallback: if the
library cannot be loaded, every call raises.

Names follow the ABI: ``symbolic`` / ``numeric`` / ``backward`` /
``two_step_symbolic`` / ``Batch``; ``PtAP`` is the autograd Function.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from . import build as _build

_c = ctypes
F64, F32 = 0, 1
MODE_AUTO, MODE_OWNER, MODE_ATOMIC = 0, 1, 2

ERRORS = {1: "PTAP_ERR_INVALID", 2: "PTAP_ERR_PATTERN", 3: "PTAP_ERR_OVERFLOW",
          4: "PTAP_ERR_OOM", 5: "PTAP_ERR_SPILL", 6: "PTAP_ERR_TIMEOUT",
          7: "PTAP_ERR_CUDA", 8: "PTAP_ERR_UNSUPPORTED"}


class PtapError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = _lib().ptap_error_string(code).decode() if _LIB is not None else ""
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({msg})")


class _Csr(_c.Structure):
    _fields_ = [("nrows", _c.c_int32), ("ncols", _c.c_int32), ("nnz", _c.c_int64),
                ("row_ptr", _c.c_void_p), ("col_idx", _c.c_void_p), ("val", _c.c_void_p),
                ("dtype", _c.c_int32)]


_ALLOC_FN = _c.CFUNCTYPE(_c.c_void_p, _c.c_size_t, _c.c_void_p, _c.c_void_p)
_FREE_FN = _c.CFUNCTYPE(None, _c.c_void_p, _c.c_size_t, _c.c_void_p, _c.c_void_p)


class _Allocator(_c.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", _c.c_void_p)]


class _Config(_c.Structure):
    _fields_ = [("mode", _c.c_int32), ("chunk_entries", _c.c_int32),
                ("block_threads", _c.c_int32), ("group_lanes", _c.c_int32),
                ("ap_slots", _c.c_int32), ("debug_checks", _c.c_int32),
                ("force_spill", _c.c_int32), ("class_programs", _c.c_int32),
                ("visit_block_log2", _c.c_int32), ("specialize", _c.c_int32),
                ("cache_indices", _c.c_int32), ("general_kernel", _c.c_int32),
                ("compact_chunks", _c.c_int32), ("specialize_scope", _c.c_int32),
                ("specialize_async", _c.c_int32), ("reserved", _c.c_int32 * 1)]


class _Stats(_c.Structure):
    _fields_ = [("n", _c.c_int32), ("m", _c.c_int32), ("nnz_a", _c.c_int64),
                ("nnz_p", _c.c_int64), ("nnz_c", _c.c_int64), ("plan_bytes", _c.c_int64),
                ("peak_bytes", _c.c_int64), ("symbolic_peak_bytes", _c.c_int64),
                ("n_chunks", _c.c_int32), ("n_heavy_chunks", _c.c_int32),
                ("chunk_fine_rows", _c.c_int64), ("n_spill_rows_symbolic", _c.c_int32),
                ("mode", _c.c_int32), ("chunk_entries", _c.c_int32),
                ("block_threads", _c.c_int32), ("group_lanes", _c.c_int32),
                ("ap_slots", _c.c_int32), ("kind", _c.c_int32), ("fast_path", _c.c_int32),
                ("n_classes", _c.c_int32), ("n_segments", _c.c_int32),
                ("n_pieces", _c.c_int32), ("n_specialized", _c.c_int32),
                ("specialized_permille", _c.c_int32), ("specialize_us", _c.c_int32),
                ("compact_chunks", _c.c_int32), ("cache_indices", _c.c_int32),
                ("cached_index_bytes", _c.c_int64)]


_LIB = None
_VP = _c.c_void_p
_PP = _c.POINTER(_c.c_void_p)

SYMBOLS = ["ptap_symbolic", "ptap_plan_pattern", "ptap_numeric", "ptap_backward",
           "ptap_two_step_symbolic", "ptap_batch_create", "ptap_batch_numeric",
           "ptap_batch_destroy", "ptap_plan_stats", "ptap_plan_check", "ptap_plan_destroy",
           "ptap_error_string", "ptap_version", "ptap_gather", "ptap_scatter_add",
           "ptap_numeric_host", "ptap_batch_numeric_noalloc", "ptap_aggregate",
           "ptap_prolongator_symbolic", "ptap_prolongator_pattern", "ptap_prolongator_numeric",
           "ptap_prolongator_check", "ptap_prolongator_destroy"]


def lib_path() -> str:
    return _build.LIB


def _lib():
    """Load libptap.so (building it first if missing); raises if it cannot."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path) or os.environ.get("PTAP_REBUILD"):
            path = _build.build()
        L = _c.CDLL(path)
        L.ptap_symbolic.argtypes = [_c.POINTER(_Csr), _c.POINTER(_Csr), _c.POINTER(_Config),
                                    _c.POINTER(_Allocator), _VP, _PP]
        L.ptap_two_step_symbolic.argtypes = L.ptap_symbolic.argtypes
        L.ptap_plan_pattern.argtypes = [_VP, _c.POINTER(_c.c_int32), _c.POINTER(_c.c_int64),
                                        _PP, _PP]
        L.ptap_numeric.argtypes = [_VP, _c.POINTER(_Csr), _c.POINTER(_Csr), _VP, _VP]
        L.ptap_backward.argtypes = [_VP, _c.POINTER(_Csr), _c.POINTER(_Csr), _VP, _VP, _VP, _VP]
        L.ptap_batch_create.argtypes = [_c.POINTER(_VP), _c.POINTER(_Csr), _c.POINTER(_Csr),
                                        _c.POINTER(_VP), _c.c_int32, _c.POINTER(_Allocator),
                                        _VP, _PP]
        L.ptap_batch_numeric.argtypes = [_VP, _VP]
        L.ptap_batch_destroy.argtypes = [_VP]
        L.ptap_batch_destroy.restype = None
        L.ptap_plan_stats.argtypes = [_VP, _c.POINTER(_Stats)]
        L.ptap_plan_check.argtypes = [_VP, _VP]
        L.ptap_plan_destroy.argtypes = [_VP]
        L.ptap_plan_destroy.restype = None
        L.ptap_error_string.argtypes = [_c.c_int]
        L.ptap_error_string.restype = _c.c_char_p
        L.ptap_version.argtypes = []
        L.ptap_gather.argtypes = [_VP, _VP, _c.c_int64, _c.c_int32, _VP, _VP]
        L.ptap_scatter_add.argtypes = [_VP, _VP, _VP, _c.c_int64, _c.c_int32, _VP, _VP]
        missing = [name for name in SYMBOLS if not hasattr(L, name)]
        if missing:
            raise RuntimeError(f"{path} lacks {missing}")
        _LIB = L
    return _LIB


def _check(rc: int, where: str):
    if rc != 0:
        raise PtapError(rc, where)


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


# ---------------------------------------------------------------------------
# torch caching allocator handed to the library
# ---------------------------------------------------------------------------
def _py_alloc(nbytes, stream, ctx):
    try:
        return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                  int(stream or 0))
    except Exception:  # out of memory: the library reports PTAP_ERR_OOM
        return None


def _py_free(ptr, nbytes, stream, ctx):
    torch.cuda.caching_allocator_delete(int(ptr))


_ALLOC_CB = _ALLOC_FN(_py_alloc)
_FREE_CB = _FREE_FN(_py_free)
_TORCH_ALLOCATOR = _Allocator(_ALLOC_CB, _FREE_CB, None)


# ---------------------------------------------------------------------------
# matrices
# ---------------------------------------------------------------------------
@dataclass
class Csr:
    """A device CSR matrix held in torch tensors (int32 indices, f32/f64 values)."""

    nrows: int
    ncols: int
    row_ptr: torch.Tensor
    col_idx: torch.Tensor
    val: torch.Tensor | None

    @property
    def nnz(self) -> int:
        return int(self.col_idx.numel())

    @property
    def dtype_code(self) -> int:
        v = self.val
        if v is None or v.dtype == torch.float64:
            return F64
        if v.dtype == torch.float32:
            return F32
        raise TypeError(f"unsupported value dtype {v.dtype}")

    def c(self, dtype_code: int | None = None) -> _Csr:
        for t in (self.row_ptr, self.col_idx):
            assert t.is_cuda and t.dtype == torch.int32 and t.is_contiguous()
        if self.val is not None:
            assert self.val.is_cuda and self.val.is_contiguous() and self.val.numel() == self.nnz
        return _Csr(self.nrows, self.ncols, self.nnz, self.row_ptr.data_ptr(),
                    self.col_idx.data_ptr(), self.val.data_ptr() if self.val is not None else None,
                    self.dtype_code if dtype_code is None else dtype_code)

    def with_values(self, val: torch.Tensor) -> "Csr":
        return Csr(self.nrows, self.ncols, self.row_ptr, self.col_idx, val)

    @staticmethod
    def from_host(M, device="cuda", dtype=torch.float64) -> "Csr":
        """From any host CSR with nrows/ncols/row_ptr/col_idx/val (numpy)."""
        rp = torch.as_tensor(M.row_ptr, dtype=torch.int32).to(device)
        ci = torch.as_tensor(M.col_idx, dtype=torch.int32).to(device)
        v = torch.as_tensor(M.val).to(device=device, dtype=dtype)
        return Csr(M.nrows, M.ncols, rp.contiguous(), ci.contiguous(), v.contiguous())


def make_config(mode=MODE_OWNER, chunk_entries=0, block_threads=0, group_lanes=0, ap_slots=0,
                debug_checks=False, force_spill=False, class_programs=True,
                visit_block_log2=0, specialize=False, cache_indices=False, general_kernel=0,
                compact_chunks=False, specialize_in_batch=False, specialize_async=False) -> _Config:
    """A ptap_config (fields as in include/ptap.h).  specialize: True for 8 classes or a count;
    cache_indices: False, True (P row starts per entry of A) or "visits" (piece records: the
    indices cached per visit of a fine row to a chunk); specialize_in_batch: leave the compile
    to a Batch over this plan; specialize_async: compile in a background thread."""
    cfg = _Config()
    cfg.mode = mode
    cfg.chunk_entries = chunk_entries
    cfg.block_threads = block_threads
    cfg.group_lanes = group_lanes
    cfg.ap_slots = ap_slots
    cfg.debug_checks = int(bool(debug_checks))
    cfg.force_spill = int(bool(force_spill))
    cfg.class_programs = 0 if class_programs else -1
    cfg.visit_block_log2 = visit_block_log2
    cfg.specialize = 8 if specialize is True else (-1 if not specialize else int(specialize))
    cfg.cache_indices = 2 if cache_indices in ("visits", 2) else int(bool(cache_indices))
    cfg.general_kernel = int(general_kernel)
    cfg.compact_chunks = 1 if compact_chunks is True else int(compact_chunks)
    cfg.specialize_scope = 1 if specialize_in_batch else 0
    cfg.specialize_async = int(bool(specialize_async))
    return cfg


class _DevArray:
    """Zero-copy view of library-owned device memory for torch.as_tensor."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr,
                                         "data": (ptr, False), "version": 3}


class Plan:
    """A symbolic result (C's pattern and the numeric schedule), library-owned."""

    def __init__(self, handle, dtype_code: int, n: int, m: int):
        self._h = handle
        self.dtype_code = dtype_code
        self.n, self.m = n, m
        s = self.stats()
        self.nnz = s["nnz_c"]

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("plan already destroyed")
        return self._h

    @property
    def torch_dtype(self):
        return torch.float64 if self.dtype_code == F64 else torch.float32

    def pattern(self):
        """(row_ptr, col_idx) of C as int32 tensors (copies)."""
        m, nnz = _c.c_int32(), _c.c_int64()
        rp, ci = _c.c_void_p(), _c.c_void_p()
        _check(_lib().ptap_plan_pattern(self.handle, _c.byref(m), _c.byref(nnz), _c.byref(rp),
                                        _c.byref(ci)), "ptap_plan_pattern")
        dev = torch.device("cuda", torch.cuda.current_device())
        r = torch.as_tensor(_DevArray(rp.value, m.value + 1, "<i4"), device=dev).clone()
        c = (torch.as_tensor(_DevArray(ci.value, nnz.value, "<i4"), device=dev).clone()
             if nnz.value > 0 else torch.zeros(0, dtype=torch.int32, device=dev))
        return r, c

    def stats(self) -> dict:
        st = _Stats()
        _check(_lib().ptap_plan_stats(self.handle, _c.byref(st)), "ptap_plan_stats")
        return {k: getattr(st, k) for k, _ in _Stats._fields_ if k != "reserved"}

    def check(self, stream=None):
        _check(_lib().ptap_plan_check(self.handle, _stream(stream)), "device status")

    def destroy(self):
        if self._h:
            _lib().ptap_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def symbolic(A: Csr, P: Csr, config: _Config | None = None, stream=None,
             dtype=None) -> Plan:
    """ptap_symbolic: pattern of C = P^T A P and the numeric schedule."""
    code = A.dtype_code if dtype is None else (F64 if dtype == torch.float64 else F32)
    h = _c.c_void_p()
    _check(_lib().ptap_symbolic(_c.byref(A.c(code)), _c.byref(P.c(code)),
                                _c.byref(config) if config is not None else None,
                                _c.byref(_TORCH_ALLOCATOR), _stream(stream), _c.byref(h)),
           "ptap_symbolic")
    return Plan(h, code, A.nrows, P.ncols)


def two_step_symbolic(A: Csr, P: Csr, config: _Config | None = None, stream=None,
                      dtype=None) -> Plan:
    """ptap_two_step_symbolic: the GPU two-step comparator (holds A P and P^T)."""
    code = A.dtype_code if dtype is None else (F64 if dtype == torch.float64 else F32)
    h = _c.c_void_p()
    _check(_lib().ptap_two_step_symbolic(_c.byref(A.c(code)), _c.byref(P.c(code)),
                                         _c.byref(config) if config is not None else None,
                                         _c.byref(_TORCH_ALLOCATOR), _stream(stream),
                                         _c.byref(h)), "ptap_two_step_symbolic")
    return Plan(h, code, A.nrows, P.ncols)


def numeric(plan: Plan, A: Csr, P: Csr, out: torch.Tensor | None = None, stream=None):
    """ptap_numeric: values of C on the plan's pattern."""
    if out is None:
        out = torch.empty(plan.nnz, dtype=plan.torch_dtype, device=A.row_ptr.device)
    assert out.is_contiguous() and out.numel() == plan.nnz and out.dtype == plan.torch_dtype
    _check(_lib().ptap_numeric(plan.handle, _c.byref(A.c()), _c.byref(P.c()), out.data_ptr(),
                               _stream(stream)), "ptap_numeric")
    return out


def numeric_host(plan: Plan, A: Csr, P: Csr, A_val: torch.Tensor, P_val: torch.Tensor,
                 out: torch.Tensor, stream=None):
    """ptap_numeric_host: C's values from host-resident values of A and P into host ``out``.

    A and P supply the device patterns (their values are not read).  All three
    value tensors live on the host (pinned for overlapped copies) with the
    plan's dtype; ``out`` is complete once ``stream`` has been synchronised.
    """
    for t, n in ((A_val, A.nnz), (P_val, P.nnz), (out, plan.nnz)):
        assert t.device.type == "cpu" and t.is_contiguous() and t.numel() == n
        assert t.dtype == plan.torch_dtype
    f = _lib().ptap_numeric_host
    f.argtypes = [_VP, _c.POINTER(_Csr), _c.POINTER(_Csr), _VP, _VP, _VP, _VP]
    _check(f(plan.handle, _c.byref(A.c()), _c.byref(P.c()), A_val.data_ptr(), P_val.data_ptr(),
             out.data_ptr(), _stream(stream)), "ptap_numeric_host")
    return out


def backward(plan: Plan, A: Csr, P: Csr, G: torch.Tensor, need_dA=True, need_dP=True,
             stream=None):
    """ptap_backward: (dL/dA on pat(A), dL/dP on pat(P)) given G = dL/dC on pat(C)."""
    G = G.contiguous()
    assert G.numel() == plan.nnz and G.dtype == plan.torch_dtype
    dA = torch.empty(A.nnz, dtype=plan.torch_dtype, device=G.device) if need_dA else None
    dP = torch.empty(P.nnz, dtype=plan.torch_dtype, device=G.device) if need_dP else None
    _check(_lib().ptap_backward(plan.handle, _c.byref(A.c()), _c.byref(P.c()), G.data_ptr(),
                                dA.data_ptr() if dA is not None else None,
                                dP.data_ptr() if dP is not None else None, _stream(stream)),
           "ptap_backward")
    return dA, dP


def _check_outputs(plans, Cs, where: str):
    """Each C must be a contiguous CUDA tensor of its plan's dtype with room for nnz(C) values:
    the library writes through the raw pointers."""
    if len(plans) != len(Cs):
        raise PtapError(1, f"{where}: {len(plans)} plans but {len(Cs)} outputs")
    for q, (p, C) in enumerate(zip(plans, Cs)):
        if not (isinstance(C, torch.Tensor) and C.is_cuda and C.is_contiguous()
                and C.dtype == p.torch_dtype and C.numel() >= p.nnz):
            raise PtapError(1, f"{where}: output {q} must be a contiguous CUDA {p.torch_dtype} "
                               f"tensor of at least {p.nnz} values")


class Batch:
    """ptap_batch_create / ptap_batch_numeric: many products in one persistent launch."""

    def __init__(self, plans, As, Ps, Cs, stream=None):
        n = len(plans)
        _check_outputs(plans, Cs, "ptap_batch_create")
        self._keep = (list(plans), list(As), list(Ps), list(Cs))
        hp = (_VP * n)(*[p.handle for p in plans])
        ca = (_Csr * n)(*[a.c() for a in As])
        cp = (_Csr * n)(*[p.c() for p in Ps])
        cc = (_VP * n)(*[c.data_ptr() for c in Cs])
        h = _c.c_void_p()
        _check(_lib().ptap_batch_create(hp, ca, cp, cc, n, _c.byref(_TORCH_ALLOCATOR),
                                        _stream(stream), _c.byref(h)), "ptap_batch_create")
        self._h = h

    def numeric(self, stream=None):
        _check(_lib().ptap_batch_numeric(self._h, _stream(stream)), "ptap_batch_numeric")

    def destroy(self):
        if self._h:
            _lib().ptap_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class PtAP(torch.autograd.Function):
    """C_val = ptap_numeric(plan, A(A_val), P(P_val)), differentiable in A_val and P_val.

    ``plan`` fixes the patterns; A and P carry the index tensors (their
    ``val`` fields are ignored in favour of the differentiable arguments).
    """

    @staticmethod
    def forward(ctx, A_val, P_val, plan: Plan, A: Csr, P: Csr):
        Aw, Pw = A.with_values(A_val.contiguous()), P.with_values(P_val.contiguous())
        C = numeric(plan, Aw, Pw)
        ctx.plan, ctx.A, ctx.P = plan, A, P
        ctx.save_for_backward(A_val, P_val)
        return C

    @staticmethod
    def backward(ctx, G):
        A_val, P_val = ctx.saved_tensors
        Aw, Pw = ctx.A.with_values(A_val.contiguous()), ctx.P.with_values(P_val.contiguous())
        dA, dP = backward(ctx.plan, Aw, Pw, G.contiguous(), ctx.needs_input_grad[0],
                          ctx.needs_input_grad[1])
        return dA, dP, None, None, None


def batch_numeric_noalloc(plans, As, Ps, Cs, stream=None):
    """ptap_batch_numeric_noalloc: the batched numeric products with no device allocation.

    For callers that cannot allocate device memory while the products run
    (a fixed device footprint reserved up front, or no room for the implicit
    synchronisation of an allocation).  The library keeps its work queue in a
    fixed 8 MiB device array; calls that overlap on the GPU race on it.
    """
    L = _lib()
    f = L.ptap_batch_numeric_noalloc
    f.argtypes = [_c.POINTER(_VP), _c.POINTER(_Csr), _c.POINTER(_Csr), _c.POINTER(_VP),
                  _c.c_int32, _VP]
    n = len(plans)
    _check_outputs(plans, Cs, "ptap_batch_numeric_noalloc")
    hp = (_VP * n)(*[p.handle for p in plans])
    ca = (_Csr * n)(*[a.c() for a in As])
    cp = (_Csr * n)(*[p.c() for p in Ps])
    cc = (_VP * n)(*[c.data_ptr() for c in Cs])
    _check(f(hp, ca, cp, cc, n, _stream(stream)), "ptap_batch_numeric_noalloc")



def _vcode(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError(f"unsupported value dtype {t.dtype}")


def gather(src: torch.Tensor, idx: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """ptap_gather: out[e] = src[idx[e]] (packing exchanged values of the row partition)."""
    assert src.is_cuda and src.is_contiguous() and idx.is_cuda and idx.dtype == torch.int32
    idx = idx.contiguous()
    if out is None:
        out = torch.empty(idx.numel(), dtype=src.dtype, device=src.device)
    assert out.is_contiguous() and out.dtype == src.dtype and out.numel() >= idx.numel()
    _check(_lib().ptap_gather(src.data_ptr(), idx.data_ptr(), idx.numel(), _vcode(src), out.data_ptr(),
                              _stream(stream)), "ptap_gather")
    return out


def scatter_add(dst: torch.Tensor, dst_idx: torch.Tensor, src: torch.Tensor,
                src_idx: torch.Tensor | None = None, stream=None):
    """ptap_scatter_add: dst[dst_idx[e]] += src[src_idx[e] or e] (distinct dst_idx in one call)."""
    assert dst.is_cuda and dst.is_contiguous() and src.is_cuda and src.is_contiguous()
    assert src.dtype == dst.dtype and dst_idx.dtype == torch.int32
    n = dst_idx.numel()
    if src_idx is not None:
        assert src_idx.dtype == torch.int32 and src_idx.numel() == n
        src_idx = src_idx.contiguous()
    else:
        assert src.numel() >= n
    dst_idx = dst_idx.contiguous()
    _check(_lib().ptap_scatter_add(src.data_ptr(), src_idx.data_ptr() if src_idx is not None else None,
                                   dst_idx.data_ptr(), n, _vcode(dst), dst.data_ptr(), _stream(stream)),
           "ptap_scatter_add")
    return dst


# ---------------------------------------------------------------------------
# levels of an algebraic multigrid hierarchy (aggregation, smoothed prolongator)
# ---------------------------------------------------------------------------
def _amg_sigs(L):
    if getattr(L, "_amg_sigs", False):
        return
    L.ptap_aggregate.argtypes = [_c.POINTER(_Csr), _c.c_int32, _c.c_int32, _VP, _c.POINTER(_c.c_int32),
                                 _c.POINTER(_Allocator), _VP]
    L.ptap_prolongator_symbolic.argtypes = [_c.POINTER(_Csr), _VP, _c.c_int32, _c.c_double,
                                            _c.POINTER(_Allocator), _VP, _PP]
    L.ptap_prolongator_pattern.argtypes = [_VP, _c.POINTER(_c.c_int32), _c.POINTER(_c.c_int32),
                                           _c.POINTER(_c.c_int64), _PP, _PP]
    L.ptap_prolongator_numeric.argtypes = [_VP, _c.POINTER(_Csr), _c.c_double, _VP, _VP]
    L.ptap_prolongator_check.argtypes = [_VP, _VP]
    L.ptap_prolongator_destroy.argtypes = [_VP]
    L.ptap_prolongator_destroy.restype = None
    L._amg_sigs = True


def aggregate(A: Csr, passes: int = 2, rounds: int = 16, stream=None):
    """ptap_aggregate: (agg, n_agg) -- the aggregate of every row of A (int32 device tensor)."""
    L = _lib()
    _amg_sigs(L)
    agg = torch.empty(max(A.nrows, 1), dtype=torch.int32, device=A.row_ptr.device)
    n = _c.c_int32()
    _check(L.ptap_aggregate(_c.byref(A.c()), passes, rounds, agg.data_ptr(), _c.byref(n),
                            _c.byref(_TORCH_ALLOCATOR), _stream(stream)), "ptap_aggregate")
    return agg[:A.nrows], n.value


class Prolongator:
    """ptap_prolongator_*: the pattern of P = (I - omega D^-1 A_F) T (A_F: A filtered by
    strength theta, D = diag(A)), and its values on demand."""

    def __init__(self, A: Csr, agg: torch.Tensor, n_agg: int, theta: float = 0.0, stream=None):
        L = _lib()
        _amg_sigs(L)
        assert agg.dtype == torch.int32 and agg.is_cuda and agg.numel() == A.nrows
        h = _c.c_void_p()
        _check(L.ptap_prolongator_symbolic(_c.byref(A.c()), agg.contiguous().data_ptr(), n_agg, float(theta),
                                           _c.byref(_TORCH_ALLOCATOR), _stream(stream), _c.byref(h)),
               "ptap_prolongator_symbolic")
        self._h = h
        self.n, self.m = A.nrows, n_agg
        nr, nc, nnz, rp, ci = _c.c_int32(), _c.c_int32(), _c.c_int64(), _c.c_void_p(), _c.c_void_p()
        _check(L.ptap_prolongator_pattern(h, _c.byref(nr), _c.byref(nc), _c.byref(nnz), _c.byref(rp),
                                          _c.byref(ci)), "ptap_prolongator_pattern")
        self.nnz = nnz.value
        dev = A.row_ptr.device
        self.row_ptr = torch.as_tensor(_DevArray(rp.value, nr.value + 1, "<i4"), device=dev).clone()
        self.col_idx = (torch.as_tensor(_DevArray(ci.value, self.nnz, "<i4"), device=dev).clone()
                        if self.nnz > 0 else torch.zeros(0, dtype=torch.int32, device=dev))

    def numeric(self, A: Csr, omega: float = 2.0 / 3.0, out: torch.Tensor | None = None, stream=None):
        if out is None:
            out = torch.empty(self.nnz, dtype=A.val.dtype, device=A.val.device)
        assert out.is_contiguous() and out.numel() == self.nnz and out.dtype == A.val.dtype
        _check(_lib().ptap_prolongator_numeric(self._h, _c.byref(A.c()), float(omega), out.data_ptr(),
                                               _stream(stream)), "ptap_prolongator_numeric")
        return out

    def csr(self, val: torch.Tensor) -> Csr:
        return Csr(self.n, self.m, self.row_ptr, self.col_idx, val)

    def check(self, stream=None):
        _check(_lib().ptap_prolongator_check(self._h, _stream(stream)), "prolongator status")

    def destroy(self):
        if self._h:
            _lib().ptap_prolongator_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
