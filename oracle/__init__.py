"""Oracle for the sparse triple product C = P^T A P.

TEST INFRASTRUCTURE ONLY.  A plain, slow, single-threaded CPU implementation in
FP64 (``ptap_oracle.c``) used to check the CUDA library.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference legs may
import it.  It shares no code with the CUDA path and imports nothing from it.

What each function follows (Kong, "Parallel memory-efficient all-at-once
algorithms for the sparse matrix triple products in multigrid methods"):

* ``spgemm``      -- row-wise product, Section 2, Alg. 3-4 (pattern: Alg. 1-2).
* ``transpose``   -- explicit transpose of the two-step method, Alg. 5-6.
* ``ptap``        -- two-step triple product, Section 3, Eq. 6, Alg. 5-6.
* ``ptap_rows``   -- rows of C from the definition, Section 3, Eq. 7-8.
* ``ptap_row_block`` -- the contribution of a block of fine rows, i.e. the
  1D block-row partition of Section 2 (Eq. 1-3) applied to Eq. 9.
* ``ptap_backward`` -- gradients of a scalar loss through C = P^T A P:
  dA = (P G P^T) on pat(A), dP = (A P G^T + A^T P G) on pat(P), composed from
  the same products; this is not in the paper (its pins are central finite
  differences and a dense reference).

All products are structural: every reached entry is kept, including exact
cancellations (Section 2: the symbolic phase uses no floating point).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ptap_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain -O2, no FP contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_spgemm.argtypes = [ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, _f64p,
                                      ctypes.c_int32, _i32p, _i32p, _f64p,
                                      ctypes.POINTER(_i32p), ctypes.POINTER(_i32p),
                                      ctypes.POINTER(_f64p), ctypes.POINTER(ctypes.c_int64)]
        lib.oracle_transpose.argtypes = [ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, _f64p,
                                         ctypes.POINTER(_i32p), ctypes.POINTER(_i32p),
                                         ctypes.POINTER(_f64p)]
        lib.oracle_ptap_two_step.argtypes = [ctypes.c_int32, ctypes.c_int32, _i32p, _i32p,
                                             _f64p, _i32p, _i32p, _f64p,
                                             ctypes.POINTER(_i32p), ctypes.POINTER(_i32p),
                                             ctypes.POINTER(_f64p),
                                             ctypes.POINTER(ctypes.c_int64)]
        lib.oracle_ptap_rows.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _i32p, _i32p,
                                         _f64p, _i32p, _i32p, _f64p, ctypes.c_int32, _i32p,
                                         ctypes.POINTER(_i32p), ctypes.POINTER(_i32p),
                                         ctypes.POINTER(_f64p), ctypes.POINTER(ctypes.c_int64)]
        lib.oracle_sample.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _i32p, _i32p, _f64p]
        lib.oracle_free.argtypes = [ctypes.c_void_p]
        for f in ("oracle_spgemm", "oracle_transpose", "oracle_ptap_two_step",
                  "oracle_ptap_rows", "oracle_sample"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclass
class OCSR:
    """CSR result of the oracle (int32 indices, float64 values)."""

    nrows: int
    ncols: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.nrows, self.ncols))
        rows = np.repeat(np.arange(self.nrows), np.diff(self.row_ptr.astype(np.int64)))
        np.add.at(d, (rows, self.col_idx), self.val)
        return d


def _arr_i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_i32p)


def _arr_f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_f64p)


def _csr_args(M):
    rp, rpp = _arr_i32(M.row_ptr)
    ci, cip = _arr_i32(M.col_idx)
    v, vp = _arr_f64(M.val)
    return (rp, ci, v), (rpp, cip, vp)


def _take(lib, rows: int, ncols: int, p, j, x, nnz: int) -> OCSR:
    rp = np.ctypeslib.as_array(p, shape=(rows + 1,)).copy()
    ci = np.ctypeslib.as_array(j, shape=(max(nnz, 1),))[:nnz].copy()
    v = np.ctypeslib.as_array(x, shape=(max(nnz, 1),))[:nnz].copy()
    for ptr in (p, j, x):
        lib.oracle_free(ctypes.cast(ptr, ctypes.c_void_p))
    return OCSR(rows, ncols, rp, ci, v)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def spgemm(A, B) -> OCSR:
    """Row-wise structural product A * B (Alg. 3-4)."""
    assert A.ncols == B.nrows
    lib = _load()
    keepA, (ap, aj, ax) = _csr_args(A)
    keepB, (bp, bj, bx) = _csr_args(B)
    p, j, x, nnz = _i32p(), _i32p(), _f64p(), ctypes.c_int64()
    _check(lib.oracle_spgemm(A.nrows, A.ncols, ap, aj, ax, B.ncols, bp, bj, bx,
                             ctypes.byref(p), ctypes.byref(j), ctypes.byref(x),
                             ctypes.byref(nnz)), "spgemm")
    return _take(lib, A.nrows, B.ncols, p, j, x, nnz.value)


def transpose(M) -> OCSR:
    """Explicit transpose by counting sort (the two-step method's P^T)."""
    lib = _load()
    keep, (mp, mj, mx) = _csr_args(M)
    p, j, x = _i32p(), _i32p(), _f64p()
    _check(lib.oracle_transpose(M.nrows, M.ncols, mp, mj, mx, ctypes.byref(p),
                                ctypes.byref(j), ctypes.byref(x)), "transpose")
    return _take(lib, M.ncols, M.nrows, p, j, x, int(M.row_ptr[-1]))


def ptap(A, P) -> OCSR:
    """Two-step C = P^T (A P) (Eq. 6, Alg. 5-6), FP64, structural pattern."""
    assert A.nrows == A.ncols == P.nrows
    lib = _load()
    keepA, (ap, aj, ax) = _csr_args(A)
    keepP, (pp, pj, px) = _csr_args(P)
    p, j, x, nnz = _i32p(), _i32p(), _f64p(), ctypes.c_int64()
    _check(lib.oracle_ptap_two_step(A.nrows, P.ncols, ap, aj, ax, pp, pj, px,
                                    ctypes.byref(p), ctypes.byref(j), ctypes.byref(x),
                                    ctypes.byref(nnz)), "ptap_two_step")
    return _take(lib, P.ncols, P.ncols, p, j, x, nnz.value)


class _Abs:
    def __init__(self, M):
        self.nrows, self.ncols = M.nrows, M.ncols
        self.row_ptr, self.col_idx = M.row_ptr, M.col_idx
        self.val = np.abs(np.asarray(M.val, dtype=np.float64))


def ptap_bound(A, P) -> OCSR:
    """B = |P|^T |A| |P|: the entrywise bound the tolerance is measured against."""
    return ptap(_Abs(A), _Abs(P))


def ptap_rows(A, P, rows, PT: OCSR | None = None) -> OCSR:
    """Rows ``rows`` of C evaluated from the definition C(i,:) = sum_I P(I,i) (A P)(I,:)."""
    assert A.nrows == A.ncols == P.nrows
    lib = _load()
    if PT is None:
        PT = transpose(P)
    keepA, (ap, aj, ax) = _csr_args(A)
    keepP, (pp, pj, px) = _csr_args(P)
    keepT, (tp, tj, tx) = _csr_args(PT)
    r, rp = _arr_i32(np.asarray(rows))
    p, j, x, nnz = _i32p(), _i32p(), _f64p(), ctypes.c_int64()
    _check(lib.oracle_ptap_rows(P.ncols, ap, aj, ax, pp, pj, px, tp, tj, tx, len(r), rp,
                                ctypes.byref(p), ctypes.byref(j), ctypes.byref(x),
                                ctypes.byref(nnz)), "ptap_rows")
    return _take(lib, len(r), P.ncols, p, j, x, nnz.value)


def _row_slice(M, r0: int, r1: int) -> OCSR:
    rp = np.asarray(M.row_ptr, dtype=np.int64)
    s, e = rp[r0], rp[r1]
    return OCSR(r1 - r0, M.ncols, (rp[r0:r1 + 1] - s).astype(np.int32),
                np.asarray(M.col_idx[s:e], dtype=np.int32),
                np.asarray(M.val[s:e], dtype=np.float64))


def ptap_row_block(A, P, r0: int, r1: int) -> OCSR:
    """Contribution of fine rows [r0, r1) to C: P(r0:r1,:)^T (A(r0:r1,:) P).

    Summing this over a partition of the fine rows gives C (Eq. 9 split by the
    1D block-row partition of Eq. 1).
    """
    Ab = _row_slice(A, r0, r1)
    Pb = _row_slice(P, r0, r1)
    APb = spgemm(Ab, P)
    return spgemm(transpose(Pb), APb)


def sample(M, S) -> np.ndarray:
    """Values of M at the stored entries of S (0 where M has no entry)."""
    assert M.nrows == S.nrows
    lib = _load()
    keepM, (mp, mj, mx) = _csr_args(M)
    sp_, spp = _arr_i32(S.row_ptr)
    sj, sjp = _arr_i32(S.col_idx)
    out = np.zeros(int(S.row_ptr[-1]), dtype=np.float64)
    _check(lib.oracle_sample(M.nrows, mp, mj, mx, spp, sjp,
                             out.ctypes.data_as(_f64p)), "sample")
    return out


def ptap_backward(A, P, G):
    """Gradients of L through C = P^T A P, given G = dL/dC on C's pattern.

    Returns (dA on pat(A), dP on pat(P)) with dA = P G P^T and
    dP = A P G^T + A^T P G, each restricted to the pattern.
    """
    PT = transpose(P)
    PG = spgemm(P, G)
    dA = sample(spgemm(PG, PT), A)
    AP = spgemm(A, P)
    APGt = spgemm(AP, transpose(G))
    AtPG = spgemm(transpose(A), PG)
    dP = sample(APGt, P) + sample(AtPG, P)
    return dA, dP
