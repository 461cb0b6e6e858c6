"""C ABI checks that need no GPU: the library loads, exports every entry point
declared in include/*.h, and rejects malformed calls on the host (before any
device work) with the documented error codes."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(ptap_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1905_08423_gb300 import build
    return ctypes.CDLL(build.build())


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 14
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_error_strings_and_version(lib):
    lib.ptap_error_string.restype = ctypes.c_char_p
    for code in range(0, 9):
        s = lib.ptap_error_string(code).decode()
        assert s and "unknown" not in s
    assert "unknown" in lib.ptap_error_string(99).decode()
    assert lib.ptap_version() >= 100


class Csr(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int32), ("ncols", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p),
                ("val", ctypes.c_void_p), ("dtype", ctypes.c_int32)]


def _fake(nrows, ncols, nnz, dtype=0):
    # device pointers are never dereferenced on the host; these calls must be
    # rejected before any device work
    return Csr(nrows, ncols, nnz, 0x1000, 0x2000, 0x3000, dtype)


def test_host_validation(lib):
    out = ctypes.c_void_p()
    sym = lib.ptap_symbolic
    sym.argtypes = [ctypes.POINTER(Csr), ctypes.POINTER(Csr), ctypes.c_void_p, ctypes.c_void_p,
                    ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    A, P = _fake(10, 12, 30), _fake(10, 4, 10)          # A not square
    assert sym(ctypes.byref(A), ctypes.byref(P), None, None, None, ctypes.byref(out)) == 1
    A, P = _fake(10, 10, 30), _fake(9, 4, 10)           # ncols(A) != nrows(P)
    assert sym(ctypes.byref(A), ctypes.byref(P), None, None, None, ctypes.byref(out)) == 1
    A, P = _fake(10, 10, 30, 0), _fake(10, 4, 10, 1)    # dtype mismatch
    assert sym(ctypes.byref(A), ctypes.byref(P), None, None, None, ctypes.byref(out)) == 1
    A, P = _fake(10, 10, 30, 7), _fake(10, 4, 10, 7)    # unknown dtype
    assert sym(ctypes.byref(A), ctypes.byref(P), None, None, None, ctypes.byref(out)) == 1
    A, P = _fake(10, 10, 2**31), _fake(10, 4, 10)       # nnz beyond int32 indexing
    assert sym(ctypes.byref(A), ctypes.byref(P), None, None, None, ctypes.byref(out)) == 1
    assert sym(None, ctypes.byref(P), None, None, None, ctypes.byref(out)) == 1
    assert sym(ctypes.byref(A), ctypes.byref(P), None, None, None, None) == 1
    lib.ptap_numeric.argtypes = [ctypes.c_void_p] * 5
    assert lib.ptap_numeric(None, None, None, None, None) == 1
    lib.ptap_backward.argtypes = [ctypes.c_void_p] * 7
    assert lib.ptap_backward(None, None, None, None, None, None, None) == 1
    lib.ptap_plan_stats.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.ptap_plan_stats(None, None) == 1
    lib.ptap_batch_numeric.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.ptap_batch_numeric(None, None) == 1
    lib.ptap_batch_create.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int32] + [ctypes.c_void_p] * 3
    assert lib.ptap_batch_create(None, None, None, None, 0, None, None, None) == 1
    lib.ptap_plan_destroy.argtypes = [ctypes.c_void_p]
    lib.ptap_plan_destroy(None)   # no-op on NULL



def _struct_fields(name):
    """Field names, in order, of `typedef struct { ... } name;` in include/ptap.h."""
    txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "ptap.h")).read(), flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", txt)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        for part in decl.split(","):
            fields.append(re.sub(r"\[.*\]", "", part).split()[-1].lstrip("*"))
    return fields


def test_binding_structs_mirror_the_header():
    """The Python binding's ctypes mirrors list the header's fields in the same order and
    with the same sizes (a mismatch would shift every later field across the ABI)."""
    from paper_1905_08423_gb300 import ptap
    for name, mirror in (("ptap_config", ptap._Config), ("ptap_stats", ptap._Stats)):
        assert [f for f, _ in mirror._fields_] == _struct_fields(name), name
    assert ctypes.sizeof(ptap._Config) == 16 * 4       # the config keeps its size
    cfg = ptap.make_config(compact_chunks=True)
    assert cfg.compact_chunks == 1
    assert ptap.make_config(compact_chunks=32).compact_chunks == 32
    assert ptap.make_config().compact_chunks == 0


def test_exchange_calls_validate_on_host(lib):
    """ptap_gather / ptap_scatter_add reject bad sizes, dtypes and NULL pointers before
    any device work, and accept n = 0 as a no-op."""
    g, s = lib.ptap_gather, lib.ptap_scatter_add
    g.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                  ctypes.c_void_p]
    s.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                  ctypes.c_void_p, ctypes.c_void_p]
    assert g(0x1000, 0x2000, -1, 0, 0x3000, None) == 1
    assert g(0x1000, 0x2000, 4, 7, 0x3000, None) == 1
    assert g(None, 0x2000, 4, 0, 0x3000, None) == 1
    assert g(None, None, 0, 0, None, None) == 0
    assert s(0x1000, None, None, 4, 1, 0x3000, None) == 1
    assert s(0x1000, None, 0x2000, -2, 1, 0x3000, None) == 1
    assert s(None, None, None, 0, 1, None, None) == 0
