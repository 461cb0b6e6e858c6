"""Builds libptap.so (the CUDA library behind include/ptap.h) in-tree for sm_103a.

Each .cu file of csrc/ compiles to an object in parallel with nvcc
(-gencode arch=compute_103a,code=sm_103a), then the objects link into
``_build/libptap.so``.  Nothing here needs PyTorch.  Rebuilds only what is
older than its sources.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libptap.so")
# Measurement tool beside the library: the part's FMA peaks (not on the product's path).
PROBE_SRC = os.path.join(PKG, "probe", "fma_peak.cu")
PROBE_LIB = os.path.join(OUT, "libptap_probe.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-O3",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC, "-I", OUT]
# Device header that the library also hands to NVRTC at run time (jit.cu).
JIT_HEADER = os.path.join(CSRC, "fastkern.cuh")
JIT_INC = os.path.join(OUT, "fastkern_src.inc")


def _embed_jit_header() -> None:
    """Writes fastkern.cuh into a C string literal that jit.cu compiles in."""
    if not _stale(JIT_INC, [JIT_HEADER]):
        return
    text = open(JIT_HEADER).read()
    assert ")PTAPSRC\"" not in text
    tmp = JIT_INC + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        f.write('static const char kFastKernSource[] = R"PTAPSRC(' + text + ')PTAPSRC";\n')
    os.replace(tmp, JIT_INC)


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libptap")
    return exe


def _deps() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(INCLUDE, "ptap.h")])


def _stale(target: str, sources: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def build(verbose: bool = False, extra: list[str] | None = None) -> str:
    """Compile (if stale) and return the path of libptap.so."""
    os.makedirs(OUT, exist_ok=True)
    _embed_jit_header()
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    deps = _deps() + [JIT_INC]
    cc = nvcc()
    extra = list(extra or [])
    jobs = []
    objs = []
    for src in sources:
        obj = os.path.join(OUT, os.path.basename(src).replace(".cu", ".o"))
        objs.append(obj)
        if _stale(obj, [src] + deps):
            jobs.append([cc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {cmd[-3]}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr.strip():
            print(r.stderr, flush=True)
        return cmd[-1]

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            list(ex.map(run, jobs))
    if _stale(LIB, objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        run([cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-ldl"])
        os.replace(tmp, LIB)
    if _stale(PROBE_LIB, [PROBE_SRC]):
        tmp = PROBE_LIB + f".{os.getpid()}.tmp"
        run([cc, *ARCH, *FLAGS, "-shared", PROBE_SRC, "-o", tmp, "-lcudart"])
        os.replace(tmp, PROBE_LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
