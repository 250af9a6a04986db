"""Build libdsm.so in-tree for sm_103a (GB300) with nvcc.

Each .cu translation unit compiles in parallel into csrc/_build/, then nvcc
links them into paper_2504_19941_gb300/libdsm.so (static CUDA runtime, no
torch dependency).  Rebuilds only what changed.

``build(checked=True)`` makes the bounds-checked library instead
(libdsm_checked.so from csrc/_build_checked/, compiled with -DDSM_CHECKED):
the same kernels with every index they form tested against its buffer.  The
loader takes it when the environment sets DSM_LIB=checked.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(CSRC, "_build")
LIB = os.path.join(HERE, "libdsm.so")
BUILD_CHECKED = os.path.join(CSRC, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libdsm_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xptxas", "-O3"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdsm")


def _deps(src: str):
    deps = [src]
    deps += glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
    deps.append(os.path.join(os.path.dirname(HERE), "include", "dsm.h"))
    return deps


def _stale(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.exists(d) and os.path.getmtime(d) > t for d in deps)


def _compile(src: str, bdir: str, extra, verbose: bool) -> str:
    obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
    if _stale(obj, _deps(src)):
        cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj + ".tmp"]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.check_call(cmd)
        os.replace(obj + ".tmp", obj)
    return obj


def build(verbose: bool = False, extra=(), force: bool = False, checked: bool = False) -> str:
    """Compile every CUDA source of the library and link libdsm.so
    (libdsm_checked.so with ``checked``)."""
    bdir, lib = (BUILD_CHECKED, LIB_CHECKED) if checked else (BUILD, LIB)
    extra = list(extra) + (["-DDSM_CHECKED"] if checked else [])
    os.makedirs(bdir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    if force:
        for o in glob.glob(os.path.join(bdir, "*.o")):
            os.remove(o)
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, bdir, extra, verbose), srcs))
    if _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.check_call(cmd)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    args = sys.argv[1:]
    chk = "--checked" in args
    print(build(verbose=True, extra=[a for a in args if a != "--checked"], checked=chk))
