"""Build the CUDA library (sm_103a) in-tree: paper_2002_11529_gb300/_lib/libutcompass.so.

Every translation unit is compiled by nvcc in parallel, then linked into
one shared library with the C ABI declared in include/ut_compass.h.
Floating point: -fmad=false on the device and -ffp-contract=off on the
host, so every float operation of the decode and the Compass decisions is
a single IEEE-rounded operation in the written order.

With the environment variable UT_CHECKED=1 the bounds-checked variant is
built and loaded instead (-DUT_CHECKED, _lib/libutcompass_checked.so):
every checked access compares its index with its array's extent and
records UT_ERR_BOUNDS in the status word instead of touching memory out of
bounds.  It computes the same results, more slowly.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libutcompass.so")
LIB_CHECKED = os.path.join(LIBDIR, "libutcompass_checked.so")


def checked() -> bool:
    """The bounds-checked variant is selected (UT_CHECKED=1)."""
    return os.environ.get("UT_CHECKED", "") == "1"


def lib_path() -> str:
    return LIB_CHECKED if checked() else LIB
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC,-ffp-contract=off",
              "-Xptxas", "-warn-spills"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(lib) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(
        os.path.join(HERE, "..", "include", "*.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Build the selected variant (the bounds-checked one under UT_CHECKED=1)."""
    chk = checked()
    lib = LIB_CHECKED if chk else LIB
    if not force and not _stale(lib):
        return lib
    objdir = os.path.join(LIBDIR, "obj_checked" if chk else "obj")
    os.makedirs(objdir, exist_ok=True)
    nv = nvcc()
    inc = ["-I", os.path.join(HERE, "..", "include")]
    defs = ["-DUT_CHECKED"] if chk else []

    def compile_one(src):
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        cmd = [nv, *ARCH, *NVCC_FLAGS, *defs, *inc, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nv, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
