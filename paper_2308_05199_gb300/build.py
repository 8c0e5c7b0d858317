"""Build the CUDA library libzc.so in-tree for sm_103a.

Every translation unit under csrc/ is compiled by nvcc in parallel and linked
into ``_build/libzc.so``.  ``-fmad=false`` keeps the quantizer's multiplies
and adds as separate roundings (the codec states its arithmetic step by step;
intrinsic FMAs are written where one rounding is meant).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libzc.so")
# The bounds-checked variant (-DZC_DEBUG): every checked kernel access is
# tested against its buffer; a failed check reports ZC_ERR_BOUNDS and skips
# the access.  Loaded instead of the release library when ZC_LIBRARY=debug.
DEBUG_BUILD = os.path.join(HERE, "_build_debug")
DEBUG_LIB = os.path.join(DEBUG_BUILD, "libzc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libzc.so")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC",
                   "-I", os.path.join(ROOT, "include"), "-I", CSRC] + list(extra)


# Sources compiled more than once, with one macro value per object: the
# encoder kernels once per block size, the batch kernel once per tile size
# (the heavy instantiations then compile in parallel).
VARIANTS = {
    "zc_kenc.cu": [("zc_kenc_l%d" % (1 << lg), ["-DZC_LOG2L=%d" % lg]) for lg in (4, 5, 6, 7)],
    "zc_kbatch.cu": [("zc_kbatch_u%d" % u, ["-DZC_BATCH_U=%d" % u]) for u in (32, 64, 128)],
}


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _units():
    """(source, object name, extra flags) of every object of the library."""
    out = []
    for src in _sources():
        name = os.path.basename(src)
        for obj, defs in VARIANTS.get(name, [(name[:-3], [])]):
            out.append((src, obj, defs))
    return out


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(CSRC, "*.h")) + [os.path.join(ROOT, "include", "zc.h")]


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra=(), debug: bool = False) -> str:
    """Compile the library (the bounds-checked variant when `debug`) unless it
    is newer than every source; returns its path."""
    out_dir, lib = (DEBUG_BUILD, DEBUG_LIB) if debug else (BUILD, LIB)
    if not force and not extra and up_to_date(lib):
        return lib
    if debug:
        extra = ["-DZC_DEBUG"] + list(extra)
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    objs = []

    def compile_one(unit):
        src, name, defs = unit
        obj = os.path.join(out_dir, name + ".o")
        cmd = [cc, "-c", src, "-o", obj] + _flags(list(defs) + list(extra))
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    units = _units()
    with cf.ThreadPoolExecutor(max_workers=min(len(units), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, units))
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static", "-lrt", "-ldl",
                                                         "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    v = "-v" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(force=True, verbose=v or bool(extra), extra=extra))
