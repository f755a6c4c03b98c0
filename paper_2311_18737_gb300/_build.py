"""Build the CUDA library ``lib/libisr.so`` in-tree (nvcc, sm_103a only).

The translation units are compiled in parallel (one nvcc per unit) and linked with the
static CUDA runtime, so the library needs no CUDA shared objects beyond the driver.
"""
from __future__ import annotations

import concurrent.futures
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "lib")
OBJDIR = os.path.join(LIBDIR, "obj")
LIB = os.path.join(LIBDIR, "libisr.so")
# debug build: the kernels check every gate's staged window against its echo row
# (-DISR_DEBUG; a failed check is reported as ISR_ERR_OUT_OF_RANGE, never a trap)
OBJDIR_DEBUG = os.path.join(LIBDIR, "obj_debug")
LIB_DEBUG = os.path.join(LIBDIR, "libisr_debug.so")
INCLUDE = os.path.join(ROOT, "include")

UNITS = ["isr_api.cu", "isr_linefit.cu", "isr_peak.cu", "isr_estimator.cu", "isr_batch.cu", "isr_k_small.cu", "isr_k_mid.cu", "isr_k_8192.cu", "isr_k_16384.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", f"-I{INCLUDE}", f"-I{CSRC}"]


def _deps():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return hdrs + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]


def _stale(target, srcs):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in srcs)


def _compile(unit, verbose, debug=False):
    src = os.path.join(CSRC, unit)
    obj = os.path.join(OBJDIR_DEBUG if debug else OBJDIR, unit.replace(".cu", ".o"))
    if not _stale(obj, [src] + _deps()):
        return obj, ""
    cmd = ["nvcc", *ARCH, *FLAGS, *(["-DISR_DEBUG=1"] if debug else []), "-c", src, "-o", obj + ".tmp"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {unit}:\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return obj, r.stderr


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Build lib/libisr.so (or, with debug=True, lib/libisr_debug.so) and return its path."""
    objdir, lib = (OBJDIR_DEBUG, LIB_DEBUG) if debug else (OBJDIR, LIB)
    os.makedirs(objdir, exist_ok=True)
    if force:
        for f in os.listdir(objdir):
            os.remove(os.path.join(objdir, f))
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        results = list(ex.map(lambda u: _compile(u, verbose, debug), UNITS))
    objs = [o for o, _ in results]
    if verbose:
        for (_, log), u in zip(results, UNITS):
            if log:
                print(f"--- {u}\n{log}")
    if force or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.run(["nvcc", *ARCH, "-shared", "-cudart", "static", *objs, "-o", tmp], check=True)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
