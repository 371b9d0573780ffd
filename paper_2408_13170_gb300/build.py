"""Builds the CUDA library libscstat.so in-tree (sm_103a only).

Each translation unit is compiled by its own nvcc process (in parallel) and
linked with ``nvcc -shared``; the CUDA runtime is linked statically so the
library loads without a GPU (for the ABI checks on a CPU-only host).
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libscstat.so")
LIB_DEBUG = os.path.join(OUT, "libscstat_debug.so")   # -DSCS_DEBUG: index checks
UNITS = ["scs_api", "scs_setup", "scs_mixed", "scs_fp64", "scs_pso", "scs_peaks", "scs_spline"]
HEADERS = ["scs_device.cuh", "scs_internal.cuh", "scs_anchor.cuh", "scs_setup.cuh", "scs_df.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libscstat")


def _newest_input() -> float:
    paths = [os.path.join(SRC, u + ".cu") for u in UNITS]
    paths += [os.path.join(SRC, h) for h in HEADERS]
    inc = os.path.join(HERE, "..", "include")
    paths += [os.path.join(inc, h) for h in os.listdir(inc) if h.endswith(".h")]
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile (if stale) and return the path of libscstat.so, or with
    debug=True of libscstat_debug.so (the kernels' index checks compiled in,
    read by scs_debug_error)."""
    lib = LIB_DEBUG if debug else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _newest_input():
        return lib
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    tag = f"{os.getpid()}{'d' if debug else ''}"
    flags = FLAGS + (["-DSCS_DEBUG"] if debug else [])

    def compile_unit(u):
        obj = os.path.join(OUT, f"{u}.{tag}.o")
        cmd = [nvcc, *ARCH, *flags, "-c", os.path.join(SRC, u + ".cu"), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {u}.cu:\n{r.stderr}")
        return obj, r.stderr

    try:
        with ThreadPoolExecutor(len(UNITS)) as ex:
            results = list(ex.map(compile_unit, UNITS))
    except RuntimeError:
        for u in UNITS:   # objects of the units that did compile
            o = os.path.join(OUT, f"{u}.{tag}.o")
            if os.path.exists(o):
                os.remove(o)
        raise
    objs = [o for o, _ in results]
    tmp = lib + f".{tag}.tmp"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True,
                       text=True)
    for o in objs:
        os.remove(o)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    if verbose:
        for _, log in results:
            print(log)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
