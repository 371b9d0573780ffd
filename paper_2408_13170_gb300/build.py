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


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if stale) and return the path of libscstat.so."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    tag = f"{os.getpid()}"

    def compile_unit(u):
        obj = os.path.join(OUT, f"{u}.{tag}.o")
        cmd = [nvcc, *ARCH, *FLAGS, "-c", os.path.join(SRC, u + ".cu"), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {u}.cu:\n{r.stderr}")
        return obj, r.stderr

    with ThreadPoolExecutor(len(UNITS)) as ex:
        results = list(ex.map(compile_unit, UNITS))
    objs = [o for o, _ in results]
    tmp = LIB + f".{tag}.tmp"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True,
                       text=True)
    for o in objs:
        os.remove(o)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        for _, log in results:
            print(log)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
