"""Measured issue rates of the pipes the statistic's kernels use (FP32 FMA,
MUFU, FP64 FMA, integer ALU), through ``scs_peak_probe`` of libscstat.so
(include/scs_peaks.h).  They are the roofline denominators of the benchmark:
per SM and clock, so that they scale to the SM clock seen under load.

``python -m paper_2408_13170_gb300.peaks`` prints them as one JSON line.
"""
from __future__ import annotations

import ctypes
import json

from . import scstat

KINDS = {"ffma": 0, "mufu": 1, "dfma": 2, "iadd": 3}
# rounds per probe, sized for a few tens of milliseconds each on a GB300
ITERS = {"ffma": 40000, "mufu": 5000, "dfma": 600, "iadd": 20000}


def probe(kind: str, device: int = 0, iters: int | None = None) -> dict:
    """One probe: ops/s, the in-kernel SM clock and lanes per clock per SM."""
    L = scstat.lib()
    fn = L.scs_peak_probe
    fn.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int
    ops, mhz, per = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    rc = fn(device, KINDS[kind], int(iters or ITERS[kind]), ctypes.byref(ops),
            ctypes.byref(mhz), ctypes.byref(per))
    if rc != 0:
        raise RuntimeError(f"scs_peak_probe({kind}) failed with {rc}")
    return {"ops_per_s": ops.value, "sm_mhz": mhz.value, "ops_per_clk_sm": per.value}


def measure(device: int = 0, repeats: int = 3) -> dict:
    """Best of `repeats` runs of every probe (lanes per clock per SM)."""
    out = {}
    for kind in KINDS:
        runs = [probe(kind, device) for _ in range(repeats)]
        best = max(runs, key=lambda r: r["ops_per_clk_sm"])
        out[kind] = best
    return out


if __name__ == "__main__":
    print(json.dumps(measure()))
