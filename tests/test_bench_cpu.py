"""The bench on the CPU: its reference arm (the oracle on the host cores)
with the third TDI channel gives one JSON line naming the channels, and the
roofline arithmetic of its line checked by hand."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_three_channels():
    env = dict(os.environ, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--channels", "AET", "--steps",
           "1", "--warmup", "0", "--cpu-sample", "4"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0
    assert "TDI A,E,T" in d["config"]["workload"]
    assert d["cpu_baseline"]["cores"] == 2      # the threads the oracle used


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_roofline_legs_bound_and_fraction():
    """The roofline of the JSON line by hand: each leg is the algorithmic work
    over the measured pipe rate at the clock under load; the slowest leg
    bounds the kernel and frac = that leg's time / the measured time (for the
    FP32 leg also achieved / peak)."""
    b = _bench()
    peaks = {"ffma": {"ops_per_clk_sm": 128.0}, "mufu": {"ops_per_clk_sm": 32.0},
             "dfma": {"ops_per_clk_sm": 2.0}}
    sms, mhz = 100, 1000.0                        # 1e11 SM-cycles per second
    bin_evals = np.array([1.0e8, 1.0e8])
    anchors = np.array([1.0e5, 1.0e5])
    t = np.array([1.0e-3, 1.0e-3])
    r = b.roofline(peaks, sms, mhz, bin_evals, anchors, 1000, t, False, 1000.0)
    legs = r["legs_ms"]
    assert np.isclose(legs["fp32"], 1e3 * 1.0e8 * 55 / 1.28e13)
    assert np.isclose(legs["mufu"], 1e3 * 1.0e8 * 2 / 3.2e12)
    assert np.isclose(legs["fp64"], 1e3 * 1.0e5 * b.FP64_OPS_PER_ANCHOR / 2.0e11)
    assert np.isclose(legs["hbm"], 1e3 * 1000 * 24 / 1.0e12)
    assert r["bound"] == "alu" and r["unit"] == "TFP32-slots/s"
    assert np.isclose(r["frac"], legs["fp32"] / 1e3 / 1.0e-3)
    assert np.isclose(r["achieved"] / r["peak"], r["frac"])
    # many anchors: the FP64 leg bounds the kernel
    r = b.roofline(peaks, sms, mhz, bin_evals, 1000 * anchors, 1000, t, False, 1000.0)
    assert r["bound"] == "fp64"
    assert np.isclose(r["frac"], r["legs_ms"]["fp64"] / 1e3 / 1.0e-3)
    # the third channel counts its own slots per bin
    r = b.roofline(peaks, sms, mhz, bin_evals, anchors, 1000, t, True, 1000.0)
    assert np.isclose(r["legs_ms"]["fp32"], 1e3 * 1.0e8 * 72 / 1.28e13)
    assert np.isclose(r["legs_ms"]["hbm"], 1e3 * 1000 * 40 / 1.0e12)


def test_clock_samples_parsed():
    """The clock record of the JSON line from nvidia-smi's CSV samples: the
    median SM clock, the maximum clock, the sample count and every throttle
    reason seen active; lines that are not samples are skipped."""
    b = _bench()
    cs = b.ClockSampler(0)

    class Finished:   # stands in for the sampling process
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    cs.proc = Finished()
    with open(cs.path, "w") as f:
        f.write("0, 2070, 2070, 900.50, 0x0000000000000000, Not Active, Not Active, "
                "Not Active, Not Active\n")
        f.write("0, 1980, 2070, 1390.00, 0x0000000000000004, Not Active, Not Active, "
                "Not Active, Active\n")
        f.write("[N/A]\n")
        f.write("0, 2070, 2070, 1200.00, 0x0000000000000000, Not Active, Not Active, "
                "Not Active, Not Active\n")
    r = cs.stop()
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "samples": 3,
                 "reasons": ["sw_power_cap"]}
    assert not os.path.exists(cs.path)
