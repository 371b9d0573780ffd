"""Cases run by tests/test_gpu_debug.py twice: in the test process with the
normal library and in a child process with the debug build (SCS_DEBUG=1).
Not collected by pytest (no test_ prefix); imports nothing of the oracle but
its injection, like the other GPU tests' streams."""
import sys

import numpy as np

import oracle
from paper_2408_13170_gb300 import scstat, synth


def _stream(seed, channels="AE", T=3e6, fmin=0.0175, fmax=0.0200):
    d = synth.make_stream(dict(T_obs=T, f_min=fmin, f_max=fmax, seed=seed), channels=channels)
    inj = synth.injection_params(d["rng"], 30.0, 1.5, 0.018)
    oracle.inject(inj, d["f_first"], d["df"], d["K"], d["T_obs"], d["SA"], d["SE"], 18.0,
                  d["A"], d["E"], T=d.get("T"), ST=d.get("ST"))
    rng = np.random.default_rng(seed)
    th = np.vstack([inj, synth.draw_particles(
        70, rng, lo=[10, 1, 0.0176, 0, -1.5, 0, 0, 0], hi=[100, 8, 0.019, 6.28, 1.5, 3.14, 3.14, 0.1]),
        synth.draw_particles(30, rng)])   # the whole prior box: short and long supports
    return d, th


def run():
    """Statistics of every path and segmentation, a two-stream batch with the
    third channel and two swarm iterations; returns (results, debug record)."""
    out = {}
    d, th = _stream(21)
    d3, th3 = _stream(22, channels="AET", T=2e6, fmin=0.0150, fmax=0.0190)
    with scstat.Context(0, scstat.SCS_MIXED) as ctx:
        ctx.set_data(0, d)
        ctx.set_data(1, d3)
        for path, name in ((scstat.SCS_MIXED, "mixed"), (scstat.SCS_FP64, "fp64"),
                           (scstat.SCS_SPLINE, "spline")):
            ctx.set_path(path)
            for mode, N in ((scstat.SCS_EQUAL_SNR2, 64), (scstat.SCS_EQUAL_WIDTH, 8),
                            (scstat.SCS_EQUAL_SNR2, 1)):
                ctx.set_segments(0, N, mode)
                out[f"{name}_{mode}_{N}"] = ctx.eval(0, th)
        ctx.set_path(scstat.SCS_MIXED)
        ctx.set_segments(0, 16, scstat.SCS_EQUAL_SNR2)
        ctx.set_segments(1, 5, scstat.SCS_EQUAL_WIDTH)
        b = ctx.batch_eval([0, 1], [th, th3])
        out["batch0"], out["batch1"] = b[0], b[1]
        out["edges"] = ctx.edges(0, th, 16)
        lo = synth.PRIOR_BOX["lo"].copy()
        hi = synth.PRIOR_BOX["hi"].copy()
        lo[2], hi[2] = 0.0176, 0.019
        ctx.pso_create([0, 1], [40, 24], lo, hi, 5)
        ctx.pso_run(2, use_graph=False)
        st = ctx.pso_get()
        out["pso_stat"], out["pso_pos"] = st["stat"], st["pos"]
        dbg = scstat.scs_debug_error(ctx.h)
    return out, dbg


if __name__ == "__main__":
    res, dbg = run()
    np.savez(sys.argv[1], dbg=np.array([int(dbg[0]), dbg[1], dbg[2]], dtype=np.int64), **res)
