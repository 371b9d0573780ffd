"""The background campaign of the FAP estimate (Sec. V) on the device: the
hierarchical search on signal-free streams gives one Upsilon_{N=1} maximum
per stream; a loud injection searched the same way stands far above them."""
import math

import numpy as np
import pytest

import oracle
from paper_2408_13170_gb300 import fap, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scstat():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2408_13170_gb300 import scstat as m
    return m


def test_background_campaign_and_candidate(scstat):
    cfg = dict(T_obs=3e6, f_min=0.0175, f_max=0.0200)
    th = np.array([30.0, 1.5, 0.018, 1.1, 0.4, 1.2, 0.7, 0.0])
    lo = th.copy()
    hi = th.copy()
    lo[:3] = th[:3] * np.array([0.9, 0.8, 0.999])
    hi[:3] = th[:3] * np.array([1.1, 1.2, 1.001])
    lo[3:7] = [0, -math.pi / 2, 0, 0]
    hi[3:7] = [2 * math.pi, math.pi / 2, math.pi, math.pi]
    with scstat.Context(0, scstat.SCS_MIXED) as ctx:
        bg, iters = fap.noise_background(ctx, [101, 102, 103, 104], cfg, lo, hi, [128, 128],
                                         ladder=(16, 4, 1), chunk_iters=10, max_iters=60)
        assert bg.shape == (4,) and np.all(np.isfinite(bg)) and np.all(bg > 0)
        assert all(len(i) == 3 and np.all(i >= 1) for i in iters)
        # every maximum is a genuine Upsilon_1 of some particle: re-evaluate
        # the best swarm position of the last campaign stream with the oracle
        st = ctx.pso_get()
        best = st["swarm_pos"][int(np.argmax(st["swarm_val"]))]
        d = synth.make_stream(dict(cfg, seed=104))
        ref = oracle.evaluate(d, best[None], 1, mode=oracle.EQUAL_SNR2)[0]
        assert bg[-1] == pytest.approx(ref, rel=1e-5)
        # a loud candidate: the same search on an injection at SNR 30
        d = synth.make_stream(dict(cfg, seed=105))
        oracle.inject(th, d["f_first"], d["df"], d["K"], d["T_obs"], d["SA"], d["SE"], 30.0,
                      d["A"], d["E"])
        ctx.set_data(0, d)
        ctx.pso_create([0, 0], [128, 128], lo, hi, 105)
        ctx.pso_search([16, 4, 1], chunk_iters=10, max_iters=60)
        cand = float(np.max(ctx.pso_get()["swarm_val"]))
    assert cand > bg.max()
    row = fap.fap_table(bg, [cand], x_min=float(np.min(bg)))[0]
    assert row["empirical"] == 0.0 and row["empirical_bound"]
    assert row["gumbel"] < row["floor"] and row["power_law"] < row["floor"]
