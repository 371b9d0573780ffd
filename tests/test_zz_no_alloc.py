"""scs_eval_stat_noalloc: the evaluation entry point for callers that cannot
allocate device memory at call time (device memory owned by another
allocator, loops that must not pay an allocation's latency or
synchronisation).  It must give the same statistic as scs_eval_stat, on two
calls in a row (the shared scratch array keeps the previous call's
contents), leave the device's free memory unchanged, and refuse sizes beyond
its fixed scratch.

This file is collected last on purpose; it also passes on its own."""
import numpy as np
import pytest

import oracle
from paper_2408_13170_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2408_13170_gb300 import scstat
    d = synth.make_stream(dict(T_obs=3e6, f_min=0.0175, f_max=0.0200, seed=41))
    inj = synth.injection_params(d["rng"], 30.0, 1.5, 0.018)
    oracle.inject(inj, d["f_first"], d["df"], d["K"], d["T_obs"], d["SA"], d["SE"], 18.0,
                  d["A"], d["E"])
    rng = np.random.default_rng(77)
    th = np.vstack([inj, synth.draw_particles(
        90, rng, lo=[10, 1, 0.0176, 0, -1.5, 0, 0, 0], hi=[100, 8, 0.019, 6.28, 1.5, 3.14, 3.14, 0])])
    ctx = scstat.Context(0, scstat.SCS_MIXED)
    ctx.set_data(0, d)
    yield scstat, torch, ctx, th
    ctx.close()


@pytest.mark.parametrize("path,tol", [("mixed", 1e-5), ("fp64", 1e-10)])
@pytest.mark.parametrize("mode,N", [(0, 8), (1, 16)])
def test_noalloc_matches_eval_stat(env, path, tol, mode, N):
    scstat, torch, ctx, th = env
    ctx.set_path(scstat.SCS_MIXED if path == "mixed" else scstat.SCS_FP64)
    ctx.set_segments(0, N, mode)
    P = len(th)
    dev_th = torch.tensor(th, device="cuda")
    ref = torch.empty(P, dtype=torch.float64, device="cuda")
    scstat.scs_eval_stat(ctx.h, 0, dev_th, P, ref)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    for call in range(2):   # the second call starts from the first call's scratch
        out = torch.full((P,), np.nan, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        scstat.scs_eval_stat_noalloc(ctx.h, 0, dev_th, P, out)
        torch.cuda.synchronize()
        if call == 1:   # (the first call may load kernel code on first use)
            assert torch.cuda.mem_get_info()[0] == free0
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)) <= tol


def test_noalloc_refuses_oversized_calls(env):
    scstat, torch, ctx, th = env
    ctx.set_path(scstat.SCS_MIXED)
    ctx.set_segments(0, 8, 0)
    P = 300_000
    big = torch.tensor(np.repeat(th[:1], P, axis=0), device="cuda")
    out = torch.empty(P, dtype=torch.float64, device="cuda")
    with pytest.raises(scstat.ScsError) as e:
        scstat.scs_eval_stat_noalloc(ctx.h, 0, big, P, out)
    assert e.value.code == scstat.SCS_EINVAL
    assert "scratch" in str(e.value)
    # host pointers are refused too (nothing would be there to stage them)
    with pytest.raises(scstat.ScsError):
        scstat.scs_eval_stat_noalloc(ctx.h, 0, th, len(th), np.empty(len(th)))
