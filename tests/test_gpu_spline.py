"""The sparse-grid spline path (SCS_SPLINE), built like the paper's own GPU
design (Sec. IV: waveform and response on a grid ~1000 times coarser than
the FFT grid, cubic-spline interpolated onto it), against the FP64 oracle.

Its stated tolerance is the mixed path's, 1e-5 relative on Upsilon_N: the
node spacing is chosen per particle so that the phase spline stays within
1e-6 turns, and the products and sums are FP32 with Kahan compensation.
"""
import numpy as np
import pytest

import oracle
from paper_2408_13170_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def scstat():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2408_13170_gb300 import scstat as m
    return m


def rel_err(got, ref):
    ref = np.asarray(ref)
    return np.max(np.abs(np.asarray(got) - ref) / np.maximum(np.abs(ref), 1.0))


def stream(T, fmin, fmax, seed, snr, channels="AE"):
    d = synth.make_stream(dict(T_obs=T, f_min=fmin, f_max=fmax, seed=seed), channels=channels)
    inj = synth.injection_params(d["rng"], 30.0, 1.5, fmin + 0.3 * (fmax - fmin))
    oracle.inject(inj, d["f_first"], d["df"], d["K"], d["T_obs"], d["SA"], d["SE"], snr,
                  d["A"], d["E"], T=d.get("T"), ST=d.get("ST"))
    return d, inj


@pytest.fixture(scope="module")
def month(scstat):
    """A 35-day stream over 0.0175-0.02 Hz (short supports, few nodes)."""
    d, inj = stream(3e6, 0.0175, 0.0200, 31, 18.0)
    rng = np.random.default_rng(8)
    th = np.vstack([inj, synth.draw_particles(60, rng, lo=[10, 1, 0.0176, 0, -1.5, 0, 0, 0],
                                              hi=[100, 8, 0.0195, 6.28, 1.5, 3.14, 3.14, 0])])
    return d, th


@pytest.mark.parametrize("mode,N", [(oracle.EQUAL_WIDTH, 1), (oracle.EQUAL_WIDTH, 8),
                                    (oracle.EQUAL_SNR2, 8), (oracle.EQUAL_SNR2, 100)])
def test_spline_path_matches_oracle(scstat, month, mode, N):
    d, th = month
    ref, rx, rh = oracle.evaluate(d, th, N, mode=mode, want_segments=True)
    with scstat.Context(0, scstat.SCS_SPLINE) as ctx:
        ctx.set_data(0, d)
        ctx.set_segments(0, N, mode)
        stat, sx, sh = ctx.eval(0, th, N, segments=True)
    assert rel_err(stat, ref) <= TOL
    scale = np.maximum(rh.max(axis=1, keepdims=True), 1e-300)
    assert np.max(np.abs(sh - rh) / scale) <= TOL


def test_spline_path_long_stream_and_many_nodes(scstat):
    """A 0.4-year stream over 0.01-0.03 Hz: supports of up to ~250k bins,
    hundreds of spline nodes per particle, the last interval ragged."""
    d, inj = stream(1.26e7, 0.010, 0.030, 32, 20.0)
    rng = np.random.default_rng(9)
    th = np.vstack([inj, synth.draw_particles(40, rng, lo=[10, 1, 0.0101, 0, -1.5, 0, 0, 0],
                                              hi=[100, 8, 0.0250, 6.28, 1.5, 3.14, 3.14, 0])])
    N = 64
    ref = oracle.evaluate(d, th, N, mode=oracle.EQUAL_SNR2)
    with scstat.Context(0, scstat.SCS_SPLINE) as ctx:
        ctx.set_data(0, d)
        ctx.set_segments(0, N, scstat.SCS_EQUAL_SNR2)
        got = ctx.eval(0, th)
        lo, hi, _ = ctx.support(0, th)
    assert np.max(hi - lo) > 100000
    assert rel_err(got, ref) <= TOL


def test_spline_path_three_channels(scstat):
    d, inj = stream(3e6, 0.0175, 0.0200, 33, 18.0, channels="AET")
    rng = np.random.default_rng(10)
    th = np.vstack([inj, synth.draw_particles(30, rng, lo=[10, 1, 0.0176, 0, -1.5, 0, 0, 0],
                                              hi=[100, 8, 0.0195, 6.28, 1.5, 3.14, 3.14, 0])])
    ref = oracle.evaluate(d, th, 8, mode=oracle.EQUAL_SNR2)
    with scstat.Context(0, scstat.SCS_SPLINE) as ctx:
        ctx.set_data(0, d)
        ctx.set_segments(0, 8, scstat.SCS_EQUAL_SNR2)
        got = ctx.eval(0, th)
    assert rel_err(got, ref) <= TOL


def test_spline_spacing_cap_changes_nodes_not_results(scstat, month):
    """A smaller spacing cap adds nodes; the statistic stays within the
    tolerance of the oracle either way."""
    d, th = month
    ref = oracle.evaluate(d, th, 8, mode=oracle.EQUAL_SNR2)
    with scstat.Context(0, scstat.SCS_SPLINE) as ctx:
        ctx.set_data(0, d)
        ctx.set_segments(0, 8, scstat.SCS_EQUAL_SNR2)
        for l2 in (10, 6, 3):
            scstat.scs_set_spline(ctx.h, l2)
            assert rel_err(ctx.eval(0, th), ref) <= TOL
        with pytest.raises(scstat.ScsError):
            scstat.scs_set_spline(ctx.h, 2)


def test_spline_batch_equals_single_calls(scstat, month):
    d, th = month
    d2, inj2 = stream(3e6, 0.0175, 0.0200, 34, 15.0)
    with scstat.Context(0, scstat.SCS_SPLINE) as ctx:
        ctx.set_data(0, d)
        ctx.set_data(1, d2)
        ctx.set_segments(0, 8, scstat.SCS_EQUAL_SNR2)
        ctx.set_segments(1, 16, scstat.SCS_EQUAL_WIDTH)
        a = ctx.eval(0, th)
        b = ctx.eval(1, th[:20])
        ba, bb = ctx.batch_eval([0, 1], [th, th[:20]])
    np.testing.assert_array_equal(ba, a)
    np.testing.assert_array_equal(bb, b)


def test_spline_path_refuses_swarm_and_noalloc(scstat, month):
    import torch
    d, th = month
    with scstat.Context(0, scstat.SCS_MIXED) as ctx:
        ctx.set_data(0, d)
        ctx.set_segments(0, 8, scstat.SCS_EQUAL_SNR2)
        ctx.pso_create([0], [32], synth.PRIOR_BOX["lo"], synth.PRIOR_BOX["hi"], 5)
        ctx.set_path(scstat.SCS_SPLINE)
        with pytest.raises(scstat.ScsError) as e:
            ctx.pso_run(1)
        assert e.value.code == scstat.SCS_EUNSUPPORTED
        dev = torch.tensor(th, device="cuda")
        out = torch.empty(len(th), dtype=torch.float64, device="cuda")
        with pytest.raises(scstat.ScsError) as e:
            scstat.scs_eval_stat_noalloc(ctx.h, 0, dev, len(th), out)
        assert e.value.code == scstat.SCS_EUNSUPPORTED


def test_spline_path_short_supports_near_band_end(scstat):
    """The C1 band (0.015-0.03 Hz, 35 days) with particles up to the band's
    end: supports of a few bins to a few thousand, where a spline with fewer
    than four nodes would degrade to a parabola or a line."""
    d, inj = stream(3e6, 0.015, 0.030, 35, 20.0)
    rng = np.random.default_rng(12)
    th = np.vstack([inj, synth.draw_particles(120, rng)])
    for mode, N in ((oracle.EQUAL_WIDTH, 8), (oracle.EQUAL_SNR2, 16)):
        ref = oracle.evaluate(d, th, N, mode=mode)
        with scstat.Context(0, scstat.SCS_SPLINE) as ctx:
            ctx.set_data(0, d)
            ctx.set_segments(0, N, mode)
            got = ctx.eval(0, th)
        assert rel_err(got, ref) <= TOL
