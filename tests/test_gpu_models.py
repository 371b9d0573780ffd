"""The closed-form test models on the CUDA path (scs_debug_set_model).

The oracle's closed-form pins (a Newtonian power-law chirp seen through an
identity response in white noise, and App. A's constant-amplitude linear
chirp) are checked here on the GPU: the same closed forms hold for the
library's edges and segment powers, both evaluation paths agree with the
oracle run in the same model, and the templates agree bin by bin.
"""
import numpy as np
import pytest

import oracle
from paper_2408_13170_gb300 import synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-5


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


def white(T, fmin, fmax, S0, seed=None):
    """White PSD S0; zero data, or Gaussian noise of that PSD if seeded."""
    f_first, df, K = synth.grid(fmin, fmax, T)
    S = np.full(K, S0)
    if seed is None:
        A = np.zeros(K, np.complex128)
        E = np.zeros(K, np.complex128)
    else:
        rng = np.random.default_rng(seed)
        A = synth.noise(S, T, rng)
        E = synth.noise(S, T, rng)
    return dict(f_first=f_first, df=df, K=K, T_obs=T, A=A, E=E, SA=S, SE=S.copy())


def test_power_law_closed_form_on_gpu(scstat):
    """Newtonian + identity response + white PSD: the summed segment powers
    [h|h]_n equal (4/S)(3/4)(f_a^{-4/3} - f_b^{-4/3}) (midpoint rule), and the
    equal-SNR^2 edges sit at f_n^{-4/3} = f_lo^{-4/3} - (n/N)(f_lo^{-4/3} -
    f_hi^{-4/3}) within one bin plus the anchor rule's bound; on both paths,
    and the edges are the oracle's."""
    T = 3e6
    d = white(T, 0.0175, 0.0300, 2.0)
    th = np.array([[100.0, 1.0, 0.018, 0, 0, 0, 0, 0]])
    N = 16
    st, lo, hi = oracle.support(th[0], d["f_first"], d["df"], d["K"], T, oracle.NEWTONIAN)
    assert st == oracle.OK and hi - lo > 5000
    _, kap = oracle.evaluate(d, th, N, mode=oracle.EQUAL_SNR2, waveform=oracle.NEWTONIAN,
                             response=oracle.IDENTITY, want_kappa=True)
    f_first, df = d["f_first"], d["df"]
    fa = f_first + (lo - 0.5) * df
    fb = f_first + (hi + 0.5) * df
    closed = 4.0 / 2.0 * 0.75 * (fa ** (-4 / 3) - fb ** (-4 / 3))
    B = oracle.SNR2_STRIDE
    tol = 1.0 + 1.05 * B * B / 8.0 * (7.0 / 3.0) * df / (f_first + lo * df)
    for path in (scstat.SCS_FP64, scstat.SCS_MIXED):
        with scstat.Context(0, path) as ctx:
            ctx.set_model(scstat.SCS_MODEL_NEWTONIAN, scstat.SCS_RESPONSE_IDENTITY)
            ctx.set_data(0, d)
            ctx.set_segments(0, N, scstat.SCS_EQUAL_SNR2)
            glo, ghi, _ = ctx.support(0, th)
            assert (glo[0], ghi[0]) == (lo, hi)
            e = ctx.edges(0, th, N)[0]
            np.testing.assert_array_equal(e, np.ceil(kap[0]).astype(np.int64))
            for n in range(1, N):
                fn = (fa ** (-4 / 3) - n / N * (fa ** (-4 / 3) - fb ** (-4 / 3))) ** (-3 / 4)
                assert abs(e[n] - ((fn - f_first) / df - 0.5)) <= tol + 1.0
            stat, sx, sh = ctx.eval(0, th, N, segments=True)
            assert sh.sum() == pytest.approx(closed, rel=1e-6)
            assert stat[0] == 0.0 and np.all(sx == 0.0)   # zero data


@pytest.mark.parametrize("N", [4, 10, 50])
def test_linear_chirp_equal_time_segments_on_gpu(scstat, N):
    """App. A: a constant-amplitude linear chirp in white noise has
    equal-SNR^2 boundaries at equal times, i.e. equal numbers of bins."""
    T = 2e6
    d = white(T, 0.0100, 0.0120, 1.0)
    fdot = 5e-10
    th = np.array([[fdot, 1.0, 0.0101, 0, 0, 0, 0, 0]])
    st, lo, hi = oracle.support(th[0], d["f_first"], d["df"], d["K"], T, oracle.LINEAR_CHIRP)
    assert st == oracle.OK
    _, kap = oracle.evaluate(d, th, N, mode=oracle.EQUAL_SNR2, waveform=oracle.LINEAR_CHIRP,
                             response=oracle.IDENTITY, want_kappa=True)
    with scstat.Context(0, scstat.SCS_FP64) as ctx:
        ctx.set_model(scstat.SCS_MODEL_LINEAR_CHIRP, scstat.SCS_RESPONSE_IDENTITY)
        ctx.set_data(0, d)
        ctx.set_segments(0, N, scstat.SCS_EQUAL_SNR2)
        glo, ghi, _ = ctx.support(0, th)
        assert (glo[0], ghi[0]) == (lo, hi)
        e = ctx.edges(0, th, N)[0]
    np.testing.assert_array_equal(e, np.ceil(kap[0]).astype(np.int64))
    expect = lo + (hi + 1 - lo) * np.arange(N + 1) / N
    assert np.max(np.abs(e - expect)) <= 1.0 + 1e-9
    # equal time: t(f) at the edges evenly spaced (to a bin)
    tb = (d["f_first"] + e * d["df"] - th[0, 2]) / fdot
    assert np.max(np.abs(np.diff(tb) - T / N)) <= 2 * d["df"] / fdot


MODELS = [("NEWTONIAN", "TDI_AE"), ("NEWTONIAN", "IDENTITY"), ("LINEAR_CHIRP", "IDENTITY"),
          ("LINEAR_CHIRP", "TDI_AE"), ("TF2", "IDENTITY")]


def model_particles(wave, rng, n):
    if wave == "LINEAR_CHIRP":   # theta[0] = fdot
        return synth.draw_particles(n, rng, lo=[2e-10, 1, 0.0101, 0, -1.5, 0, 0, 0],
                                    hi=[8e-10, 1, 0.0110, 6.28, 1.5, 3.14, 3.14, 0])
    return synth.draw_particles(n, rng, lo=[20, 1, 0.0101, 0, -1.5, 0, 0, 0],
                                hi=[100, 4, 0.0115, 6.28, 1.5, 3.14, 3.14, 0])


@pytest.mark.parametrize("wave,resp", MODELS)
def test_templates_match_oracle_in_test_models(scstat, wave, resp):
    T = 2e6
    d = white(T, 0.0100, 0.0120, 1.0)
    rng = np.random.default_rng(5)
    th = model_particles(wave, rng, 3)
    W, R = getattr(oracle, wave), getattr(oracle, resp)
    with scstat.Context(0, scstat.SCS_FP64) as ctx:
        ctx.set_model(getattr(scstat, f"SCS_MODEL_{wave}"),
                      scstat.SCS_RESPONSE_IDENTITY if resp == "IDENTITY" else scstat.SCS_RESPONSE_TDI)
        ctx.set_data(0, d)
        for t in th:
            st, rA, rE = oracle.template(t, d["f_first"], d["df"], d["K"], T, waveform=W,
                                         response=R)
            assert st == oracle.OK
            hA, hE = ctx.waveform(0, t, d["K"])
            scale = np.max(np.abs(rA)) + np.max(np.abs(rE))
            assert np.max(np.abs(hA - rA)) <= 1e-11 * scale
            assert np.max(np.abs(hE - rE)) <= 1e-11 * scale


@pytest.mark.parametrize("wave,resp", MODELS)
@pytest.mark.parametrize("mode,N", [(oracle.EQUAL_WIDTH, 8), (oracle.EQUAL_SNR2, 12)])
def test_stat_parity_in_test_models(scstat, wave, resp, mode, N):
    """Both paths against the oracle in the same model, on noisy data with
    an injection drawn by the oracle in that model."""
    T = 2e6
    d = white(T, 0.0100, 0.0120, 1.0, seed=9)
    rng = np.random.default_rng(6)
    th = model_particles(wave, rng, 40)
    W, R = getattr(oracle, wave), getattr(oracle, resp)
    # inject the first particle's template at SNR ~ 20 (oracle template)
    st, hA, hE = oracle.template(th[0], d["f_first"], d["df"], d["K"], T, waveform=W,
                                 response=R)
    hh = 4 * d["df"] * np.sum((np.abs(hA) ** 2 + np.abs(hE) ** 2) / d["SA"])
    d["A"] = d["A"] + 20.0 / np.sqrt(hh) * hA
    d["E"] = d["E"] + 20.0 / np.sqrt(hh) * hE
    ref = oracle.evaluate(d, th, N, mode=mode, waveform=W, response=R)
    assert ref[0] > 100.0
    for path, tol in ((scstat.SCS_FP64, TOL64), (scstat.SCS_MIXED, TOL32)):
        with scstat.Context(0, path) as ctx:
            ctx.set_model(getattr(scstat, f"SCS_MODEL_{wave}"),
                          scstat.SCS_RESPONSE_IDENTITY if resp == "IDENTITY"
                          else scstat.SCS_RESPONSE_TDI)
            ctx.set_data(0, d)
            ctx.set_segments(0, N, mode)
            got = ctx.eval(0, th)
        assert rel_err(got, ref) <= tol, (path, rel_err(got, ref))


def test_model_switch_refuses_unknown_models(scstat):
    with scstat.Context(0, scstat.SCS_MIXED) as ctx:
        with pytest.raises(scstat.ScsError):
            ctx.set_model(3, 0)
        with pytest.raises(scstat.ScsError):
            ctx.set_model(0, 2)
        ctx.set_model(scstat.SCS_MODEL_TF2, scstat.SCS_RESPONSE_TDI)
