"""Parity of the CUDA paths with the FP64 CPU oracle on streams with the third
TDI channel T (scs_set_data_aet; the search uses A, E and T, Sec. I).

Same tolerances as the two-channel parity tests: relative to
max(|Upsilon_oracle|, 1), FP64 path 1e-10, mixed path 1e-5; integer outputs
(segment edges) identical.
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


def stream(T=3e6, fmin=0.0175, fmax=0.0200, seed=41, snr=18.0, inj=(30.0, 1.5, 0.018),
           channels="AET", noise_free=False):
    d = synth.make_stream(dict(T_obs=T, f_min=fmin, f_max=fmax, seed=seed), channels=channels,
                          noise_free=noise_free)
    th = synth.injection_params(d["rng"], *inj)
    hh = oracle.inject(th, d["f_first"], d["df"], d["K"], d["T_obs"], d["SA"], d["SE"], snr,
                       d["A"], d["E"], T=d.get("T"), ST=d.get("ST"))
    return d, th, hh


def particles(rng, n, f_lo=0.0176, f_hi=0.019):
    return synth.draw_particles(n, rng, lo=[10, 1, f_lo, 0, -1.5, 0, 0, 0],
                                hi=[100, 8, f_hi, 6.28, 1.5, 3.14, 3.14, 0])


@pytest.fixture(scope="module")
def small(scstat):
    d, inj, _ = stream()
    rng = np.random.default_rng(14)
    th = np.vstack([inj, particles(rng, 70)])
    ctx = scstat.Context(0, scstat.SCS_FP64)
    ctx.set_data(0, d)
    yield d, th, ctx
    ctx.close()


def test_aet_waveform_matches_oracle(scstat, small):
    d, th, ctx = small
    for p in th[:6]:
        hA, hE, hT = ctx.waveform(0, p, d["K"], want_T=True)
        _, oA, oE, oT = oracle.template(p, d["f_first"], d["df"], d["K"], d["T_obs"],
                                        want_T=True)
        scale = max(np.abs(oA).max(), np.abs(oE).max())
        assert np.max(np.abs(hA - oA)) <= 1e-11 * scale
        assert np.max(np.abs(hE - oE)) <= 1e-11 * scale
        assert np.max(np.abs(hT - oT)) <= 1e-10 * np.abs(oT).max()
        # the two-channel call gives the same A and E
        a2, e2 = ctx.waveform(0, p, d["K"])
        np.testing.assert_array_equal(a2, hA)
        np.testing.assert_array_equal(e2, hE)


@pytest.mark.parametrize("N", [1, 7, 64])
def test_aet_snr2_edges_are_exact(scstat, small, N):
    """The equal-SNR^2 cut uses the template power of all three channels."""
    d, th, ctx = small
    ctx.set_segments(0, N, scstat.SCS_EQUAL_SNR2)
    e = ctx.edges(0, th, N)
    _, kap = oracle.evaluate(d, th, N, mode=oracle.EQUAL_SNR2, want_kappa=True)
    np.testing.assert_array_equal(e, np.ceil(kap).astype(np.int64))


@pytest.mark.parametrize("path", ["fp64", "mixed"])
@pytest.mark.parametrize("mode", [oracle.EQUAL_WIDTH, oracle.EQUAL_SNR2])
@pytest.mark.parametrize("N", [1, 8, 100])
def test_aet_stat_parity(scstat, small, path, mode, N):
    d, th, ctx = small
    ctx.set_path(scstat.SCS_FP64 if path == "fp64" else scstat.SCS_MIXED)
    ctx.set_segments(0, N, mode)
    stat, sx, sh = ctx.eval(0, th, N, segments=True)
    ref, rx, rh = oracle.evaluate(d, th, N, mode=mode, want_segments=True)
    tol = TOL64 if path == "fp64" else TOL32
    assert rel_err(stat, ref) <= tol
    scale = np.maximum(rh.max(axis=1, keepdims=True), 1e-300)
    assert np.max(np.abs(sh - rh) / scale) <= tol
    xs = np.maximum(rx.max(axis=1, keepdims=True), 1e-300)
    assert np.max(np.abs(sx - rx) / xs) <= 10 * tol
    assert np.argmax(stat) == np.argmax(ref)
    # the T channel changes the statistic: the two-channel oracle differs
    ae = {k: v for k, v in d.items() if k not in ("T", "ST")}
    ref2 = oracle.evaluate(ae, th[:1], N, mode=mode)
    assert abs(ref2[0] - ref[0]) > 100 * tol * max(abs(ref[0]), 1.0)


def test_aet_batch_with_two_channel_streams(scstat):
    """One call over two-channel and three-channel streams: each particle
    gives its single-stream bits (one main kernel per channel set) and the
    oracle's value."""
    specs = [(3e6, 0.0175, 0.0200, 51, 8, oracle.EQUAL_SNR2, "AE"),
             (2e6, 0.0150, 0.0190, 52, 5, oracle.EQUAL_WIDTH, "AET"),
             (4e6, 0.0120, 0.0220, 53, 64, oracle.EQUAL_SNR2, "AET")]
    rng = np.random.default_rng(5)
    with scstat.Context(0, scstat.SCS_MIXED) as ctx:
        datas, ths = [], []
        for i, (T, f0, f1, seed, N, mode, ch) in enumerate(specs):
            d, inj, _ = stream(T=T, fmin=f0, fmax=f1, seed=seed, channels=ch)
            ctx.set_data(i, d)
            ctx.set_segments(i, N, mode)
            datas.append(d)
            ths.append(np.vstack([inj, particles(rng, 25 + 11 * i, f0 * 1.01, f1 * 0.95)]))
        for path, tol in ((scstat.SCS_MIXED, TOL32), (scstat.SCS_FP64, TOL64)):
            ctx.set_path(path)
            single = [ctx.eval(i, th) for i, th in enumerate(ths)]
            batched = ctx.batch_eval([0, 1, 2], ths)
            for i in range(3):
                np.testing.assert_array_equal(batched[i], single[i])
                ref = oracle.evaluate(datas[i], ths[i], specs[i][4], mode=specs[i][5])
                assert rel_err(batched[i], ref) <= tol
        # reloading a slot with two channels drops T
        ctx.set_path(scstat.SCS_MIXED)
        ae = {k: v for k, v in datas[1].items() if k not in ("T", "ST")}
        ctx.set_data(1, ae)
        ref = oracle.evaluate(ae, ths[1], specs[1][4], mode=specs[1][5])
        assert rel_err(ctx.eval(1, ths[1]), ref) <= TOL32


def test_aet_injection_and_loglike(scstat):
    """The library's injection on a three-channel stream equals the
    oracle's; the log-likelihood (with <d|d> over A, E, T) matches the
    oracle's and vanishes at the noise-free truth with the injected
    amplitude."""
    d0, inj, _ = stream(noise_free=True, snr=0.0, seed=61)
    d = dict(d0)
    for key in ("A", "E", "T"):
        d[key] = d0[key].copy()
    hh0 = oracle.inject(inj, d["f_first"], d["df"], d["K"], d["T_obs"], d["SA"], d["SE"], 12.0,
                        d["A"], d["E"], T=d["T"], ST=d["ST"])
    rng = np.random.default_rng(6)
    th = np.vstack([inj, particles(rng, 30)])
    with scstat.Context(0, scstat.SCS_FP64) as ctx:
        ctx.set_data(0, d0)                 # noise-free, no signal
        hh = ctx.inject(0, inj, 12.0)
        assert hh == pytest.approx(hh0, rel=1e-10)
        ctx.set_segments(0, 8, scstat.SCS_EQUAL_SNR2)
        ref = oracle.evaluate(d, th, 8, mode=oracle.EQUAL_SNR2)
        assert rel_err(ctx.eval(0, th), ref) <= TOL64
        a = 12.0 / np.sqrt(hh0)
        L, O, H = ctx.loglike(0, inj[None, :], [a])
        assert abs(L[0]) <= 1e-8 * 144.0
        assert H[0] == pytest.approx(hh0, rel=1e-10)
        amp = np.linspace(0.5, 2.0, len(th)) * a
        for path, tol in ((scstat.SCS_FP64, TOL64), (scstat.SCS_MIXED, TOL32)):
            ctx.set_path(path)
            L, O, H = ctx.loglike(0, th, amp)
            rL, rO, rH = oracle.loglike(d, th, 8, mode=oracle.EQUAL_SNR2, amp=amp)
            ok = np.isfinite(rL)
            scale = 0.5 * oracle.inner_dd(d) + np.abs(amp * rO) + amp * amp * rH
            assert np.max(np.abs(L[ok] - rL[ok]) / scale[ok]) <= tol


def test_aet_mid_size_and_call_independence(scstat):
    """A 2e7 s stream (50 001 bins, several tiles) with 300 particles and
    N = 64 equal-SNR^2 segments on the mixed path against the oracle; a
    large call, small calls and the no-allocation entry point give the same
    bits."""
    import torch
    d, inj, _ = stream(T=2e7, seed=71, snr=20.0)
    rng = np.random.default_rng(7)
    th = np.vstack([inj, particles(rng, 299)])
    with scstat.Context(0, scstat.SCS_MIXED) as ctx:
        ctx.set_data(0, d)
        ctx.set_segments(0, 64, scstat.SCS_EQUAL_SNR2)
        stat = ctx.eval(0, th)
        ref = oracle.evaluate(d, th, 64, mode=oracle.EQUAL_SNR2)
        assert rel_err(stat, ref) <= TOL32
        assert np.argmax(stat) == np.argmax(ref) == 0
        pieces = np.concatenate([ctx.eval(0, th[i:i + 70]) for i in range(0, len(th), 70)])
        np.testing.assert_array_equal(stat, pieces)
        dev = torch.tensor(th, device="cuda")
        out = torch.empty(len(th), dtype=torch.float64, device="cuda")
        scstat.scs_eval_stat_noalloc(ctx.h, 0, dev, len(th), out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), stat)


def test_aet_swarm_iteration(scstat):
    """One device swarm iteration (CUDA graph) on a three-channel stream
    equals the reference update applied to the library's own statistic."""
    from oracle import pso as rpso
    d, _, _ = stream(seed=81)
    lo = np.array([20, 1, 0.0176, 0, -np.pi / 2, 0, 0, 0], float)
    hi = np.array([80, 4, 0.019, 2 * np.pi, np.pi / 2, np.pi, np.pi, 0], float)
    with scstat.Context(0, scstat.SCS_MIXED) as ctx:
        ctx.set_data(0, d)
        ctx.set_segments(0, 8, scstat.SCS_EQUAL_SNR2)
        ctx.pso_create([0], [64], lo, hi, 5)
        s0 = ctx.pso_get()
        ctx.pso_run(1, use_graph=True)
        s1 = ctx.pso_get()
        ref = oracle.evaluate(d, s0["pos"], 8, mode=oracle.EQUAL_SNR2)
        assert rel_err(s1["stat"], ref) <= TOL32
    hyper = np.concatenate([[0.5, 0.2, 0.3], [0.1, 0.05, 5e-8, 0.1, 0.1, 0.2, 0.1, 0.1]])[None]
    bp, bv, sp, sv = rpso.pso_bests(s1["stat"], s0["pos"], s0["best_pos"], s0["best_val"],
                                    s0["swarm_pos"], s0["swarm_val"], [0, 64])
    pos, vel = rpso.pso_step(s0["pos"], s0["vel"], bp, sp, np.zeros(64, int), hyper, lo, hi, 5, 0)
    assert np.array_equal(s1["pos"], pos) and np.array_equal(s1["vel"], vel)
