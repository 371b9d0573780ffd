"""Parity of the CUDA paths with the FP64 CPU oracle, through the C ABI.

Tolerances (relative to max(|Upsilon_oracle|, 1), the statistic's natural
scale: noise alone gives Upsilon ~ 2N >= 2):
  FP64 path  1e-10   (both compute the waveform phase in double-double)
  mixed path 1e-5    (FP32 split phase; the bound stated for the method)
Integer outputs (supports, segment edges) must be identical.
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


def stream(T=3e6, fmin=0.0175, fmax=0.0200, seed=21, snr=18.0, inj=(30.0, 1.5, 0.018)):
    d = synth.make_stream(dict(T_obs=T, f_min=fmin, f_max=fmax, seed=seed))
    th = synth.injection_params(d["rng"], *inj)
    oracle.inject(th, d["f_first"], d["df"], d["K"], d["T_obs"], d["SA"], d["SE"], snr,
                  d["A"], d["E"])
    return d, th


def particles(rng, n, f_lo=0.0176, f_hi=0.019, mc=(10, 100), q=(1, 8), e0=(0.0, 0.1)):
    return synth.draw_particles(n, rng, lo=[mc[0], q[0], f_lo, 0, -1.5, 0, 0, e0[0]],
                                hi=[mc[1], q[1], f_hi, 6.28, 1.5, 3.14, 3.14, e0[1]])


@pytest.fixture(scope="module")
def small(scstat):
    d, inj = stream()
    rng = np.random.default_rng(4)
    th = np.vstack([inj, particles(rng, 70)])
    ctx = scstat.Context(0, scstat.SCS_FP64)
    ctx.set_data(0, d)
    yield d, th, ctx
    ctx.close()


def test_waveform_matches_oracle(scstat, small):
    d, th, ctx = small
    for p in th[:6]:
        hA, hE = ctx.waveform(0, p, d["K"])
        _, oA, oE = oracle.template(p, d["f_first"], d["df"], d["K"], d["T_obs"])
        scale = max(np.abs(oA).max(), np.abs(oE).max())
        assert np.max(np.abs(hA - oA)) <= 1e-11 * scale
        assert np.max(np.abs(hE - oE)) <= 1e-11 * scale


def test_support_is_exact(scstat, small):
    d, th, ctx = small
    rng = np.random.default_rng(9)
    extra = synth.draw_particles(200, rng)            # full prior box
    bad = np.array([[-1, 1.5, .018, 0, 0, 0, 0, 0], [30, .5, .018, 0, 0, 0, 0, 0],
                    [30, 1.5, .05, 0, 0, 0, 0, 0], [2e5, 1, .018, 0, 0, 0, 0, 0],
                    [30, 1.5, .018, 0, 0, 0, 0, 0.1]], float)
    allp = np.vstack([th, extra, bad])
    lo, hi, _ = ctx.support(0, allp)
    for i, p in enumerate(allp):
        st, olo, ohi = oracle.support(p, d["f_first"], d["df"], d["K"], d["T_obs"])
        if st == oracle.INVALID:
            assert lo[i] == -1 and hi[i] == -1, i
        elif st == oracle.EMPTY:
            assert hi[i] < lo[i], i
        else:
            assert (lo[i], hi[i]) == (olo, ohi), i


@pytest.mark.parametrize("N", [1, 7, 64])
def test_snr2_edges_are_exact(scstat, small, N):
    d, th, ctx = small
    ctx.set_segments(0, N, scstat.SCS_EQUAL_SNR2)
    e = ctx.edges(0, th, N)
    _, kap = oracle.evaluate(d, th, N, mode=oracle.EQUAL_SNR2, want_kappa=True)
    np.testing.assert_array_equal(e, np.ceil(kap).astype(np.int64))


@pytest.mark.parametrize("path", ["fp64", "mixed"])
@pytest.mark.parametrize("mode", [oracle.EQUAL_WIDTH, oracle.EQUAL_SNR2])
@pytest.mark.parametrize("N", [1, 8, 100])
def test_stat_parity(scstat, small, path, mode, N):
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
    # the injected particle is the best one on both sides
    assert np.argmax(stat) == np.argmax(ref)


def test_edge_cases(scstat, small):
    """Non-physical particles -> -inf, empty support -> 0, single particle,
    a ragged particle count, and the largest segment count N = K."""
    d, th, ctx = small
    ctx.set_path(scstat.SCS_MIXED)
    bad = np.array([[-1, 1.5, .018, 0, 0, 0, 0, 0], [30, 1.5, np.inf, 0, 0, 0, 0, 0],
                    [30, 1.5, 0.025, 0, 0, 0, 0, 0], [30, 1.5, .018, 0, 0, 0, 0, 0.35],
                    [30, 1.5, .018, 0, 0, 0, 0, -0.01], [30, 1.5, .018, 0, 0, 0, 0, 0.3]])
    ctx.set_segments(0, 4, scstat.SCS_EQUAL_WIDTH)
    s = ctx.eval(0, bad)
    assert np.isneginf(s[0]) and np.isneginf(s[1]) and s[2] == 0.0 and np.isneginf(s[3])
    assert np.isneginf(s[4]) and s[5] > 0.0   # e0 in [0, 0.3]
    ref = oracle.evaluate(d, bad, 4)
    assert np.array_equal(np.isneginf(s), np.isneginf(ref))
    assert abs(s[5] - ref[5]) <= TOL32 * abs(ref[5])
    for path in (scstat.SCS_FP64, scstat.SCS_MIXED):
        ctx.set_path(path)
        one = ctx.eval(0, th[:1])
        ref = oracle.evaluate(d, th[:1], 4)
        assert rel_err(one, ref) <= (TOL64 if path == scstat.SCS_FP64 else TOL32)
    # N = K: every bin its own segment (equal width)
    small_d = synth.make_stream(dict(T_obs=3e6, f_min=0.0179, f_max=0.01815, seed=5))
    ctx.set_data(1, small_d)
    K = small_d["K"]
    ctx.set_segments(1, K, scstat.SCS_EQUAL_WIDTH)
    p = np.array([[30.0, 1.5, 0.018, 1.0, 0.2, 0.5, 0.3, 0.0]])
    ref = oracle.evaluate(small_d, p, K)
    for path in (scstat.SCS_FP64, scstat.SCS_MIXED):
        ctx.set_path(path)
        got = ctx.eval(1, p)
        assert rel_err(got, ref) <= (TOL64 if path == scstat.SCS_FP64 else TOL32)


def test_slow_and_fast_chirps(scstat):
    """Particles from the whole prior box (slow chirps with a few bins of
    support up to signals reaching the last stable orbit) over a band that
    spans several work chunks."""
    d, inj = stream(T=4e6, fmin=0.012, fmax=0.03, seed=33)
    rng = np.random.default_rng(12)
    th = np.vstack([inj, synth.draw_particles(96, rng)])
    with scstat.Context(0, scstat.SCS_MIXED) as ctx:
        ctx.set_data(0, d)
        for mode, N in ((scstat.SCS_EQUAL_SNR2, 16), (scstat.SCS_EQUAL_WIDTH, 32)):
            ctx.set_segments(0, N, mode)
            ref = oracle.evaluate(d, th, N, mode=mode)
            ctx.set_path(scstat.SCS_MIXED)
            assert rel_err(ctx.eval(0, th), ref) <= TOL32
            ctx.set_path(scstat.SCS_FP64)
            assert rel_err(ctx.eval(0, th), ref) <= TOL64


def test_device_pointers_and_streams(scstat, small):
    """torch CUDA tensors in, results on the device, on a user stream; the
    same numbers as the host-pointer call."""
    import torch
    d, th, ctx = small
    ctx.set_path(scstat.SCS_MIXED)
    ctx.set_segments(0, 8, scstat.SCS_EQUAL_SNR2)
    host = ctx.eval(0, th)
    dev_th = torch.tensor(th, device="cuda")
    out = torch.empty(len(th), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        scstat.scs_eval_stat(ctx.h, 0, dev_th, len(th), out, cuda_stream=s)
    s.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), host)


def test_argument_errors(scstat):
    ctx = scstat.Context(0, scstat.SCS_MIXED)
    with pytest.raises(scstat.ScsError) as e:
        ctx.eval(0, np.zeros((1, 8)))
    assert e.value.code == scstat.SCS_ENODATA
    d = synth.make_stream(dict(T_obs=3e6, f_min=0.0179, f_max=0.0181, seed=5))
    bad = dict(d)
    bad["SA"] = d["SA"].copy()
    bad["SA"][3] = -1.0
    with pytest.raises(scstat.ScsError) as e:
        ctx.set_data(0, bad)
    assert e.value.code == scstat.SCS_EINVAL
    bad = dict(d)
    bad["df"] = d["df"] * 1.001
    with pytest.raises(scstat.ScsError):
        ctx.set_data(0, bad)
    ctx.set_data(0, d)
    with pytest.raises(scstat.ScsError):
        ctx.set_segments(0, d["K"] + 1, scstat.SCS_EQUAL_WIDTH)
    with pytest.raises(scstat.ScsError):
        ctx.set_segments(0, 4, 9)
    with pytest.raises(scstat.ScsError) as e:
        ctx.eval(0, np.zeros((1, 8)))
    assert e.value.code == scstat.SCS_ENODATA
    ctx.close()


def test_c1_full(scstat):
    """The small published configuration in full: 256 particles, 45 001 bins,
    N = 8 equal-width segments; both paths against the oracle."""
    d = synth.make_stream("C1")
    cfg = d["cfg"]
    inj = synth.injection_params(d["rng"], *cfg["inj"])
    oracle.inject(inj, d["f_first"], d["df"], d["K"], d["T_obs"], d["SA"], d["SE"],
                  cfg["snr"], d["A"], d["E"])
    th = synth.draw_particles(cfg["P"], d["rng"])
    th[0] = inj
    ref = oracle.evaluate(d, th, cfg["N"], mode=oracle.EQUAL_WIDTH)
    with scstat.Context(0, scstat.SCS_FP64) as ctx:
        ctx.set_data(0, d)
        ctx.set_segments(0, cfg["N"], scstat.SCS_EQUAL_WIDTH)
        s64 = ctx.eval(0, th)
        ctx.set_path(scstat.SCS_MIXED)
        s32 = ctx.eval(0, th)
    assert rel_err(s64, ref) <= TOL64
    assert rel_err(s32, ref) <= TOL32
    assert np.argmax(s32) == np.argmax(ref) == 0


def test_batch_eval_matches_single_streams(scstat):
    """One persistent launch over three streams with different durations,
    bands, segment counts and segmentations gives, particle by particle, the
    single-stream results (and the oracle's)."""
    specs = [(3e6, 0.0175, 0.0200, 31, 8, oracle.EQUAL_SNR2),
             (2e6, 0.0150, 0.0190, 32, 5, oracle.EQUAL_WIDTH),
             (4e6, 0.0120, 0.0220, 33, 64, oracle.EQUAL_SNR2)]
    rng = np.random.default_rng(3)
    with scstat.Context(0, scstat.SCS_MIXED) as ctx:
        datas, ths = [], []
        for i, (T, f0, f1, seed, N, mode) in enumerate(specs):
            d, inj = stream(T=T, fmin=f0, fmax=f1, seed=seed)
            ctx.set_data(i, d)
            ctx.set_segments(i, N, mode)
            th = np.vstack([inj, particles(rng, 20 + 17 * i, f_lo=f0 * 1.01, f_hi=f1 * 0.95)])
            datas.append(d)
            ths.append(th)
        for path, tol in ((scstat.SCS_MIXED, TOL32), (scstat.SCS_FP64, TOL64)):
            ctx.set_path(path)
            single = [ctx.eval(i, th) for i, th in enumerate(ths)]
            batched = ctx.batch_eval([0, 1, 2], ths)
            for i in range(3):
                np.testing.assert_array_equal(batched[i], single[i])
                ref = oracle.evaluate(datas[i], ths[i], specs[i][4], mode=specs[i][5])
                assert rel_err(batched[i], ref) <= tol
        # the same stream twice, and an empty item
        ctx.set_path(scstat.SCS_MIXED)
        b = ctx.batch_eval([2, 0, 2], [ths[2][:5], np.zeros((0, 8)), ths[2][5:]])
        np.testing.assert_array_equal(np.concatenate([b[0], b[2]]), ctx.eval(2, ths[2]))


def test_large_call_matches_small_calls(scstat, small):
    """A particle's result does not depend on the other particles of its
    call (its work-item grouping, chunk-list order and batch): a large
    equal-SNR^2 call, small calls, the no-allocation entry point and a
    batch split all give the same bits."""
    import torch
    d, th, ctx = small
    rng = np.random.default_rng(17)
    big = np.vstack([th, particles(rng, 2600 - len(th))])
    ctx.set_path(scstat.SCS_MIXED)
    ctx.set_segments(0, 64, oracle.EQUAL_SNR2)
    stat = ctx.eval(0, big)
    pieces = np.concatenate([ctx.eval(0, big[i:i + 700]) for i in range(0, len(big), 700)])
    np.testing.assert_array_equal(stat, pieces)
    dev = torch.tensor(big, device="cuda")
    out = torch.empty(len(big), dtype=torch.float64, device="cuda")
    scstat.scs_eval_stat_noalloc(ctx.h, 0, dev, len(big), out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), stat)
    b = ctx.batch_eval([0, 0], [big[:1300], big[1300:]])
    np.testing.assert_array_equal(np.concatenate(b), stat)
    sample = np.arange(0, len(big), 97)
    ref = oracle.evaluate(d, big[sample], 64, mode=oracle.EQUAL_SNR2)
    assert rel_err(stat[sample], ref) <= TOL32


def test_tiles_give_same_bits_and_autotune(scstat, small):
    """The work tile (bins per chunk) moves where FP32 block sums are handed
    to the FP64 merge, so results agree across tiles to FP32 rounding (and
    with the oracle to the mixed tolerance); the autotuner times every tile
    and keeps the fastest; a given tile always gives the same bits."""
    d, th, ctx = small
    rng = np.random.default_rng(23)
    ps = np.vstack([th, particles(rng, 300)])
    ctx.set_path(scstat.SCS_MIXED)
    ctx.set_segments(0, 16, oracle.EQUAL_SNR2)
    outs = []
    for l2 in (11, 12, 13, 14):
        scstat.scs_set_tile(ctx.h, 0, l2)
        outs.append(ctx.eval(0, ps))
    ref = oracle.evaluate(d, ps, 16, mode=oracle.EQUAL_SNR2)
    for o in outs:
        assert rel_err(o, outs[0]) <= 1e-6
        assert rel_err(o, ref) <= TOL32
    best, ms = scstat.scs_autotune(ctx.h, 0, ps, len(ps))
    assert 11 <= best <= 14 and np.all(ms > 0)
    np.testing.assert_array_equal(ctx.eval(0, ps), outs[best - 11])
    with pytest.raises(scstat.ScsError):
        scstat.scs_set_tile(ctx.h, 0, 10)
    scstat.scs_set_tile(ctx.h, 0, 12)


@pytest.mark.parametrize("path", ["fp64", "mixed"])
@pytest.mark.parametrize("N", [1, 16])
def test_loglike_parity(scstat, small, path, N):
    """Semi-coherent log-likelihood (Sec. II.B) against the oracle; zero at the
    noise-free truth with the injected amplitude."""
    d, th, ctx = small
    ctx.set_path(scstat.SCS_FP64 if path == "fp64" else scstat.SCS_MIXED)
    ctx.set_segments(0, N, oracle.EQUAL_SNR2)
    amp = np.linspace(0.5, 2.0, len(th)) * 1e-20
    L, O, H = ctx.loglike(0, th, amp)
    rL, rO, rH = oracle.loglike(d, th, N, mode=oracle.EQUAL_SNR2, amp=amp)
    tol = TOL64 if path == "fp64" else TOL32
    ok = np.isfinite(rL)
    assert np.array_equal(np.isfinite(L), ok)
    assert rel_err(O[ok], rO[ok]) <= tol * 10 and rel_err(H[ok], rH[ok]) <= tol
    scale = 0.5 * oracle.inner_dd(d) + np.abs(amp * rO) + amp * amp * rH
    assert np.max(np.abs(L[ok] - rL[ok]) / scale[ok]) <= tol


def test_loglike_zero_at_noise_free_truth(scstat):
    d = synth.make_stream(dict(T_obs=3e6, f_min=0.0175, f_max=0.0200, seed=8), noise_free=True)
    th = synth.injection_params(d["rng"], 30.0, 1.5, 0.018)
    hh0 = oracle.inject(th, d["f_first"], d["df"], d["K"], d["T_obs"], d["SA"], d["SE"], 12.0,
                        d["A"], d["E"])
    a = 12.0 / np.sqrt(hh0)
    with scstat.Context(0, scstat.SCS_FP64) as ctx:
        ctx.set_data(0, d)
        for N in (1, 8):
            ctx.set_segments(0, N, scstat.SCS_EQUAL_SNR2)
            L, O, H = ctx.loglike(0, th[None, :], [a])
            assert abs(L[0]) <= 1e-8 * 144.0
            assert H[0] == pytest.approx(hh0, rel=1e-10)


@pytest.mark.parametrize("N", [1500, 5000])
def test_snr2_segments_outnumber_support_bins(scstat, small, N):
    """Equal-SNR^2 segmentations finer than the supports: most segments hold
    zero or one bin (coinciding edges, empty segments), on both paths, with
    per-segment outputs."""
    d, th, ctx = small
    ctx.set_segments(0, N, scstat.SCS_EQUAL_SNR2)
    ref, rx, rh = oracle.evaluate(d, th, N, mode=oracle.EQUAL_SNR2, want_segments=True)
    for path, tol in ((scstat.SCS_FP64, TOL64), (scstat.SCS_MIXED, TOL32)):
        ctx.set_path(path)
        stat, sx, sh = ctx.eval(0, th, N, segments=True)
        assert rel_err(stat, ref) <= tol
        scale = np.maximum(rh.max(axis=1, keepdims=True), 1e-300)
        assert np.max(np.abs(sh - rh) / scale) <= tol
