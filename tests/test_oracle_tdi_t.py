"""Pins of the oracle's third TDI channel T (the search uses A, E and T,
Sec. I; the response model of Sec. IV).

T = (X + Y + Z)/sqrt 3 is checked against facts derived independently of the
oracle's code: A, E, T are an orthonormal recombination of X, Y, Z; T's
response vanishes as (f L)^3 relative to A at low frequency; and the
three-channel statistic keeps the exact identities and the sampling law of
Sec. II.B-C that the two-channel one has.
"""
import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2408_13170_gb300 import synth

THETA_STAR = np.array([30.0, 1.5, 0.018, 1.1, 0.4, 1.2, 0.7, 0.0])
ANGLES = [np.array([1.0, 1.0, 0.01, 2.01, 0.785, 2.498, 1.3, 0.0]),
          np.array([1.0, 1.0, 0.01, 5.5, -1.1, 0.3, 2.9, 0.0]),
          np.array([1.0, 1.0, 0.01, 0.3, 1.2, 1.9, 0.1, 0.0])]


def stream(T=3e6, fmin=0.0175, fmax=0.0200, seed=11, noise_free=False):
    cfg = dict(T_obs=T, f_min=fmin, f_max=fmax, seed=seed)
    return synth.make_stream(cfg, noise_free=noise_free, channels="AET")


def inner3(d, a, b):
    """<a|b> over the three channels (Sec. II.A, Eq. inner_prod without Re);
    a, b: (h_A, h_E, h_T)."""
    out = 0.0
    for x, y, S in zip(a, b, (d["SA"], d["SE"], d["ST"])):
        out = out + np.sum(4.0 * d["df"] / S * x * np.conj(y))
    return out


@pytest.mark.parametrize("th", ANGLES)
@pytest.mark.parametrize("f", [0.004, 0.019, 0.047])
@pytest.mark.parametrize("t", [0.0, 1.1e7])
def test_aet_orthonormal(th, f, t):
    """A, E, T are orthonormal combinations of X, Y, Z, so the total
    response power is the same in both bases."""
    R, _ = oracle.response(th, f, t)
    X, Y, Z, A, E, T = R[6:12]
    xyz = abs(X) ** 2 + abs(Y) ** 2 + abs(Z) ** 2
    assert abs(A) ** 2 + abs(E) ** 2 + abs(T) ** 2 == pytest.approx(xyz, rel=1e-13)
    # and T is the symmetric one: it sees no X - Z or X - 2Y + Z part
    assert T == pytest.approx((X + Y + Z) / math.sqrt(3.0), rel=1e-13)


@pytest.mark.parametrize("th", ANGLES)
def test_t_long_wavelength_cubic(th):
    """Long-wavelength limit: X + Y + Z = W (1 - D) sum over the arms of
    (G_sr - G_rs); the two directions of an arm share phase and n.P.n and
    differ only in sinc(a(1 - k.n)) - sinc(a(1 + k.n)) = O(a^2), a = pi f L,
    and 1 - D = O(a), while A = W O(a).  So |T|/|A| falls as f^3: halving
    f divides it by 8."""
    def ratio(f):
        R, _ = oracle.response(th, f, 7.7e6)
        return abs(R[11]) / math.hypot(abs(R[9]), abs(R[10]))
    for f in (1e-4, 5e-5):
        assert ratio(f) / ratio(f / 2) == pytest.approx(8.0, rel=2e-3)
    # in the search band (f L / c ~ 1) T is small but not zero
    assert 1e-3 < ratio(0.02) < 1.0


@pytest.mark.parametrize("mode", [oracle.EQUAL_WIDTH, oracle.EQUAL_SNR2])
@pytest.mark.parametrize("N", [1, 8, 64])
def test_aet_noise_free_identity(mode, N):
    """d = h(theta*) in all three channels: Upsilon_N(theta*) = <h|h> over
    A, E, T for any N, the [h|h]_n partition it and x_n = [h|h]_n."""
    d = stream(noise_free=True)
    st, hA, hE, hT = oracle.template(THETA_STAR, d["f_first"], d["df"], d["K"],
                                     d["T_obs"], want_T=True)
    assert st == oracle.OK
    d["A"], d["E"], d["T"] = hA.copy(), hE.copy(), hT.copy()
    hh = inner3(d, (hA, hE, hT), (hA, hE, hT)).real
    hh_ae = hh - inner3(d, (0 * hA, 0 * hE, hT), (0 * hA, 0 * hE, hT)).real
    assert hh > hh_ae * (1.0 + 1e-6)    # T carries a share of the power
    stat, sx, sh = oracle.evaluate(d, THETA_STAR[None], N, mode=mode,
                                   want_segments=True)
    assert stat[0] == pytest.approx(hh, rel=1e-13)
    assert sh.sum() == pytest.approx(hh, rel=1e-13)
    np.testing.assert_allclose(sx[0], sh[0], rtol=1e-12, atol=1e-300)


def test_aet_reduces_to_ae():
    """A T channel with no data and an enormous PSD carries no weight: the
    statistic (and the equal-SNR^2 boundaries) equal the two-channel ones."""
    d = stream()
    oracle.inject(THETA_STAR, d["f_first"], d["df"], d["K"], d["T_obs"], d["SA"],
                  d["SE"], 14.0, d["A"], d["E"])
    rng = np.random.default_rng(4)
    th = np.vstack([THETA_STAR, synth.draw_particles(
        7, rng, lo=[20, 1, 0.0176, 0, -1.5, 0, 0, 0], hi=[80, 4, 0.019, 6.2, 1.5, 3.1, 3.1, 0])])
    ae = {k: v for k, v in d.items() if k not in ("T", "ST")}
    d["T"] = np.zeros(d["K"], np.complex128)
    d["ST"] = d["SA"] * 1e250
    for mode in (oracle.EQUAL_WIDTH, oracle.EQUAL_SNR2):
        s3, k3 = oracle.evaluate(d, th, 16, mode=mode, want_kappa=True)
        s2, k2 = oracle.evaluate(ae, th, 16, mode=mode, want_kappa=True)
        np.testing.assert_allclose(s3, s2, rtol=1e-14)
        np.testing.assert_array_equal(k3, k2)


def test_aet_coherent_reduction_and_injection():
    """N = 1: Upsilon_1 = |<d|h>|^2/<h|h> with the three-channel inner
    product; the injection scales the template to the requested SNR over
    the three channels."""
    d = stream(noise_free=True)
    hh0 = oracle.inject(THETA_STAR, d["f_first"], d["df"], d["K"], d["T_obs"], d["SA"],
                        d["SE"], 13.0, d["A"], d["E"], T=d["T"], ST=d["ST"])
    _, hA, hE, hT = oracle.template(THETA_STAR, d["f_first"], d["df"], d["K"], d["T_obs"],
                                    want_T=True)
    assert hh0 == pytest.approx(inner3(d, (hA, hE, hT), (hA, hE, hT)).real, rel=1e-12)
    assert oracle.evaluate(d, THETA_STAR[None], 1)[0] == pytest.approx(169.0, rel=1e-12)
    rng = np.random.Generator(np.random.PCG64(8))
    for a, S in (("A", "SA"), ("E", "SE"), ("T", "ST")):
        d[a] = d[a] + synth.noise(d[S], d["T_obs"], rng)
    th = np.vstack([THETA_STAR, synth.draw_particles(
        5, rng, lo=[20, 1, 0.0176, 0, -1.5, 0, 0, 0], hi=[80, 4, 0.019, 6.2, 1.5, 3.1, 3.1, 0])])
    stat = oracle.evaluate(d, th, 1, mode=oracle.EQUAL_SNR2)
    for i, p in enumerate(th):
        _, a, e, t = oracle.template(p, d["f_first"], d["df"], d["K"], d["T_obs"], want_T=True)
        dh = inner3(d, (d["A"], d["E"], d["T"]), (a, e, t))
        hh = inner3(d, (a, e, t), (a, e, t)).real
        assert stat[i] == pytest.approx(abs(dh) ** 2 / hh if hh > 0 else 0.0, rel=1e-12)


def test_aet_noise_only_sampling_law():
    """Sec. II.C at any fixed template: with noise of PSD S_alpha in each
    channel, every segment's |z_n|^2/[h|h]_n is chi^2_2 whatever the
    channels, so noise-only Upsilon_10 has mean 20 and variance 40."""
    base = stream(T=1e6, fmin=0.0179, fmax=0.0190, noise_free=True)
    th = np.array([60.0, 2.0, 0.018, 1.0, 0.3, 1.0, 0.5, 0.0])
    N, n = 10, 1500

    def one(i):
        rng = np.random.Generator(np.random.PCG64(300 + i))
        dd = dict(base)
        for a, S in (("A", "SA"), ("E", "SE"), ("T", "ST")):
            dd[a] = synth.noise(base[S], base["T_obs"], rng)
        return oracle.evaluate(dd, th[None], N, mode=oracle.EQUAL_SNR2, nthreads=1)[0]

    with ThreadPoolExecutor(8) as ex:
        u = np.array(list(ex.map(one, range(n))))
    mean, var = 2.0 * N, 4.0 * N
    assert abs(u.mean() - mean) < 5 * math.sqrt(var / n)
    assert abs(u.var(ddof=1) - var) < 5 * var * math.sqrt((2 + 12 / (2 * N)) / n)


@pytest.mark.parametrize("mode", [oracle.EQUAL_WIDTH, oracle.EQUAL_SNR2])
def test_aet_loglike_zero_at_noise_free_truth(mode):
    """log L_N = -<d|d>/2 - a^2<h|h>/2 + a O_N (Sec. II.B) over A, E, T: zero
    at the noise-free truth with the injected amplitude, -(a - a')^2<h|h>/2
    at another amplitude a' (so <d|d> carries T's term too)."""
    d = stream(noise_free=True)
    hh0 = oracle.inject(THETA_STAR, d["f_first"], d["df"], d["K"], d["T_obs"], d["SA"],
                        d["SE"], 11.0, d["A"], d["E"], T=d["T"], ST=d["ST"])
    a = 11.0 / math.sqrt(hh0)
    assert oracle.inner_dd(d) == pytest.approx(121.0, rel=1e-12)
    for N in (1, 8):
        L, O, H = oracle.loglike(d, THETA_STAR[None], N, mode=mode, amp=[a])
        assert abs(L[0]) <= 1e-10 * 121.0
        L2, _, _ = oracle.loglike(d, THETA_STAR[None], N, mode=mode, amp=[1.3 * a])
        assert L2[0] == pytest.approx(-0.5 * (0.3 * a) ** 2 * hh0, rel=1e-9)
