"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: an exact
identity of the statistic, a closed form, a brute-force definition, a
time-domain simulation, a value printed in the paper, or the sampling law of
Sec. II.C.  A plausible mistake in the oracle (a dropped conjugate, a wrong
sign of the phase, a missing factor 4 in the inner product, a segment
off-by-one, a transposed TDI combination) fails at least one of them.
"""
import json
import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2408_13170_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TSUN = 4.925490947641267e-6
YEAR = 3.15581497632e7


def small_stream(T=3e6, fmin=0.0175, fmax=0.0200, seed=11, noise_free=False):
    cfg = dict(T_obs=T, f_min=fmin, f_max=fmax, seed=seed)
    return synth.make_stream(cfg, noise_free=noise_free)


def inner(data, a_A, a_E, b_A, b_E):
    """<a|b> as a complex sum (Sec. II.A, Eq. inner_prod without Re)."""
    w = 4.0 * data["df"] / data["SA"]
    wE = 4.0 * data["df"] / data["SE"]
    return np.sum(w * a_A * np.conj(b_A)) + np.sum(wE * a_E * np.conj(b_E))


THETA_STAR = np.array([30.0, 1.5, 0.018, 1.1, 0.4, 1.2, 0.7, 0.0])


# ---------------------------------------------------------------- identities
@pytest.mark.parametrize("mode", [oracle.EQUAL_WIDTH, oracle.EQUAL_SNR2])
@pytest.mark.parametrize("N", [1, 2, 8, 64])
def test_noise_free_identity(mode, N):
    """d = h(theta*): every segment has z_n = [h|h]_n real, so
    Upsilon_N(theta*) = <h|h> for any N and any segmentation (Sec. II.B)."""
    d = small_stream(noise_free=True)
    st, hA, hE = oracle.template(THETA_STAR, d["f_first"], d["df"], d["K"],
                                 d["T_obs"])
    assert st == oracle.OK
    d["A"], d["E"] = hA.copy(), hE.copy()
    hh = inner(d, hA, hE, hA, hE)
    assert abs(hh.imag) < 1e-12 * hh.real
    stat, sx, sh = oracle.evaluate(d, THETA_STAR[None], N, mode=mode,
                                   want_segments=True)
    assert stat[0] == pytest.approx(hh.real, rel=1e-13)
    # segment partition: the [h|h]_n add up to the full-band <h|h>
    assert sh.sum() == pytest.approx(hh.real, rel=1e-13)
    # x_n = [h|h]_n in every segment
    np.testing.assert_allclose(sx[0], sh[0], rtol=1e-12, atol=1e-300)


def _segment_bins(kappa, k_lo, k_hi, N):
    k = np.arange(k_lo, k_hi + 1)
    seg = np.searchsorted(kappa, k, side="right") - 1
    return k, seg


@pytest.mark.parametrize("mode", [oracle.EQUAL_WIDTH, oracle.EQUAL_SNR2])
def test_phase_max_brute_force(mode):
    """x_n = max over phi of [d|h e^{i phi}]_n (Sec. II.B, Eq.
    semi-coherent_O), by a 2^20-point grid over phi, with the segmented inner
    products formed bin by bin from the template and the boundaries."""
    d = small_stream()
    oracle.inject(THETA_STAR, d["f_first"], d["df"], d["K"], d["T_obs"],
                  d["SA"], d["SE"], 15.0, d["A"], d["E"])
    th = THETA_STAR.copy()
    th[0] *= 1.0 + 2e-4           # slightly off the injection
    N = 16
    stat, sx, sh, kap = oracle.evaluate(d, th[None], N, mode=mode,
                                        want_segments=True, want_kappa=True)
    st, lo, hi = oracle.support(th, d["f_first"], d["df"], d["K"], d["T_obs"])
    _, hA, hE = oracle.template(th, d["f_first"], d["df"], d["K"], d["T_obs"])
    k, seg = _segment_bins(kap[0], lo, hi, N)
    w = 4.0 * d["df"] / d["SA"]
    phis = np.linspace(0.0, 2 * np.pi, 1 << 20, endpoint=False)
    ups = 0.0
    for n in range(N):
        kk = k[seg == n]
        if kk.size == 0:
            assert sx[0, n] == 0.0 and sh[0, n] == 0.0
            continue
        c = (np.sum(w[kk] * d["A"][kk] * np.conj(hA[kk]))
             + np.sum(w[kk] * d["E"][kk] * np.conj(hE[kk])))
        # [d|h e^{i phi}]_n = 4 Re sum d conj(h) e^{-i phi} / S
        vals = np.real(c * np.exp(-1j * phis))
        xmax = vals.max()
        assert sx[0, n] == pytest.approx(xmax, rel=2e-11)
        hh = np.sum(w[kk] * (np.abs(hA[kk]) ** 2 + np.abs(hE[kk]) ** 2))
        assert sh[0, n] == pytest.approx(hh, rel=1e-12)
        ups += xmax ** 2 / hh
    assert stat[0] == pytest.approx(ups, rel=1e-10)


def test_coherent_reduction():
    """N = 1: Upsilon_1 = |<d|h>|^2 / <h|h>, the phase-maximised squared
    matched-filter SNR (Sec. II.B, last sentence before Sec. II.C)."""
    d = small_stream()
    oracle.inject(THETA_STAR, d["f_first"], d["df"], d["K"], d["T_obs"],
                  d["SA"], d["SE"], 12.0, d["A"], d["E"])
    rng = np.random.default_rng(5)
    th = synth.draw_particles(6, rng, lo=[20, 1, 0.0176, 0, -1.5, 0, 0, 0],
                              hi=[80, 4, 0.019, 6.2, 1.5, 3.1, 3.1, 0])
    th = np.vstack([THETA_STAR, th])
    for mode in (oracle.EQUAL_WIDTH, oracle.EQUAL_SNR2):
        stat = oracle.evaluate(d, th, 1, mode=mode)
        for i, p in enumerate(th):
            _, hA, hE = oracle.template(p, d["f_first"], d["df"], d["K"],
                                        d["T_obs"])
            dh = inner(d, d["A"], d["E"], hA, hE)
            hh = inner(d, hA, hE, hA, hE).real
            expect = abs(dh) ** 2 / hh if hh > 0 else 0.0
            assert stat[i] == pytest.approx(expect, rel=1e-12)


# --------------------------------------------------------------- invariances
def test_amplitude_and_phase_invariance():
    """Upsilon_N does not change when the template is multiplied by
    c e^{i phi0} (D_L and the orbital phase drop out, Sec. IV)."""
    d = small_stream()
    oracle.inject(THETA_STAR, d["f_first"], d["df"], d["K"], d["T_obs"],
                  d["SA"], d["SE"], 15.0, d["A"], d["E"])
    rng = np.random.default_rng(2)
    th = np.vstack([THETA_STAR, synth.draw_particles(
        5, rng, lo=[20, 1, 0.0176, 0, -1.5, 0, 0, 0],
        hi=[80, 4, 0.019, 6.2, 1.5, 3.1, 3.1, 0])])
    for mode in (oracle.EQUAL_WIDTH, oracle.EQUAL_SNR2):
        base = oracle.evaluate(d, th, 32, mode=mode)
        other = oracle.evaluate(d, th, 32, mode=mode, amp_scale=3.7,
                                phase0=1.234)
        np.testing.assert_allclose(other, base, rtol=1e-12)


def test_polarisation_shift_invariance():
    """psi -> psi + pi/2 flips the sign of both polarisation tensors, i.e.
    multiplies h by -1; psi -> psi + pi leaves h unchanged."""
    d = small_stream()
    oracle.inject(THETA_STAR, d["f_first"], d["df"], d["K"], d["T_obs"],
                  d["SA"], d["SE"], 15.0, d["A"], d["E"])
    th = np.vstack([THETA_STAR] * 3)
    th[1, 6] += np.pi / 2
    th[2, 6] += np.pi
    stat = oracle.evaluate(d, th, 8, mode=oracle.EQUAL_SNR2)
    np.testing.assert_allclose(stat[1:], stat[0], rtol=1e-12)
    _, a0, e0 = oracle.template(th[0], d["f_first"], d["df"], d["K"], d["T_obs"])
    _, a1, e1 = oracle.template(th[1], d["f_first"], d["df"], d["K"], d["T_obs"])
    np.testing.assert_allclose(a1, -a0, rtol=1e-9, atol=1e-12 * np.abs(a0).max())


@pytest.mark.parametrize("mode", [oracle.EQUAL_WIDTH, oracle.EQUAL_SNR2])
def test_refinement_monotone(mode):
    """Nested segmentations (factor 2): each N-segment splits into two
    2N-segments and |z_a + z_b|^2/(h_a + h_b) <= |z_a|^2/h_a + |z_b|^2/h_b
    (Cauchy-Schwarz), so Upsilon_2N >= Upsilon_N."""
    d = small_stream()
    oracle.inject(THETA_STAR, d["f_first"], d["df"], d["K"], d["T_obs"],
                  d["SA"], d["SE"], 15.0, d["A"], d["E"])
    rng = np.random.default_rng(3)
    th = np.vstack([THETA_STAR, synth.draw_particles(
        8, rng, lo=[20, 1, 0.0176, 0, -1.5, 0, 0, 0],
        hi=[80, 4, 0.019, 6.2, 1.5, 3.1, 3.1, 0])])
    prev = None
    for N in (1, 2, 4, 8, 16, 32, 64):
        s, kap = oracle.evaluate(d, th, N, mode=mode, want_kappa=True)
        if prev is not None:
            assert np.all(s >= prev[0] * (1 - 1e-12))
            # exact nesting of boundaries
            np.testing.assert_array_equal(kap[:, ::2], prev[1])
        prev = (s, kap)



def test_snr2_edges_of_short_supports_are_exact_rationals():
    """A support no longer than one anchor stride (1024 bins) has two anchors,
    so the trapezoid cumulative is linear and kappa_n = k_lo + n span / N
    exactly: the edges must be k_lo + ceil(n span / N) in integer arithmetic,
    also where n span / N is an integer (there the FP64 kappa may round to
    either side of it; the 2^-20-bin snap of the definition takes the
    integer)."""
    d = small_stream()
    rng = np.random.default_rng(17)
    th = synth.draw_particles(400, rng, lo=[10, 1, 0.0176, 0, -1.5, 0, 0, 0],
                              hi=[100, 8, 0.0195, 6.28, 1.5, 3.14, 3.14, 0.1])
    short = []
    for p in th:
        st, lo, hi = oracle.support(p, d["f_first"], d["df"], d["K"], d["T_obs"])
        if st == oracle.OK and 100 < hi - lo <= 1024:
            short.append((p, lo, hi))
    assert len(short) >= 5
    hits = 0
    for N in (4, 10, 12, 100):   # N = 12 meets an FP64 kappa just above its integer
        ps = np.array([p for p, _, _ in short])
        _, kap = oracle.evaluate(d, ps, N, mode=oracle.EQUAL_SNR2, want_kappa=True)
        for (p, lo, hi), k in zip(short, kap):
            span = hi - lo
            want = [lo + (-(-n * span // N)) for n in range(N)] + [hi + 1]
            np.testing.assert_array_equal(np.ceil(k).astype(np.int64), want)
            hits += sum(1 for n in range(1, N) if n * span % N == 0)
    assert hits >= 10   # the integer cases occur

# ----------------------------------------------------------------- waveform
def test_newtonian_time_closed_form():
    """Newtonian chirp: t_c - t(f) = (5/256) (G Mc/c^3)^{-5/3} (pi f)^{-8/3}."""
    for Mc, q, f0 in [(30.0, 1.5, 0.018), (10.0, 1.0, 0.012), (95.0, 3.0, 0.0175)]:
        th = np.array([Mc, q, f0, 0, 0, 0, 0, 0])
        st, eta, M, tc = oracle.derive(th, oracle.NEWTONIAN)
        assert st == oracle.OK
        assert eta == pytest.approx(q / (1 + q) ** 2, rel=1e-15)
        assert M == pytest.approx(Mc * eta ** -0.6 * TSUN, rel=1e-14)
        for f in (f0, 1.3 * f0, 2.0 * f0):
            t = oracle.time_of_freq(th, f, oracle.NEWTONIAN)
            tau = 5.0 / 256.0 * (Mc * TSUN) ** (-5.0 / 3.0) * (np.pi * f) ** (-8.0 / 3.0)
            assert tc - t == pytest.approx(tau, rel=1e-12)


@pytest.mark.parametrize("theta", [
    (10.0, 1.0, 0.0101, 0.3, -0.2, 1.0, 0.4, 0.0),   # the largest phase on the grid
    (30.0, 1.5, 0.018, 1.1, 0.4, 1.2, 0.7, 0.0),
    (70.0, 6.0, 0.013, 4.0, 1.0, 2.5, 2.9, 0.0),
    (30.0, 1.5, 0.018, 1.1, 0.4, 1.2, 0.7, 0.1),     # eccentric
    (10.0, 1.0, 0.0101, 0.3, -0.2, 1.0, 0.4, 0.3),   # the largest eccentric term
])
def test_tf2_time_is_phase_derivative(theta):
    """t(f) is defined as Psi'(f)/(2 pi) (Sec. IV reading of the SPA): over
    one grid bin the phase in turns must advance by the integral of t, which
    the midpoint rule gives as t(f_k + df/2) df up to t'' df^3/24 (< 1e-11
    turns here).  The phase (pn_phase_turns, weights 1) and the time
    (pn_time_offset, weights k - 5) come from separate series, so a wrong
    weight, sign or power on any PN term of t(f), or on the eccentric term,
    shows as a mismatch of order 1e-5 turns or more; the tolerance is 1e-9
    turns."""
    th = np.array(theta)
    f_first, df, K = synth.grid(0.01, 0.05, 3.15e7)
    st, lo, hi = oracle.support(th, f_first, df, K, 3.15e7)
    assert st == oracle.OK and hi - lo > 1000
    worst = 0.0
    for k in np.linspace(lo, hi - 1, 7).astype(int):
        a = oracle.phase_turns(th, f_first, df, int(k))
        b = oracle.phase_turns(th, f_first, df, int(k) + 1)
        t_mid = oracle.time_of_freq(th, f_first + (k + 0.5) * df)
        d = (b - a) - t_mid * df
        d -= round(d)
        worst = max(worst, abs(d))
    assert worst < 1e-9


def test_table1_time_to_merger():
    """Table I: the GW150914-like source (Mc = 28.095555, eta = 0.2471,
    f_low = 0.018 Hz) merges 43.28 months after the start.  The PN t(f)
    must land within a few per cent (at v ~ 0.03 the orders beyond 1PN and
    the eccentricity move t_c by < 0.1%); the Newtonian value is lower
    still."""
    g = json.load(open(os.path.join(GOLDEN, "table1_gw150914.json")))
    eta = g["eta"]
    q = ((1 - 2 * eta) + math.sqrt(1 - 4 * eta)) / (2 * eta)
    th = np.array([g["Mc"], q, g["f_low"], 0, 0, 0, 0, 0])
    month = YEAR / 12.0
    _, _, _, tc = oracle.derive(th, oracle.TF2)
    _, _, _, tcN = oracle.derive(th, oracle.NEWTONIAN)
    assert tc / month == pytest.approx(g["t_c_months"], rel=0.03)
    assert tcN / month == pytest.approx(g["t_c_months"], rel=0.03)
    assert tcN < tc   # 1PN terms lengthen the inspiral at this mass ratio


def _spa_from_energy_balance():
    """TaylorF2 derived here from scratch, not from the oracle's coefficients:
    the 3PN binding energy E(v) and the 3.5PN flux F(v) of a non-spinning
    circular binary (Blanchet, Living Rev. Relativ. 17 (2014) 2), the balance
    dE/dt = -F, and the SPA phase Psi = 2 pi f t(f) - 2 phi(f) - pi/4 with
    dphi/dt = v^3/M and 2 pi f = 2 v^3/M.  Returns, per order k = 0..7,
    functions (v, eta) -> the phase term Psi_k/(2 pi) [turns] and the time
    term t_k [units of M], both without the integration constants."""
    sp = pytest.importorskip("sympy")
    v, eta, L = sp.symbols("v eta L")   # L stands for ln v
    R, pi, gE = sp.Rational, sp.pi, sp.EulerGamma
    e = [1, -R(3, 4) - eta / 12, -R(27, 8) + R(19, 8) * eta - eta ** 2 / 24,
         -R(675, 64) + (R(34445, 576) - R(205, 96) * pi ** 2) * eta
         - R(155, 96) * eta ** 2 - R(35, 5184) * eta ** 3]
    fl = [1, 0, -R(1247, 336) - R(35, 12) * eta, 4 * pi,
          -R(44711, 9072) + R(9271, 504) * eta + R(65, 18) * eta ** 2,
          (-R(8191, 672) - R(583, 24) * eta) * pi,
          R(6643739519, 69854400) + R(16, 3) * pi ** 2 - R(1712, 105) * gE
          - R(856, 105) * (sp.log(16) + 2 * L)
          + (-R(134543, 7776) + R(41, 48) * pi ** 2) * eta - R(94403, 3024) * eta ** 2
          - R(775, 324) * eta ** 3,
          (-R(16285, 504) + R(214745, 1728) * eta + R(193385, 3024) * eta ** 2) * pi]
    # -dE/dv = eta v sum_j (j+1) e_j v^{2j};  F = (32/5) eta^2 v^10 sum_k fl_k v^k
    num = [0] * 8
    for j in range(4):
        num[2 * j] = (j + 1) * e[j]
    qs = []   # dt/dv = (5/(32 eta)) v^{-9} sum_k q_k v^k   (M = 1)
    for k in range(8):
        qs.append(sp.expand(num[k] - sum(qs[j] * fl[k - j] for j in range(k))))

    def integ(c, n):   # int c(L) v^n dv, L = ln v, n != -1
        c1 = sp.expand(c).coeff(L, 1)
        c0 = sp.expand(c - c1 * L)
        return c0 * v ** (n + 1) / (n + 1) + c1 * v ** (n + 1) / (n + 1) * (L - R(1, n + 1))

    def integ_log(c):  # n = -1 (only the 2.5PN phase term meets it)
        return sp.expand(c) * L

    pre = R(5, 32) / eta
    out = []
    for k in range(8):
        tk = pre * integ(qs[k], k - 9)
        phik = pre * (integ_log(qs[k]) if k == 5 else integ(qs[k], k - 6))
        psik = sp.expand(2 * v ** 3 * tk - 2 * phik) / (2 * pi)
        lam = [sp.lambdify((v, eta), expr.subs(L, sp.log(v)), "math") for expr in (psik, tk)]
        out.append(lam)
    return out


@pytest.mark.parametrize("theta,fs", [
    ((30.0, 1.5, 0.018, 0, 0, 0, 0, 0.0), (0.018, 0.021, 0.03)),     # LISA band
    ((1.2188, 1.0, 10.0, 0, 0, 0, 0, 0.0), (10.0, 100.0, 1000.0)),   # 1.4 + 1.4 Msun
    ((8.0, 3.0, 30.0, 0, 0, 0, 0, 0.0), (30.0, 120.0, 300.0)),       # v up to ~0.36
])
def test_pn_orders_follow_from_energy_balance(theta, fs):
    """Every PN order of the oracle's phase and time (orders 0 to 3.5PN, each
    returned separately by orc_pn_terms) equals the term the SPA derivation
    from the binding energy and the flux gives (above), to 1e-12 relative.
    The 2.5PN phase term is a constant plus a logarithm; its constant is a
    phase convention (absorbed in phi_c), so that order compares the phase
    difference between two frequencies."""
    terms = _spa_from_energy_balance()
    th = np.array(theta)
    st, eta, M, _ = oracle.derive(th)
    assert st == oracle.OK
    idx = {0: 0, 2: 1, 3: 2, 4: 3, 5: 4, 6: 5, 7: 6}
    ref = {}
    for f in fs:
        v = (math.pi * M * f) ** (1.0 / 3.0)
        st, F, T = oracle.pn_terms(th, f)
        assert st == oracle.OK and F[7] == 0.0 and T[7] == 0.0
        for k, j in idx.items():
            psi_k, t_k = terms[k]
            assert T[j] == pytest.approx(t_k(v, eta) * M, rel=1e-12, abs=1e-300)
            if k != 5:
                assert F[j] == pytest.approx(psi_k(v, eta), rel=1e-12, abs=1e-300)
        ref[f] = (F[4], terms[5][0](v, eta))
    f1, f2 = fs[0], fs[-1]
    assert ref[f2][0] - ref[f1][0] == pytest.approx(ref[f2][1] - ref[f1][1], rel=1e-11)


def test_eccentric_term_follows_peters_mathews():
    """The leading-order eccentric correction against a direct integration of
    the Peters-Mathews orbit-averaged evolution (Peters 1964): da/dt and de/dt
    of the quadrupole inspiral with the full enhancement functions of e, the
    dominant harmonic at f = 2 x orbital frequency = sqrt(M/a^3)/pi.  The
    time from f0 to f with e(f0) = e0, minus the circular time, must equal
    the oracle's eccentric time term T_e(f) - T_e(f0) to O(e0^2) relative
    (1% at e0 = 0.01), and the circular (e0 = 0) integral must equal its
    Newtonian time term to 1e-9.  The eccentric phase term is then fixed by
    t = dF/df (test_tf2_time_is_phase_derivative)."""
    integrate = pytest.importorskip("scipy.integrate")
    for e0 in (0.01, 0.02):
        th = np.array([30.0, 1.5, 0.018, 0, 0, 0, 0, e0])
        st, eta, M, _ = oracle.derive(th)
        assert st == oracle.OK
        f0 = th[2]

        def a_of(f):
            return (M / (math.pi * f) ** 2) ** (1.0 / 3.0)

        def rhs(a, y):
            ecc = y[1]
            e2 = ecc * ecc
            dadt = -64.0 / 5.0 * eta * M ** 3 / a ** 3 * (
                1 + 73.0 / 24.0 * e2 + 37.0 / 96.0 * e2 * e2) / (1 - e2) ** 3.5
            dedt = -304.0 / 15.0 * eta * M ** 3 * ecc / a ** 4 * (
                1 + 121.0 / 304.0 * e2) / (1 - e2) ** 2.5
            return [1.0 / dadt, dedt / dadt]

        for f in (0.021, 0.03, 0.05):
            span = (a_of(f0), a_of(f))
            te = integrate.solve_ivp(rhs, span, [0.0, e0], rtol=1e-12, atol=1e-30,
                                     method="DOP853").y[0, -1]
            tc0 = integrate.solve_ivp(rhs, span, [0.0, 0.0], rtol=1e-12, atol=1e-30,
                                      method="DOP853").y[0, -1]
            _, _, T = oracle.pn_terms(th, f)
            _, _, T0 = oracle.pn_terms(th, f0)
            assert T[0] - T0[0] == pytest.approx(tc0, rel=1e-9)
            assert T[7] - T0[7] == pytest.approx(te - tc0, rel=0.01)
            assert T[7] < T0[7] and te < tc0   # eccentric binaries merge sooner


def test_spa_sign_against_time_domain_chirp():
    """The frequency-domain template e^{-i Psi} with Psi' = 2 pi t(f) is the
    stationary-phase transform (h~(f) = int h(t) e^{-2 pi i f t} dt) of a
    time-domain Newtonian chirp h(t) = f(t)^{2/3} cos(phi(t)) started at
    f0 at t = 0: normalised overlap >= 0.99; the opposite sign convention
    (conjugated template) gives almost none."""
    Mc, f0 = 4000.0, 0.02
    Mcs = Mc * TSUN
    tau0 = 5.0 / 256.0 * Mcs ** (-5 / 3) * (np.pi * f0) ** (-8 / 3)
    fs = 0.25
    n = int(0.8 * tau0 * fs)
    T = n / fs
    t = np.arange(n) / fs
    tau = tau0 - t
    theta_c = tau / (5 * Mcs)
    phi = -2.0 * theta_c ** (5 / 8)
    f = (5 / 256 * Mcs ** (-5 / 3) / tau) ** (3 / 8) / np.pi
    h = f ** (2 / 3) * np.cos(phi)
    H = np.fft.rfft(h) / fs
    th = np.array([Mc, 1.0, f0, 0, 0, 0, 0, 0])
    K = H.size - 1
    st, hA, _ = oracle.template(th, 1.0 / T, 1.0 / T, K, T,
                                waveform=oracle.NEWTONIAN,
                                response=oracle.IDENTITY)
    _, lo, hi = oracle.support(th, 1.0 / T, 1.0 / T, K, T, oracle.NEWTONIAN)
    assert hi - lo > 200
    a, b = H[1:][lo:hi + 1], hA[lo:hi + 1]
    norm = math.sqrt(np.vdot(a, a).real * np.vdot(b, b).real)
    assert abs(np.vdot(b, a)) / norm >= 0.99
    assert abs(np.vdot(np.conj(b), a)) / norm < 0.15


def test_power_law_closed_form():
    """Newtonian + identity response + white PSD: [h|h] over the support is
    the Riemann sum of (4/S) f^{-7/3}; against the integral
    (4/S)(3/4)(f_a^{-4/3} - f_b^{-4/3}) over the bin-centred interval
    (midpoint rule, O(df^2)).  Equal-SNR^2 boundaries sit at
    f_n^{-4/3} = f_lo^{-4/3} - (n/N)(f_lo^{-4/3} - f_hi^{-4/3}) within one
    bin plus the error bound of the anchor rule: linear inverse
    interpolation of the cumulative over an anchor interval of B bins is off
    by at most (B^2/8) max|d ln(h^2)/dk| bins (here h^2 ~ f^{-7/3})."""
    T = 3e6
    f_first, df, K = synth.grid(0.0175, 0.0300, T)
    S = np.full(K, 2.0)
    data = dict(f_first=f_first, df=df, K=K, T_obs=T,
                A=np.zeros(K, np.complex128), E=np.zeros(K, np.complex128),
                SA=S, SE=S)
    th = np.array([100.0, 1.0, 0.018, 0, 0, 0, 0, 0])
    st, lo, hi = oracle.support(th, f_first, df, K, T, oracle.NEWTONIAN)
    assert st == oracle.OK and hi - lo > 5000
    N = 16
    _, _, sh, kap = oracle.evaluate(data, th[None], N, mode=oracle.EQUAL_SNR2,
                                    waveform=oracle.NEWTONIAN,
                                    response=oracle.IDENTITY,
                                    want_segments=True, want_kappa=True)
    fa = f_first + (lo - 0.5) * df
    fb = f_first + (hi + 0.5) * df
    closed = 4.0 / 2.0 * 0.75 * (fa ** (-4 / 3) - fb ** (-4 / 3))
    assert sh.sum() == pytest.approx(closed, rel=1e-6)
    flo, fhi = fa, fb
    B = oracle.SNR2_STRIDE
    tol = 1.0 + 1.05 * B * B / 8.0 * (7.0 / 3.0) * df / (f_first + lo * df)
    for n in range(1, N):
        fn = (flo ** (-4 / 3) - n / N * (flo ** (-4 / 3) - fhi ** (-4 / 3))) ** (-3 / 4)
        kn = (fn - f_first) / df - 0.5
        assert abs(kap[0, n] - kn) <= tol


def test_linear_chirp_equal_time_segments():
    """Appendix A: for a constant-amplitude linear chirp in white noise the
    equal-SNR^2 boundaries split the signal into equal durations, i.e.
    (t linear in f) equal numbers of bins."""
    T = 2e6
    f_first, df, K = synth.grid(0.0100, 0.0120, T)
    S = np.ones(K)
    data = dict(f_first=f_first, df=df, K=K, T_obs=T,
                A=np.zeros(K, np.complex128), E=np.zeros(K, np.complex128),
                SA=S, SE=S)
    fdot = 5e-10
    th = np.array([fdot, 1.0, 0.0101, 0, 0, 0, 0, 0])
    st, lo, hi = oracle.support(th, f_first, df, K, T, oracle.LINEAR_CHIRP)
    assert st == oracle.OK
    assert hi - lo + 1 == pytest.approx(fdot * T / df, abs=2)
    for N in (4, 10, 50):
        _, kap = oracle.evaluate(data, th[None], N, mode=oracle.EQUAL_SNR2,
                                 waveform=oracle.LINEAR_CHIRP,
                                 response=oracle.IDENTITY, want_kappa=True)
        expect = lo + (hi + 1 - lo) * np.arange(N + 1) / N
        assert np.max(np.abs(kap[0] - expect)) <= 1.0
        # equal time: t(f) at the boundaries is evenly spaced
        tb = (f_first + kap[0] * df - th[2]) / fdot
        assert np.max(np.abs(np.diff(tb) - T / N)) <= 2 * df / fdot


# ----------------------------------------------------------------- response
ANGLES = [np.array([1.0, 1.0, 0.01, 2.01, 0.785, 2.498, 1.3, 0.0]),
          np.array([1.0, 1.0, 0.01, 5.5, -1.1, 0.3, 2.9, 0.0])]


@pytest.mark.parametrize("t", [0.0, 1.3e7, 2.9e7])
def test_orbit_rigid_triangle(t):
    """Craft positions: exactly equal arms L, centroid on the 1 AU circle
    at angle Omega t, constellation plane inclined by 60 degrees."""
    _, pos = oracle.response(ANGLES[0], 0.02, t)
    L = 2.5e9 / 299792458.0
    R = 149597870700.0 / 299792458.0
    for i, j in ((0, 1), (1, 2), (2, 0)):
        assert np.linalg.norm(pos[i] - pos[j]) == pytest.approx(L, rel=1e-12)
    a = 2 * np.pi / YEAR * t
    np.testing.assert_allclose(pos.mean(axis=0),
                               [R * np.cos(a), R * np.sin(a), 0.0], atol=1e-9)
    nrm = np.cross(pos[1] - pos[0], pos[2] - pos[0])
    nrm /= np.linalg.norm(nrm)
    assert abs(nrm[2]) == pytest.approx(0.5, abs=1e-12)


@pytest.mark.parametrize("th", ANGLES)
@pytest.mark.parametrize("f", [0.011, 0.037])
def test_link_and_tdi_from_two_pulse_model(th, f):
    """Single-link transfer against the two-pulse definition: for a plane
    wave H(t, x) = P e^{2 pi i f (t - k.x)}, the link s->r reads
    y(t) = n.[H(t - L, p_s) - H(t, p_r)].n / (2 (1 - k.n)); and first
    generation X(t) = y31 + y13(t-L) + y21(t-2L) + y12(t-3L)
    - [y21 + y12(t-L) + y31(t-2L) + y13(t-3L)], Y, Z cyclic,
    A = (Z - X)/sqrt 2, E = (X - 2Y + Z)/sqrt 6, T = (X + Y + Z)/sqrt 3
    (static constellation, delays applied to the plane-wave time
    dependence)."""
    t0 = 7.7e6
    T, pos = oracle.response(th, f, t0)
    lam, bet, inc, psi = th[3], th[4], th[5], th[6]
    k = -np.array([np.cos(bet) * np.cos(lam), np.cos(bet) * np.sin(lam), np.sin(bet)])
    u = np.array([np.sin(lam), -np.cos(lam), 0.0])
    v = np.array([-np.sin(bet) * np.cos(lam), -np.sin(bet) * np.sin(lam), np.cos(bet)])
    ep = np.outer(u, u) - np.outer(v, v)
    ex = np.outer(u, v) + np.outer(v, u)
    Ep = np.cos(2 * psi) * ep + np.sin(2 * psi) * ex
    Ex = -np.sin(2 * psi) * ep + np.cos(2 * psi) * ex
    P = 0.5 * (1 + np.cos(inc) ** 2) * Ep - 1j * np.cos(inc) * Ex
    L = 2.5e9 / 299792458.0

    def H(t, x):
        return P * np.exp(2j * np.pi * f * (t - k @ x))

    def y(s, r, t):
        n = (pos[r] - pos[s]) / np.linalg.norm(pos[r] - pos[s])
        return n @ (H(t - L, pos[s]) - H(t, pos[r])) @ n / (2 * (1 - k @ n))

    tt = 123.0
    carrier = np.exp(2j * np.pi * f * tt)
    links = [(0, 1), (1, 0), (0, 2), (2, 0), (1, 2), (2, 1)]
    for i, (s, r) in enumerate(links):
        assert T[i] == pytest.approx(y(s, r, tt) / carrier, rel=1e-9, abs=1e-12)

    def X_td(a, b, c, t):   # a: vertex; b, c: the two far craft
        return (y(c, a, t) + y(a, c, t - L) + y(b, a, t - 2 * L) + y(a, b, t - 3 * L)
                - y(b, a, t) - y(a, b, t - L) - y(c, a, t - 2 * L) - y(a, c, t - 3 * L))

    X = X_td(0, 1, 2, tt) / carrier
    Y = X_td(1, 2, 0, tt) / carrier
    Z = X_td(2, 0, 1, tt) / carrier
    scale = max(abs(X), abs(Y), abs(Z))
    for got, want in ((T[6], X), (T[7], Y), (T[8], Z),
                      (T[9], (Z - X) / np.sqrt(2)),
                      (T[10], (X - 2 * Y + Z) / np.sqrt(6)),
                      (T[11], (X + Y + Z) / np.sqrt(3))):
        assert abs(got - want) <= 1e-10 * scale


# -------------------------------------------------------------- statistics
def _mc(nreal, signal_snr, N, mode, seed0=100):
    base = small_stream(T=1e6, fmin=0.0179, fmax=0.0190, noise_free=True)
    th = np.array([60.0, 2.0, 0.018, 1.0, 0.3, 1.0, 0.5, 0.0])
    _, hA, hE = oracle.template(th, base["f_first"], base["df"], base["K"],
                                base["T_obs"])
    hh = inner(base, hA, hE, hA, hE).real
    s = signal_snr / math.sqrt(hh)

    def one(i):
        rng = np.random.Generator(np.random.PCG64(seed0 + i))
        d = dict(base)
        d["A"] = synth.noise(base["SA"], base["T_obs"], rng) + s * hA
        d["E"] = synth.noise(base["SE"], base["T_obs"], rng) + s * hE
        return oracle.evaluate(d, th[None], N, mode=mode, nthreads=1)[0]

    with ThreadPoolExecutor(8) as ex:
        return np.array(list(ex.map(one, range(nreal))))


@pytest.mark.parametrize("N", [1, 10])
def test_noise_only_sampling_law(N):
    """Sec. II.C, Eq. CLTdist_noise with mu_k = 2, sigma_k^2 = 2: noise-only
    Upsilon_N has mean 2N and variance 4N (exact for chi^2_2 segments);
    Upsilon_1 ~ chi^2_2 (Kolmogorov-Smirnov)."""
    g = json.load(open(os.path.join(GOLDEN, "clt_moments.json")))
    n = 2000
    u = _mc(n, 0.0, N, oracle.EQUAL_SNR2)
    mean, var = N * g["mu_k"], 2 * N * g["sigma_k_sq"]
    assert abs(u.mean() - mean) < 5 * math.sqrt(var / n)
    # variance of the sample variance for chi^2_{2N}: 2 var^2/(n-1) + kurtosis
    assert abs(u.var(ddof=1) - var) < 5 * var * math.sqrt((2 + 12 / (2 * N)) / n)
    if N == 1:
        from scipy import stats
        assert stats.kstest(u, stats.chi2(2).cdf).pvalue > 1e-4


def test_signal_sampling_law_and_table4():
    """Sec. II.C, Eq. CLTdist_signal at the true parameters: mean
    rho^2 + 2N, variance 4N + 4 rho^2; and the four Upsilon_1 values of
    Table IV at rho = 38 are consistent with chi^2_2(rho^2)."""
    N, rho, n = 10, 20.0, 1500
    u = _mc(n, rho, N, oracle.EQUAL_SNR2, seed0=5000)
    mean, var = rho ** 2 + 2 * N, 4 * N + 4 * rho ** 2
    assert abs(u.mean() - mean) < 5 * math.sqrt(var / n)
    assert abs(u.var(ddof=1) - var) < 5 * var * math.sqrt(2.5 / n)
    g = json.load(open(os.path.join(GOLDEN, "table4_upsilon1_rho38.json")))
    r = g["rho"]
    m1, s1 = r ** 2 + 2, math.sqrt(4 + 4 * r ** 2)
    vals = np.array(g["upsilon_1"])
    assert np.all(np.abs(vals - m1) < 3 * s1)
    assert abs(vals.mean() - m1) < 3 * s1 / 2
    u1 = _mc(400, r, 1, oracle.EQUAL_SNR2, seed0=9000)
    assert abs(u1.mean() - m1) < 5 * s1 / math.sqrt(400)


# ------------------------------------------------------------- conventions
def test_invalid_and_empty_particles():
    d = small_stream()
    bad = np.array([
        [-1.0, 1.5, 0.018, 0, 0, 0, 0, 0],         # Mc <= 0
        [30.0, 0.5, 0.018, 0, 0, 0, 0, 0],         # q < 1
        [30.0, 1.5, -0.01, 0, 0, 0, 0, 0],         # f0 <= 0
        [30.0, 1.5, np.nan, 0, 0, 0, 0, 0],        # not finite
        [30.0, 1.5, 0.018, 0, 0, 0, 0, 0.35],      # e0 beyond 0.3
        [30.0, 1.5, 0.018, 0, 0, 0, 0, -0.05],     # e0 < 0
        [2.0e5, 1.0, 0.018, 0, 0, 0, 0, 0],        # past the last stable orbit
        [30.0, 1.5, 0.025, 0, 0, 0, 0, 0],         # starts above the band
    ])
    s = oracle.evaluate(d, bad, 4)
    assert np.all(np.isneginf(s[:7]))
    assert s[7] == 0.0


def test_support_matches_linear_scan():
    """The bisection for the last in-band bin agrees with a plain scan of
    t(f_k) <= T_obs and pi M f_k <= 6^{-3/2}."""
    d = small_stream(T=2e6, fmin=0.012, fmax=0.03)
    rng = np.random.default_rng(8)
    th = synth.draw_particles(20, rng)
    for p in th:
        st, lo, hi = oracle.support(p, d["f_first"], d["df"], d["K"], d["T_obs"])
        if st != oracle.OK:
            continue
        _, eta, M, _ = oracle.derive(p)
        ks = np.arange(lo, min(d["K"], hi + 3))
        fk = d["f_first"] + ks * d["df"]
        inb = np.array([oracle.time_of_freq(p, f) <= d["T_obs"] for f in fk])
        inb &= np.pi * M * fk <= 6 ** -1.5
        last = ks[inb][-1]
        assert last == hi
        assert d["f_first"] + lo * d["df"] >= p[2]
        assert lo == 0 or d["f_first"] + (lo - 1) * d["df"] < p[2]


def test_phase_precision_floor():
    """The reduced phase carries double-double accuracy: against a 40-digit
    evaluation of the same Psi/(2 pi) (all orders to 3.5PN and the eccentric
    term), the turn fraction agrees to 1e-13 turns although Psi reaches ~1e7
    turns (without double-double, ~1e-9)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    th = np.array([12.0, 1.3, 0.0121, 0, 0, 0, 0, 0.08])
    T = 1.26e8
    f_first, df, K = synth.grid(0.01, 0.05, T)
    mpf = mpmath.mpf
    q = mpf(th[1])
    eta = q / (1 + q) ** 2
    M = mpf(th[0]) * eta ** (mpf(-3) / 5) * mpf(TSUN)
    pi, gE = mpmath.pi, mpmath.euler
    phi = {0: mpf(1), 2: mpf(3715) / 756 + mpf(55) / 9 * eta, 3: -16 * pi,
           4: mpf(15293365) / 508032 + mpf(27145) / 504 * eta + mpf(3085) / 72 * eta ** 2,
           7: pi * (mpf(77096675) / 254016 + mpf(378515) / 1512 * eta
                    - mpf(74045) / 756 * eta ** 2)}
    phi5 = pi * (mpf(38645) / 756 - mpf(65) / 9 * eta)
    phi6c = (mpf(11583231236531) / 4694215680 - mpf(640) / 3 * pi ** 2
             - mpf(6848) / 21 * gE
             + (mpf(-15737765635) / 3048192 + mpf(2255) / 12 * pi ** 2) * eta
             + mpf(76055) / 1728 * eta ** 2 - mpf(127825) / 1296 * eta ** 3)
    phi6l = mpf(-6848) / 21
    e0, f0 = mpf(th[7]), mpf(th[2])
    P = 3 / (256 * pi * eta)

    def Fpn(f):
        v = (pi * M * f) ** (mpf(1) / 3)
        s = sum(c * v ** (k - 5) for k, c in phi.items())
        s += phi5 * (1 + 3 * mpmath.log(v * mpmath.sqrt(6)))
        s += v * (phi6c + phi6l * mpmath.log(4 * v))
        s += -mpf(2355) / 1462 * e0 ** 2 * v ** -5 * (f / f0) ** (mpf(-19) / 9)
        return P * s

    tc = -mpmath.diff(Fpn, f0)
    for k in (150000, 900000, 4000000):
        f = mpf(f_first) + k * mpf(df)
        F = f * tc - mpf(1) / 8 + Fpn(f)
        frac = float(F - mpmath.nint(F))
        got = oracle.phase_turns(th, f_first, df, k)
        assert abs(got - frac) < 1e-13
        assert abs(float(F)) > 1e5


@pytest.mark.parametrize("mode", [oracle.EQUAL_WIDTH, oracle.EQUAL_SNR2])
def test_loglike_zero_at_noise_free_truth_and_quadratic_in_amplitude(mode):
    """log L_N = -<d|d>/2 - <h|h>/2 + O_N (Sec. II.B): for noise-free d = a h(theta)
    every segment has x_n = a [h|h]_n, so log L_N(theta, a) = 0 for every N, and
    log L_N(theta, a') = -(a - a')^2 <h|h> / 2 exactly."""
    d = synth.make_stream(dict(T_obs=3e6, f_min=0.0175, f_max=0.0200, seed=3), noise_free=True)
    th = synth.injection_params(d["rng"], 30.0, 1.5, 0.018)
    hh0 = oracle.inject(th, d["f_first"], d["df"], d["K"], d["T_obs"], d["SA"], d["SE"], 12.0,
                        d["A"], d["E"])
    a = 12.0 / math.sqrt(hh0)
    for N in (1, 7, 64):
        L, O, H = oracle.loglike(d, th[None, :], N, mode=mode, amp=[a])
        assert abs(L[0]) <= 1e-9 * 144.0
        assert H[0] == pytest.approx(hh0, rel=1e-12)
        for a2 in (0.5 * a, 1.7 * a):
            L2, _, _ = oracle.loglike(d, th[None, :], N, mode=mode, amp=[a2])
            assert L2[0] == pytest.approx(-0.5 * (a - a2) ** 2 * hh0, rel=1e-9, abs=1e-9)
