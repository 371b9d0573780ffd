"""The false-alarm-probability estimates (Sec. V: empirical CCDF of the
noise background, power-law and Gumbel extrapolations), pinned to closed
forms: exact quantile samples of a Pareto and a Gumbel law, the maximum of
M chi^2_2 draws (whose law tends to a Gumbel law of scale 2 at 2 ln M, the
paper's motivation for the Gumbel fit), and the campaign's orchestration on
a stand-in context."""
import math

import numpy as np
import pytest

from paper_2408_13170_gb300 import fap


def test_ccdf_and_floor():
    bg = [10.0, 20.0, 20.0, 35.0, 50.0]
    np.testing.assert_allclose(fap.ccdf(bg, [5.0, 10.0, 15.0, 20.0, 50.0, 51.0]),
                               [1.0, 1.0, 0.8, 0.8, 0.2, 0.0])
    assert fap.fap_floor(bg) == 0.2
    # the paper's bound with 60 background searches
    assert fap.fap_floor(np.zeros(60)) == pytest.approx(1 / 60)
    with pytest.raises(ValueError):
        fap.ccdf([], 1.0)
    for f in (fap.ccdf, lambda b, x: fap.PowerLawTail.fit(b, x), lambda b, x: fap.Gumbel.fit(b)):
        with pytest.raises(ValueError):
            f([40.0, np.nan, 50.0, 60.0], 30.0)


@pytest.mark.parametrize("alpha", [3.48, 1.5])
def test_power_law_recovers_a_pareto_tail(alpha):
    """Below-threshold values plus exact Pareto quantiles above 30
    (x = 30 u^(-1/alpha) at u = (i - 1/2)/n): the fit returns alpha (3.48 is
    the CCDF exponent of the paper's density exponent 4.48), the tail
    fraction, and equals the empirical CCDF at the threshold."""
    n = 4000
    u = (np.arange(n) + 0.5) / n
    tail = 30.0 * u ** (-1.0 / alpha)
    below = np.linspace(2.0, 29.0, 1000)
    bg = np.concatenate([below, tail])
    pl = fap.PowerLawTail.fit(bg, 30.0)
    assert pl.alpha == pytest.approx(alpha, rel=2e-3)
    assert pl.pdf_exponent == pytest.approx(alpha + 1.0, rel=2e-3)
    assert pl.frac == pytest.approx(n / (n + 1000))
    assert pl.fap(30.0) == pytest.approx(fap.ccdf(bg, 30.0))
    # the model's CCDF tracks the sample's inside the tail
    for q in (0.5, 0.1, 0.01):
        x = 30.0 * q ** (-1.0 / alpha)
        assert pl.fap(x) == pytest.approx(fap.ccdf(bg, x), rel=0.02)
    with pytest.raises(ValueError):
        fap.PowerLawTail.fit(below, 30.0)


@pytest.mark.parametrize("mu,beta", [(25.0, 3.0), (-4.0, 0.5)])
def test_gumbel_recovers_its_parameters(mu, beta):
    """Exact Gumbel quantiles x = mu - beta ln(-ln u): the maximum-likelihood
    fit returns (mu, beta), satisfies the score equation, and no nearby
    parameter pair has a higher likelihood."""
    n = 3000
    u = (np.arange(n) + 0.5) / n
    x = mu - beta * np.log(-np.log(u))
    g = fap.Gumbel.fit(x)
    assert g.mu == pytest.approx(mu, abs=2e-3 * beta)
    assert g.beta == pytest.approx(beta, rel=2e-3)
    assert abs(fap.Gumbel._score(g.beta, x)) < 1e-9 * beta
    best = g.loglike(x)
    for dm, db in ((1e-3, 0), (-1e-3, 0), (0, 1e-3), (0, -1e-3)):
        assert fap.Gumbel(g.mu + dm * beta, g.beta * (1 + db)).loglike(x) < best
    # FAP = 1 - CDF, accurate far into the tail
    assert g.fap(g.mu) == pytest.approx(1 - math.exp(-1.0))
    z = 40.0
    assert g.fap(g.mu + z * g.beta) == pytest.approx(math.exp(-z), rel=1e-12)


def test_gumbel_fit_reports_an_unbracketed_score(monkeypatch):
    """If the bracket search cannot enclose a root of the score equation,
    the fit says so (instead of handing the root finder a bracket without a
    sign change)."""
    monkeypatch.setattr(fap.Gumbel, "_score", staticmethod(lambda beta, x: -1.0))
    with pytest.raises(ValueError, match="not bracketed"):
        fap.Gumbel.fit(np.array([1.0, 2.0, 4.0, 8.0]))


def test_gumbel_of_chi2_maxima():
    """Noise-only Upsilon_1 at a fixed template is chi^2_2 (Sec. II.C): the
    maximum of M independent draws has CDF (1 - e^(-x/2))^M -> Gumbel with
    beta = 2 and mu = 2 ln M.  The fit to simulated maxima finds that law,
    and the power law fitted above the 70th percentile is the more
    conservative extrapolation far in the tail (Sec. V)."""
    rng = np.random.default_rng(12)
    M, reps = 4000, 1500
    maxima = np.array([rng.exponential(2.0, M).max() for _ in range(reps)])
    g = fap.Gumbel.fit(maxima)
    assert g.beta == pytest.approx(2.0, rel=0.06)
    assert g.mu == pytest.approx(2.0 * math.log(M), abs=0.15)
    thr = float(np.quantile(maxima, 0.7))
    pl = fap.PowerLawTail.fit(maxima, thr)
    far = thr + 40.0
    assert pl.fap(far) > 100 * g.fap(far)
    # both agree with the empirical CCDF where the background resolves it
    x = float(np.quantile(maxima, 0.9))
    assert g.fap(x) == pytest.approx(0.1, abs=0.02)
    assert pl.fap(x) == pytest.approx(0.1, abs=0.02)


def test_fap_table():
    rng = np.random.default_rng(3)
    bg = np.array([rng.exponential(2.0, 3000).max() for _ in range(300)]) + 10.0
    rows = fap.fap_table(bg, [bg.max() + 30.0, np.median(bg)], x_min=float(np.median(bg)))
    top, mid = rows
    assert top["empirical"] == 0.0 and top["empirical_bound"] and top["floor"] == 1 / 300
    assert 0.0 < top["gumbel"] < top["power_law"] < top["floor"]
    assert mid["empirical"] == pytest.approx(0.5, abs=0.01)
    assert mid["power_law"] == pytest.approx(mid["empirical"], abs=0.01)


class FakeContext:
    """Stand-in for scstat.Context recording what the campaign asks of it;
    its swarm best is a function of the data it was given."""

    def __init__(self):
        self.calls = []
        self.data = None

    def set_data(self, sid, d):
        self.calls.append(("set_data", sid, d["K"]))
        self.data = d

    def set_segments(self, sid, N, mode):
        self.calls.append(("set_segments", sid, N, mode))

    def pso_create(self, sids, sizes, lo, hi, seed):
        self.calls.append(("pso_create", tuple(sids), tuple(sizes), seed))

    def pso_search(self, ladder, n_clusters, chunk_iters, max_iters):
        self.calls.append(("pso_search", tuple(ladder), n_clusters, chunk_iters, max_iters))
        return np.full(len(ladder), chunk_iters)

    def pso_get(self):
        a = self.data["A"]
        return {"swarm_val": np.array([float(np.abs(a[:10]).sum()), -1.0])}


def test_noise_background_campaign():
    """One signal-free stream per seed (different noise), the full ladder
    ending at N = 1, one search each; the background is the best swarm value
    of every search."""
    from paper_2408_13170_gb300 import synth
    cfg = dict(T_obs=1e6, f_min=0.0179, f_max=0.0190)
    lo = synth.PRIOR_BOX["lo"]
    hi = synth.PRIOR_BOX["hi"]
    ctx = FakeContext()
    maxima, iters = fap.noise_background(ctx, [1, 2, 3], cfg, lo, hi, [64, 64],
                                         ladder=(16, 4, 1), chunk_iters=5, max_iters=50)
    assert maxima.shape == (3,) and len(set(maxima)) == 3
    for s, m in zip([1, 2, 3], maxima):
        d = synth.make_stream(dict(cfg, seed=s))
        assert m == pytest.approx(np.abs(d["A"][:10]).sum())
    searches = [c for c in ctx.calls if c[0] == "pso_search"]
    assert searches == [("pso_search", (16, 4, 1), 0, 5, 50)] * 3
    creates = [c for c in ctx.calls if c[0] == "pso_create"]
    assert [c[3] for c in creates] == [1, 2, 3] and creates[0][1:3] == ((0, 0), (64, 64))
    assert all(len(i) == 3 for i in iters)
    with pytest.raises(ValueError):
        fap.noise_background(ctx, [1], cfg, lo, hi, [8], ladder=(16, 4))
