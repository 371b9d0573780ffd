"""False-alarm probability of search candidates (Sec. V, estimating the FAP).

A candidate's significance is the complementary CDF of the noise background
at its optimised coherent statistic Upsilon*_{N=1}; the background is the set
of maxima of Upsilon_{N=1} that the same hierarchical search finds on
signal-free data streams.  M background searches resolve FAPs down to about
1/M; below that the background is extrapolated two ways, as in the paper: a
power law fitted to the background above Upsilon_1 = 30 (conservative: it
decays slowly) and a Gumbel law fitted to the whole background (optimistic:
the maximum of many chi^2 draws tends to a Gumbel law).

Readings where the paper is silent: both fits are maximum likelihood; the
power law is a Pareto tail, CCDF(x) = f_30 (x / 30)^(-alpha) with f_30 the
fraction of the background at or above 30 (its density falls as
x^-(alpha + 1): the paper quotes the density exponent); the Gumbel law is the
one for maxima, CDF(x) = exp(-exp(-(x - mu) / beta)).

Host-side statistics over a few hundred numbers; the background itself comes
from the device search (`noise_background`).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def _finite(background):
    bg = np.asarray(background, dtype=np.float64).ravel()
    if bg.size == 0:
        raise ValueError("empty background")
    if not np.all(np.isfinite(bg)):
        raise ValueError("background values must be finite")
    return bg


def ccdf(background, x):
    """Empirical complementary CDF: the fraction of background values >= x
    (x scalar or array)."""
    bg = np.sort(_finite(background))
    x = np.asarray(x, dtype=np.float64)
    return (bg.size - np.searchsorted(bg, x, side="left")) / bg.size


def fap_floor(background):
    """The smallest FAP the background resolves: a candidate above every
    background maximum has FAP <~ 1/M."""
    return 1.0 / len(background)


@dataclass
class PowerLawTail:
    """Pareto tail CCDF(x) = frac (x / x_min)^(-alpha) for x >= x_min."""
    x_min: float
    alpha: float       # exponent of the CCDF
    frac: float        # fraction of the background at or above x_min
    n_tail: int

    @property
    def pdf_exponent(self):
        """The density falls as x^-(alpha + 1)."""
        return self.alpha + 1.0

    @classmethod
    def fit(cls, background, x_min=30.0):
        """Maximum likelihood (Hill): alpha = n / sum ln(x_i / x_min) over the n
        background values at or above x_min."""
        bg = _finite(background)
        tail = bg[bg >= x_min]
        n = tail.size
        if n < 2:
            raise ValueError(f"{n} background values at or above {x_min}: too few to fit")
        s = float(np.sum(np.log(tail / x_min)))
        if not s > 0.0:
            raise ValueError("degenerate tail (all values equal x_min)")
        return cls(float(x_min), n / s, n / bg.size, int(n))

    def fap(self, x):
        """Extrapolated FAP at x >= x_min (values below x_min are clipped to
        x_min, where the model equals the empirical fraction)."""
        x = np.maximum(np.asarray(x, dtype=np.float64), self.x_min)
        return self.frac * (x / self.x_min) ** (-self.alpha)


@dataclass
class Gumbel:
    """Gumbel law of maxima: CDF(x) = exp(-exp(-(x - mu) / beta))."""
    mu: float
    beta: float

    @staticmethod
    def _score(beta, x):
        # d log L / d beta = 0 after eliminating mu:
        # beta = mean(x) - sum x e^{-x/beta} / sum e^{-x/beta}
        w = np.exp(-(x - x.min()) / beta)
        return beta - x.mean() + float(np.sum(x * w) / np.sum(w))

    @classmethod
    def fit(cls, background):
        """Maximum likelihood: beta solves the score equation (bracketed root),
        then mu = -beta ln mean(e^{-x/beta})."""
        from scipy.optimize import brentq
        x = _finite(background)
        if x.size < 3:
            raise ValueError("too few background values to fit")
        sd = float(np.std(x))
        if not sd > 0.0:
            raise ValueError("degenerate background (all values equal)")
        b0 = sd * math.sqrt(6.0) / math.pi        # moment estimate
        # the score rises from mean - min < 0 (beta -> 0) to +inf: bracket it
        lo, hi = b0, b0
        for _ in range(200):
            if cls._score(lo, x) <= 0.0:
                break
            lo *= 0.5
        for _ in range(200):
            if cls._score(hi, x) >= 0.0:
                break
            hi *= 2.0
        if not (cls._score(lo, x) <= 0.0 <= cls._score(hi, x)):
            raise ValueError("Gumbel score not bracketed: no maximum-likelihood scale "
                             f"found in [{lo:.3g}, {hi:.3g}]")
        beta = brentq(cls._score, lo, hi, args=(x,), xtol=1e-14 * b0, rtol=1e-14)
        mu = float(x.min() - beta * math.log(np.mean(np.exp(-(x - x.min()) / beta))))
        return cls(mu, float(beta))

    def loglike(self, x):
        z = (np.asarray(x, dtype=np.float64) - self.mu) / self.beta
        return float(np.sum(-math.log(self.beta) - z - np.exp(-z)))

    def fap(self, x):
        """1 - CDF(x), without cancellation in the far tail."""
        z = (np.asarray(x, dtype=np.float64) - self.mu) / self.beta
        return -np.expm1(-np.exp(-z))


def fap_table(background, candidates, x_min=30.0):
    """Per candidate Upsilon*_{N=1}: the empirical FAP (with the 1/M floor
    where no background value reaches it), the power-law FAP and the Gumbel
    FAP.  Returns a list of dicts."""
    pl = PowerLawTail.fit(background, x_min)
    gb = Gumbel.fit(background)
    floor = fap_floor(background)
    rows = []
    for c in np.atleast_1d(np.asarray(candidates, dtype=np.float64)):
        emp = float(ccdf(background, c))
        rows.append({"upsilon": float(c), "empirical": emp, "empirical_bound": emp == 0.0,
                     "floor": floor, "power_law": float(pl.fap(c)),
                     "gumbel": float(gb.fap(c))})
    return rows


def noise_background(ctx, seeds, stream_cfg, prior_lo, prior_hi, swarm_sizes,
                     ladder=(100, 50, 10, 1), n_clusters=0, chunk_iters=10, max_iters=200):
    """The background campaign: for every seed, a signal-free stream of the
    configuration (noise drawn with that seed), the hierarchical search of
    `ladder` (last rung N = 1) with swarms of `swarm_sizes` particles over
    the prior box, and the largest Upsilon_{N=1} any swarm found.
    ctx is a `scstat.Context` (stream slot 0 is used).  Returns the maxima
    (one per seed) and the iterations each search ran per rung."""
    from . import scstat, synth
    if ladder[-1] != 1:
        raise ValueError("the ladder must end at the coherent rung N = 1")
    maxima, iters = [], []
    for seed in seeds:
        d = synth.make_stream(dict(stream_cfg, seed=int(seed)))
        ctx.set_data(0, d)
        ctx.set_segments(0, ladder[0], scstat.SCS_EQUAL_SNR2)
        ctx.pso_create([0] * len(swarm_sizes), list(swarm_sizes), prior_lo, prior_hi,
                       int(seed))
        its = ctx.pso_search(list(ladder), n_clusters=n_clusters, chunk_iters=chunk_iters,
                             max_iters=max_iters)
        maxima.append(float(np.max(ctx.pso_get()["swarm_val"])))
        iters.append(np.asarray(its))
    return np.array(maxima), iters
