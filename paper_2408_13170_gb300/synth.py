"""Seeded synthetic inputs shaped like the paper's mock LISA streams.

This module is the one piece shared by the CUDA path's tests/bench and the
CPU oracle: it draws random numbers and builds the data grid, the noise PSD
and particle populations.  It holds none of the statistic's arithmetic (no
waveform, no response, no inner product); injections are added by whoever
owns a template (the oracle in tests, the library's own injection call in the
benchmark).

Workload shapes follow Sec. IV of arXiv:2408.13170 (analytic instrumental
PSD, stationary Gaussian noise generated directly in the frequency domain,
one injected inspiral whose amplitude sets the SNR, uniform priors) and the
benchmark configurations below.
"""
from __future__ import annotations

import math

import numpy as np

CLIGHT = 299792458.0
ARM_M = 2.5e9


def grid(f_min: float, f_max: float, T_obs: float):
    """FFT frequency grid f_k = f_first + k df, df = 1/T_obs, covering the
    Fourier frequencies j/T_obs with ceil(f_min T) <= j <= floor(f_max T)."""
    j0 = math.ceil(f_min * T_obs - 1e-9)
    j1 = math.floor(f_max * T_obs + 1e-9)
    df = 1.0 / T_obs
    return j0 * df, df, j1 - j0 + 1


def psd_AE(f):
    """Analytic instrumental one-sided PSD of TDI A (= E), first generation,
    in the SciRD form (Babak et al. 2021, the model the paper cites in
    Sec. IV).  Fractional-frequency units; only ratios matter here."""
    f = np.asarray(f, dtype=np.float64)
    L = ARM_M / CLIGHT
    x = 2.0 * np.pi * f * L
    s_oms = (15e-12) ** 2 * (1.0 + (2e-3 / f) ** 4) * (2.0 * np.pi * f / CLIGHT) ** 2
    s_acc = ((3e-15) ** 2 * (1.0 + (4e-4 / f) ** 2) * (1.0 + (f / 8e-3) ** 4)
             / (2.0 * np.pi * f * CLIGHT) ** 2)
    return 8.0 * np.sin(x) ** 2 * ((2.0 + np.cos(x)) * s_oms
                                   + 2.0 * (3.0 + 2.0 * np.cos(x) + np.cos(2.0 * x)) * s_acc)


def psd_T(f):
    """Analytic instrumental one-sided PSD of TDI T in the same model and
    units as psd_AE (first generation): the test-mass and optical-path
    terms enter through 1 - cos x, so T is quiet at low frequency."""
    f = np.asarray(f, dtype=np.float64)
    L = ARM_M / CLIGHT
    x = 2.0 * np.pi * f * L
    s_oms = (15e-12) ** 2 * (1.0 + (2e-3 / f) ** 4) * (2.0 * np.pi * f / CLIGHT) ** 2
    s_acc = ((3e-15) ** 2 * (1.0 + (4e-4 / f) ** 2) * (1.0 + (f / 8e-3) ** 4)
             / (2.0 * np.pi * f * CLIGHT) ** 2)
    omc = 1.0 - np.cos(x)
    return 16.0 * np.sin(x) ** 2 * omc * (s_oms + 2.0 * omc * s_acc)


def noise(S, T_obs, rng):
    """Stationary Gaussian FD noise: Re, Im ~ N(0, S T_obs / 4) per bin, so
    that E|n|^2 = S T_obs / 2 (one-sided PSD convention)."""
    S = np.asarray(S, dtype=np.float64)
    sig = np.sqrt(S * T_obs / 4.0)
    return rng.normal(size=S.shape) * sig + 1j * (rng.normal(size=S.shape) * sig)


PRIOR_BOX = {
    # Mc [Msun], q, f0 [Hz], lambda, beta, iota, psi, e0
    "lo": np.array([10.0, 1.0, 0.012, 0.0, -np.pi / 2, 0.0, 0.0, 0.005]),
    "hi": np.array([100.0, 8.0, 0.03, 2 * np.pi, np.pi / 2, np.pi, np.pi, 0.1]),
}


def draw_particles(P: int, rng, lo=None, hi=None):
    """P particles uniform in the prior box (uniform-in-parameter priors,
    Table I, e0 in [0.005, 0.1]); a box with lo[7] = hi[7] = 0 gives
    circular particles."""
    lo = PRIOR_BOX["lo"] if lo is None else np.asarray(lo, dtype=np.float64)
    hi = PRIOR_BOX["hi"] if hi is None else np.asarray(hi, dtype=np.float64)
    u = rng.random((P, 8))
    return lo + u * (hi - lo)


def injection_params(rng, Mc, q, f0, e0=0.01):
    """Injected source: intrinsic parameters fixed (e0 = 0.01 as Table I's
    GW150914-like source), sky / inclination / polarisation uniform (the
    phase is maximised away)."""
    return np.array([Mc, q, f0, rng.uniform(0, 2 * np.pi),
                     rng.uniform(-np.pi / 2, np.pi / 2), rng.uniform(0, np.pi),
                     rng.uniform(0, np.pi), e0])


# Benchmark / test configurations (sizes, segment counts, seeds).
CONFIGS = {
    "C1": dict(T_obs=3.0e6, f_min=0.015, f_max=0.030, P=256, N=8,
               mode="equal_width", inj=(30.0, 1.5, 0.018), snr=20.0, seed=0),
    "C2": dict(T_obs=3.15e7, f_min=0.01, f_max=0.05, P=4096, N=2048,
               mode="equal_snr2", inj=(30.0, 1.5, 0.018), snr=17.0, seed=0),
    "C3": dict(T_obs=1.26e8, f_min=0.01, f_max=0.05, P=16384,
               N=(16384, 4096, 1024, 256, 64, 16, 1), mode="equal_snr2",
               inj=(30.0, 1.5, 0.018), snr=25.0, seed=0),
    # the false-alarm campaign: 128 four-year streams (noise seeds 1-64;
    # seeds 65-128 carry an injection at SNR ~ U[15, 30]), 65 536 particles
    # per ladder level
    "C5": dict(T_obs=1.26e8, f_min=0.01, f_max=0.05, P=65536,
               N=(16384, 4096, 1024, 256, 64, 16, 1), mode="equal_snr2",
               inj=(30.0, 1.5, 0.018), snr=(15.0, 30.0), seed=0, streams=128),
}


def c5_stream(j: int):
    """Stream j of the false-alarm campaign, in an order that alternates the
    two kinds so that any prefix holds both: (seed, injected, snr).  Even j:
    noise-only seed 1 + j/2; odd j: seed 65 + (j-1)/2 with an injection whose
    SNR is drawn from U[15, 30] by a generator of its own seed."""
    if j % 2 == 0:
        return 1 + j // 2, False, 0.0
    seed = 65 + j // 2
    lo, hi = CONFIGS["C5"]["snr"]
    return seed, True, float(np.random.Generator(np.random.PCG64(5000 + seed)).uniform(lo, hi))


YEAR = 3.15e7          # seconds (the one-year stream's duration)
C4_YEARS = (1.0, 1.5, 2.0, 2.5, 3.0, 3.5, 4.0, 4.0)
C4_LADDER = (100, 50, 10, 1)   # segment ladder of the search (App. B)


def c4_streams(seed: int = 0):
    """The uneven batch: eight independent streams (noise seeds 1-8) of
    1-4 years, each with a band of width >= 0.01 Hz inside 0.01-0.05 Hz, one
    injection at SNR 20, a swarm of 2048-32768 particles (log-uniform) and a
    segment count from the search ladder.  Returns one config dict per
    stream, with its particle prior box under "lo" / "hi"."""
    rng = np.random.Generator(np.random.PCG64(1000 + seed))
    out = []
    for s, years in enumerate(C4_YEARS):
        w = rng.uniform(0.01, 0.04)
        f_lo = rng.uniform(0.01, 0.05 - w)
        P = int(round(math.exp(rng.uniform(math.log(2048), math.log(32768)))))
        lo = PRIOR_BOX["lo"].copy()
        hi = PRIOR_BOX["hi"].copy()
        lo[2], hi[2] = f_lo, f_lo + 0.5 * w
        out.append(dict(T_obs=years * YEAR, f_min=f_lo, f_max=f_lo + w, P=P,
                        N=C4_LADDER[s % len(C4_LADDER)], mode="equal_snr2",
                        inj=(30.0, 1.5, f_lo + 0.2 * w), snr=20.0, seed=s + 1, lo=lo, hi=hi))
    return out


def make_stream(name_or_cfg, seed=None, noise_free=False, channels="AE"):
    """Noise-only data stream of a configuration.

    Returns a dict: f_first, df, K, T_obs, A, E (complex128[K]), SA, SE
    (float64[K]), rng (the generator, positioned after the noise draws, for
    drawing the injection and the particles), cfg; with channels="AET" also
    the third TDI channel T (complex128[K]) and its PSD ST, its noise drawn
    after that of A and E (so A and E equal those of the two-channel stream).
    """
    if channels not in ("AE", "AET"):
        raise ValueError("channels must be 'AE' or 'AET'")
    cfg = CONFIGS[name_or_cfg] if isinstance(name_or_cfg, str) else name_or_cfg
    seed = cfg["seed"] if seed is None else seed
    rng = np.random.Generator(np.random.PCG64(seed))
    f_first, df, K = grid(cfg["f_min"], cfg["f_max"], cfg["T_obs"])
    f = f_first + np.arange(K) * df
    S = psd_AE(f)
    if noise_free:
        A = np.zeros(K, np.complex128)
        E = np.zeros(K, np.complex128)
    else:
        A = noise(S, cfg["T_obs"], rng)
        E = noise(S, cfg["T_obs"], rng)
    out = dict(f_first=f_first, df=df, K=K, T_obs=cfg["T_obs"], A=A, E=E,
               SA=S, SE=S.copy(), rng=rng, cfg=cfg)
    if channels == "AET":
        ST = psd_T(f)
        out["ST"] = ST
        out["T"] = (np.zeros(K, np.complex128) if noise_free
                    else noise(ST, cfg["T_obs"], rng))
    return out
