"""Reference particle-swarm update (test infrastructure only).

One PSO iteration as the paper defines it (Sec. III.A, Eqs. PSO_velocity_rule
and PSO_min_velocity), in numpy, for checking the device-side swarm:

  u = Omega v + Phi_P r_P (Psi - theta) + Phi_G r_G (Xi - theta)
  v = max(eps, |u|) u / |u|          (sign(0) taken as +1)
  theta <- theta + v

with r_P, r_G uniform on (0, 1), drawn independently per particle, dimension
and iteration.  Readings (where the paper is silent): the random numbers are
Philox4x32-10 (Salmon et al. 2011, "Parallel random numbers: as easy as
1, 2, 3") with key (seed low, seed high) and counter (particle, iteration,
dimension, 0), outputs 0 and 1 mapped to (x + 1/2) 2^-32; positions leaving
the prior box wrap in lambda (dimension 3) and psi (dimension 6) and reflect
(with the velocity component negated) in the other dimensions; dimension 7
(e0) is searched like the others when its prior range has width (Table I
gives it a prior), and otherwise stays at its lower bound and draws no
random numbers.
"""
from __future__ import annotations

import numpy as np

M0, M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
W0, W1 = np.uint32(0x9E3779B9), np.uint32(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)
WRAP_DIMS = (3, 6)
SEARCH_DIMS = 7          # without e0


def search_dims(lo, hi):
    """Searched dimensions: 0-6, and e0 (7) when its prior range has width."""
    return 8 if hi[7] > lo[7] else SEARCH_DIMS


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds on uint32 arrays: ctr (..., 4), key (..., 2)."""
    c = [np.asarray(ctr[..., i], dtype=np.uint32) for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint32)
    k1 = np.asarray(key[..., 1], dtype=np.uint32)
    for r in range(10):
        if r:
            k0 = (k0 + W0).astype(np.uint32)
            k1 = (k1 + W1).astype(np.uint32)
        p0 = M0 * c[0].astype(np.uint64)
        p1 = M1 * c[2].astype(np.uint64)
        hi0, lo0 = (p0 >> np.uint64(32)).astype(np.uint32), (p0 & MASK).astype(np.uint32)
        hi1, lo1 = (p1 >> np.uint64(32)).astype(np.uint32), (p1 & MASK).astype(np.uint32)
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack(c, axis=-1)


def uniforms(seed, particles, iteration, dim):
    """(r_P, r_G) for the given particle indices at one iteration and dimension."""
    n = len(particles)
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = particles
    ctr[:, 1] = iteration
    ctr[:, 2] = dim
    key = np.zeros((n, 2), np.uint32)
    key[:, 0] = seed & 0xFFFFFFFF
    key[:, 1] = (seed >> 32) & 0xFFFFFFFF
    out = philox4x32_10(ctr, key)
    scale = 2.0 ** -32
    return (out[:, 0] + 0.5) * scale, (out[:, 1] + 0.5) * scale


def pso_init(P, lo, hi, seed):
    """Initial positions and velocities (readings: theta uniform in the prior
    box, as the paper's swarms are initialised from the prior; v uniform in
    +-0.1 of the box width).  Uniforms from counter (p, 2^32 - 1, d, 1)."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    pos = np.tile(lo, (P, 1))
    vel = np.zeros((P, 8))
    idx = np.arange(P)
    for d in range(search_dims(lo, hi)):
        ctr = np.zeros((P, 4), np.uint32)
        ctr[:, 0] = idx
        ctr[:, 1] = 0xFFFFFFFF
        ctr[:, 2] = d
        ctr[:, 3] = 1
        key = np.zeros((P, 2), np.uint32)
        key[:, 0] = seed & 0xFFFFFFFF
        key[:, 1] = (seed >> 32) & 0xFFFFFFFF
        out = philox4x32_10(ctr, key)
        u0 = (out[:, 0] + 0.5) * 2.0 ** -32
        u1 = (out[:, 1] + 0.5) * 2.0 ** -32
        w = hi[d] - lo[d]
        pos[:, d] = lo[d] + u0 * w
        vel[:, d] = (u1 - 0.5) * 0.2 * w
    return pos, vel


def pso_bests(stat, pos, best_pos, best_val, swarm_pos, swarm_val, offsets):
    """Personal and swarm bests after an evaluation (strict improvement; the
    lowest particle index wins among equal personal bests of a swarm)."""
    best_pos = best_pos.copy()
    best_val = best_val.copy()
    swarm_pos = swarm_pos.copy()
    swarm_val = swarm_val.copy()
    for p in range(len(stat)):
        if stat[p] > best_val[p]:
            best_val[p] = stat[p]
            best_pos[p] = pos[p]
    for s in range(len(offsets) - 1):
        b, e = offsets[s], offsets[s + 1]
        i = b
        for p in range(b, e):
            if best_val[p] > best_val[i]:
                i = p
        if best_val[i] > swarm_val[s]:
            swarm_val[s] = best_val[i]
            swarm_pos[s] = best_pos[i]
    return best_pos, best_val, swarm_pos, swarm_val


def pso_step(pos, vel, best_pos, swarm_best_pos, swarm_of, hyper, lo, hi, seed, iteration):
    """Velocity and position update of every particle (one iteration).

    pos, vel, best_pos: (P, 8); swarm_best_pos: (S, 8); swarm_of: (P,) swarm
    index; hyper: (S, 11) rows (Omega, Phi_P, Phi_G, eps[8]); lo, hi: (8,).
    Returns new (pos, vel).
    """
    pos = pos.copy()
    vel = vel.copy()
    P = pos.shape[0]
    idx = np.arange(P)
    h = hyper[swarm_of]
    for d in range(search_dims(lo, hi)):
        rp, rg = uniforms(seed, idx, iteration, d)
        th = pos[:, d]
        u = (h[:, 0] * vel[:, d] + h[:, 1] * rp * (best_pos[:, d] - th)
             + h[:, 2] * rg * (swarm_best_pos[swarm_of, d] - th))
        eps = h[:, 3 + d]
        a = np.abs(u)
        v = np.where(a >= eps, u, np.where(u < 0.0, -eps, eps))
        x = th + v
        width = hi[d] - lo[d]
        if d in WRAP_DIMS:
            x = lo[d] + np.mod(x - lo[d], width)
        else:
            below, above = x < lo[d], x > hi[d]
            x = np.where(below, 2.0 * lo[d] - x, np.where(above, 2.0 * hi[d] - x, x))
            v = np.where(below | above, -v, v)
            x = np.clip(x, lo[d], hi[d])
        pos[:, d] = x
        vel[:, d] = v
    return pos, vel


def km_features(pos, lo, hi):
    """k-means features of positions: M_c, q, f0, beta, iota normalised to the
    prior box; lambda and psi as points on circles of circumference one."""
    pos = np.asarray(pos, np.float64).reshape(-1, 8)
    f = np.empty((len(pos), 9))
    for i, d in enumerate((0, 1, 2, 4, 5)):
        f[:, i] = (pos[:, d] - lo[d]) / (hi[d] - lo[d])
    for j, d in enumerate((3, 6)):
        u = (pos[:, d] - lo[d]) / (hi[d] - lo[d])
        f[:, 5 + 2 * j] = np.cos(2 * np.pi * u) / (2 * np.pi)
        f[:, 6 + 2 * j] = np.sin(2 * np.pi * u) / (2 * np.pi)
    return f


def _nearest(f, cent):
    d2 = np.stack([np.sum((f - c) ** 2, axis=1) for c in cent], axis=1)
    return np.argmin(d2, axis=1), np.min(d2, axis=1)


def kmeans(pos, lo, hi, k, iters, seeds=None):
    """Farthest-point seeded Lloyd k-means (labels, centroids): centroids from
    `seeds` (positions) first, then particle 0 if there is none, then the
    particle farthest from the centroids so far (first among equals); each
    Lloyd step assigns to the nearest centroid (first among equals) and moves
    each non-empty cluster's centroid to its members' mean."""
    f = km_features(pos, lo, hi)
    cent = [] if seeds is None else list(km_features(seeds, lo, hi))[:k]
    while len(cent) < k:
        if not cent:
            cent.append(f[0].copy())
        else:
            _, d2 = _nearest(f, cent)
            cent.append(f[int(np.argmax(d2))].copy())
    cent = np.array(cent)
    for _ in range(iters):
        lab, _ = _nearest(f, cent)
        for j in range(k):
            m = lab == j
            if m.any():
                cent[j] = f[m].mean(axis=0)
    lab, _ = _nearest(f, cent)
    return lab, cent


def converged_flags(history, delta, window):
    """The convergence rule on a record of swarm best values (one row per
    evaluation): converged after E evaluations when the best has not grown by
    more than delta since evaluation E - 1 - window."""
    history = np.asarray(history, np.float64)
    E, S = history.shape
    ref = np.full(S, -np.inf)
    ref_it = np.zeros(S, np.int64)
    out = []
    for e in range(E):
        up = history[e] > ref + delta
        ref = np.where(up, history[e], ref)
        ref_it = np.where(up, e, ref_it)
        out.append(np.isfinite(ref) & (e - ref_it >= window))
    return np.array(out)
