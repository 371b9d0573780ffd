"""Pins of the reference swarm update (oracle/pso.py) on the CPU.

The random numbers are pinned to the published Philox4x32-10 known-answer
vectors; the update rule (Sec. III.A, Eqs. PSO_velocity_rule and
PSO_min_velocity) to hand-derived special cases and to the behaviour any
correct PSO has on a concave objective (it climbs to the maximum).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import pso

HERE = os.path.dirname(os.path.abspath(__file__))
TWO_PI = 2 * math.pi
LO = np.array([10.0, 1.0, 0.012, 0.0, -math.pi / 2, 0.0, 0.0, 0.0])
HI = np.array([100.0, 8.0, 0.03, TWO_PI, math.pi / 2, math.pi, math.pi, 0.0])


def _kat():
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.json")) as f:
        return json.load(f)["vectors"]


@pytest.mark.parametrize("vec", _kat())
def test_philox_known_answers(vec):
    ctr = np.array([[int(x, 16) for x in vec["ctr"]]], np.uint32)
    key = np.array([[int(x, 16) for x in vec["key"]]], np.uint32)
    out = pso.philox4x32_10(ctr, key)[0]
    assert [f"{int(x):08x}" for x in out] == vec["out"]


def test_uniform_mapping_of_first_draw():
    # seed 0, particle 0, iteration 0, dimension 0 is the all-zero counter and key
    rp, rg = pso.uniforms(0, np.array([0]), 0, 0)
    assert rp[0] == (0x6627E8D5 + 0.5) / 2 ** 32
    assert rg[0] == (0xE169C58D + 0.5) / 2 ** 32


def test_uniforms_open_interval_and_moments():
    r = np.concatenate([np.concatenate(pso.uniforms(7, np.arange(20000), it, d))
                        for it in range(3) for d in range(7)])
    assert r.min() > 0.0 and r.max() < 1.0
    n = r.size
    assert abs(r.mean() - 0.5) < 5 * math.sqrt(1 / 12 / n)
    assert abs(r.var() - 1 / 12) < 5 * math.sqrt(1 / 180 / n)
    # independent per particle, iteration and dimension: no repeated streams
    a = pso.uniforms(7, np.arange(1000), 0, 0)[0]
    b = pso.uniforms(7, np.arange(1000), 1, 0)[0]
    c = pso.uniforms(7, np.arange(1000), 0, 1)[0]
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.15 and abs(np.corrcoef(a, c)[0, 1]) < 0.15


def _state(P=6, seed=3):
    rng = np.random.default_rng(seed)
    pos = LO + (HI - LO) * rng.uniform(0.3, 0.7, (P, 8))
    pos[:, 7] = 0.0
    vel = (HI - LO) * rng.uniform(-0.01, 0.01, (P, 8))
    vel[:, 7] = 0.0
    return pos, vel


def _hyper(S, omega, pp, pg, eps):
    return np.tile(np.concatenate([[omega, pp, pg], eps]), (S, 1))


def test_pure_inertia():
    pos, vel = _state()
    h = _hyper(1, 0.7, 0.0, 0.0, np.zeros(8))
    p2, v2 = pso.pso_step(pos, vel, pos + 1.0, pos[:1] - 1.0, np.zeros(6, int), h, LO, HI, 1, 0)
    assert np.array_equal(v2[:, :7], 0.7 * vel[:, :7])
    assert np.array_equal(p2[:, :7], pos[:, :7] + 0.7 * vel[:, :7])
    assert np.array_equal(p2[:, 7], pos[:, 7])


def test_minimum_speed_and_sign_of_zero():
    pos, vel = _state()
    eps = np.array([0.1, 0.05, 5e-8, 0.1, 0.1, 0.2, 0.1, 0.1])
    # u = 0 exactly: v = +eps in every searched dimension
    p2, v2 = pso.pso_step(pos, vel, pos, pos[:1], np.zeros(6, int),
                          _hyper(1, 0.0, 0.5, 0.0, eps), LO, HI, 1, 0)
    assert np.array_equal(v2[:, :7], np.tile(eps[:7], (6, 1)))
    # small negative u keeps its sign
    vneg = -np.abs(vel) * 1e-6
    _, v3 = pso.pso_step(pos, vneg, pos, pos[:1], np.zeros(6, int),
                         _hyper(1, 1.0, 0.0, 0.0, eps), LO, HI, 1, 0)
    assert np.array_equal(v3[:, :7], -np.tile(eps[:7], (6, 1)))
    # speeds above eps are untouched
    vbig = np.sign(vel) * (eps * 3 + 1e-3)
    _, v4 = pso.pso_step(pos, vbig, pos, pos[:1], np.zeros(6, int),
                         _hyper(1, 1.0, 0.0, 0.0, eps), LO, HI, 1, 0)
    assert np.array_equal(v4[:, :7], vbig[:, :7])


def test_single_component_by_hand():
    # particle 0, dimension 0, iteration 0, seed 0: r_P, r_G are the first KAT outputs
    rp = (0x6627E8D5 + 0.5) / 2 ** 32
    rg = (0xE169C58D + 0.5) / 2 ** 32
    pos = np.tile((LO + HI) / 2, (1, 1))
    pos[0, 7] = 0.0
    vel = np.zeros((1, 8))
    vel[0, 0] = 1.5
    best = pos.copy()
    best[0, 0] = 60.0
    xi = pos.copy()
    xi[0, 0] = 40.0
    om, pp, pg = 0.5, 0.2, 0.3
    p2, v2 = pso.pso_step(pos, vel, best, xi, np.zeros(1, int),
                          _hyper(1, om, pp, pg, np.zeros(8)), LO, HI, 0, 0)
    u = om * 1.5 + pp * rp * (60.0 - 55.0) + pg * rg * (40.0 - 55.0)
    assert v2[0, 0] == pytest.approx(u, rel=1e-15, abs=0)
    assert p2[0, 0] == pytest.approx(55.0 + u, rel=1e-15, abs=0)


def test_wrap_and_reflect():
    pos = np.tile((LO + HI) / 2, (1, 1))
    pos[0, 3] = TWO_PI - 0.05     # lambda wraps
    pos[0, 6] = 0.02              # psi wraps below 0
    pos[0, 0] = 99.0              # Mc reflects at 100
    pos[0, 4] = -math.pi / 2 + 0.01   # beta reflects at -pi/2
    vel = np.zeros((1, 8))
    vel[0, 3], vel[0, 6], vel[0, 0], vel[0, 4] = 0.2, -0.05, 3.0, -0.03
    p2, v2 = pso.pso_step(pos, vel, pos, pos, np.zeros(1, int),
                          _hyper(1, 1.0, 0.0, 0.0, np.zeros(8)), LO, HI, 0, 0)
    assert p2[0, 3] == pytest.approx(0.15, abs=1e-12) and v2[0, 3] == 0.2
    assert p2[0, 6] == pytest.approx(math.pi - 0.03, abs=1e-12) and v2[0, 6] == -0.05
    assert p2[0, 0] == pytest.approx(98.0, abs=1e-12) and v2[0, 0] == -3.0
    assert p2[0, 4] == pytest.approx(-math.pi / 2 + 0.02, abs=1e-12) and v2[0, 4] == 0.03
    assert np.all(p2[0, :7] >= LO[:7]) and np.all(p2[0, :7] <= HI[:7])


def test_bests_strict_and_lowest_index_on_ties():
    P = 6
    pos = np.arange(P * 8, dtype=float).reshape(P, 8)
    bp = np.zeros((P, 8))
    bv = np.array([5.0, 1.0, 1.0, -np.inf, 2.0, 2.0])
    stat = np.array([5.0, 3.0, 0.5, -np.inf, 7.0, 7.0])
    sp = np.zeros((2, 8))
    sv = np.array([-np.inf, 9.0])
    bp2, bv2, sp2, sv2 = pso.pso_bests(stat, pos, bp, bv, sp, sv, [0, 3, 6])
    assert list(bv2) == [5.0, 3.0, 1.0, -np.inf, 7.0, 7.0]
    assert np.array_equal(bp2[0], bp[0])            # equal is not an improvement
    assert np.array_equal(bp2[1], pos[1]) and np.array_equal(bp2[2], bp[2])
    assert np.array_equal(bp2[3], bp[3])            # -inf never becomes a best
    assert sv2[0] == 5.0 and np.array_equal(sp2[0], bp2[0])
    assert sv2[1] == 9.0 and np.array_equal(sp2[1], sp[1])   # 7 does not beat 9
    # ties inside a swarm: the lowest index
    sv[1] = -np.inf
    _, _, sp3, sv3 = pso.pso_bests(stat, pos, bp, bv, sp, sv, [0, 3, 6])
    assert sv3[1] == 7.0 and np.array_equal(sp3[1], pos[4])


def test_init_inside_box():
    pos, vel = pso.pso_init(5000, LO, HI, 11)
    w = HI - LO
    assert np.all(pos[:, :7] > LO[:7]) and np.all(pos[:, :7] < HI[:7])
    assert np.all(pos[:, 7] == LO[7]) and np.all(vel[:, 7] == 0.0)
    assert np.all(np.abs(vel[:, :7]) <= 0.1 * w[:7])
    assert np.allclose(pos[:, :7].mean(0), (LO + HI)[:7] / 2, atol=0.02 * w[:7].max())



def test_e0_is_searched_when_its_prior_has_width():
    """Table I gives e0 a prior range: with lo[7] < hi[7] dimension 7 is
    drawn, moved and reflected like the others, from its own counters
    (dimension 7), so dimensions 0-6 are bit for bit those of the run with
    e0 held fixed."""
    lo8, hi8 = LO.copy(), HI.copy()
    lo8[7], hi8[7] = 0.005, 0.1
    p7, v7 = pso.pso_init(300, LO, HI, 11)
    p8, v8 = pso.pso_init(300, lo8, hi8, 11)
    np.testing.assert_array_equal(p7[:, :7], p8[:, :7])
    np.testing.assert_array_equal(v7[:, :7], v8[:, :7])
    assert np.all(p8[:, 7] > lo8[7]) and np.all(p8[:, 7] < hi8[7])
    assert np.all(np.abs(v8[:, 7]) <= 0.1 * (hi8[7] - lo8[7])) and np.all(v8[:, 7] != 0.0)
    h = _hyper(1, 0.5, 0.2, 0.3, np.array([0.1, 0.05, 5e-8, 0.1, 0.1, 0.2, 0.1, 0.1]))
    s7, s8 = (p7, v7), (p8, v8)
    for it in range(5):
        s7 = pso.pso_step(s7[0], s7[1], s7[0], s7[0][:1], np.zeros(300, int), h, LO, HI, 11, it)
        s8 = pso.pso_step(s8[0], s8[1], s8[0], s8[0][:1], np.zeros(300, int), h, lo8, hi8, 11, it)
        np.testing.assert_array_equal(s7[0][:, :7], s8[0][:, :7])
        assert np.all(s7[0][:, 7] == LO[7])
        assert np.all(s8[0][:, 7] >= lo8[7]) and np.all(s8[0][:, 7] <= hi8[7])
        assert np.all(np.abs(s8[1][:, 7]) >= 0.1)   # eps_e0 = 0.1 (Table III)

def test_swarm_climbs_a_concave_objective():
    """Any correct PSO update climbs to the maximum of a smooth concave
    function; a sign error in a pull term or in the bests makes it wander."""
    lo, hi = np.zeros(8), np.ones(8)
    hi[7] = 0.0
    target = np.array([0.3, 0.7, 0.55, 0.2, 0.8, 0.4, 0.6, 0.0])
    f = lambda x: -np.sum((x[:, :7] - target[:7]) ** 2, axis=1)
    P, S = 64, 2
    off = [0, 32, 64]
    swarm_of = np.repeat([0, 1], 32)
    pos, vel = pso.pso_init(P, lo, hi, 5)
    bp, bv = pos.copy(), np.full(P, -np.inf)
    sp, sv = np.zeros((S, 8)), np.full(S, -np.inf)
    h = _hyper(S, 0.72, 1.193, 1.193, np.zeros(8))
    for it in range(150):
        bp, bv, sp, sv = pso.pso_bests(f(pos), pos, bp, bv, sp, sv, off)
        pos, vel = pso.pso_step(pos, vel, bp, sp, swarm_of, h, lo, hi, 5, it)
    assert np.all(np.abs(sp[:, :7] - target[:7]) < 1e-4)


def test_kmeans_reference_separates_blobs():
    rng = np.random.default_rng(5)
    centers = np.array([[20, 2, 0.014, 1.0, -0.5, 0.5, 0.3, 0],
                        [80, 6, 0.025, 5.5, 0.8, 2.5, 2.8, 0],
                        [50, 4, 0.020, 3.0, 0.0, 1.5, 1.5, 0]], float)
    pos = np.vstack([c + rng.normal(0, 0.01, (40, 8)) * (HI - LO) for c in centers])
    pos[:, 7] = 0
    lab, cent = pso.kmeans(pos, LO, HI, 3, 5)
    # each blob is one cluster
    for b in range(3):
        assert len(set(lab[40 * b:40 * (b + 1)])) == 1
    assert len(set(lab)) == 3
    # periodic dimension: lambda near 0 and near 2 pi are neighbours
    f = pso.km_features(np.array([[50, 4, 0.02, 0.01, 0, 1, 1, 0],
                                  [50, 4, 0.02, 2 * np.pi - 0.01, 0, 1, 1, 0]]), LO, HI)
    assert np.sum((f[0] - f[1]) ** 2) < 2e-5   # (0.02 / 2 pi)^2, not ~1


def test_convergence_rule_reference():
    h = np.array([[1.0], [2.0], [3.5], [3.6], [3.7], [3.8], [6.0], [6.1], [6.2], [6.3]])
    flags = pso.converged_flags(h, 2.0, 3)[:, 0]
    # improvements by > 2: at 0 (-inf -> 1), 2 (1 -> 3.5), 6 (3.5 -> 6.0)
    assert list(flags) == [False, False, False, False, False, True, False, False, False, True]
