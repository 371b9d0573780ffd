"""Device-side particle swarm (Sec. III.A), through the C ABI.

The statistic of each iteration is checked against the FP64 oracle; the
bests and the move, which are exact floating-point sequences, are checked
bit for bit against the reference swarm update (oracle/pso.py) fed with the
same pre-iteration state and the statistic the device computed.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import pso as rpso
from paper_2408_13170_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-5}
LO = np.array([10.0, 1.0, 0.0176, 0.0, -math.pi / 2, 0.0, 0.0, 0.005])   # e0 searched
HI = np.array([100.0, 8.0, 0.0190, 2 * math.pi, math.pi / 2, math.pi, math.pi, 0.1])
SIZES = [40, 72]
SEED = 0x1234_5678_9ABC


@pytest.fixture(scope="module")
def scstat():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2408_13170_gb300 import scstat as m
    return m


def _stream(T, fmin, fmax, seed, snr=18.0):
    d = synth.make_stream(dict(T_obs=T, f_min=fmin, f_max=fmax, seed=seed))
    th = synth.injection_params(d["rng"], 30.0, 1.5, 0.018)
    oracle.inject(th, d["f_first"], d["df"], d["K"], d["T_obs"], d["SA"], d["SE"], snr,
                  d["A"], d["E"])
    return d


STREAMS = [(3e6, 0.0175, 0.0200, 41, 8, oracle.EQUAL_SNR2),
           (2e6, 0.0170, 0.0195, 42, 5, oracle.EQUAL_WIDTH)]


@pytest.fixture(scope="module")
def datas():
    return [_stream(T, f0, f1, seed) for T, f0, f1, seed, _, _ in STREAMS]


def _ctx(scstat, datas, path):
    ctx = scstat.Context(0, path)
    for i, d in enumerate(datas):
        ctx.set_data(i, d)
        ctx.set_segments(i, STREAMS[i][4], STREAMS[i][5])
    return ctx


def _hyper_rows(scstat):
    rows = []
    for N in (100, 10):
        om, pp, pg, eps = scstat.table3_hyper(N)
        rows.append(np.concatenate([[om, pp, pg], eps]))
    return np.array(rows)


def _setup(scstat, ctx):
    ctx.pso_create([0, 1], SIZES, LO, HI, SEED)
    for s, row in enumerate(_hyper_rows(scstat)):
        ctx.pso_set_hyper(row[0], row[1], row[2], row[3:], swarm=s)


def _same(a, b):
    for k in ("pos", "vel", "best_pos", "best_val", "swarm_pos", "swarm_val", "stat"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    assert a["iteration"] == b["iteration"]


def test_init_matches_reference(scstat, datas):
    with _ctx(scstat, datas, scstat.SCS_MIXED) as ctx:
        _setup(scstat, ctx)
        st = ctx.pso_get()
    pos, vel = rpso.pso_init(sum(SIZES), LO, HI, SEED)
    np.testing.assert_array_equal(st["pos"], pos)
    np.testing.assert_array_equal(st["vel"], vel)
    np.testing.assert_array_equal(st["best_pos"], pos)
    assert np.all(st["best_val"] == -np.inf) and np.all(st["swarm_val"] == -np.inf)
    assert st["iteration"] == 0


@pytest.mark.parametrize("path", ["mixed", "fp64"])
def test_iterations_match_reference(scstat, datas, path):
    P = sum(SIZES)
    offs = np.concatenate([[0], np.cumsum(SIZES)])
    swarm_of = np.repeat(np.arange(len(SIZES)), SIZES)
    hyper = _hyper_rows(scstat)
    with _ctx(scstat, datas, scstat.SCS_MIXED if path == "mixed" else scstat.SCS_FP64) as ctx:
        _setup(scstat, ctx)
        prev = ctx.pso_get()
        for it in range(3):
            ctx.pso_run(1, use_graph=False)
            cur = ctx.pso_get()
            assert cur["iteration"] == it + 1
            # statistic of the pre-move positions, per swarm against the oracle
            for s in range(len(SIZES)):
                b, e = offs[s], offs[s + 1]
                ref = oracle.evaluate(datas[s], prev["pos"][b:e], STREAMS[s][4],
                                      mode=STREAMS[s][5])
                err = np.max(np.abs(cur["stat"][b:e] - ref) / np.maximum(np.abs(ref), 1.0))
                assert err <= TOL[path]
            bp, bv, sp, sv = rpso.pso_bests(cur["stat"], prev["pos"], prev["best_pos"],
                                            prev["best_val"], prev["swarm_pos"],
                                            prev["swarm_val"], offs)
            np.testing.assert_array_equal(cur["best_pos"], bp)
            np.testing.assert_array_equal(cur["best_val"], bv)
            np.testing.assert_array_equal(cur["swarm_pos"], sp)
            np.testing.assert_array_equal(cur["swarm_val"], sv)
            pos, vel = rpso.pso_step(prev["pos"], prev["vel"], bp, sp, swarm_of, hyper, LO, HI,
                                     SEED, it)
            np.testing.assert_array_equal(cur["pos"], pos)
            np.testing.assert_array_equal(cur["vel"], vel)
            assert np.all(cur["pos"] >= LO) and np.all(cur["pos"] <= HI)
            prev = cur
        assert P == len(cur["stat"])


def test_graph_equals_direct_launches(scstat, datas):
    with _ctx(scstat, datas, scstat.SCS_MIXED) as a, _ctx(scstat, datas, scstat.SCS_MIXED) as b:
        _setup(scstat, a)
        _setup(scstat, b)
        last = None
        for _ in range(3):
            a.pso_run(4, use_graph=True)
            for _ in range(4):
                b.pso_run(1, use_graph=False)
            sa, sb = a.pso_get(), b.pso_get()
            _same(sa, sb)
            if last is not None:    # swarm records never decrease
                assert np.all(sa["swarm_val"] >= last)
            last = sa["swarm_val"]
        assert sa["iteration"] == 12
        # a new segmentation of a swarm's stream re-captures the graph
        for c in (a, b):
            c.set_segments(0, 16, oracle.EQUAL_SNR2)
        a.pso_run(4, use_graph=True)
        b.pso_run(4, use_graph=False)
        _same(a.pso_get(), b.pso_get())
        # as does a different iteration count
        a.pso_run(2, use_graph=True)
        b.pso_run(2, use_graph=False)
        _same(a.pso_get(), b.pso_get())


def test_checkpoint_resume_is_bitwise(scstat, datas):
    with _ctx(scstat, datas, scstat.SCS_MIXED) as a:
        _setup(scstat, a)
        a.pso_run(3)
        blob = a.pso_save()
        a.pso_run(4)
        ref = a.pso_get()
        with _ctx(scstat, datas, scstat.SCS_MIXED) as b:
            b.pso_load(blob)
            assert b.pso_get()["iteration"] == 3
            b.pso_run(4, use_graph=False)
            _same(b.pso_get(), ref)
        a.pso_load(blob)       # back in time, in the same context
        a.pso_run(4)
        _same(a.pso_get(), ref)


def test_corrupt_checkpoint_is_refused(scstat, datas):
    """A checkpoint whose swarm coefficients or convergence rule fail the
    setters' checks is refused, and the context keeps its swarm."""
    with _ctx(scstat, datas, scstat.SCS_MIXED) as ctx:
        _setup(scstat, ctx)
        ctx.pso_run(2, use_graph=False)
        blob = ctx.pso_save()
        before = ctx.pso_get()
        S = int(np.frombuffer(blob, np.int64, 1, 16)[0])
        hyper_at = 40 + 8 * (S + 1) + 8 * ((4 * S + 7) // 8) + 16 * 8
        n = len(blob)   # the last 16 bytes: the rule's delta (double) and window (int64)
        for at, raw in ((hyper_at, np.float64(np.nan)), (hyper_at + 8 * 3, np.float64(-1.0)),
                        (n - 16, np.float64(-0.5)), (n - 8, np.int64(0))):
            bad = bytearray(blob)
            bad[at:at + 8] = raw.tobytes()
            with pytest.raises(scstat.ScsError) as e:
                ctx.pso_load(bytes(bad))
            assert e.value.code == scstat.SCS_EINVAL
            _same(ctx.pso_get(), before)
        ctx.pso_load(blob)   # the checkpoint holds the state, not the last statistic
        after = ctx.pso_get()
        for k in ("pos", "vel", "best_pos", "best_val", "swarm_pos", "swarm_val"):
            np.testing.assert_array_equal(after[k], before[k], err_msg=k)
        assert after["iteration"] == before["iteration"]


def test_swarm_best_ties_take_lowest_index(scstat, datas):
    with _ctx(scstat, datas, scstat.SCS_MIXED) as ctx:
        _setup(scstat, ctx)
        st = ctx.pso_get()
        st["best_val"][[3, 5, 9]] = [1e300, 1e300, 1e299]
        st["best_pos"][5] = st["best_pos"][3][::-1]
        ctx.pso_set(st)
        ctx.pso_run(1, use_graph=False)
        out = ctx.pso_get()
        assert out["swarm_val"][0] == 1e300
        np.testing.assert_array_equal(out["swarm_pos"][0], st["best_pos"][3])


def test_swarm_errors(scstat, datas):
    with _ctx(scstat, datas, scstat.SCS_MIXED) as ctx:
        with pytest.raises(scstat.ScsError) as e:
            ctx.pso_run(1)
        assert e.value.code == scstat.SCS_ENODATA
        with pytest.raises(scstat.ScsError) as e:
            scstat.scs_pso_create(ctx.h, [0, 1], [0, 10, 10], LO, HI, 1)
        assert e.value.code == scstat.SCS_EINVAL
        with pytest.raises(scstat.ScsError) as e:
            scstat.scs_pso_create(ctx.h, [0, 7], [0, 10, 20], LO, HI, 1)
        assert e.value.code == scstat.SCS_ENODATA
        bad = HI.copy()
        bad[2] = LO[2]
        with pytest.raises(scstat.ScsError) as e:
            scstat.scs_pso_create(ctx.h, [0], [0, 10], LO, bad, 1)
        assert e.value.code == scstat.SCS_EINVAL
        _setup(scstat, ctx)
        with pytest.raises(scstat.ScsError) as e:
            ctx.pso_set_hyper(0.5, 0.2, 0.3, [-1.0] + [0.0] * 7)
        assert e.value.code == scstat.SCS_EINVAL
        with pytest.raises(scstat.ScsError) as e:
            ctx.pso_load(b"not a checkpoint at all, not at all......")
        assert e.value.code == scstat.SCS_EINVAL


def test_two_hundred_iterations_in_one_graph(scstat, datas):
    """200 whole iterations captured as one CUDA graph and launched once give
    the state of 200 directly launched iterations."""
    with _ctx(scstat, datas, scstat.SCS_MIXED) as a, _ctx(scstat, datas, scstat.SCS_MIXED) as b:
        _setup(scstat, a)
        _setup(scstat, b)
        a.pso_run(200, use_graph=True)
        b.pso_run(200, use_graph=False)
        sa, sb = a.pso_get(), b.pso_get()
        _same(sa, sb)
        assert sa["iteration"] == 200
        assert np.all(np.isfinite(sa["swarm_val"]))


def test_kmeans_matches_reference(scstat, datas):
    rng = np.random.default_rng(5)
    centers = np.array([[20, 2, 0.0178, 1.0, -0.5, 0.5, 0.3, 0],
                        [80, 6, 0.0186, 5.5, 0.8, 2.5, 2.8, 0],
                        [50, 4, 0.0182, 6.2, 0.0, 1.5, 0.05, 0]], float)
    pos = np.vstack([c + rng.normal(0, 0.02, (300, 8)) * (HI - LO) for c in centers])
    pos = np.vstack([pos, LO + rng.random((60, 8)) * (HI - LO)])   # scatter
    pos[:, 3] %= 2 * math.pi
    pos[:, 6] %= math.pi
    pos[:, 7] = 0.0
    with scstat.Context(0, scstat.SCS_MIXED) as ctx:
        for k in (3, 5):
            lab, cen = scstat.scs_kmeans(ctx.h, pos, LO, HI, k, 8)
            rlab, rcen = rpso.kmeans(pos, LO, HI, k, 8)
            np.testing.assert_array_equal(lab, rlab)
            np.testing.assert_allclose(cen, rcen, rtol=0, atol=1e-12)


def test_convergence_record_follows_the_rule(scstat, datas):
    with _ctx(scstat, datas, scstat.SCS_MIXED) as ctx:
        _setup(scstat, ctx)
        scstat.scs_pso_set_convergence(ctx.h, 1.0, 3)
        hist, flags = [], []
        for _ in range(30):
            ctx.pso_run(1, use_graph=False)
            hist.append(ctx.pso_get()["swarm_val"].copy())
            flags.append(scstat.scs_pso_status(ctx.h)[1])
        ref = rpso.converged_flags(np.array(hist), 1.0, 3)
        np.testing.assert_array_equal(np.array(flags), ref)
        assert ref.any()


def test_regroup_keeps_particles_and_streams(scstat, datas):
    with _ctx(scstat, datas, scstat.SCS_MIXED) as ctx:
        ctx.pso_create([0, 1, 0], [30, 50, 40], LO, HI, 3)
        ctx.pso_run(5, use_graph=True)
        before = ctx.pso_get()
        scstat.scs_pso_regroup(ctx.h, 4, 6)
        sids, offs = scstat.scs_pso_layout(ctx.h)
        after = ctx.pso_get()
        assert offs[-1] == 120 and np.all(np.diff(offs) > 0)
        # stream 0's 70 particles first (up to 4 swarms), then stream 1's 50
        n0 = sum(offs[i + 1] - offs[i] for i in range(len(sids)) if sids[i] == 0)
        assert n0 == 70 and list(sids) == sorted(sids, key=lambda s: s != 0)
        key = lambda a: a[np.lexsort(a.T[::-1])]
        np.testing.assert_array_equal(key(after["pos"][:70]),
                                      key(np.vstack([before["pos"][:30], before["pos"][80:]])))
        np.testing.assert_array_equal(key(after["pos"][70:]), key(before["pos"][30:80]))
        assert np.all(after["best_val"] == -np.inf) and np.all(after["swarm_val"] == -np.inf)
        ctx.pso_run(3, use_graph=True)   # the new layout runs (graph re-captured)
        assert np.all(np.isfinite(ctx.pso_get()["swarm_val"]))


def test_search_ladder_finds_the_injection(scstat):
    """The hierarchical search (ladder 16 -> 4 -> 1, re-clustering between
    rungs) on a loud injection climbs to the coherent statistic of the
    injected parameters."""
    d = synth.make_stream(dict(T_obs=3e6, f_min=0.0175, f_max=0.0200, seed=51))
    th = synth.injection_params(d["rng"], 30.0, 1.5, 0.018)
    oracle.inject(th, d["f_first"], d["df"], d["K"], d["T_obs"], d["SA"], d["SE"], 30.0,
                  d["A"], d["E"])
    lo = th.copy()
    hi = th.copy()
    lo[:3] = th[:3] * np.array([0.9, 0.8, 0.999])
    hi[:3] = th[:3] * np.array([1.1, 1.2, 1.001])
    lo[3:7] = [0, -math.pi / 2, 0, 0]
    hi[3:7] = [2 * math.pi, math.pi / 2, math.pi, math.pi]
    lo[7] = hi[7] = th[7]   # e0 held at the injected value
    with scstat.Context(0, scstat.SCS_MIXED) as ctx:
        ctx.set_data(0, d)
        ctx.set_segments(0, 1, scstat.SCS_EQUAL_SNR2)
        target = ctx.eval(0, th)[0]
        ctx.pso_create([0, 0], [256, 256], lo, hi, 11)
        its = ctx.pso_search([16, 4, 1], n_clusters=2, chunk_iters=10, max_iters=150)
        assert np.all(its >= 10)
        st = ctx.pso_get()
        assert st["swarm_val"].max() >= 0.8 * target
