"""The seeded input recipes: grid sizes of the configurations, the noise
convention, the uneven batch's stream shapes, and the three-channel stream
keeping the two-channel stream's A and E."""
import numpy as np
import pytest

from paper_2408_13170_gb300 import synth


@pytest.mark.parametrize("name,K", [("C1", 45001), ("C2", 1260001), ("C3", 5040001),
                                    ("C5", 5040001)])
def test_config_grids(name, K):
    cfg = synth.CONFIGS[name]
    f_first, df, k = synth.grid(cfg["f_min"], cfg["f_max"], cfg["T_obs"])
    assert k == K
    assert df * cfg["T_obs"] == pytest.approx(1.0, abs=1e-15)
    assert f_first == pytest.approx(cfg["f_min"], abs=df)


LADDER7 = (16384, 4096, 1024, 256, 64, 16, 1)


@pytest.mark.parametrize("name,P,N,mode,snr", [
    ("C1", 256, 8, "equal_width", 20.0),
    ("C2", 4096, 2048, "equal_snr2", 17.0),
    ("C3", 16384, LADDER7, "equal_snr2", 25.0),
    ("C5", 65536, LADDER7, "equal_snr2", (15.0, 30.0))])
def test_config_sizes(name, P, N, mode, snr):
    """Particles (per level), segment counts, segmentation and injection SNR
    of the named workloads; every injection is M_c = 30, q = 1.5, f0 = 0.018 Hz."""
    cfg = synth.CONFIGS[name]
    assert (cfg["P"], cfg["N"], cfg["mode"], cfg["snr"]) == (P, N, mode, snr)
    assert cfg["inj"] == (30.0, 1.5, 0.018)


def test_noise_convention():
    """One-sided PSD: Re and Im ~ N(0, S T/4), so E|n|^2 = S T/2."""
    rng = np.random.Generator(np.random.PCG64(1))
    S = np.full(200000, 3.0)
    n = synth.noise(S, 8.0, rng)
    assert np.mean(np.abs(n) ** 2) == pytest.approx(3.0 * 8.0 / 2.0, rel=0.01)
    assert abs(np.mean(n.real * n.imag)) < 0.02 * 6.0


def test_uneven_batch_shapes():
    streams = synth.c4_streams()
    assert len(streams) == 8
    assert [s["T_obs"] / synth.YEAR for s in streams] == list(synth.C4_YEARS)
    assert sum(s["P"] for s in streams) == 86911
    for i, s in enumerate(streams):
        w = s["f_max"] - s["f_min"]
        assert 0.01 <= w <= 0.04 and 0.01 <= s["f_min"] and s["f_max"] <= 0.05
        assert 2048 <= s["P"] <= 32768
        assert s["N"] == synth.C4_LADDER[i % len(synth.C4_LADDER)]
        assert s["seed"] == i + 1
        assert s["lo"][2] == s["f_min"] and s["hi"][2] == pytest.approx(s["f_min"] + w / 2)


def test_three_channel_stream_extends_the_two_channel_one():
    cfg = dict(T_obs=1e6, f_min=0.0179, f_max=0.0190, seed=4)
    d2 = synth.make_stream(cfg)
    d3 = synth.make_stream(cfg, channels="AET")
    np.testing.assert_array_equal(d3["A"], d2["A"])
    np.testing.assert_array_equal(d3["E"], d2["E"])
    assert d3["T"].shape == d2["A"].shape and np.all(d3["ST"] > 0)
    assert "T" not in d2
    z = synth.make_stream(cfg, channels="AET", noise_free=True)
    assert not np.any(z["T"])
    with pytest.raises(ValueError):
        synth.make_stream(cfg, channels="XYZ")


def test_false_alarm_campaign_order():
    """The campaign's 128 streams: seeds 1-64 noise-only, 65-128 injected at
    SNR in [15, 30], each seed once, the two kinds alternating."""
    st = [synth.c5_stream(j) for j in range(synth.CONFIGS["C5"]["streams"])]
    assert sorted(s for s, _, _ in st) == list(range(1, 129))
    assert all(inj == (s > 64) for s, inj, _ in st)
    assert all(15.0 <= snr <= 30.0 for s, inj, snr in st if inj)
    assert [inj for _, inj, _ in st[:4]] == [False, True, False, True]
