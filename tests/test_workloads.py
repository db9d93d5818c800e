"""The seeded synthetic inputs follow the stated recipe (units of Sec. 2: lambda = 0.8 um,
rho = lambda_r / lambda_C), on the CPU: ranges and laws of every config, the head-on
geometry, the plane wave's phase advance of 2 omega_r dt per step, and determinism."""
import math

import numpy as np
import pytest

from paper_2301_07684_gb300 import workloads as W


def test_units_and_phase_advance():
    assert W.RHO == pytest.approx(3.2972e5, rel=1e-4)
    assert W.DT == pytest.approx(0.01 * 2 * math.pi)
    # head-on with beta ~ 1 the phase advances by 2 omega_r dt per step: 128 of 6400 entries
    assert W.K_STEP == round(2 * W.DT / (2 * math.pi / W.K_TABLE))
    t = W.cos_table(np.float64)
    assert t[0] == 1.0 and t[W.K_TABLE // 2] == -1.0 and t.shape == (W.K_TABLE,)


def test_config1_ranges():
    d = W.config1(n=4096)
    for k, lo, hi in (("gamma_e", 10, 1e4), ("chi_e", 1e-3, 10), ("gamma_g", 1e2, 1e5), ("chi_g", 0.1, 100)):
        v = d[k]
        assert v.min() >= lo and v.max() <= hi
        # log-uniform: the mean of the log sits mid-range
        assert abs(np.log(v).mean() - 0.5 * (math.log(lo) + math.log(hi))) < 0.05 * math.log(hi / lo)
    # E_y is set so that gamma |E_y| / rho = chi for momentum along +x, B = 0
    np.testing.assert_allclose(d["gamma_e"] * d["ey_e"] / W.RHO, d["chi_e"], rtol=1e-12)


def test_config2_recipe():
    n = 1 << 16
    d = W.config2(n=n, seed=0, dtype=np.float64)
    pm = -d["px"]
    g = np.sqrt(1 + pm * pm)
    assert abs(g.mean() - 2000) < 3 and abs(g.std() / 2000 - 0.05) < 0.002
    assert (d["py"] == 0).all() and (d["pz"] == 0).all() and (pm > 0).all()        # head-on, along -x
    assert (d["flags"] == W.ALIVE).all() and (d["tau"] < 0).all()                  # electrons, tau drawn later
    assert d["k0"].min() >= 0 and d["k0"].max() < W.K_TABLE and d["amp0"] == 100.0
    # peak chi of the head-on electron: 2 gamma a0 / rho ~ 1.2 at gamma = 2000
    assert 2 * 2000 * 100 / W.RHO == pytest.approx(1.213, rel=1e-3)
    e = W.config2(n=n, seed=0, dtype=np.float64)
    assert np.array_equal(d["px"], e["px"]) and np.array_equal(d["k0"], e["k0"])          # seeded
    assert not np.array_equal(d["px"], W.config2(n=n, seed=1, dtype=np.float64)["px"])


def test_config3_amplitude_gives_the_peak_chi():
    n = 1 << 14
    d = W.config3(n=n, seed=0, dtype=np.float64)
    gam = -d["px"]
    assert (((d["flags"] >> W.SPECIES_SHIFT) & 3) == W.SP_PHOTON).all()
    # chi of a head-on photon at the wave's crest: 2 gamma a / rho
    np.testing.assert_allclose(2 * gam * d["amp"] / W.RHO, d["chi_peak"], rtol=1e-12)
    assert d["chi_peak"].min() >= 0.1 and d["chi_peak"].max() <= 100


def test_config4_beams():
    d = W.config4(seed=0, scale=0.01)
    assert len(d["counts"]) == 64 and d["px"].size == d["counts"].sum()
    assert set(np.unique(d["species"])) <= {0, 1, 2}
    assert d["a0"].min() >= 10 and d["a0"].max() <= 300
    assert d["gamma0"].min() >= 200 and d["gamma0"].max() <= 1e4
    beam = np.repeat(np.arange(64), d["counts"])
    np.testing.assert_array_equal((d["flags"] >> W.SPECIES_SHIFT) & 3, d["species"][beam])


def test_plane_wave_fields():
    t = W.cos_table(np.float64)
    k0 = np.array([0, 100, 6399], dtype=np.uint32)
    (ex, ey, ez), (bx, by, bz) = W.plane_wave_fields(k0, 2.0, t, step=3)
    idx = (k0.astype(np.int64) + 3 * W.K_STEP) % W.K_TABLE
    np.testing.assert_array_equal(ey, 2.0 * t[idx])
    np.testing.assert_array_equal(bz, ey)                          # E_y = B_z (a plane wave along +x)
    assert not ex.any() and not ez.any() and not bx.any() and not by.any()


def test_sample_ids_are_distinct_and_seeded():
    a = W.sample_ids(1000, 100, seed=3)
    assert len(np.unique(a)) == 100 and a.min() >= 0 and a.max() < 1000
    assert np.array_equal(a, W.sample_ids(1000, 100, seed=3))
    assert len(W.sample_ids(10, 100)) == 10
