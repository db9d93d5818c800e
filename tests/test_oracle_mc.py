"""Statistical and structural pins of the oracle's Monte Carlo step.

The counting laws of Sec. 2 (Montefiori & Tamburini, arXiv:2301.07684) fix
what the optical-depth and local methods must produce for a constant rate:
Poisson photon counts in the soft-photon limit (Eq. final_sol), survival
exp(-int R) for pair creation (Eq. solution_simp_pre) and a per-step event
probability R dt for the local method.  They are checked here on the oracle,
which never sees a fitted function.
"""
import math

import numpy as np
import pytest

RHO = 0.8e-6 / (2 * math.pi) / 3.8615926796e-13


def _const_fields(n, nsteps, Ey):
    f = np.zeros((n, nsteps, 6))
    f[:, :, 1] = Ey
    return f


def test_soft_photon_counts_are_poisson(oracle):
    n, nsteps = 400, 40
    gamma, chi = 100.0, 1e-3
    pref = oracle.rate_prefactor(RHO)
    R = oracle.photon_rate([gamma], [chi], pref)[0]
    lam = 2.0
    dt = lam / (R * nsteps)
    pm = math.sqrt(gamma ** 2 - 1)
    out = oracle.mc_run(np.tile([pm, 0, 0], (n, 1)), -np.ones(n), np.arange(n, dtype=np.uint64),
                        np.ones(n, np.uint8), np.zeros(n, np.uint8),
                        _const_fields(n, nsteps, chi * RHO / gamma), rho=RHO, dt=dt, seed=99,
                        nsteps=nsteps)
    counts = np.bincount(out["products"]["parent_id"].astype(np.int64), minlength=n)
    assert counts.sum() == out["n_events"].sum()
    m = counts.mean()
    assert abs(m - lam) < 4 * math.sqrt(lam / n)
    assert abs(counts.var() / m - 1) < 0.3
    assert np.all(out["products"]["species"] == oracle.SP_PHOTON)
    # the emitted photons are collinear with the emitter and carry xi < 1
    pp = out["products"]["p"]
    assert np.all(pp[:, 1:] == 0) and np.all(pp[:, 0] > 0)


def test_pair_survival_is_exponential(oracle):
    n, nsteps = 1000, 20
    gg, chi = 1000.0, 1.0
    pref = oracle.rate_prefactor(RHO)
    R = oracle.pair_rate([gg], [chi], pref)[0]
    dt = 1.0 / (R * nsteps)                      # int R dt = 1
    out = oracle.mc_run(np.tile([gg, 0, 0], (n, 1)), -np.ones(n), np.arange(n, dtype=np.uint64),
                        np.ones(n, np.uint8), np.full(n, oracle.SP_PHOTON, np.uint8),
                        _const_fields(n, nsteps, chi * RHO / gg), rho=RHO, dt=dt, seed=5,
                        nsteps=nsteps)
    alive = (out["flags"] & oracle.FL_ALIVE).astype(bool)
    p_surv = alive.mean()
    q = math.exp(-1.0)
    assert abs(p_surv - q) < 4 * math.sqrt(q * (1 - q) / n)
    prods = out["products"]
    assert len(prods) == 2 * (~alive).sum()
    # energy is conserved by each conversion: gamma_e + gamma_p = gamma_gamma (|p| = sqrt(g^2-1))
    ge = np.sqrt(1 + (prods["p"] ** 2).sum(1))
    by_parent = {}
    for pid, g in zip(prods["parent_id"], ge):
        by_parent[int(pid)] = by_parent.get(int(pid), 0.0) + g
    assert all(abs(v / gg - 1) < 1e-12 for v in by_parent.values())
    # mean electron share is 1/2 (Sec. 4.4, symmetry of Eq. pp_dp)
    xe = ge[prods["member"] == 1] / gg
    assert abs(xe.mean() - 0.5) < 4 * xe.std() / math.sqrt(len(xe))


def test_local_method_event_probability(oracle):
    # beyond-LCFA leptons in a constant field: delta = 0, the gate is off and the
    # local test fires with probability R dt per step
    n, nsteps = 400, 40
    gamma, chi = 100.0, 1e-3
    pref = oracle.rate_prefactor(RHO)
    R = oracle.photon_rate([gamma], [chi], pref)[0]
    dt = 0.05 / R
    pm = math.sqrt(gamma ** 2 - 1)
    F0 = [0.0, chi * RHO / gamma, 0.0]
    out = oracle.mc_run(np.tile([pm, 0, 0], (n, 1)), np.zeros(n), np.arange(n, dtype=np.uint64),
                        np.ones(n, np.uint8), np.zeros(n, np.uint8),
                        _const_fields(n, nsteps, F0[1]), rho=RHO, dt=dt, seed=3, nsteps=nsteps,
                        fprev=np.tile(F0, (n, 1)), dfprev=np.zeros((n, 3)),
                        lepton_mode=oracle.MODE_BLCFA_LOCAL)
    k = out["n_events"]
    expect = nsteps * 0.05
    assert abs(k.mean() - expect) < 4 * math.sqrt(expect * 0.95 / n)
    assert len(out["products"]) == k.sum()          # gate off: every local event emits


def test_just_created_skips_emission(oracle):
    # Sec. 5 / App. A: the first update after creation only stores the force
    n, nsteps = 50, 1
    gamma, chi = 100.0, 1.0
    pm = math.sqrt(gamma ** 2 - 1)
    out = oracle.mc_run(np.tile([pm, 0, 0], (n, 1)), np.zeros(n), np.arange(n, dtype=np.uint64),
                        np.full(n, oracle.FL_ALIVE | oracle.FL_JUST_CREATED, np.uint8),
                        np.zeros(n, np.uint8), _const_fields(n, nsteps, chi * RHO / gamma), rho=RHO,
                        dt=1e3, seed=3, nsteps=nsteps, fprev=np.zeros((n, 3)), dfprev=np.zeros((n, 3)),
                        lepton_mode=oracle.MODE_BLCFA_LOCAL)
    assert len(out["products"]) == 0
    assert np.all(out["flags"] == oracle.FL_ALIVE)
    # p along x, E along y, B = 0: F_perp = E; the stored difference is zero
    np.testing.assert_allclose(out["fprev"][:, 1], chi * RHO / gamma, rtol=1e-15)
    assert np.all(out["dfprev"] == 0)


def test_blcfa_delta_of_a_plane_wave(oracle):
    # F_perp(t) = F0 cos(omega t): Fdot^2 + |F . Fddot| -> F0^2 omega^2 as dt -> 0 (Eq. condit)
    rho, F0, omega = RHO, 50.0, 1.0
    g = 2000.0
    pm = math.sqrt(g * g - 1)
    for dt in [1e-3, 1e-4]:
        Fprev, dF, jc = [0.0] * 3, [0.0] * 3, True
        phi0 = 0.7
        res = None
        for k in range(3):
            # head-on plane wave: E_y = B_z = a cos(phi), F_y = a (1 + beta) cos(phi)
            a = F0 / (1 + pm / g)
            c = math.cos(phi0 + omega * k * dt)
            gate, ev, Fprev, dF, jc = oracle.blcfa_update((-pm, 0, 0), (0, a * c, 0), (0, 0, a * c),
                                                           dt, rho, Fprev, dF, jc)
            res = (gate, ev)
        gate, ev = res
        want = (F0 * omega / rho) ** 2
        assert gate == 1
        assert ev.delta == pytest.approx(want, rel=3 * omega * dt)
        assert ev.chi == pytest.approx(g * abs(ev.F[1]) / rho, rel=1e-14)
