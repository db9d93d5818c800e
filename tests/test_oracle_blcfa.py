"""Pins of the oracle's photon spectrum (Eq. pe_dp) and of its beyond-LCFA decision logic
(Sec. 5: the gate below Eq. condit, the threshold of Eq. gammaLCFA, the 0.75 gamma_e rule
and the rejection of Eq. rej_cond).

Eq. pe_dp is the one oracle function the rest of the oracle does not integrate: the
rejection test evaluates it pointwise.  It is pinned by what the mathematics fixes:
  - its integral over the photon energy is the rate of Eq. pe_rate_3, which the oracle
    computes from a different integrand (Eq. wtilde);
  - its first moment is the radiated power, whose small-chi series is the classical
    (Larmor) power (2/3) alpha m^2 c^4 chi^2 / hbar times the textbook quantum factor
    1 - (55 sqrt 3 / 16) chi + 48 chi^2 + O(chi^3);
  - its soft-photon end is the synchrotron law 2 K-leading term ~ gamma_gamma^{-2/3} with
    the constant -Ki_{1/3}(0) = -pi/sqrt 3 of the integral term next to it.
The decision logic is pinned by its stated behaviour: the gate's two inequalities at their
boundaries, the threshold formula's bound (it never exceeds 0.7 gamma_e, so the 0.75 rule
cannot fire), and the law of the accepted photons: flat at S(gamma_LCFA) below the
threshold and the LCFA spectrum above it.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special, stats

RHO = 0.8e-6 / (2 * math.pi) / 3.8615926796e-13
ALPHA = 7.2973525693e-3                       # CODATA 2018 fine-structure constant
ZETA = 2.0 ** -52
A23 = 2 ** (-1 / 3) * special.gamma(2 / 3)    # K_2/3(x) ~ A23 x^{-2/3}, x -> 0 (DLMF 10.30.2)


def _spectrum(oracle):
    L = oracle.lib()
    pref = oracle.rate_prefactor(RHO)
    return (lambda gg, ge, chi: L.orc_spectrum_pe(gg, ge, chi, pref)), pref


def _moment(S, ge, chi, k):
    """int_0^ge gamma_gamma^k S d gamma_gamma with gamma_gamma = ge t^3 (removes the
    gamma_gamma^{-2/3} end point)."""
    f = lambda t: (ge * t ** 3) ** k * S(ge * t ** 3, ge, chi) * 3 * ge * t * t
    return integrate.quad(f, 0.0, 1.0, epsabs=0.0, epsrel=1e-13, limit=400)[0]


# --- Eq. pe_dp ------------------------------------------------------------------
@pytest.mark.parametrize("ge,chi", [(10.0, 1e-3), (2000.0, 0.3), (2000.0, 1.0), (1e4, 10.0), (50.0, 200.0)])
def test_spectrum_integrates_to_the_rate(oracle, ge, chi):
    # Eq. pe_rate: the rate is the integral of Eq. pe_dp over the photon energy; the oracle
    # computes the rate from Eq. wtilde, a different integrand
    S, pref = _spectrum(oracle)
    R = oracle.photon_rate([ge], [chi], pref)[0]
    assert _moment(S, ge, chi, 0) == pytest.approx(R, rel=1e-10)


def test_spectrum_radiated_power_small_chi(oracle):
    # first moment = power in units of m c^2 omega_r; classical limit (2/3) alpha rho chi^2
    # (rho = 1/(omega_r tau_C)), quantum factor g = 1 - (55 sqrt3/16) chi + 48 chi^2 + O(chi^3)
    S, _ = _spectrum(oracle)
    for chi in (1e-4, 1e-3):
        g = _moment(S, 1000.0, chi, 1) / (2 / 3 * ALPHA * RHO * chi ** 2)
        c2 = (g - 1 + 55 * math.sqrt(3) / 16 * chi) / chi ** 2
        assert c2 == pytest.approx(48.0, abs=600 * chi), (chi, g, c2)


def test_spectrum_power_is_independent_of_the_lepton_energy(oracle):
    # at fixed chi the spectrum scales as S(x ge, ge) = f(x)/ge, so the power does not depend on ge
    S, _ = _spectrum(oracle)
    p = [_moment(S, ge, 0.5, 1) for ge in (20.0, 2000.0, 2e5)]
    assert p[1] == pytest.approx(p[0], rel=1e-10) and p[2] == pytest.approx(p[0], rel=1e-10)


def test_spectrum_soft_photon_end(oracle):
    # gamma_gamma -> 0: S = C gamma_gamma^{-2/3} - (pi/sqrt 3) pref/ge^2 + O(gamma_gamma^{1/3}),
    # C = 2 A23 pref/ge^2 (2/(3 chi ge))^{-2/3} -- the leading synchrotron law from
    # 2 K_2/3 and the constant from the integral term -(1 + u) Ki_1/3(0)
    S, pref = _spectrum(oracle)
    for ge, chi in [(1000.0, 1.0), (300.0, 0.05)]:
        C = 2 * A23 * pref / ge ** 2 * (2 / (3 * chi * ge)) ** (-2 / 3)
        const = -math.pi / math.sqrt(3) * pref / ge ** 2
        for x in (1e-9, 1e-10):
            gg = x * ge
            assert S(gg, ge, chi) * gg ** (2 / 3) / C == pytest.approx(1.0, rel=1e-4)
            assert S(gg, ge, chi) - C * gg ** (-2 / 3) == pytest.approx(const, rel=2e-2)


def test_spectrum_against_scipy_restatement(oracle):
    # a cross-check of the variable map and Bessel calls (not a pin of the formula itself):
    # Eq. pe_dp with scipy's K_nu and a quadrature of K_1/3 for the integral term
    S, pref = _spectrum(oracle)
    ki = lambda x: integrate.quad(lambda y: special.kv(1 / 3, y), x, np.inf, epsabs=0, epsrel=1e-12)[0]
    for gg, ge, chi in [(1.0, 1000.0, 1.0), (400.0, 1000.0, 1.0), (990.0, 1000.0, 5.0), (0.02, 50.0, 0.01)]:
        u = gg / (ge - gg)
        x = 2 * u / (3 * chi)
        ref = pref / ge ** 2 / (1 + u) * ((1 + (1 + u) ** 2) * special.kv(2 / 3, x) - (1 + u) * ki(x))
        assert S(gg, ge, chi) == pytest.approx(ref, rel=1e-9)


# --- the gate below Eq. condit ------------------------------------------------------
def _gate(oracle, F, gamma, d, dt, dd=None):
    """One update of a lepton moving along x in E = (0, F, 0), B = 0 (so F_perp = F y-hat),
    whose stored force is F - d and stored difference dd (default d: no second difference)."""
    pm = math.sqrt(gamma * gamma - 1)
    dd = d if dd is None else dd
    gate, ev, _, _, _ = oracle.blcfa_update((pm, 0, 0), (0, F, 0), (0, 0, 0), dt, RHO, [0, F - d, 0],
                                            [0, dd, 0], False)
    return gate, ev


def test_gate_constant_field_is_off(oracle):
    # a locally constant field: no first or second difference, delta = 0, the LCFA holds
    gate, ev = _gate(oracle, 200.0, 1000.0, 0.0, 0.01)
    assert gate == 0 and ev.delta == 0.0


def test_gate_boundary_delta(oracle):
    # gamma^2 delta / zeta^2 > chi^2 F^2 with chi = tau_C gamma F: delta > zeta^2 tau_C^2 F^4.
    # With no second difference delta = tau_C^2 d^2/dt^2, so the boundary is d = zeta F^2 dt
    F, g, dt = 2.0 ** 20, 1000.0, 1.0
    d0 = ZETA * F * F * dt
    for lam, want in [(4.0, 1), (0.25, 0)]:
        gate, ev = _gate(oracle, F, g, lam * d0, dt)
        assert ev.delta == pytest.approx((lam * d0 / dt / RHO) ** 2, rel=1e-6)
        assert gate == want, lam


def test_gate_boundary_chi(oracle):
    # chi > zeta: a field so weak that chi <= zeta keeps the gate off however fast it varies
    g = 1000.0
    for chi, want in [(1e-15, 1), (1e-16, 0)]:
        F = chi * RHO / g
        gate, ev = _gate(oracle, F, g, 0.5 * F, 1e-3)
        assert ev.chi == pytest.approx(chi, rel=1e-12)
        assert gate == want, chi


# --- Eq. gammaLCFA and the 0.75 rule ----------------------------------------------
def test_threshold_never_reaches_the_no_emission_rule(oracle):
    # the denominator of Eq. gammaLCFA is 1 + (positive), so gamma_LCFA <= 0.7 gamma_e < 0.75
    # gamma_e: the no-emission rule of Sec. 5 cannot fire; gamma_LCFA -> 0.7 gamma_e as tau -> 0
    rng = np.random.default_rng(4)
    for _ in range(2000):
        F = 10 ** rng.uniform(-3, 6, size=3) * rng.choice([-1, 1], size=3)
        delta = 10 ** rng.uniform(-40, 10)
        g = 10 ** rng.uniform(0.5, 6)
        chi = 10 ** rng.uniform(-6, 3)
        gL = oracle.blcfa_threshold(tuple(F), delta, g, chi)
        assert 0.0 <= gL <= 0.7 * g
    gL = oracle.blcfa_threshold((1.0, 0, 0), 1e30, 1000.0, 1.0)   # tau/tau_C = 2 pi 1e-15
    assert gL == pytest.approx(700.0, rel=1e-12)


# --- Eq. rej_cond: the law of the accepted photons ------------------------------
def _z_for_threshold(q, chi):
    """z with 0.7/(1 + 4/(3 pi chi) (3z + 4z^3)) = q: 3z + 4z^3 = sinh(3 asinh z) = c,
    so z = sinh(asinh(c)/3) (triple-angle identity)."""
    c = (0.7 / q - 1) * 3 * math.pi * chi / 4
    return math.sinh(math.asinh(c) / 3)


def _gated_emitters(oracle, q, n, chi=1.0, gamma=1000.0, seed=11):
    """n beyond-LCFA electrons, one step each, with the gate on, gamma_LCFA = q gamma and
    R dt > 1 (every local test fires): the emitted photons' energies and the oracle's run."""
    pref = oracle.rate_prefactor(RHO)
    R = oracle.photon_rate([gamma], [chi], pref)[0]
    dt = 1.5 / R
    F = chi * RHO / gamma
    z = _z_for_threshold(q, chi)
    # tau/tau_C = 8 gamma z / chi = 2 pi rho F dt / d  (delta = tau_C^2 d^2/dt^2, no second difference)
    d = 2 * math.pi * RHO * F * dt * chi / (8 * gamma * z)
    pm = math.sqrt(gamma * gamma - 1)
    # the state gives the intended threshold through Eqs. condit and gammaLCFA
    gate, ev = _gate(oracle, F, gamma, d, dt)
    assert gate == 1
    assert oracle.blcfa_threshold(tuple(ev.F), ev.delta, ev.gamma, ev.chi) == pytest.approx(q * gamma, rel=1e-9)
    fields = np.zeros((n, 1, 6))
    fields[:, 0, 1] = F
    out = oracle.mc_run(np.tile([pm, 0, 0], (n, 1)), np.zeros(n), np.arange(n, dtype=np.uint64),
                        np.full(n, oracle.FL_ALIVE, np.uint8), np.zeros(n, np.uint8), fields, rho=RHO, dt=dt,
                        seed=seed, nsteps=1, fprev=np.tile([0, F - d, 0], (n, 1)), dfprev=np.tile([0, d, 0], (n, 1)),
                        lepton_mode=oracle.MODE_BLCFA_LOCAL, cap_products=2 * n)
    pr = out["products"]
    e = np.linalg.norm(pr["p"], axis=1)
    return e, out


def _fractions(oracle, gL, gamma, chi):
    """LCFA probabilities (of an event's photon) of the region above gL and the flat mass
    gL S(gL) below it, from the oracle's spectrum (pinned above)."""
    S, pref = _spectrum(oracle)
    W = oracle.photon_rate([gamma], [chi], pref)[0]
    f = lambda t: S(gamma * t ** 3, gamma, chi) * 3 * gamma * t * t
    above = integrate.quad(f, (gL / gamma) ** (1 / 3), 1.0, epsabs=0, epsrel=1e-11, limit=400)[0] / W
    flat = gL * S(gL, gamma, chi) / W
    return above, flat


@pytest.mark.parametrize("q", [0.01, 0.1])
def test_rejection_law_of_accepted_photons(oracle, q, n=3000):
    # 3000 events: the oracle samples each photon energy by Brent's method on a nested
    # quadrature (~50 ms a sample on one core)
    gamma, chi = 1000.0, 1.0
    e, out = _gated_emitters(oracle, q, n, chi, gamma)
    gL = q * gamma
    assert np.all(out["n_events"] == 1) and np.all(out["n_gated"] == 1)
    assert out["n_no_emission"].sum() == 0
    assert out["n_rejected"].sum() + len(e) == n
    above, flat = _fractions(oracle, gL, gamma, chi)
    lo, hi = e[e <= gL], e[e > gL]
    # above the threshold every LCFA sample is kept: the count is binomial(n, above)
    assert abs(len(hi) - n * above) < 4.5 * math.sqrt(n * above * (1 - above)), (len(hi), n * above)
    # below it the kept photons have the density S(gL)/W: count binomial(n, gL S(gL)/W) ...
    assert abs(len(lo) - n * flat) < 4.5 * math.sqrt(n * flat * (1 - flat)), (len(lo), n * flat)
    # ... spread uniformly over (0, gL)
    ks = stats.kstest(lo / gL, "uniform")
    assert ks.statistic < 1.95 / math.sqrt(len(lo)), ks
    # and the LCFA law above it: the kept photons' CDF against the spectrum's
    S, _ = _spectrum(oracle)
    f = lambda t: S(gamma * t ** 3, gamma, chi) * 3 * gamma * t * t
    t0 = (gL / gamma) ** (1 / 3)
    tot = integrate.quad(f, t0, 1.0, epsabs=0, epsrel=1e-10, limit=400)[0]
    xs = np.quantile(hi, [0.1, 0.3, 0.5, 0.7, 0.9])
    for p, x in zip([0.1, 0.3, 0.5, 0.7, 0.9], xs):
        F = integrate.quad(f, t0, (x / gamma) ** (1 / 3), epsabs=0, epsrel=1e-10, limit=400)[0] / tot
        assert abs(F - p) < 4.5 * math.sqrt(p * (1 - p) / len(hi)), (p, F)


def test_threshold_below_the_rule_still_emits(oracle, n=1500):
    # gamma_LCFA = 0.65 gamma_e (the gate on, below 0.7 gamma_e): the event is not stopped
    # by the 0.75 rule, and the kept fraction is the law above
    gamma, chi = 1000.0, 1.0
    e, out = _gated_emitters(oracle, 0.65, n, chi, gamma)
    above, flat = _fractions(oracle, 0.65 * gamma, gamma, chi)
    assert out["n_no_emission"].sum() == 0
    p = above + flat
    assert abs(len(e) - n * p) < 4.5 * math.sqrt(n * p * (1 - p)), (len(e), n * p)
