"""Pins of the oracle's Boris push (oracle/sfq_oracle.c, orc_boris_push), on the CPU, by the
algorithm's textbook properties (Boris 1970):

- in a magnetic field alone the push is a rotation: |u| is conserved to rounding and the
  angle turned per step is 2 atan(|t|), t = q B dt / (2 gamma);
- in an electric field alone the momentum changes by exactly q E dt;
- the push is time-reversible: a step with -dt undoes a step with dt;
- q = 0 (photons) leaves the momentum unchanged.
"""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.build()
    return oracle


def test_magnetic_rotation(O):
    g = np.random.default_rng(1)
    n = 256
    u = g.normal(0.0, 50.0, (n, 3))
    B = g.normal(0.0, 30.0, (n, 3))
    q = np.where(g.random(n) < 0.5, -1.0, 1.0)
    dt = 0.0628
    un = O.boris_push(u.copy(), np.zeros((n, 3)), B, q, dt)
    # |u| conserved
    assert np.max(np.abs(np.linalg.norm(un, axis=1) / np.linalg.norm(u, axis=1) - 1.0)) < 1e-14
    # angle about B: the components perpendicular to B turn by 2 atan(|t|)
    gam = np.sqrt(1.0 + np.sum(u * u, axis=1))
    tmag = 0.5 * dt * np.linalg.norm(B, axis=1) / gam
    bh = B / np.linalg.norm(B, axis=1)[:, None]
    perp = lambda v: v - np.sum(v * bh, axis=1)[:, None] * bh
    a, b = perp(u), perp(un)
    cosang = np.sum(a * b, axis=1) / (np.linalg.norm(a, axis=1) * np.linalg.norm(b, axis=1))
    ang = np.arccos(np.clip(cosang, -1.0, 1.0))
    assert np.max(np.abs(ang - 2.0 * np.arctan(tmag))) < 1e-9
    # the component along B is untouched
    assert np.max(np.abs(np.sum(un * bh, axis=1) - np.sum(u * bh, axis=1))) < 1e-12 * np.abs(u).max()


def test_electric_kick(O):
    g = np.random.default_rng(2)
    n = 128
    u = g.normal(0.0, 10.0, (n, 3))
    E = g.normal(0.0, 5.0, (n, 3))
    q = np.where(g.random(n) < 0.5, -1.0, 1.0)
    dt = 0.03
    un = O.boris_push(u.copy(), E, np.zeros((n, 3)), q, dt)
    np.testing.assert_allclose(un, u + q[:, None] * E * dt, rtol=0, atol=1e-13)


def test_time_reversible(O):
    g = np.random.default_rng(3)
    n = 128
    u = g.normal(0.0, 100.0, (n, 3))
    E, B = g.normal(0.0, 50.0, (n, 3)), g.normal(0.0, 50.0, (n, 3))
    q = -np.ones(n)
    dt = 0.05
    back = O.boris_push(O.boris_push(u.copy(), E, B, q, dt), E, B, q, -dt)
    assert np.max(np.abs(back - u)) < 1e-12 * np.abs(u).max()


def test_photons_unchanged(O):
    u = np.array([[1.0, 2.0, 3.0]])
    un = O.boris_push(u.copy(), [[1.0, 1.0, 1.0]], [[2.0, 0.0, 1.0]], [0.0], 0.1)
    np.testing.assert_array_equal(un, u)


def test_pushed_force_in_a_magnetic_field(O):
    """With the pusher, F_L = (p^(n+1/2) - p^(n-1/2)) / dt (Eqs. fl).  In a magnetic field
    alone the Boris push is the implicit midpoint rule, so F_L = q p_L x B / gamma(p) with
    p_L the mid-point momentum, exactly; it is perpendicular to p_L, so F_perp = F_L, and
    chi_p = tau_C gamma(p_L) |F_perp|."""
    g = np.random.default_rng(7)
    rho, dt = 3.2972e5, 0.0628
    for _ in range(32):
        p = g.normal(0.0, 300.0, 3)
        B = g.normal(0.0, 80.0, 3)
        pn = O.boris_push(p.copy(), np.zeros(3), B, -1.0, dt)[0]
        _, ev, _, _, _ = O.blcfa_update_pushed(p, pn, dt, rho, [0.0] * 3, [0.0] * 3, True)
        pL = 0.5 * (p + pn)
        F = -np.cross(pL, B) / np.sqrt(1.0 + p @ p)
        np.testing.assert_allclose(np.array(ev.F[:]), F, rtol=1e-9, atol=1e-12 * np.abs(F).max())
        assert ev.chi == pytest.approx(np.sqrt(1.0 + pL @ pL) * np.linalg.norm(F) / rho, rel=1e-12)
