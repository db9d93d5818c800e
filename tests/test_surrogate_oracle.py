"""Pins of the surrogate's oracle (oracle/surrogate.py), on the CPU.

- The dense CDF table (logit F from the oracle's quadrature, bicubic spline) against
  direct quadrature of Eq. pe_eff_int_2 at off-grid points and against the oracle's
  Brent inversion of Eq. again, on a coarse grid (the interpolation error falls as
  the fourth power of the spacing; the fine grid of the GPU tests is checked there).
- The network's gradient (chain rule written out) against central finite
  differences of its loss, and its bfloat16 rounding against torch's conversion.
- The small-u law xi ~ chi u^3 carried by the output variable.
"""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def S():
    from oracle import oracle as O
    O.build()
    from oracle import surrogate
    return surrogate


@pytest.fixture(scope="module")
def coarse(S):
    return S.DenseCDF(dx=0.2, dy=0.1)


def test_dense_cdf_matches_direct_quadrature(S, coarse):
    from oracle import oracle as O
    g = np.random.default_rng(3)
    m = 120
    chi = np.exp(g.uniform(np.log(1e-3), np.log(100.0), m))
    w = O.photon_wbar(g.uniform(0.001, 0.999, m), chi)       # points spread over the bulk of F
    lo, up = O.itilde_pe_batch(w, chi), O.itilde_pe_upper_batch(w, chi)
    F = lo / (lo + up)
    Ft = coarse.cdf_w(chi, w)
    assert np.max(np.abs(Ft - F)) < 5e-6
    # the two halves are the oracle's complementary integrals: they add up to W~_rad
    W = O.wtilde_rad(chi)
    assert np.max(np.abs((lo + up) / W - 1.0)) < 1e-12


def test_dense_cdf_inverse_matches_brent(S, coarse):
    from oracle import oracle as O
    g = np.random.default_rng(4)
    m = 80
    chi = np.exp(g.uniform(np.log(1e-3), np.log(100.0), m))
    u = g.uniform(0.0005, 0.9995, m)
    s = O.photon_s(u, chi)
    xo = s / (1.0 + s)
    xt = coarse.inverse_xi(chi, u)
    assert np.max(np.abs(xt - xo) / xo) < 1e-4
    # PIT of the inverse returns u
    assert np.max(np.abs(coarse.pit(chi, xt) - u)) < 1e-9


def test_small_u_law(S, coarse):
    """For u -> 0, I~_pe ~ 9 Gamma(2/3) w / 2^(1/3) (Eq. pe_eff_int_approx_w_small), so
    w-bar = u W~_rad / (9 Gamma(2/3) / 2^(1/3)) and ln w-bar - ln u is a function of chi."""
    from math import gamma
    from oracle import oracle as O
    chi = np.array([1e-3, 0.1, 10.0])
    u = np.full(3, 1e-6)
    lnw = coarse.inverse_lnw(chi, u)
    expect = np.log(u * O.wtilde_rad(chi) / (9.0 * gamma(2.0 / 3.0) / 2.0 ** (1.0 / 3.0)))
    assert np.max(np.abs(lnw - expect)) < 1e-6


def test_gradient_matches_finite_differences(S):
    g = np.random.default_rng(5)
    theta = g.uniform(-0.5, 0.5, S.N_PARAMS)
    n = 16
    lnchi = g.uniform(np.log(1e-3), np.log(100.0), n)
    u = g.uniform(0.01, 0.99, n)
    target = g.normal(0.0, 1.0, n)
    loss, grad = S.mlp_loss_grad(theta, lnchi, u, target)
    idx = np.concatenate([g.choice(S.N_PARAMS, 60, replace=False), [0, 1, 128, 191, 8511, 8576]])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (S.mlp_loss_grad(tp, lnchi, u, target)[0] - S.mlp_loss_grad(tm, lnchi, u, target)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(grad[i])), (i, fd, grad[i])
    # the loss is the mean squared error of ln w-bar
    lnw = S.surrogate_lnw(theta, lnchi, u)
    assert abs(loss - np.mean((lnw - target) ** 2)) < 1e-12


def test_bf16_rounding_matches_torch(S):
    torch = pytest.importorskip("torch")
    g = np.random.default_rng(6)
    x = np.concatenate([g.normal(0, 3, 2000), [1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 0.0, 1e-30]])
    x32 = x.astype(np.float32)
    ref = torch.tensor(x32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(S.bf16(x32), ref)


@pytest.fixture(scope="module")
def coarse_pair(S):
    return S.DensePairCDF(ds=0.1, dx=0.2)


def test_dense_pair_cdf_matches_brent(S, coarse_pair):
    """The pair-share CDF table (logit of I~_pp over its complement, Eq. tilde_I_pp) against
    the oracle's Brent roots of Eq. again_pp: the CDF at the root returns |r'|, and the
    table's inverse returns the root."""
    from oracle import oracle as O
    g = np.random.default_rng(7)
    m = 200
    chi = np.exp(g.uniform(np.log(0.1), np.log(100.0), m))
    a = g.uniform(2.0 ** -24, 1.0 - 2.0 ** -24, m)
    v, y = O.pair_vbar(a, chi)
    at = coarse_pair.cdf_y(chi, y)
    assert np.max(np.abs(at - a)) < 5e-6
    assert np.max(np.abs((1.0 - at) - (1.0 - a)) / (1.0 - a)) < 1e-4
    yt = np.exp(coarse_pair.inverse_lny(chi, a))
    assert np.max(np.abs(yt / y - 1.0)) < 1e-4
    # shares built from the root: the PIT returns |r'|
    xe, xp = 1.0 - 0.5 * y, 0.5 * y
    assert np.max(np.abs(coarse_pair.pit(chi, xe, xp) - a)) < 5e-6
    # the two halves are independent integrals that add up to W~_pair
    lo, up = O.itilde_pp_batch(v, chi), O.itilde_pp_upper_y_batch(y, chi)
    assert np.max(np.abs((lo + up) / O.wtilde_pair(chi) - 1.0)) < 1e-10


def test_pair_kind_features(S):
    """The pair kind maps chi in [0.1, 100] onto [-1, 1] and u = |r'| as the photon kind maps u."""
    x = S.features(np.log([0.1, 100.0]), [0.5, 0.5], kind="pair")
    assert np.allclose(x[:, 0], [-1.0, 1.0], atol=1e-15)
    assert np.allclose(x[:, 1], S.features([0.0, 0.0], [0.5, 0.5])[:, 1])
