"""Independent FP64 evaluation of the defining integrals, for table generation.

This is the generator's own numerics and shares nothing with the test oracle:
K_nu and Ki_nu use the trapezoidal rule on the integral representations
K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt and
Ki_nu(x) = int_x^inf K_nu = int_0^inf exp(-x cosh t) cosh(nu t)/cosh t dt
(DLMF 10.32.9 and its x-integral; both integrands are even and analytic in a
strip, so the rule converges exponentially), and the outer integrals of the
paper (Eqs. wtilde, wtilde_pair, pe_eff_int_2, tilde_I_pp of Montefiori &
Tamburini, arXiv:2301.07684) use composite Gauss-Legendre panels.
"""
from __future__ import annotations

import numpy as np

H_T = 0.02           # trapezoid step in t: error ~ exp(-2 pi^2/(H_T^2 x)) < 1e-28 up to x = 745


def _t_grid(xmin: float) -> np.ndarray:
    tmax = np.arccosh(1.0 + 760.0 / max(xmin, 1e-300)) + 1.0
    return np.arange(0.0, tmax + H_T, H_T)


def besselk_scaled(nu: float, x) -> np.ndarray:
    """exp(x) K_nu(x) for x > 0 (array)."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    out = np.empty_like(x)
    order = np.argsort(x)
    # chunk by magnitude so that each chunk uses a grid long enough for its smallest x
    for chunk in np.array_split(order, max(1, x.size // 4096)):
        xc = x[chunk]
        t = _t_grid(xc.min())
        w = np.full(t.size, H_T)
        w[0] = 0.5 * H_T
        sh = np.sinh(0.5 * t)
        e = np.exp(-np.outer(xc, 2.0 * sh * sh))
        out[chunk] = e @ (w * np.cosh(nu * t))
    return out


def besselk_int_scaled(nu: float, x) -> np.ndarray:
    """exp(x) Ki_nu(x), Ki_nu(x) = int_x^inf K_nu(y) dy, x > 0 (array)."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    out = np.empty_like(x)
    order = np.argsort(x)
    for chunk in np.array_split(order, max(1, x.size // 4096)):
        xc = x[chunk]
        t = _t_grid(xc.min())
        w = np.full(t.size, H_T)
        w[0] = 0.5 * H_T
        sh = np.sinh(0.5 * t)
        e = np.exp(-np.outer(xc, 2.0 * sh * sh))
        out[chunk] = e @ (w * np.cosh(nu * t) / np.cosh(t))
    return out


def besselk(nu, x):
    x = np.asarray(x, dtype=np.float64)
    return np.where(x > 745.0, 0.0, np.exp(-np.minimum(x, 745.0)) * besselk_scaled(nu, x))


def besselk_int(nu, x):
    x = np.asarray(x, dtype=np.float64)
    return np.where(x > 745.0, 0.0, np.exp(-np.minimum(x, 745.0)) * besselk_int_scaled(nu, x))


def gl_panels(edges: np.ndarray, npts: int = 24):
    """Nodes and weights of composite Gauss-Legendre over consecutive edges."""
    xg, wg = np.polynomial.legendre.leggauss(npts)
    a, b = edges[:-1, None], edges[1:, None]
    nodes = 0.5 * (a + b) + 0.5 * (b - a) * xg[None, :]
    weights = 0.5 * (b - a) * wg[None, :]
    return nodes.ravel(), weights.ravel()


# --- photon emission -----------------------------------------------------------
T_MAX_RAD = 700.0 ** (1.0 / 3.0)


def _rad_edges(chi: float) -> np.ndarray:
    # t = v^{1/3}; refine geometrically towards t = 0 where the rational factor
    # varies on the scale v ~ 1/chi
    lo = np.geomspace(1e-4, 1.0, 25)
    return np.unique(np.concatenate([[0.0], lo, np.linspace(1.0, T_MAX_RAD, 25)]))


def wtilde_rad(chi) -> np.ndarray:
    """W~_rad(chi), Eq. wtilde (v = t^3)."""
    chi = np.atleast_1d(np.asarray(chi, dtype=np.float64))
    t, w = gl_panels(_rad_edges(1.0))
    v = t ** 3
    k = besselk(2.0 / 3.0, v) * 3.0 * t * t * w
    x = np.outer(chi, v)
    den = 2.0 + 3.0 * x
    f = (45.0 * x * x + 42.0 * x + 20.0) / (den * den * den)
    return f @ k


def pe_density(w, chi):
    """Integrand of Eq. pe_eff_int_2 at (w, chi) (broadcast)."""
    w, chi = np.broadcast_arrays(np.asarray(w, dtype=np.float64), np.asarray(chi, dtype=np.float64))
    x = w ** 3
    s = 1.5 * chi * x
    ops = 1.0 + s
    k23 = besselk(2.0 / 3.0, x.ravel()).reshape(x.shape)
    ki = besselk_int(1.0 / 3.0, x.ravel()).reshape(x.shape)
    return 9.0 * w * w / (2.0 * ops ** 3) * ((1.0 + ops * ops) * k23 - ops * ki)


# --- pair creation ---------------------------------------------------------------
def pp_density_om(v, om, chi):
    """Integrand of Eq. tilde_I_pp with om = 1 - v^2 given separately."""
    eta = 8.0 / (3.0 * chi * om)
    big = eta > 745.0
    e = np.where(big, 745.0, eta)
    k23 = besselk(2.0 / 3.0, e.ravel()).reshape(e.shape)
    ki = besselk_int(1.0 / 3.0, e.ravel()).reshape(e.shape)
    return np.where(big, 0.0, 2.0 * (1.0 + v * v) / om * k23 + ki)


def _pair_w_integrand(v, om, chi):
    """Integrand of Eq. wtilde_pair with om = 1 - v^2 given separately."""
    eta = 8.0 / (3.0 * chi * om)
    ok = eta < 745.0
    out = np.zeros_like(v)
    out[ok] = (9.0 - v[ok] ** 2) / (3.0 * om[ok]) * besselk(2.0 / 3.0, eta[ok])
    return out


def pair_lower_nodes(chi: float, vmax: float = 0.5):
    """GL nodes on [0, vmax] graded to the width sqrt(3 chi/16) of the spectrum at v = 0."""
    width = min(vmax, np.sqrt(3.0 * chi / 16.0))
    edges = np.unique(np.concatenate([np.linspace(0.0, min(vmax, 10 * width), 41),
                                      np.linspace(min(vmax, 10 * width), vmax, 9)]))
    return gl_panels(edges)


def pair_upper_nodes(zmax: float = 0.5 ** (1.0 / 3.0)):
    """GL nodes in z on [0, zmax] for v = 1 - z^3 (removes the (1-v)^(-1/3) end behaviour)."""
    edges = np.unique(np.concatenate([[0.0], np.geomspace(1e-6, zmax, 40)]))
    return gl_panels(edges)


def wtilde_pair(chi) -> np.ndarray:
    """W~_pair(chi), Eq. wtilde_pair: [0, 1/2] in v plus [1/2, 1] in z, v = 1 - z^3."""
    chi = np.atleast_1d(np.asarray(chi, dtype=np.float64))
    out = np.empty_like(chi)
    z, wz = pair_upper_nodes()
    y = z ** 3
    vu, omu, ju = 1.0 - y, y * (2.0 - y), 3.0 * z * z * wz
    for i, c in enumerate(chi):
        v, wv = pair_lower_nodes(c)
        lo = _pair_w_integrand(v, (1.0 - v) * (1.0 + v), c) @ wv
        hi = _pair_w_integrand(vu, omu, c) @ ju
        out[i] = lo + hi
    return out
