"""Inverse cumulative functions for table generation (generator numerics).

For one chi the density of Eq. pe_eff_int_2 (photon emission, variable w) or
of Eq. tilde_I_pp (pair creation, variables v near 0 and z = (1-v)^(1/3) near
v = 1) is sampled at Gauss-Legendre nodes of graded panels.  Inside a panel
the density is represented by its Legendre series (from the nodes) and its
antiderivative gives the cumulative function at any point; lower and upper
cumulative sums are kept separately so that both tails keep relative
precision.  Roots of Eq. again / Eq. again_pp (Montefiori & Tamburini,
arXiv:2301.07684, Secs. 4.3-4.4) come from Newton's method on that
representation.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg

from . import quad as Q

NGL = 24
_XG, _WG = npleg.leggauss(NGL)
# Legendre coefficients from values at the nodes: c_k = (2k+1)/2 sum_j w_j P_k(x_j) f_j
_PK = np.stack([npleg.legval(_XG, np.eye(NGL)[k]) for k in range(NGL)])     # (k, j)
_V2C = (2 * np.arange(NGL)[:, None] + 1) / 2.0 * _PK * _WG[None, :]         # (k, j)


def _antideriv_matrix():
    # coefficients of int_{-1}^{x} P_k  in the Legendre basis of degree NGL
    M = np.zeros((NGL + 1, NGL))
    for k in range(NGL):
        c = np.zeros(NGL)
        c[k] = 1.0
        M[:, k] = npleg.legint(c, lbnd=-1)
    return M


_INT = _antideriv_matrix()


class PanelCDF:
    """Piecewise Legendre representation of a density on panels [e_i, e_{i+1}]."""

    def __init__(self, edges: np.ndarray, density_at):
        self.edges = np.asarray(edges, dtype=np.float64)
        a, b = self.edges[:-1], self.edges[1:]
        self.half = 0.5 * (b - a)
        self.mid = 0.5 * (a + b)
        x = self.mid[:, None] + self.half[:, None] * _XG[None, :]
        f = density_at(x)                                   # (panels, NGL)
        self.coef = f @ _V2C.T                              # density Legendre coefficients
        self.icoef = self.coef @ _INT.T * self.half[:, None]   # antiderivative from the left edge
        mass = (f * _WG[None, :]).sum(1) * self.half
        self.mass = mass
        self.lower = np.concatenate([[0.0], np.cumsum(mass)])            # int_{e0}^{e_i}
        self.upper = np.concatenate([np.cumsum(mass[::-1])[::-1], [0.0]])  # int_{e_i}^{e_end}
        self.total = self.lower[-1]

    def _local(self, i, x):
        return (x - self.mid[i]) / self.half[i]

    def density(self, i, x):
        t = self._local(i, x)
        return _legval_rows(self.coef[i], t)

    def partial(self, i, x):
        """int from e_i to x (x inside panel i)."""
        t = self._local(i, x)
        return _legval_rows(self.icoef[i], t)

    def invert_lower(self, target):
        """x with int_{e0}^{x} = target (vectorised)."""
        target = np.asarray(target, dtype=np.float64)
        i = np.clip(np.searchsorted(self.lower, target, side="right") - 1, 0, len(self.mass) - 1)
        base = self.lower[i]
        frac = np.clip((target - base) / np.where(self.mass[i] > 0, self.mass[i], 1.0), 0.0, 1.0)
        x = self.edges[i] + frac * (self.edges[i + 1] - self.edges[i])
        for _ in range(40):
            g = base + self.partial(i, x) - target
            d = self.density(i, x)
            step = np.where(d > 0, g / np.where(d > 0, d, 1.0), 0.0)
            xn = np.clip(x - step, self.edges[i], self.edges[i + 1])
            if np.all(np.abs(xn - x) <= 1e-16 * np.abs(xn) + 1e-300):
                x = xn
                break
            x = xn
        return x

    def invert_upper(self, target):
        """x with int_{x}^{e_end} = target (vectorised)."""
        target = np.asarray(target, dtype=np.float64)
        # upper is decreasing in the panel index
        i = np.clip(np.searchsorted(-self.upper, -target, side="left") - 1, 0, len(self.mass) - 1)
        top = self.upper[i + 1]                               # int_{e_{i+1}}^{end}
        frac = np.clip((self.upper[i] - target) / np.where(self.mass[i] > 0, self.mass[i], 1.0), 0, 1)
        x = self.edges[i] + frac * (self.edges[i + 1] - self.edges[i])
        for _ in range(40):
            # int_x^{e_{i+1}} = mass_i - partial(x)
            g = top + (self.mass[i] - self.partial(i, x)) - target
            d = self.density(i, x)
            step = np.where(d > 0, -g / np.where(d > 0, d, 1.0), 0.0)
            xn = np.clip(x - step, self.edges[i], self.edges[i + 1])
            if np.all(np.abs(xn - x) <= 1e-16 * np.abs(xn) + 1e-300):
                x = xn
                break
            x = xn
        return x


def _legval_rows(c, t):
    """Legendre series with per-element coefficient rows c (n, NGL[+1]) at t (n,) (Clenshaw)."""
    n = c.shape[1]
    b1 = np.zeros_like(t)
    b2 = np.zeros_like(t)
    for k in range(n - 1, 0, -1):
        # P_{k+1} = ((2k+1) t P_k - k P_{k-1})/(k+1): Clenshaw with alpha_k = (2k+1)t/(k+1), beta_k = -(k+1)/(k+2)
        a = (2 * k + 1) * t / (k + 1)
        b = -(k + 1) / (k + 2)
        b1, b2 = c[:, k] + a * b1 + b * b2, b1
    return c[:, 0] + t * b1 - 0.5 * b2


# ----------------------------------------------------------------------------------
# photon emission: variable w of Eq. subs_altri
W_MAX = 700.0 ** (1.0 / 3.0)


def _photon_edges():
    lo = np.geomspace(1e-13, 0.05, 80)
    mid = np.linspace(0.05, 3.5, 140)
    hi = np.linspace(3.5, W_MAX, 60)
    return np.unique(np.concatenate([[0.0], lo, mid, hi]))


class _KTable:
    """K_2/3(w^3) and Ki_1/3(w^3) at the Gauss nodes of the photon w-panels (chi-independent)."""

    def __init__(self):
        self.edges = _photon_edges()
        a, b = self.edges[:-1], self.edges[1:]
        self.w = 0.5 * (a + b)[:, None] + 0.5 * (b - a)[:, None] * _XG[None, :]
        x = self.w ** 3
        self.k23 = Q.besselk(2.0 / 3.0, x.ravel()).reshape(x.shape)
        self.ki13 = Q.besselk_int(1.0 / 3.0, x.ravel()).reshape(x.shape)


_KT = None


def _kt():
    global _KT
    if _KT is None:
        _KT = _KTable()
    return _KT


class PhotonCDF:
    """I~_pe(w, chi) for one chi (Eq. pe_eff_int_2) and its inverse (Eq. again)."""

    def __init__(self, chi: float):
        kt = _kt()
        self.chi = float(chi)
        w = kt.w
        s = 1.5 * chi * w ** 3
        ops = 1.0 + s
        dens = 9.0 * w * w / (2.0 * ops ** 3) * ((1.0 + ops * ops) * kt.k23 - ops * kt.ki13)
        self.p = PanelCDF(kt.edges, lambda x: dens)
        self.W = Q.wtilde_rad(self.chi)[0]

    def wbar(self, r):
        r = np.asarray(r, dtype=np.float64)
        out = np.empty_like(r)
        lo = r < 0.5
        out[lo] = self.p.invert_lower(r[lo] * self.W)
        out[~lo] = self.p.invert_upper((1.0 - r[~lo]) * self.W)
        return out


# ----------------------------------------------------------------------------------
# pair creation: v of Eq. subs_pair on [0, 1/2], z = (1 - v)^(1/3) on [0, (1/2)^(1/3)]
Z_SPLIT = 0.5 ** (1.0 / 3.0)


class PairCDF:
    """I~_pp(v, chi) for one chi (Eq. tilde_I_pp) and its inverse (Eq. again_pp).

    Lower part in v in [0, 1/2]; upper part in z with v = 1 - z^3 (mass in the
    upper part is int_{1/2}^{1} dv = int_0^{Z_SPLIT} 3 z^2 dz)."""

    def __init__(self, chi: float):
        self.chi = c = float(chi)
        width = min(0.5, np.sqrt(3.0 * c / 16.0))
        ev = np.unique(np.concatenate([[0.0], np.geomspace(1e-12 * width, 0.01 * width, 40),
                                       np.linspace(0.01 * width, min(0.5, 12 * width), 80),
                                       np.linspace(min(0.5, 12 * width), 0.5, 20)]))

        def dv(v):
            return Q.pp_density_om(v, (1.0 - v) * (1.0 + v), c)

        def dz(z):
            y = z ** 3
            return Q.pp_density_om(1.0 - y, y * (2.0 - y), c) * 3.0 * z * z

        ez = np.unique(np.concatenate([[0.0], np.geomspace(1e-5, Z_SPLIT, 160)]))
        self.pv = PanelCDF(ev, dv)
        self.pz = PanelCDF(ez, dz)
        self.W = Q.wtilde_pair(c)[0]

    def vbar_ybar(self, a):
        """(v-bar, y-bar = 1 - v-bar) solving I~_pp(v) = a W~_pair (Eq. again_pp)."""
        a = np.asarray(a, dtype=np.float64)
        v = np.empty_like(a)
        y = np.empty_like(a)
        upper_mass = self.pz.total                     # int_{1/2}^{1}
        # target measured from v = 1 down: (1 - a) W
        tgt_hi = (1.0 - a) * self.W
        in_z = tgt_hi < upper_mass
        z = self.pz.invert_lower(tgt_hi[in_z])         # int_0^{z} in z = int_{1-z^3}^{1} in v
        y[in_z] = z ** 3
        v[in_z] = 1.0 - y[in_z]
        low = (~in_z) & (a < 0.5)
        mid = (~in_z) & (a >= 0.5)
        vv = self.pv.invert_lower(a[low] * self.W)
        v[low] = vv
        y[low] = 1.0 - vv
        # complementary form: int_v^{1/2} = (1 - a) W - int_{1/2}^{1}
        vm = self.pv.invert_upper(tgt_hi[mid] - upper_mass)
        v[mid] = vm
        y[mid] = 1.0 - vm
        return v, y
