"""Oracle side of the learned inverse-CDF surrogate (TEST INFRASTRUCTURE ONLY).

Two plain FP64 references, used only by the test-suite:

1. ``DenseCDF`` -- the photon-emission energy CDF of the oracle (``DensePairCDF``
   the same for the pair shares),
   F(xi | chi) = I~_pe(w, chi) / W~_rad(chi) with s = xi / (1 - xi) = 3 chi w^3 / 2
   (Eq. pe_eff_int_2, Eq. wtilde, Eq. subs_altri), tabulated by the oracle's own
   quadrature on a dense grid of (ln chi, ln w) and interpolated by a bicubic
   spline (a library primitive) of logit F.  The lower and upper parts of the CDF
   are integrated separately (I~_pe and its complement), so logit F keeps its
   relative precision in both tails.  It serves the probability-integral
   transform of many draws (KS test) and the inversion that produces training
   triples (chi, u, xi).  Its accuracy is pinned in the tests against direct
   quadrature and the oracle's Brent inversion.

2. ``mlp_forward`` / ``mlp_loss_grad`` -- the surrogate network written out in
   numpy FP64 (2 -> 64 -> 64 -> 64 -> 1, SiLU) with the input features, output
   variable and optional bfloat16 rounding of weights and activations that the
   GPU kernels use; the backward pass is the chain rule written out layer by
   layer.  Pinned by central finite differences.
"""
from __future__ import annotations

import hashlib
import os

import numpy as np

from . import oracle as O

_HERE = os.path.dirname(os.path.abspath(__file__))
_CACHE = os.path.join(_HERE, "_build")

# --- dense CDF -------------------------------------------------------------------
LNCHI_LO, LNCHI_HI, DX = np.log(5e-4), np.log(200.0), 0.1
LNW_LO, LNW_HI, DY = -16.5, 1.1, 0.05


class DenseCDF:
    """logit F(w | chi) on a (ln chi, ln w) grid, bicubic spline in between."""

    def __init__(self, dx=DX, dy=DY, cache=True):
        from scipy.interpolate import RectBivariateSpline
        self.x = np.arange(LNCHI_LO, LNCHI_HI + 0.5 * dx, dx)
        self.y = np.arange(LNW_LO, LNW_HI + 0.5 * dy, dy)
        key = hashlib.sha1(np.concatenate([self.x, self.y]).tobytes()).hexdigest()[:16]
        path = os.path.join(_CACHE, f"nlc_cdf_{key}.npz")
        z = None
        if cache and os.path.exists(path):
            z = np.load(path)["logit"]
        if z is None:
            X, Y = np.meshgrid(self.x, self.y, indexing="ij")
            chi, w = np.exp(X).ravel(), np.exp(Y).ravel()
            lo = O.itilde_pe_batch(w, chi)
            up = O.itilde_pe_upper_batch(w, chi)
            z = (np.log(lo) - np.log(up)).reshape(X.shape)      # logit F = ln(I / (W - I))
            if cache:
                os.makedirs(_CACHE, exist_ok=True)
                tmp = path + f".tmp{os.getpid()}.npz"
                np.savez(tmp, logit=z)
                os.replace(tmp, path)
        self.logit_grid = z
        self.spline = RectBivariateSpline(self.x, self.y, z, kx=3, ky=3, s=0)

    # logit F at (ln chi, ln w); below the grid F ~ w (Eq. pe_eff_int_approx_w_small), so
    # ln F continues with slope 1; above it 1 - F < 1e-7 and F is taken as 1.
    def logit(self, lnchi, lnw):
        lnchi = np.clip(np.asarray(lnchi, np.float64), self.x[0], self.x[-1])
        lnw = np.asarray(lnw, np.float64)
        yc = np.clip(lnw, self.y[0], self.y[-1])
        z = self.spline.ev(lnchi, yc)
        low = lnw < self.y[0]
        if np.any(low):
            lnF = -np.logaddexp(0.0, -z[low]) + (lnw[low] - self.y[0])
            z[low] = lnF - np.log1p(-np.exp(lnF))
        z[lnw > self.y[-1]] = np.inf
        return z

    def cdf_w(self, chi, w):
        z = self.logit(np.log(chi), np.log(w))
        return 1.0 / (1.0 + np.exp(-z))

    def pit(self, chi, xi):
        """F(xi | chi) for photon energy fractions xi in (0, 1)."""
        chi = np.asarray(chi, np.float64)
        xi = np.asarray(xi, np.float64)
        s = xi / (1.0 - xi)
        lnw = (np.log(2.0 * s) - np.log(3.0 * chi)) / 3.0
        z = self.logit(np.log(chi), lnw)
        return 1.0 / (1.0 + np.exp(-z))

    def inverse_lnw(self, chi, u, iters=48):
        """ln w with F(w | chi) = u: bisection on the monotone spline, then two Newton steps."""
        lnchi = np.log(np.asarray(chi, np.float64))
        u = np.asarray(u, np.float64)
        target = np.log(u) - np.log1p(-u)
        a = np.full(u.shape, self.y[0])
        b = np.full(u.shape, self.y[-1])
        for _ in range(iters):
            m = 0.5 * (a + b)
            below = self.spline.ev(lnchi, m) < target
            a = np.where(below, m, a)
            b = np.where(below, b, m)
        y = 0.5 * (a + b)
        for _ in range(2):
            f = self.spline.ev(lnchi, y) - target
            d = self.spline.ev(lnchi, y, dy=1)
            y = np.clip(y - f / np.maximum(d, 1e-300), self.y[0], self.y[-1])
        # below the grid: ln F continues with slope 1
        lowF = self.logit(lnchi, np.full(u.shape, self.y[0]))
        low = target < lowF
        if np.any(low):
            lnF0 = -np.logaddexp(0.0, -lowF[low])
            y[low] = self.y[0] + (np.log(u[low]) - lnF0)
        return y

    def inverse_xi(self, chi, u):
        """xi = s / (1 + s), s = 3 chi w^3 / 2 with F(w | chi) = u (Eq. again, Eq. subs_altri)."""
        chi = np.asarray(chi, np.float64)
        lnw = self.inverse_lnw(chi, u)
        s = 1.5 * chi * np.exp(3.0 * lnw)
        return s / (1.0 + s)


# --- dense CDF of the pair shares --------------------------------------------------------
PLNCHI_LO, PLNCHI_HI, PDX = np.log(0.05), np.log(200.0), 0.1
PS_LO, PS_HI, PDS = -8.0, 19.5, 0.05


def _expit(x):
    return 0.5 * (1.0 + np.tanh(0.5 * np.asarray(x, np.float64)))


class DensePairCDF:
    """The pair-creation CDF of the oracle in the half-domain of Eq. again_pp:
    a(y | chi) = I~_pp(1 - y, chi) / W~_pair(chi) with y = 1 - v-bar (Eq. tilde_I_pp), the
    probability that |r'| falls below the value that returns v-bar.  logit a = ln I~_pp(v)
    - ln int_{1-y}^1 (the two parts integrated separately, each in its own variable, so that
    both tails keep their relative precision) is tabulated on a (ln chi, s) grid with
    s = logit y = ln(y / v) and interpolated by a bicubic spline (a library primitive).
    Above the grid (v -> 0) a ~ v, so logit a continues with slope -1 in s.  Where the upper
    part underflows (small chi, small y) logit a is capped at 60."""

    def __init__(self, ds=PDS, dx=PDX, cache=True):
        from scipy.interpolate import RectBivariateSpline
        self.x = np.arange(PLNCHI_LO, PLNCHI_HI + 0.5 * dx, dx)
        self.s = np.arange(PS_LO, PS_HI + 0.5 * ds, ds)
        key = hashlib.sha1(np.concatenate([self.x, self.s, [60.0]]).tobytes()).hexdigest()[:16]
        path = os.path.join(_CACHE, f"nbw_cdf_{key}.npz")
        z = None
        if cache and os.path.exists(path):
            z = np.load(path)["logit"]
        if z is None:
            X, S = np.meshgrid(self.x, self.s, indexing="ij")
            chi = np.exp(X).ravel()
            y = _expit(S).ravel()
            v = _expit(-S).ravel()
            lo = O.itilde_pp_batch(v, chi)
            up = O.itilde_pp_upper_y_batch(y, chi)
            # far in the upper tail (small chi and y) the upper part underflows; logit a is
            # capped at 60 there, far beyond binary32 draws (logit a <= ln 2^24 = 16.6)
            ok = (lo > 0.0) & (up > 0.0)
            z = np.full(lo.shape, 60.0)
            z[ok] = np.minimum(np.log(lo[ok]) - np.log(up[ok]), 60.0)
            z[(lo <= 0.0) & (up > 0.0)] = -60.0
            z = z.reshape(X.shape)
            if cache:
                os.makedirs(_CACHE, exist_ok=True)
                tmp = path + f".tmp{os.getpid()}.npz"
                np.savez(tmp, logit=z)
                os.replace(tmp, path)
        self.logit_grid = z
        self.spline = RectBivariateSpline(self.x, self.s, z, kx=3, ky=3, s=0)

    def logit(self, lnchi, s):
        lnchi = np.clip(np.asarray(lnchi, np.float64), self.x[0], self.x[-1])
        s = np.asarray(s, np.float64)
        sc = np.clip(s, self.s[0], self.s[-1])
        z = self.spline.ev(lnchi, sc)
        hi = s > self.s[-1]
        if np.any(hi):
            z[hi] = z[hi] - (s[hi] - self.s[-1])
        return z

    def cdf_y(self, chi, y):
        y = np.asarray(y, np.float64)
        return _expit(self.logit(np.log(chi), np.log(y) - np.log1p(-y)))

    def pit(self, chi, xe, xp):
        """a = F(v-bar | chi) of sampled shares: y = 2 min(xe, xp), v-bar = |xe - xp|."""
        xe = np.asarray(xe, np.float64)
        xp = np.asarray(xp, np.float64)
        y = 2.0 * np.minimum(xe, xp)
        v = np.abs(xe - xp)
        return _expit(self.logit(np.log(np.asarray(chi, np.float64)), np.log(y) - np.log(v)))

    def inverse_lny(self, chi, a, iters=56):
        """ln y with a(y | chi) = a, by bisection in s on the monotone spline."""
        lnchi = np.log(np.asarray(chi, np.float64))
        a = np.asarray(a, np.float64)
        target = np.log(a) - np.log1p(-a)
        lo = np.full(a.shape, self.s[0])
        hi = np.full(a.shape, self.s[-1] + 40.0)
        for _ in range(iters):
            m = 0.5 * (lo + hi)
            above = self.logit(lnchi, m) > target          # logit a falls as s rises
            lo = np.where(above, m, lo)
            hi = np.where(above, hi, m)
        s = 0.5 * (lo + hi)
        return -np.logaddexp(0.0, -s)                     # ln y = ln expit(s)


# --- the surrogate network ------------------------------------------------------------
# It approximates the inverse CDF of Eq. again in the paper's own variable w-bar:
#   features  x1 = (ln chi - C_CHI) / S_CHI,  x2 = L / 8 - 1  with  L = -ln(1 - u),
#   output    y  = network(x1, x2),  ln w-bar = y + ln u,
#   xi = s / (1 + s),  s = 3 chi w-bar^3 / 2  (Eq. subs_altri).
# ln w-bar - ln u tends to a function of chi alone as u -> 0 (I~_pe ~ w, Eq.
# pe_eff_int_approx_w_small) and is smooth in L as u -> 1 (the upper tail falls off as
# exp(-w^3)), so the network sees a smooth function at both ends.
C_CHI = 0.5 * (np.log(1e-3) + np.log(100.0))
S_CHI = 0.5 * (np.log(100.0) - np.log(1e-3))
L_SCALE = 0.125
H = 64
SIZES = [(H, 2), (H, H), (H, H), (1, H)]          # (out, in) of each layer
N_PARAMS = sum(o * i + o for o, i in SIZES)      # 8577


def unpack(theta):
    """Flat parameter vector -> [(W, b)] (W row-major [out, in])."""
    theta = np.asarray(theta, np.float64)
    out, k = [], 0
    for o, i in SIZES:
        W = theta[k:k + o * i].reshape(o, i)
        k += o * i
        b = theta[k:k + o]
        k += o
        out.append((W, b))
    return out


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64.  Values are
    first rounded to binary32, as the GPU holds them."""
    f = np.asarray(x, np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


# the pair-creation kind: chi in [0.1, 100], input u = |r'|, sampler variable ln(-ln y)
# with y = 1 - v-bar; the network output is that variable minus ln u
P_C_CHI = 0.5 * (np.log(0.1) + np.log(100.0))
P_S_CHI = 0.5 * (np.log(100.0) - np.log(0.1))


def features(lnchi, u, kind="photon"):
    u = np.asarray(u, np.float64)
    c, sc = (P_C_CHI, P_S_CHI) if kind == "pair" else (C_CHI, S_CHI)
    return np.stack([(np.asarray(lnchi, np.float64) - c) / sc, -np.log1p(-u) * L_SCALE - 1.0], 1)


def mlp_forward(theta, lnchi, u, quantize=False, keep=False, kind="photon"):
    """The network output y for each (ln chi, u).  With quantize, the weights of every
    layer and the inputs of layers 2-4 are rounded to bfloat16 (layer 1 takes the
    binary32 features), as the inference kernel does; biases stay binary32."""
    layers = unpack(theta)
    a = features(lnchi, u, kind)
    cache = []
    for l, (W, b) in enumerate(layers):
        Wq = bf16(W) if quantize else W
        aq = bf16(a) if (quantize and l > 0) else a
        z = aq @ Wq.T + b
        cache.append((aq, Wq, z))
        a = silu(z) if l < len(layers) - 1 else z
    y = a[:, 0]
    return (y, cache) if keep else y


def surrogate_lnw(theta, lnchi, u, quantize=False):
    """ln w-bar = y + ln u."""
    return mlp_forward(theta, lnchi, u, quantize) + np.log(np.asarray(u, np.float64))


def surrogate_xi(theta, chi, u, quantize=False):
    chi = np.asarray(chi, np.float64)
    s = 1.5 * chi * np.exp(3.0 * surrogate_lnw(theta, np.log(chi), u, quantize))
    return s / (1.0 + s)


def mlp_loss_grad(theta, lnchi, u, target_lnw, quantize=False):
    """Loss = sum_i (ln w_pred,i - ln w_target,i)^2 / n and its gradient in theta; the
    rounding of the forward pass is passed straight through in the backward pass."""
    y, cache = mlp_forward(theta, lnchi, u, quantize=quantize, keep=True)
    n = y.size
    r = y - (np.asarray(target_lnw, np.float64) - np.log(np.asarray(u, np.float64)))
    loss = np.sum(r * r) / n
    d = ((2.0 / n) * r)[:, None]                     # d loss / d z of the last layer
    grads = []
    L = len(cache)
    for l in range(L - 1, -1, -1):
        aq, Wq, z = cache[l]
        if l < L - 1:
            d = d * dsilu(z)
        grads.append((d.T @ aq, d.sum(0)))
        d = d @ Wq                                     # d loss / d (input of layer l)
    grads.reverse()
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat


def surrogate_pair_shares(theta, chi, r, quantize=False):
    """Electron and positron shares of the pair-kind network: ln(-ln y) = network + ln |r'|,
    y = 1 - v-bar (-ln y ~ v-bar ~ |r'| as |r'| -> 0, and y <= 1 for any output)."""
    r = np.asarray(r, np.float64)
    rp = 2.0 * r - 1.0
    a = np.abs(rp)
    y = np.exp(-a * np.exp(mlp_forward(theta, np.log(np.asarray(chi, np.float64)), a, quantize, kind="pair")))
    small, big = 0.5 * y, 1.0 - 0.5 * y
    return np.where(rp >= 0.0, big, small), np.where(rp >= 0.0, small, big)
