"""Piecewise tensor-Chebyshev fits and their monomial (Horner) form.

A fitted function is split into pieces whose index comes from the binary
exponent and the top mantissa bits of its arguments, so that on the GPU the
piece index and the local variable in [-1, 1] are computed exactly with a few
integer operations.  Inside a piece the function is interpolated at Chebyshev
points of the first kind, and the Chebyshev series is converted exactly (in
rational arithmetic) to monomials in the local variable, then rounded once to
the table's precision.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from fractions import Fraction

import numpy as np
from numpy.polynomial import chebyshev as npcheb


# ---------------------------------------------------------------------------
# one axis: pieces by exponent
@dataclass
class Axis:
    """Piece layout along one variable.

    kind "octave":   value in [2^e_lo, 2^e_hi) split into octaves, each into 2^sub
                     equal sub-pieces; below 2^e_lo a "low" block [0, 2^e_lo) of
                     2^sub_low equal pieces (if low=True).
    kind "prob":     a uniform number in (0, 1): low block [0, 2^e0) (2^sub_low
                     pieces), octaves of r in [2^e0, 1/2) (2^sub each), then
                     octaves of q = 1 - r in [2^q_lo, 1/2] (2^sub_q each), the
                     last one closed at q = 1/2.
    """
    kind: str
    e_lo: int = 0
    e_hi: int = 0
    sub: int = 0
    low: bool = True
    sub_low: int = 0
    q_lo: int = -24
    sub_q: int = 0

    # list of (lo, hi, var) with var in {"x", "q"}: the interval in the natural
    # variable of the piece (x = value itself, q = 1 - r)
    def pieces(self):
        out = []
        if self.kind == "octave":
            if self.low:
                n = 1 << self.sub_low
                for j in range(n):
                    out.append((2.0 ** self.e_lo * j / n, 2.0 ** self.e_lo * (j + 1) / n, "x"))
            for e in range(self.e_lo, self.e_hi):
                n = 1 << self.sub
                for j in range(n):
                    out.append((2.0 ** e * (1 + j / n), 2.0 ** e * (1 + (j + 1) / n), "x"))
        elif self.kind == "prob":
            n = 1 << self.sub_low
            for j in range(n):
                out.append((2.0 ** self.e_lo * j / n, 2.0 ** self.e_lo * (j + 1) / n, "x"))
            for e in range(self.e_lo, -1):
                n = 1 << self.sub
                for j in range(n):
                    out.append((2.0 ** e * (1 + j / n), 2.0 ** e * (1 + (j + 1) / n), "x"))
            # q-octaves from the top (q in [1/4, 1/2]) down to [2^q_lo, 2^(q_lo+1))
            for e in range(-2, self.q_lo - 1, -1):
                n = 1 << self.sub_q
                for j in range(n):
                    out.append((2.0 ** e * (1 + j / n), 2.0 ** e * (1 + (j + 1) / n), "q"))
        else:
            raise ValueError(self.kind)
        return out

    def n_pieces(self):
        return len(self.pieces())


def cheb_nodes(d: int) -> np.ndarray:
    k = np.arange(d + 1)
    return np.cos((2 * k + 1) * np.pi / (2 * (d + 1)))


def _cheb_to_mono_exact(c: np.ndarray) -> list:
    """Monomial coefficients (as Fractions) of sum_k c_k T_k(x)."""
    n = len(c)
    # T_k as exact integer coefficient lists
    T = [[1], [0, 1]]
    for k in range(2, n):
        a = [0] + [2 * t for t in T[k - 1]]
        b = T[k - 2] + [0] * (len(a) - len(T[k - 2]))
        T.append([x - y for x, y in zip(a, b)])
    out = [Fraction(0)] * n
    for k in range(n):
        ck = Fraction(float(c[k]))
        for i, t in enumerate(T[k]):
            if t:
                out[i] += ck * t
    return out


def cheb2d_to_mono(C: np.ndarray) -> np.ndarray:
    """C[i, j] Chebyshev (x^i-degree i in T_i(x), j in T_j(y)) -> monomial a[i, j] (float64)."""
    dx, dy = C.shape
    # convert along y first (exact), then along x (exact)
    rows = [_cheb_to_mono_exact(C[i, :]) for i in range(dx)]          # rows[i][j] Fractions
    out = np.empty((dx, dy))
    Tx = _cheb_to_mono_exact.__wrapped__ if hasattr(_cheb_to_mono_exact, "__wrapped__") else None
    # monomial in x of sum_i rows[i][j] T_i(x): reuse the exact converter on Fractions
    T = [[1], [0, 1]]
    for k in range(2, dx):
        a = [0] + [2 * t for t in T[k - 1]]
        b = T[k - 2] + [0] * (len(a) - len(T[k - 2]))
        T.append([x - y for x, y in zip(a, b)])
    for j in range(dy):
        acc = [Fraction(0)] * dx
        for i in range(dx):
            cij = rows[i][j]
            for p, t in enumerate(T[i]):
                if t:
                    acc[p] += cij * t
        for p in range(dx):
            out[p, j] = float(acc[p])
    return out


def cheb1d_to_mono(c: np.ndarray) -> np.ndarray:
    return np.array([float(v) for v in _cheb_to_mono_exact(c)])


def cheb_coeffs_1d(vals: np.ndarray) -> np.ndarray:
    d = len(vals) - 1
    V = npcheb.chebvander(cheb_nodes(d), d)
    return np.linalg.solve(V, vals)


def cheb_coeffs_2d(vals: np.ndarray) -> np.ndarray:
    """vals[i, j] at (x-node i, y-node j) -> Chebyshev coefficients C[p, q]."""
    dx, dy = vals.shape[0] - 1, vals.shape[1] - 1
    Vx = npcheb.chebvander(cheb_nodes(dx), dx)
    Vy = npcheb.chebvander(cheb_nodes(dy), dy)
    A = np.linalg.solve(Vx, vals)              # along x
    return np.linalg.solve(Vy, A.T).T          # along y


def horner1d(a: np.ndarray, x):
    r = np.zeros_like(np.asarray(x, dtype=np.float64)) + a[-1]
    for k in range(len(a) - 2, -1, -1):
        r = r * x + a[k]
    return r


def horner2d(a: np.ndarray, x, y):
    """sum_ij a[i, j] x^i y^j, Horner in y for each i, then in x (the kernels' order)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    acc = None
    for i in range(a.shape[0] - 1, -1, -1):
        b = horner1d(a[i], y)
        acc = b if acc is None else acc * x + b
    return acc


def local(lo, hi, v):
    return 2.0 * (v - lo) / (hi - lo) - 1.0
