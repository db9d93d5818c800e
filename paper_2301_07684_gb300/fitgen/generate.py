"""Generate the kernels' approximation tables (``csrc/sfq_tables.inc``).

    python -m paper_2301_07684_gb300.fitgen.generate [--check]

Four fitted functions, each in an FP32 and an FP64 variant:
  nlc_rate  W~_rad(chi)                          Eq. wtilde            1D in chi
  nbw_rate  h(chi) = W~_pair(chi) e^{8/(3chi)}/chi   Eq. wtilde_pair   1D in chi
  nlc_inv   w-bar(r, chi) (w-bar/r in the low-r block)   Eq. again     2D
  nbw_inv   y-bar(a, chi) = 1 - v-bar, a = |r'|          Eq. again_pp  2D
(Montefiori & Tamburini, arXiv:2301.07684, Secs. 4.1-4.4).  Values come from
this package's own quadrature (``quad``, ``cdf``), never from the test oracle.
"""
from __future__ import annotations

import argparse
import os
import sys
import time
from dataclasses import dataclass

import numpy as np

from . import cdf as CDF
from . import fit as FIT
from . import quad as Q

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(os.path.dirname(HERE), "csrc", "sfq_tables.inc")            # arrays (host TU only)
OUT_LAYOUT = os.path.join(os.path.dirname(HERE), "csrc", "sfq_tables_layout.h")  # layout constants


@dataclass
class Table1D:
    name: str
    axis: FIT.Axis
    deg: int
    target: float
    coef: np.ndarray = None      # (pieces, deg+1) monomial
    err: float = 0.0


@dataclass
class Table2D:
    name: str
    xaxis: FIT.Axis              # chi
    yaxis: FIT.Axis              # probability variable
    dx: int
    dy: int
    target: float
    coef: np.ndarray = None      # (xpieces, ypieces, dx+1, dy+1)
    err: float = 0.0


# --- the functions --------------------------------------------------------------
def f_nlc_rate(chi):
    return Q.wtilde_rad(chi)


def f_k23(x):
    """x^{2/3} e^x K_2/3(x): bounded, -> 2^{-1/3} Gamma(2/3) as x -> 0."""
    x = np.asarray(x, dtype=np.float64)
    return x ** (2.0 / 3.0) * Q.besselk_scaled(2.0 / 3.0, x)


def f_ki13(x):
    """e^x Ki_1/3(x), Ki_1/3(x) = int_x^inf K_1/3: -> pi/sqrt(3) as x -> 0."""
    x = np.asarray(x, dtype=np.float64)
    return Q.besselk_int_scaled(1.0 / 3.0, x)


def f_nbw_rate(chi):
    chi = np.asarray(chi, dtype=np.float64)
    return Q.wtilde_pair(chi) * np.exp(8.0 / (3.0 * chi)) / chi


class _CDFCache:
    def __init__(self, make):
        self.make, self.d = make, {}

    def __call__(self, chi):
        k = float(chi)
        if k not in self.d:
            self.d[k] = self.make(k)
        return self.d[k]


_photon = _CDFCache(CDF.PhotonCDF)
_pair = _CDFCache(CDF.PairCDF)


def inv_nlc(chi, lo, hi, var, ys):
    """Fit target of the photon inverse at one chi for points ys of one r-piece."""
    c = _photon(chi)
    if var == "q":
        return c.p.invert_upper(ys * c.W)                  # y is q = 1 - r
    w = c.p.invert_lower(ys * c.W)
    if lo == 0.0:
        return w / ys                                      # low block: w-bar / r
    return w


def inv_nbw(chi, lo, hi, var, ys):
    c = _pair(chi)
    a = 1.0 - ys if var == "q" else ys
    if var == "q":
        # y-bar from the complementary target (1 - a) W = q W, without forming a
        v = np.empty_like(ys)
        y = np.empty_like(ys)
        tgt = ys * c.W
        in_z = tgt < c.pz.total
        z = c.pz.invert_lower(tgt[in_z])
        y[in_z] = z ** 3
        mid = ~in_z
        vm = c.pv.invert_upper(tgt[mid] - c.pz.total)
        y[mid] = 1.0 - vm
        return y
    v, y = c.vbar_ybar(a)
    return y


# --- fitting ----------------------------------------------------------------------
def fit_1d(t: Table1D, f, rng):
    pcs = t.axis.pieces()
    nodes = FIT.cheb_nodes(t.deg)
    xs = np.array([lo + (nodes + 1) / 2 * (hi - lo) for lo, hi, _ in pcs])
    vals = f(xs.ravel()).reshape(xs.shape)
    coef = np.array([FIT.cheb1d_to_mono(FIT.cheb_coeffs_1d(v)) for v in vals])
    # verification at fresh points
    xt = np.array([rng.uniform(lo, hi, 24) for lo, hi, _ in pcs])
    ref = f(xt.ravel()).reshape(xt.shape)
    app = np.array([FIT.horner1d(coef[i], FIT.local(lo, hi, xt[i])) for i, (lo, hi, _) in enumerate(pcs)])
    t.coef, t.err = coef, float(np.max(np.abs(app / ref - 1)))
    return t


def fit_2d(t: Table2D, finv, rng, verbose=False):
    xp, yp = t.xaxis.pieces(), t.yaxis.pieces()
    nx, ny = FIT.cheb_nodes(t.dx), FIT.cheb_nodes(t.dy)
    coef = np.empty((len(xp), len(yp), t.dx + 1, t.dy + 1))
    err = 0.0
    for ix, (xlo, xhi, _) in enumerate(xp):
        chis = xlo + (nx + 1) / 2 * (xhi - xlo)
        vals = np.empty((len(yp), t.dx + 1, t.dy + 1))
        for i, chi in enumerate(chis):
            for iy, (ylo, yhi, var) in enumerate(yp):
                ys = ylo + (ny + 1) / 2 * (yhi - ylo)
                vals[iy, i, :] = finv(chi, ylo, yhi, var, ys)
        for iy in range(len(yp)):
            coef[ix, iy] = FIT.cheb2d_to_mono(FIT.cheb_coeffs_2d(vals[iy]))
        # verification: fresh chi and y values
        for chi in rng.uniform(xlo, xhi, 2):
            xl = FIT.local(xlo, xhi, chi)
            for iy, (ylo, yhi, var) in enumerate(yp):
                ys = rng.uniform(ylo, yhi, 6)
                if ylo == 0.0:
                    ys[0] = ylo + 1e-3 * (yhi - ylo)
                ref = finv(chi, ylo, yhi, var, ys)
                app = FIT.horner2d(coef[ix, iy], xl, FIT.local(ylo, yhi, ys))
                e = float(np.max(np.abs(app / ref - 1)))
                err = max(err, e)
        if verbose:
            print(f"  {t.name} chi-piece {ix}/{len(xp)} [{xlo:.4g},{xhi:.4g}) err so far {err:.2e}", flush=True)
    t.coef, t.err = coef, err
    return t


# --- layouts ------------------------------------------------------------------------
def layouts():
    """(tables, precision) with the layout chosen for each."""
    L = {}
    # rates: chi up to 2^20; NLC from 0 with a low block, NBW from 2^-7
    L["nlc_rate_f64"] = Table1D("nlc_rate_f64", FIT.Axis("octave", e_lo=-10, e_hi=20, sub=1, low=True, sub_low=0), 10, 5e-12)
    L["nlc_rate_f32"] = Table1D("nlc_rate_f32", FIT.Axis("octave", e_lo=-10, e_hi=20, sub=0, low=True, sub_low=0), 8, 5e-8)
    L["nbw_rate_f64"] = Table1D("nbw_rate_f64", FIT.Axis("octave", e_lo=-7, e_hi=20, sub=1, low=False), 10, 5e-12)
    L["nbw_rate_f32"] = Table1D("nbw_rate_f32", FIT.Axis("octave", e_lo=-7, e_hi=20, sub=0, low=False), 8, 5e-8)
    # special functions of the spectrum Eq. pe_dp (beyond-LCFA rejection, Eq. rej_cond):
    # x = 2u/(3 chi) in [2^-64, 2^12), octaves in x
    L["k23_f64"] = Table1D("k23_f64", FIT.Axis("octave", e_lo=-64, e_hi=12, sub=1, low=False), 9, 5e-12)
    L["k23_f32"] = Table1D("k23_f32", FIT.Axis("octave", e_lo=-64, e_hi=12, sub=0, low=False), 8, 5e-8)
    L["ki13_f64"] = Table1D("ki13_f64", FIT.Axis("octave", e_lo=-64, e_hi=12, sub=1, low=False), 10, 5e-12)
    L["ki13_f32"] = Table1D("ki13_f32", FIT.Axis("octave", e_lo=-64, e_hi=12, sub=0, low=False), 9, 5e-8)
    # inverses: chi up to 2^12 (the paper's domain ends at 2000)
    L["nlc_inv_f64"] = Table2D("nlc_inv_f64", FIT.Axis("octave", e_lo=-10, e_hi=12, sub=1, low=True, sub_low=0),
                               FIT.Axis("prob", e_lo=-6, sub=1, sub_low=0, q_lo=-24, sub_q=1), 11, 11, 5e-12)
    L["nlc_inv_f32"] = Table2D("nlc_inv_f32", FIT.Axis("octave", e_lo=-10, e_hi=12, sub=0, low=True, sub_low=0),
                               FIT.Axis("prob", e_lo=-6, sub=0, sub_low=0, q_lo=-24, sub_q=0), 8, 8, 3e-7)
    L["nbw_inv_f64"] = Table2D("nbw_inv_f64", FIT.Axis("octave", e_lo=-7, e_hi=12, sub=1, low=False),
                               FIT.Axis("prob", e_lo=-6, sub=1, sub_low=0, q_lo=-23, sub_q=1), 11, 11, 5e-12)
    L["nbw_inv_f32"] = Table2D("nbw_inv_f32", FIT.Axis("octave", e_lo=-7, e_hi=12, sub=0, low=False),
                               FIT.Axis("prob", e_lo=-6, sub=0, sub_low=0, q_lo=-23, sub_q=0), 8, 8, 3e-7)
    return L


# --- emission ------------------------------------------------------------------------
def _axis_defines(prefix, a: FIT.Axis):
    out = [f"#define {prefix}_ELO {a.e_lo}", f"#define {prefix}_EHI {a.e_hi}", f"#define {prefix}_SUB {a.sub}",
           f"#define {prefix}_LOW {1 if (a.low or a.kind == 'prob') else 0}", f"#define {prefix}_SUBLOW {a.sub_low}",
           f"#define {prefix}_NPIECES {a.n_pieces()}"]
    if a.kind == "prob":
        out += [f"#define {prefix}_QLO {a.q_lo}", f"#define {prefix}_SUBQ {a.sub_q}"]
    return out


def _fmt(v, f32):
    if f32:
        return f"{float(np.float32(v)).hex()}f".replace("0x", "0x")
    return float(v).hex()


def emit(tables, path=OUT, layout_path=OUT_LAYOUT):
    head = ["// Generated by paper_2301_07684_gb300/fitgen/generate.py -- do not edit.",
            "// Piecewise monomial (Horner) coefficients in the local variable of each piece;",
            "// see the generator for the layout and the fitted functions.", ""]
    lay = ["#pragma once"] + head
    dat = list(head)
    for t in tables.values():
        f32 = t.name.endswith("f32")
        P = t.name.upper()
        lay.append(f"// {t.name}: max relative fit error {t.err:.3e} (target {t.target:.1e})")
        if isinstance(t, Table1D):
            lay += _axis_defines(f"{P}_X", t.axis)
            lay.append(f"#define {P}_DEG {t.deg}")
        else:
            lay += _axis_defines(f"{P}_X", t.xaxis)
            lay += _axis_defines(f"{P}_Y", t.yaxis)
            lay.append(f"#define {P}_DX {t.dx}")
            lay.append(f"#define {P}_DY {t.dy}")
        vals = t.coef.ravel()
        lay.append(f"#define {P}_COUNT {vals.size}")
        lay.append(f"#define {P}_ERR {t.err:.3e}")
        lay.append("")
        ty = "float" if f32 else "double"
        dat.append(f"static const {ty} {t.name}[{vals.size}] = {{")
        row = []
        for v in vals:
            row.append(_fmt(v, f32))
            if len(row) == 4:
                dat.append("  " + ", ".join(row) + ",")
                row = []
        if row:
            dat.append("  " + ", ".join(row) + ",")
        dat.append("};")
        dat.append("")
    for pth, lines in ((path, dat), (layout_path, lay)):
        tmp = pth + ".tmp"
        with open(tmp, "w") as fh:
            fh.write("\n".join(lines) + "\n")
        os.replace(tmp, pth)


CACHE = os.path.join(os.path.dirname(os.path.dirname(HERE)), "_build", "fitgen_cache.npz")


def _load_cache():
    if os.path.exists(CACHE):
        z = np.load(CACHE, allow_pickle=False)
        return {k: z[k] for k in z.files}
    return {}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", nargs="*", default=None)
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--out", default=OUT)
    args = ap.parse_args(argv)
    rng = np.random.default_rng(20230118)
    tables = layouts()
    cache = _load_cache()
    for name, t in tables.items():
        if args.only and name not in args.only:
            if name in cache:               # reuse a previous fit of the same layout
                t.coef = cache[name]
                t.err = float(cache[name + "__err"])
            continue
        t0 = time.time()
        if isinstance(t, Table1D):
            fn = {"nlc": f_nlc_rate, "nbw": f_nbw_rate, "k23": f_k23, "ki1": f_ki13}[name[:3]]
            fit_1d(t, fn, rng)
        else:
            fit_2d(t, inv_nlc if name.startswith("nlc") else inv_nbw, rng, verbose=args.verbose)
        ok = "ok" if t.err <= t.target else "ABOVE TARGET"
        print(f"{name}: err {t.err:.3e} target {t.target:.1e} {ok} ({time.time() - t0:.1f}s)", flush=True)
        cache[name] = t.coef
        cache[name + "__err"] = np.array(t.err)
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    np.savez(CACHE, **cache)
    if all(t.coef is not None for t in tables.values()):
        emit(tables, args.out)
        print("wrote", args.out)
    else:
        print("not all tables fitted; nothing emitted")


if __name__ == "__main__":
    main()
