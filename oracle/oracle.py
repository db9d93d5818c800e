"""Python access to the FP64 CPU oracle (``sfq_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the CPU-baseline
leg of the benchmark are the only users.  The product path never imports this
module.  The oracle follows the defining formulas of Montefiori & Tamburini,
"SFQEDtoolkit" (arXiv:2301.07684); each C function names the equation it
evaluates.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sfq_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FMA contraction) if stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-Wall", "-Wextra", "-Wno-unused-parameter", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class RunParams(C.Structure):
    _fields_ = [("rho", C.c_double), ("pref", C.c_double), ("dt", C.c_double),
                ("seed", C.c_uint64), ("step0", C.c_uint32), ("nsteps", C.c_uint32),
                ("lepton_mode", C.c_int32), ("step_children", C.c_int32),
                ("near_od", C.c_double), ("near_local", C.c_double), ("near_blcfa", C.c_double),
                ("cascade", C.c_int32), ("reserved", C.c_int32)]


PRODUCT_DTYPE = np.dtype([("p", "<f8", (3,)), ("parent_id", "<u8"), ("step", "<u4"),
                          ("parent_tag", "<u4"), ("species", "<u4"), ("member", "<u4")], align=True)

CASCADE_DTYPE = np.dtype([("p", "<f8", (3,)), ("tau", "<f8"), ("id", "<u8"), ("parent_id", "<u8"),
                          ("root", "<i8"), ("step", "<u4"), ("member", "<u4"), ("flags", "u1"),
                          ("species", "u1"), ("pad", "u1", (6,))], align=True)

_D = C.c_double
_PD = C.POINTER(C.c_double)
_I64 = C.c_int64


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            sig = {
                "orc_rho_from_ref_len": (_D, [_D]),
                "orc_rho_from_ref_freq": (_D, [_D]),
                "orc_rate_prefactor": (_D, [_D]),
                "orc_test_gk15_monomial": (_D, [_D, _D, _D]),
                "orc_test_gauss7_monomial": (_D, [_D, _D, _D]),
                "orc_besselk": (_D, [_D, _D]),
                "orc_besselk_scaled": (_D, [_D, _D]),
                "orc_besselk_int": (_D, [_D, _D]),
                "orc_besselk_int_scaled": (_D, [_D, _D]),
                "orc_wtilde_rad": (_D, [_D]),
                "orc_wtilde_pair": (_D, [_D]),
                "orc_photon_rate": (_D, [_D, _D, _D]),
                "orc_pair_rate": (_D, [_D, _D, _D]),
                "orc_itilde_pe": (_D, [_D, _D]),
                "orc_itilde_pe_upper": (_D, [_D, _D]),
                "orc_itilde_pp": (_D, [_D, _D]),
                "orc_itilde_pp_upper_y": (_D, [_D, _D]),
                "orc_photon_wbar": (_D, [_D, _D]),
                "orc_photon_s": (_D, [_D, _D]),
                "orc_pair_vbar": (None, [_D, _D, _PD, _PD]),
                "orc_pair_shares": (None, [_D, _D, _PD, _PD]),
                "orc_spectrum_pe": (_D, [_D, _D, _D, _D]),
                "orc_spectrum_pp": (_D, [_D, _D, _D, _D]),
                "orc_chi_components": (_D, [_D] * 11),
                "orc_blcfa_threshold": (_D, [_PD, _D, _D, _D]),
                "orc_uniform": (_D, [C.c_uint32]),
                "orc_num_threads": (C.c_int, []),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _f64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


# --- scalar functions -------------------------------------------------------
def rho_from_ref_len(ref_len_m: float) -> float:
    return lib().orc_rho_from_ref_len(ref_len_m)


def rho_from_ref_freq(omega_si: float) -> float:
    return lib().orc_rho_from_ref_freq(omega_si)


def rate_prefactor(rho: float) -> float:
    return lib().orc_rate_prefactor(rho)


def besselk(nu, x):
    return lib().orc_besselk(nu, x)


def besselk_int(nu, x):
    return lib().orc_besselk_int(nu, x)


def itilde_pe(w, chi):
    return lib().orc_itilde_pe(w, chi)


def itilde_pe_upper(w, chi):
    return lib().orc_itilde_pe_upper(w, chi)


def itilde_pp(v, chi):
    return lib().orc_itilde_pp(v, chi)


def itilde_pp_upper_y(y, chi):
    return lib().orc_itilde_pp_upper_y(y, chi)


def spectrum_pe(gg, ge, chi, pref):
    return lib().orc_spectrum_pe(gg, ge, chi, pref)


def spectrum_pp(ge, gg, chi, pref):
    return lib().orc_spectrum_pp(ge, gg, chi, pref)


def chi(gamma, p, E, B, rho):
    return lib().orc_chi_components(gamma, *p, *E, *B, rho)


class BlcfaEval(C.Structure):
    _fields_ = [("F", C.c_double * 3), ("gamma", C.c_double), ("chi", C.c_double),
                ("delta", C.c_double), ("gate", C.c_int)]


def blcfa_update(p, E, B, dt, rho, Fprev, dF, just_created):
    """One beyond-LCFA state update (Sec. 5).  Returns (gate, eval, Fprev', dF', just_created')."""
    L = lib()
    f = L.orc_blcfa_update
    f.restype = C.c_int
    f.argtypes = [_PD, _PD, _PD, _D, _D, _PD, _PD, C.POINTER(C.c_uint8), C.POINTER(BlcfaEval)]
    pa, Ea, Ba = (C.c_double * 3)(*p), (C.c_double * 3)(*E), (C.c_double * 3)(*B)
    fa, da = (C.c_double * 3)(*Fprev), (C.c_double * 3)(*dF)
    jc = C.c_uint8(1 if just_created else 0)
    ev = BlcfaEval()
    g = f(pa, Ea, Ba, dt, rho, fa, da, C.byref(jc), C.byref(ev))
    return g, ev, list(fa), list(da), bool(jc.value)


def blcfa_update_pushed(p, pn, dt, rho, Fprev, dF, just_created):
    """One beyond-LCFA state update with the force from the pusher (Eqs. fl): p = p^(n-1/2),
    pn = its push p_L^(n+1/2).  Returns (gate, eval, Fprev', dF', just_created')."""
    L = lib()
    f = L.orc_blcfa_update_pushed
    f.restype = C.c_int
    f.argtypes = [_PD, _PD, _D, _D, _PD, _PD, C.POINTER(C.c_uint8), C.POINTER(BlcfaEval)]
    pa, na = (C.c_double * 3)(*p), (C.c_double * 3)(*pn)
    fa, da = (C.c_double * 3)(*Fprev), (C.c_double * 3)(*dF)
    jc = C.c_uint8(1 if just_created else 0)
    ev = BlcfaEval()
    g = f(pa, na, dt, rho, fa, da, C.byref(jc), C.byref(ev))
    return g, ev, list(fa), list(da), bool(jc.value)


def blcfa_threshold(F, delta, gamma, chi_):
    Fa = (C.c_double * 3)(*F)
    return lib().orc_blcfa_threshold(Fa, delta, gamma, chi_)


def uniform(word: int) -> float:
    return lib().orc_uniform(word)


def num_threads() -> int:
    return lib().orc_num_threads()


# --- batched functions ------------------------------------------------------
def _batch1(name, x):
    x = _f64(x)
    out = np.empty_like(x)
    getattr(lib(), name)(_I64(x.size), _p(x), _p(out))
    return out


def wtilde_rad(chi):
    return _batch1("orc_batch_wtilde_rad", chi)


def wtilde_pair(chi):
    return _batch1("orc_batch_wtilde_pair", chi)


def photon_rate(gamma, chi, pref):
    g, c = np.broadcast_arrays(_f64(gamma), _f64(chi))
    g, c = _f64(g), _f64(c)
    out = np.empty_like(g)
    lib().orc_batch_photon_rate(_I64(g.size), _p(g), _p(c), _D(pref), _p(out))
    return out


def pair_rate(gamma, chi, pref):
    g, c = np.broadcast_arrays(_f64(gamma), _f64(chi))
    g, c = _f64(g), _f64(c)
    out = np.empty_like(g)
    lib().orc_batch_pair_rate(_I64(g.size), _p(g), _p(c), _D(pref), _p(out))
    return out


def photon_wbar(r, chi):
    r, c = np.broadcast_arrays(_f64(r), _f64(chi))
    r, c = _f64(r), _f64(c)
    out = np.empty_like(r)
    lib().orc_batch_photon_wbar(_I64(r.size), _p(r), _p(c), _p(out))
    return out


def photon_s(r, chi):
    """u = 3 chi w-bar^3 / 2 (Eq. subs_altri); the photon takes xi = s/(1+s) of the lepton
    energy.  The C routine the Monte Carlo step calls (orc_photon_s), batched."""
    r, c = np.broadcast_arrays(_f64(r), _f64(chi))
    r, c = _f64(r), _f64(c)
    out = np.empty_like(r)
    lib().orc_batch_photon_s(_I64(r.size), _p(r), _p(c), _p(out))
    return out


def pair_vbar(a, chi):
    a, c = np.broadcast_arrays(_f64(a), _f64(chi))
    a, c = _f64(a), _f64(c)
    v = np.empty_like(a)
    y = np.empty_like(a)
    lib().orc_batch_pair_vbar(_I64(a.size), _p(a), _p(c), _p(v), _p(y))
    return v, y


def pair_shares(r, chi):
    """Electron and positron energy shares for a uniform r (Eq. return_to_nrg): the C
    routine the Monte Carlo step calls (orc_pair_shares), batched."""
    r, c = np.broadcast_arrays(_f64(r), _f64(chi))
    r, c = _f64(r), _f64(c)
    xe = np.empty_like(r)
    xp = np.empty_like(r)
    lib().orc_batch_pair_shares(_I64(r.size), _p(r), _p(c), _p(xe), _p(xp))
    return xe, xp


def itilde_pe_batch(w, chi):
    w, c = np.broadcast_arrays(_f64(w), _f64(chi))
    w, c = _f64(w), _f64(c)
    out = np.empty_like(w)
    lib().orc_batch_itilde_pe(_I64(w.size), _p(w), _p(c), _p(out))
    return out


def itilde_pe_upper_batch(w, chi):
    w, c = np.broadcast_arrays(_f64(w), _f64(chi))
    w, c = _f64(w), _f64(c)
    out = np.empty_like(w)
    lib().orc_batch_itilde_pe_upper(_I64(w.size), _p(w), _p(c), _p(out))
    return out


def itilde_pp_batch(v, chi):
    """I~_pp(v, chi) (Eq. tilde_I_pp) for arrays."""
    v, c = np.broadcast_arrays(_f64(v), _f64(chi))
    v, c = _f64(v), _f64(c)
    out = np.empty_like(v)
    lib().orc_batch_itilde_pp(_I64(v.size), _p(v), _p(c), _p(out))
    return out


def itilde_pp_upper_y_batch(y, chi):
    """The integral of Eq. tilde_I_pp from 1 - y to 1, integrated in y, for arrays."""
    y, c = np.broadcast_arrays(_f64(y), _f64(chi))
    y, c = _f64(y), _f64(c)
    out = np.empty_like(y)
    lib().orc_batch_itilde_pp_upper_y(_I64(y.size), _p(y), _p(c), _p(out))
    return out


def boris_push(u, E, B, q, dt):
    """Boris push of momenta u (n x 3) in fields E, B (n x 3) for charges q (n; in |e|, 0 for
    photons), normalised units; returns the new momenta."""
    u = np.ascontiguousarray(np.array(u, np.float64).reshape(-1, 3))
    E = np.ascontiguousarray(np.broadcast_to(np.asarray(E, np.float64), u.shape))
    B = np.ascontiguousarray(np.broadcast_to(np.asarray(B, np.float64), u.shape))
    q = np.ascontiguousarray(np.broadcast_to(np.asarray(q, np.float64), (u.shape[0],)))
    lib().orc_batch_boris_push(_I64(u.shape[0]), _p(u), _p(E), _p(B), _p(q), _D(dt))
    return u


def philox(ids, step, tag, seed):
    ids = np.ascontiguousarray(np.asarray(ids, dtype=np.uint64))
    out = np.empty((ids.size, 4), dtype=np.uint32)
    lib().orc_batch_philox(_I64(ids.size), _p(ids), C.c_uint32(step), C.c_uint32(tag),
                           C.c_uint64(seed), _p(out))
    return out


def uniforms_from_words(words):
    """The same map as ``orc_uniform``, vectorised (for tests only)."""
    w = np.asarray(words, dtype=np.uint32)
    return ((w >> np.uint32(9)).astype(np.float64) + 0.5) * 2.0 ** -23


# --- Monte Carlo ------------------------------------------------------------
SP_ELECTRON, SP_POSITRON, SP_PHOTON = 0, 1, 2
FL_ALIVE, FL_JUST_CREATED = 1, 2
MODE_LCFA_OD, MODE_BLCFA_LOCAL, MODE_BLCFA_PUSHED = 0, 1, 2


def mc_run(p, tau, ids, flags, species, fields, *, rho, dt, seed, step0=0, nsteps,
           tag=None, fprev=None, dfprev=None, lepton_mode=MODE_LCFA_OD, step_children=False,
           near_od=1e-6, near_local=1e-6, near_blcfa=1e-4, cap_products=None):
    """Advance independent primaries through ``nsteps`` Monte Carlo steps.

    ``fields`` has shape (n, nsteps, 6): (Ex, Ey, Ez, Bx, By, Bz) seen by each
    primary at each step (children see their primary's field).  Returns a dict
    with the updated state, the products and per-primary lineage info.
    """
    L = lib()
    n = len(ids)
    p = np.ascontiguousarray(np.array(p, dtype=np.float64).reshape(n, 3))
    tau = np.ascontiguousarray(np.array(tau, dtype=np.float64).reshape(n))
    ids = np.ascontiguousarray(np.asarray(ids, dtype=np.uint64))
    flags = np.ascontiguousarray(np.array(flags, dtype=np.uint8))
    species = np.ascontiguousarray(np.asarray(species, dtype=np.uint8))
    fields = np.ascontiguousarray(np.asarray(fields, dtype=np.float64).reshape(n, nsteps, 6))
    tagp = None
    if tag is not None:
        tag = np.ascontiguousarray(np.asarray(tag, dtype=np.uint32))
        tagp = _p(tag)
    fp = dfp = None
    if fprev is not None:
        fprev = np.ascontiguousarray(np.array(fprev, dtype=np.float64).reshape(n, 3))
        dfprev = np.ascontiguousarray(np.array(dfprev, dtype=np.float64).reshape(n, 3))
        fp, dfp = _p(fprev), _p(dfprev)
    if cap_products is None:
        cap_products = max(64, 4 * n * max(1, nsteps // 4))
    prod = np.zeros(cap_products, dtype=PRODUCT_DTYPE)
    nprod = C.c_int64(0)
    first_near = np.empty(n, dtype=np.int32)
    stats = np.empty((n, 4), dtype=np.int32)
    P = RunParams(rho=rho, pref=rate_prefactor(rho), dt=dt, seed=seed, step0=step0, nsteps=nsteps,
                  lepton_mode=lepton_mode, step_children=int(step_children), near_od=near_od,
                  near_local=near_local, near_blcfa=near_blcfa)
    f = L.orc_mc_run
    f.restype = C.c_int
    f.argtypes = [_I64] + [C.c_void_p] * 9 + [C.POINTER(RunParams), C.c_void_p, _I64,
                                               C.POINTER(C.c_int64), C.c_void_p, C.c_void_p]
    f(_I64(n), _p(p), _p(tau), _p(ids), tagp, _p(flags), _p(species), fp, dfp, _p(fields),
      C.byref(P), _p(prod), _I64(cap_products), C.byref(nprod), _p(first_near), _p(stats))
    k = nprod.value
    if k > cap_products:
        raise RuntimeError(f"oracle product capacity {cap_products} < {k}")
    return dict(p=p, tau=tau, flags=flags, fprev=fprev, dfprev=dfprev, products=prod[:k].copy(),
                first_near_step=first_near, **_lineage_stats(stats))


def _lineage_stats(stats):
    """Per-lineage counts: events, beyond-LCFA events whose gate held, events stopped by the
    0.75 gamma_e rule, samples rejected by Eq. rej_cond."""
    return dict(n_events=stats[:, 0].copy(), n_gated=stats[:, 1].copy(), n_no_emission=stats[:, 2].copy(),
                n_rejected=stats[:, 3].copy())


def child_id(seed, parent, parent_tag, step, member):
    """Id of a particle created in a full cascade (orc_child_id): bit 63 set over the first
    two Philox words of the counter (parent id, step, 0x100 | parent tag << 2 | member)."""
    f = lib().orc_child_id
    f.restype = C.c_uint64
    f.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32]
    return int(f(int(seed), int(parent), int(parent_tag), int(step), int(member)))


def mc_cascade(p, tau, ids, flags, species, fields, *, rho, dt, seed, step0=0, nsteps,
               fprev=None, dfprev=None, lepton_mode=MODE_LCFA_OD, near_od=1e-6, near_local=1e-6,
               near_blcfa=1e-4, cap_products=None, cap_out=None):
    """Full cascade of independent primaries (orc_mc_cascade): every product is also a
    particle, stepped from the next step on in its primary's field.  ``fields`` has shape
    (n, nsteps, 6).  Returns the primaries' final state, the product records, every created
    particle (CASCADE_DTYPE) and per-primary lineage info."""
    L = lib()
    n = len(ids)
    p = np.ascontiguousarray(np.array(p, dtype=np.float64).reshape(n, 3))
    tau = np.ascontiguousarray(np.array(tau, dtype=np.float64).reshape(n))
    ids = np.ascontiguousarray(np.asarray(ids, dtype=np.uint64))
    flags = np.ascontiguousarray(np.array(flags, dtype=np.uint8))
    species = np.ascontiguousarray(np.asarray(species, dtype=np.uint8))
    fields = np.ascontiguousarray(np.asarray(fields, dtype=np.float64).reshape(n, nsteps, 6))
    fp = dfp = None
    if fprev is not None:
        fprev = np.ascontiguousarray(np.array(fprev, dtype=np.float64).reshape(n, 3))
        dfprev = np.ascontiguousarray(np.array(dfprev, dtype=np.float64).reshape(n, 3))
        fp, dfp = _p(fprev), _p(dfprev)
    for _ in range(2):
        cp = cap_products if cap_products is not None else max(256, 16 * n * nsteps)
        co = cap_out if cap_out is not None else max(256, 16 * n * nsteps)
        prod = np.zeros(cp, dtype=PRODUCT_DTYPE)
        out = np.zeros(co, dtype=CASCADE_DTYPE)
        nprod, nout = C.c_int64(0), C.c_int64(0)
        first_near = np.empty(n, dtype=np.int32)
        stats = np.empty((n, 4), dtype=np.int32)
        P = RunParams(rho=rho, pref=rate_prefactor(rho), dt=dt, seed=seed, step0=step0, nsteps=nsteps,
                      lepton_mode=lepton_mode, step_children=1, near_od=near_od, near_local=near_local,
                      near_blcfa=near_blcfa, cascade=1, reserved=0)
        f = L.orc_mc_cascade
        f.restype = C.c_int
        f.argtypes = [_I64] + [C.c_void_p] * 8 + [C.POINTER(RunParams), C.c_void_p, _I64, C.POINTER(C.c_int64),
                                                  C.c_void_p, _I64, C.POINTER(C.c_int64), C.c_void_p, C.c_void_p]
        p1, tau1, fl1 = p.copy(), tau.copy(), flags.copy()
        fp1 = fprev.copy() if fprev is not None else None
        dfp1 = dfprev.copy() if dfprev is not None else None
        rc = f(_I64(n), _p(p1), _p(tau1), _p(ids), _p(fl1), _p(species),
               _p(fp1) if fp1 is not None else None, _p(dfp1) if dfp1 is not None else None, _p(fields),
               C.byref(P), _p(prod), _I64(cp), C.byref(nprod), _p(out), _I64(co), C.byref(nout),
               _p(first_near), _p(stats))
        if rc != 0:
            raise RuntimeError("orc_mc_cascade failed")
        if nprod.value <= cp and nout.value <= co:
            break
        cap_products, cap_out = 2 * max(cp, nprod.value), 2 * max(co, nout.value)
    return dict(p=p1, tau=tau1, flags=fl1, fprev=fp1, dfprev=dfp1, products=prod[:nprod.value].copy(),
                particles=out[:nout.value].copy(), first_near_step=first_near, **_lineage_stats(stats))

