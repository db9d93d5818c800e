"""ctypes binding of libsfq (include/sfq.h) for PyTorch tensors.

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  Tensors must be CUDA, contiguous and of the context's precision
(float32 for SFQ_FP32, float64 for SFQ_FP64; the optical depth is float64).
Work is enqueued on the current torch stream.  When libsfq.so is missing the
import of this module fails: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("SFQ_LIB", os.path.join(_PKG, "libsfq.so"))

SFQ_FP32, SFQ_FP64 = 0, 1
SFQ_ALIVE, SFQ_JUST_CREATED = 1, 2
SFQ_SPECIES_SHIFT, SFQ_TAG_SHIFT = 2, 4
SFQ_ELECTRON, SFQ_POSITRON, SFQ_PHOTON = 0, 1, 2
SFQ_LEPTON_LCFA_OD, SFQ_LEPTON_BLCFA_LOCAL, SFQ_LEPTON_BLCFA_PUSHED = 0, 1, 2
SFQ_FIELDS_SOA, SFQ_FIELDS_PLANE_WAVE = 0, 1
SFQ_EVAL_HORNER, SFQ_EVAL_CLENSHAW = 0, 1
STATUS = {0: "SFQ_OK", 1: "SFQ_ERR_ARG", 2: "SFQ_ERR_CUDA", 3: "SFQ_ERR_CAPACITY", 4: "SFQ_ERR_TABLE",
          5: "SFQ_ERR_RANGE", 6: "SFQ_ERR_TIMEOUT"}
COUNTER_NAMES = ["updates", "events", "emitted", "pairs", "dropped", "spawn_dropped", "out_of_range",
                 "nan_input", "gamma_below_one", "large_rdt", "blcfa_no_emission", "blcfa_rejected", "timeouts",
                 "surrogate_fallbacks"]


class Config(C.Structure):
    _fields_ = [("ref_len_m", C.c_double), ("ref_omega_si", C.c_double), ("dt", C.c_double),
                ("precision", C.c_int32), ("device", C.c_int32), ("seed", C.c_uint64)]


class Particles(C.Structure):
    _fields_ = [("n", C.c_int64), ("px", C.c_void_p), ("py", C.c_void_p), ("pz", C.c_void_p),
                ("tau", C.c_void_p), ("id", C.c_void_p), ("id_base", C.c_uint64), ("flags", C.c_void_p),
                ("fprev", C.c_void_p * 3), ("dfprev", C.c_void_p * 3), ("lepton_model", C.c_int32),
                ("reserved", C.c_int32), ("n_dev", C.c_void_p)]


class Fields(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("ex", C.c_void_p), ("ey", C.c_void_p),
                ("ez", C.c_void_p), ("bx", C.c_void_p), ("by", C.c_void_p), ("bz", C.c_void_p),
                ("k0", C.c_void_p), ("amp", C.c_void_p), ("amp0", C.c_double), ("table", C.c_void_p),
                ("n_table", C.c_uint32), ("k_step", C.c_uint32)]


class Products(C.Structure):
    _fields_ = [("capacity", C.c_int64), ("px", C.c_void_p), ("py", C.c_void_p), ("pz", C.c_void_p),
                ("parent_id", C.c_void_p), ("step", C.c_void_p), ("meta", C.c_void_p), ("count", C.c_void_p)]


class Spawn(C.Structure):
    _fields_ = [("p", Particles), ("k0", C.c_void_p), ("amp", C.c_void_p), ("count", C.c_void_p)]


class EventQueueDesc(C.Structure):
    _fields_ = [("capacity", C.c_int64), ("index", C.c_void_p), ("chi", C.c_void_p), ("r", C.c_void_p),
                ("gamma", C.c_void_p), ("px", C.c_void_p), ("py", C.c_void_p), ("pz", C.c_void_p),
                ("xi", C.c_void_p), ("count", C.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2301_07684_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, i64, u32, st = C.c_void_p, C.c_int64, C.c_uint32, C.c_int
        L.sfq_init.argtypes = [C.POINTER(Config), C.POINTER(vp)]
        L.sfq_init.restype = st
        L.sfq_finalize.argtypes = [vp]
        L.sfq_finalize.restype = None
        L.sfq_last_error.argtypes = [vp]
        L.sfq_last_error.restype = C.c_char_p
        L.sfq_constants.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.sfq_constants.restype = st
        for name in ("sfq_photon_rate", "sfq_pair_rate"):
            getattr(L, name).argtypes = [vp, i64, vp, vp, vp, vp, vp]
            getattr(L, name).restype = st
        L.sfq_uniforms.argtypes = [vp, i64, vp, u32, u32, vp, vp]
        L.sfq_uniforms.restype = st
        for name in ("sfq_sample_photon_xi", "sfq_sample_pair_xi"):
            getattr(L, name).argtypes = [vp, i64, vp, vp, vp, vp, vp, vp]
            getattr(L, name).restype = st
        L.sfq_mc_step.argtypes = [vp, C.POINTER(Particles), C.POINTER(Fields), u32, C.POINTER(Products),
                                  C.POINTER(Spawn), vp, vp]
        L.sfq_mc_step.restype = st
        L.sfq_mc_run.argtypes = [vp, C.POINTER(Particles), C.POINTER(Fields), C.POINTER(Particles),
                                 C.POINTER(Fields), u32, u32, C.POINTER(Products), C.POINTER(Spawn), vp, vp]
        L.sfq_mc_run.restype = st
        L.sfq_mc_run_fused.argtypes = [vp, C.POINTER(Particles), C.POINTER(Fields), C.c_uint32, C.c_uint32,
                                       C.POINTER(Products), vp, vp]
        L.sfq_mc_run_fused.restype = st
        L.sfq_push.argtypes = [vp, C.POINTER(Particles), C.POINTER(Fields), C.c_uint32, C.c_double, vp]
        L.sfq_push.restype = st
        L.sfq_set_pair_rate_cutoff.argtypes = [vp, C.c_double]
        L.sfq_set_pair_rate_cutoff.restype = st
        L.sfq_set_sampler_coefficients.argtypes = [vp, C.c_int32]
        L.sfq_set_sampler_coefficients.restype = st
        L.sfq_sampler_coefficients.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        L.sfq_sampler_coefficients.restype = st
        L.sfq_autotune_step.argtypes = [vp, C.POINTER(Particles), C.POINTER(Fields), u32, i64,
                                        C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_double), vp]
        L.sfq_autotune_step.restype = st
        L.sfq_sort_scratch_bytes.argtypes = [i64]
        L.sfq_sort_scratch_bytes.restype = C.c_size_t
        L.sfq_sort_products.argtypes = [vp, C.POINTER(Products), i64, vp, C.c_size_t, vp]
        L.sfq_sort_products.restype = st
        L.sfq_sort_products_noalloc.argtypes = [vp, C.POINTER(Products), i64, vp]
        L.sfq_sort_products_noalloc.restype = st
        L.sfq_mlp_num_params.restype = C.c_int32
        L.sfq_mlp_create.argtypes = [vp, C.c_uint64, C.POINTER(vp)]
        L.sfq_mlp_create.restype = st
        L.sfq_mlp_destroy.argtypes = [vp]
        L.sfq_mlp_destroy.restype = None
        for name in ("sfq_mlp_get_params", "sfq_mlp_set_params"):
            getattr(L, name).argtypes = [vp, vp]
            getattr(L, name).restype = st
        L.sfq_mlp_loss_grad.argtypes = [vp, i64, vp, vp, vp, C.c_int32, vp, vp, vp]
        L.sfq_mlp_loss_grad.restype = st
        L.sfq_mlp_train.argtypes = [vp, i64, vp, vp, vp, i64, C.c_int32, C.c_float, C.c_int32, C.c_uint64, vp, vp]
        L.sfq_mlp_train.restype = st
        L.sfq_mlp_predict_lnw.argtypes = [vp, i64, vp, vp, vp, vp]
        L.sfq_mlp_predict_lnw.restype = st
        L.sfq_mlp_plain_targets.argtypes = [vp, i64, vp, vp, vp, vp]
        L.sfq_mlp_plain_targets.restype = st
        L.sfq_mlp_calibrate.argtypes = [vp, C.c_float, C.POINTER(C.c_int32), C.POINTER(C.c_float), vp]
        L.sfq_mlp_calibrate.restype = st
        L.sfq_mlp_sample_photon_xi.argtypes = [vp, i64, vp, vp, vp, vp, C.c_int32, vp, vp]
        L.sfq_mlp_create_pair.argtypes = [vp, C.c_uint64, C.POINTER(vp)]
        L.sfq_mlp_create_pair.restype = st
        L.sfq_mlp_sample_pair_xi.argtypes = [vp, i64, vp, vp, vp, vp, C.c_int32, vp, vp]
        L.sfq_mlp_sample_pair_xi.restype = st
        L.sfq_mlp_sample_photon_xi.restype = st
        L.sfq_cascade_run.argtypes = [vp, C.POINTER(Particles), C.POINTER(Fields), vp, u32, u32,
                                      C.POINTER(Products), vp, vp]
        L.sfq_cascade_run.restype = st
        L.sfq_cascade_compact_scratch_bytes.argtypes = [i64]
        L.sfq_cascade_compact_scratch_bytes.restype = C.c_size_t
        L.sfq_cascade_compact.argtypes = [vp, C.POINTER(Particles), C.POINTER(Fields), C.POINTER(Particles),
                                          C.POINTER(Fields), vp, C.c_size_t, vp]
        L.sfq_cascade_compact.restype = st
        L.sfq_set_evaluator.argtypes = [vp, C.c_int32]
        L.sfq_set_evaluator.restype = st
        L.sfq_table_pieces.argtypes = [C.c_int32, C.c_int32, C.c_int32, vp, C.POINTER(C.c_size_t)]
        L.sfq_table_pieces.restype = st
        L.sfq_set_step_shape.argtypes = [vp, C.c_int32, C.c_int32, C.c_int32]
        L.sfq_set_step_shape.restype = st
        L.sfq_set_event_queue.argtypes = [vp, C.POINTER(EventQueueDesc)]
        L.sfq_set_event_queue.restype = st
        L.sfq_set_surrogate.argtypes = [vp, vp, C.POINTER(EventQueueDesc), C.c_int32]
        L.sfq_set_surrogate.restype = st
        L.sfq_counters_check.argtypes = [vp]
        L.sfq_counters_check.restype = st
        L.sfq_check_bounded_wait.argtypes = [vp, u32, vp, vp]
        L.sfq_check_bounded_wait.restype = st
        L.sfq_check_sqrt.argtypes = [vp, i64, vp, vp, vp, vp]
        L.sfq_check_sqrt.restype = st
        L.sfq_version.restype = C.c_char_p
        _lib = L
    return _lib


EXPORTED = ["sfq_init", "sfq_finalize", "sfq_last_error", "sfq_constants", "sfq_photon_rate", "sfq_pair_rate",
            "sfq_uniforms", "sfq_sample_photon_xi", "sfq_sample_pair_xi", "sfq_mc_step", "sfq_mc_run",
            "sfq_mc_run_fused", "sfq_push", "sfq_set_pair_rate_cutoff", "sfq_set_sampler_coefficients",
            "sfq_sampler_coefficients", "sfq_autotune_step", "sfq_sort_scratch_bytes", "sfq_sort_products", "sfq_sort_products_noalloc", "sfq_set_step_shape",
            "sfq_mlp_num_params", "sfq_mlp_create", "sfq_mlp_destroy", "sfq_mlp_get_params", "sfq_mlp_set_params",
            "sfq_mlp_loss_grad", "sfq_mlp_train", "sfq_mlp_predict_lnw", "sfq_mlp_plain_targets", "sfq_mlp_calibrate",
            "sfq_mlp_sample_photon_xi", "sfq_mlp_create_pair", "sfq_mlp_sample_pair_xi",
            "sfq_cascade_run", "sfq_cascade_compact_scratch_bytes", "sfq_cascade_compact", "sfq_set_evaluator",
            "sfq_table_pieces", "sfq_counters_check", "sfq_check_bounded_wait", "sfq_check_sqrt", "sfq_set_surrogate",
            "sfq_set_event_queue",
            "sfq_version"]


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class SfqError(RuntimeError):
    pass


def counters_tensor(device="cuda"):
    """Zeroed sfq_counters on the device (16 uint64 words)."""
    return torch.zeros(16, dtype=torch.int64, device=device)


def counters_dict(t):
    v = t.cpu().tolist()
    return {k: int(v[i]) for i, k in enumerate(COUNTER_NAMES)}


def counters_status(t):
    """sfq_counters_check on a copy of the counters (a device tensor, a host tensor or 16
    integers): "SFQ_OK", "SFQ_ERR_TIMEOUT", "SFQ_ERR_CAPACITY" or "SFQ_ERR_RANGE"."""
    import numpy as np
    h = np.ascontiguousarray(np.asarray(t.cpu() if hasattr(t, "cpu") else t, dtype=np.int64).reshape(16))
    return STATUS[lib().sfq_counters_check(h.ctypes.data_as(C.c_void_p))]


class Context:
    """One libsfq context (sfq_init / sfq_finalize)."""

    def __init__(self, *, ref_len_m=0.0, ref_omega_si=0.0, dt, precision="fp32", device=None, seed=0):
        self.precision = SFQ_FP64 if precision in ("fp64", SFQ_FP64) else SFQ_FP32
        self.dtype = torch.float64 if self.precision == SFQ_FP64 else torch.float32
        dev = torch.cuda.current_device() if device is None else int(device)
        self.device = torch.device("cuda", dev)
        cfg = Config(ref_len_m=ref_len_m, ref_omega_si=ref_omega_si, dt=dt, precision=self.precision,
                     device=dev, seed=seed)
        h = C.c_void_p()
        st = lib().sfq_init(C.byref(cfg), C.byref(h))
        if st != 0:
            raise SfqError(f"sfq_init: {STATUS.get(st, st)}")
        self._h = h
        self.dt = dt
        self.seed = seed
        rho, pref = C.c_double(), C.c_double()
        lib().sfq_constants(h, C.byref(rho), C.byref(pref))
        self.rho, self.pref = rho.value, pref.value

    def close(self):
        if getattr(self, "_h", None):
            lib().sfq_finalize(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != 0:
            msg = lib().sfq_last_error(self._h).decode()
            raise SfqError(f"{what}: {STATUS.get(st, st)}: {msg}")

    def _real(self, t, name):
        if t.dtype != self.dtype or not t.is_cuda or not t.is_contiguous():
            raise SfqError(f"{name}: expected a contiguous CUDA {self.dtype} tensor")
        return t

    def set_step_shape(self, variant=0, ppt=0, grid_blocks=0):
        """variant 0 = automatic, 1 = warp-streaming kernel, 2 = TMA-staged kernel."""
        self._check(lib().sfq_set_step_shape(self._h, variant, ppt, grid_blocks), "sfq_set_step_shape")

    # --- entry points -------------------------------------------------------
    def photon_rate(self, gamma, chi, out=None, counters=None):
        out = torch.empty_like(chi) if out is None else out
        self._check(lib().sfq_photon_rate(self._h, chi.numel(), _ptr(self._real(gamma, "gamma")),
                                          _ptr(self._real(chi, "chi")), _ptr(self._real(out, "rate")),
                                          _ptr(counters), _stream()), "sfq_photon_rate")
        return out

    def pair_rate(self, gamma, chi, out=None, counters=None):
        out = torch.empty_like(chi) if out is None else out
        self._check(lib().sfq_pair_rate(self._h, chi.numel(), _ptr(self._real(gamma, "gamma")),
                                        _ptr(self._real(chi, "chi")), _ptr(self._real(out, "rate")),
                                        _ptr(counters), _stream()), "sfq_pair_rate")
        return out

    def uniforms(self, ids, step, tag=0):
        u = torch.empty(ids.numel(), 4, dtype=self.dtype, device=ids.device)
        self._check(lib().sfq_uniforms(self._h, ids.numel(), _ptr(ids), step, tag, _ptr(u), _stream()),
                    "sfq_uniforms")
        return u

    def sample_photon_xi(self, chi, r, counters=None):
        xi = torch.empty_like(chi)
        xic = torch.empty_like(chi)
        self._check(lib().sfq_sample_photon_xi(self._h, chi.numel(), _ptr(self._real(chi, "chi")),
                                               _ptr(self._real(r, "r")), _ptr(xi), _ptr(xic), _ptr(counters),
                                               _stream()), "sfq_sample_photon_xi")
        return xi, xic

    def sample_pair_xi(self, chi, r, counters=None):
        xe = torch.empty_like(chi)
        xp = torch.empty_like(chi)
        self._check(lib().sfq_sample_pair_xi(self._h, chi.numel(), _ptr(self._real(chi, "chi")),
                                             _ptr(self._real(r, "r")), _ptr(xe), _ptr(xp), _ptr(counters),
                                             _stream()), "sfq_sample_pair_xi")
        return xe, xp

    def mc_step(self, particles: "ParticleBuffers", fields: "FieldSource", step: int, products: "ProductBuffers",
                spawn: "SpawnBuffers" = None, counters=None):
        P = particles.descriptor()
        F = fields.descriptor()
        O = products.descriptor()
        S = spawn.descriptor() if spawn is not None else None
        self._check(lib().sfq_mc_step(self._h, C.byref(P), C.byref(F), step, C.byref(O),
                                      C.byref(S) if S is not None else None, _ptr(counters), _stream()),
                    "sfq_mc_step")

    def mc_run(self, particles: "ParticleBuffers", fields: "FieldSource", step0: int, nsteps: int,
               products: "ProductBuffers", children: "ParticleBuffers" = None, children_fields: "FieldSource" = None,
               spawn: "SpawnBuffers" = None, counters=None):
        """nsteps steps in one CUDA graph (children first, then `particles`, every step)."""
        P, F, O = particles.descriptor(), fields.descriptor(), products.descriptor()
        Cp = children.descriptor() if children is not None else None
        Cf = children_fields.descriptor() if children_fields is not None else None
        S = spawn.descriptor() if spawn is not None else None
        ref = lambda x: C.byref(x) if x is not None else None
        self._check(lib().sfq_mc_run(self._h, C.byref(P), C.byref(F), ref(Cp), ref(Cf), step0, nsteps, C.byref(O),
                                     ref(S), _ptr(counters), _stream()), "sfq_mc_run")

    def mc_run_fused(self, particles: "ParticleBuffers", fields: "FieldSource", step0: int, nsteps: int,
                     products: "ProductBuffers", counters=None):
        """nsteps steps in one launch of the fused plane-wave kernel (no children)."""
        P, F, O = particles.descriptor(), fields.descriptor(), products.descriptor()
        self._check(lib().sfq_mc_run_fused(self._h, C.byref(P), C.byref(F), step0, nsteps, C.byref(O),
                                           _ptr(counters), _stream()), "sfq_mc_run_fused")

    def cascade_run(self, particles: "ParticleBuffers", fields: "FieldSource", next_count, step0: int, nsteps: int,
                    products: "ProductBuffers", counters=None):
        """nsteps steps of a population that grows by its own products (particles.n_dev holds the
        live count, particles.n the capacity; next_count is a device scratch counter)."""
        P, F, O = particles.descriptor(), fields.descriptor(), products.descriptor()
        self._check(lib().sfq_cascade_run(self._h, C.byref(P), C.byref(F), _ptr(next_count), step0, nsteps,
                                          C.byref(O), _ptr(counters), _stream()), "sfq_cascade_run")

    def cascade_compact(self, src: "ParticleBuffers", fsrc: "FieldSource", dst: "ParticleBuffers",
                        fdst: "FieldSource", scratch):
        """Moves the alive particles of src, in order, to the front of dst (dst.n_dev = their number)."""
        S, FS, D, FD = src.descriptor(), fsrc.descriptor(), dst.descriptor(), fdst.descriptor()
        self._check(lib().sfq_cascade_compact(self._h, C.byref(S), C.byref(FS), C.byref(D), C.byref(FD),
                                              _ptr(scratch), scratch.numel() * scratch.element_size(), _stream()),
                    "sfq_cascade_compact")

    def push(self, particles: "ParticleBuffers", fields: "FieldSource", step: int, dt: float):
        """One Boris push of the leptons' momenta in the fields at `step`."""
        P, F = particles.descriptor(), fields.descriptor()
        self._check(lib().sfq_push(self._h, C.byref(P), C.byref(F), step, float(dt), _stream()), "sfq_push")

    def set_pair_rate_cutoff(self, chi_min: float):
        """NBW rate zero below chi_min (0.01 by default; 0.3 gives the paper's "fast" rate)."""
        self._check(lib().sfq_set_pair_rate_cutoff(self._h, float(chi_min)), "sfq_set_pair_rate_cutoff")

    def set_sampler_coefficients(self, k: int):
        """Use the leading k x k Chebyshev coefficients of each inverse-CDF piece (k = n, n-1, n-2)."""
        self._check(lib().sfq_set_sampler_coefficients(self._h, int(k)), "sfq_set_sampler_coefficients")

    def set_evaluator(self, kind: int):
        """SFQ_EVAL_HORNER (default) or SFQ_EVAL_CLENSHAW for the rate and sampler entry points."""
        self._check(lib().sfq_set_evaluator(self._h, kind), "sfq_set_evaluator")

    def sampler_coefficients(self):
        """(n, k): coefficients per variable of the tables and those in use."""
        n, k = C.c_int32(0), C.c_int32(0)
        self._check(lib().sfq_sampler_coefficients(self._h, C.byref(n), C.byref(k)), "sfq_sampler_coefficients")
        return n.value, k.value

    def autotune_step(self, particles: "ParticleBuffers", fields: "FieldSource", step=0, sample_n=0):
        """Times every launch shape on a copy of the population; returns (variant, shape, ms)."""
        P, F = particles.descriptor(), fields.descriptor()
        v, sh, ms = C.c_int32(0), C.c_int32(0), C.c_double(0.0)
        self._check(lib().sfq_autotune_step(self._h, C.byref(P), C.byref(F), step, sample_n, C.byref(v),
                                            C.byref(sh), C.byref(ms), _stream()), "sfq_autotune_step")
        return v.value, sh.value, ms.value

    def sort_products(self, products: "ProductBuffers", n=None, scratch=None):
        """Sorts the first n records by (parent id, step, member, parent tag) in place."""
        n = min(products.n(), products.capacity) if n is None else n
        need = sort_scratch_bytes(n)
        if scratch is None:
            scratch = torch.empty(need, dtype=torch.uint8, device=products.px.device)
        O = products.descriptor()
        self._check(lib().sfq_sort_products(self._h, C.byref(O), n, _ptr(scratch), scratch.numel(), _stream()),
                    "sfq_sort_products")

    def sort_products_noalloc(self, products: "ProductBuffers", n=None):
        """As sort_products, with the library's fixed scratch (n <= SORT_NOALLOC_MAX_N)."""
        n = min(products.n(), products.capacity) if n is None else n
        O = products.descriptor()
        self._check(lib().sfq_sort_products_noalloc(self._h, C.byref(O), n, _stream()),
                    "sfq_sort_products_noalloc")

    def set_surrogate(self, net, queue=None, use_flags=True):
        """sfq_set_surrogate: photon emissions of the step drawn from `net` (a calibrated photon
        Surrogate of this context) through `queue` (an EventQueue); net=None detaches."""
        if net is None:
            self._check(lib().sfq_set_surrogate(self._h, None, None, 0), "sfq_set_surrogate")
            self._surrogate = None
            return
        D = queue.descriptor()
        self._check(lib().sfq_set_surrogate(self._h, net._h, C.byref(D), int(bool(use_flags))), "sfq_set_surrogate")
        self._surrogate = (net, queue)          # keep both alive while attached

    def set_event_queue(self, queue=None):
        """sfq_set_event_queue: the deferred event path (step kernel, then an event pass) with
        `queue` (an EventQueue); None restores the inline path."""
        if queue is None:
            self._check(lib().sfq_set_event_queue(self._h, None), "sfq_set_event_queue")
            self._event_queue = None
            return
        D = queue.descriptor()
        self._check(lib().sfq_set_event_queue(self._h, C.byref(D)), "sfq_set_event_queue")
        self._event_queue = queue

    def check_bounded_wait(self, polls, counters):
        """sfq_check_bounded_wait: a wait that nothing completes gives up after `polls` polls
        and adds 1 to counters' timeouts word (counters: a device counters_tensor)."""
        self._check(lib().sfq_check_bounded_wait(self._h, int(polls), _ptr(counters), _stream()),
                    "sfq_check_bounded_wait")

    def check_sqrt(self, x):
        """sfq_check_sqrt: the kernels' binary32 sqrt and 1/sqrt of the float32 device tensor x;
        returns (sqrt, rsqrt)."""
        import torch
        if x.dtype != torch.float32 or not x.is_contiguous():
            raise TypeError("x must be a contiguous float32 tensor")
        so, ro = torch.empty_like(x), torch.empty_like(x)
        self._check(lib().sfq_check_sqrt(self._h, x.numel(), _ptr(x), _ptr(so), _ptr(ro), _stream()), "sfq_check_sqrt")
        return so, ro


SORT_NOALLOC_MAX_N = 1 << 20
SORT_NOALLOC_SCRATCH_BYTES = 44 << 20


class EventQueue:
    """Caller-owned queue of a step's photon emissions for the surrogate pass (sfq_event_queue)."""

    def __init__(self, capacity, device="cuda"):
        self.capacity = int(capacity)
        pad = max(self.capacity, 1)
        f = lambda: torch.empty(pad, dtype=torch.float32, device=device)
        self.index = torch.empty(pad, dtype=torch.int64, device=device)
        self.chi, self.r, self.gamma, self.px, self.py, self.pz, self.xi = (f() for _ in range(7))
        self.count = torch.zeros(2, dtype=torch.int64, device=device)

    def n(self):
        return min(int(self.count[0].item()), self.capacity)

    def descriptor(self):
        D = EventQueueDesc()
        D.capacity = self.capacity
        D.index, D.chi, D.r, D.gamma = _ptr(self.index), _ptr(self.chi), _ptr(self.r), _ptr(self.gamma)
        D.px, D.py, D.pz, D.xi = _ptr(self.px), _ptr(self.py), _ptr(self.pz), _ptr(self.xi)
        D.count = _ptr(self.count)
        return D


class Surrogate:
    """The learned inverse-CDF surrogate (sfq_mlp_*) of one binary32 context: kind "photon"
    (Eq. again; input u = r, output ln w-bar) or "pair" (Eq. again_pp; input u = |2r - 1|,
    output ln y, y = 1 - v-bar)."""

    def __init__(self, ctx: Context, seed=0, kind="photon"):
        self.ctx = ctx
        self.kind = kind
        h = C.c_void_p()
        if kind == "pair":
            ctx._check(lib().sfq_mlp_create_pair(ctx._h, seed, C.byref(h)), "sfq_mlp_create_pair")
        elif kind == "photon":
            ctx._check(lib().sfq_mlp_create(ctx._h, seed, C.byref(h)), "sfq_mlp_create")
        else:
            raise SfqError(f"unknown surrogate kind {kind!r}")
        self._h = h

    def close(self):
        if self._h:
            lib().sfq_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def num_params():
        return int(lib().sfq_mlp_num_params())

    def get_params(self):
        import numpy as np
        out = np.empty(self.num_params(), np.float32)
        self.ctx._check(lib().sfq_mlp_get_params(self._h, out.ctypes.data_as(C.c_void_p)), "sfq_mlp_get_params")
        return out

    def set_params(self, theta):
        import numpy as np
        theta = np.ascontiguousarray(theta, np.float32)
        assert theta.size == self.num_params()
        self.ctx._check(lib().sfq_mlp_set_params(self._h, theta.ctypes.data_as(C.c_void_p)), "sfq_mlp_set_params")

    def loss_grad(self, chi, u, lnw, quantize=False):
        grad = torch.empty(self.num_params(), dtype=torch.float32, device=chi.device)
        loss = torch.empty(1, dtype=torch.float32, device=chi.device)
        self.ctx._check(lib().sfq_mlp_loss_grad(self._h, chi.numel(), _ptr(chi), _ptr(u), _ptr(lnw), int(quantize),
                                                _ptr(grad), _ptr(loss), _stream()), "sfq_mlp_loss_grad")
        return loss, grad

    def train(self, chi, u, lnw, steps, batch=8192, lr=3e-3, quantize=True, seed=0, history=False):
        hist = torch.empty(steps, dtype=torch.float32, device=chi.device) if history else None
        self.ctx._check(lib().sfq_mlp_train(self._h, chi.numel(), _ptr(chi), _ptr(u), _ptr(lnw), steps, batch, lr,
                                            int(quantize), seed, _ptr(hist), _stream()), "sfq_mlp_train")
        return hist

    def predict_lnw(self, chi, u):
        out = torch.empty_like(chi)
        self.ctx._check(lib().sfq_mlp_predict_lnw(self._h, chi.numel(), _ptr(chi), _ptr(u), _ptr(out), _stream()),
                        "sfq_mlp_predict_lnw")
        return out

    def plain_targets(self, chi, u):
        out = torch.empty_like(chi)
        self.ctx._check(lib().sfq_mlp_plain_targets(self._h, chi.numel(), _ptr(chi), _ptr(u), _ptr(out), _stream()),
                        "sfq_mlp_plain_targets")
        return out

    def calibrate(self, tol_u=1e-3):
        nf, mx = C.c_int32(0), C.c_float(0.0)
        self.ctx._check(lib().sfq_mlp_calibrate(self._h, tol_u, C.byref(nf), C.byref(mx), _stream()),
                        "sfq_mlp_calibrate")
        return nf.value, mx.value

    def sample_photon_xi(self, chi, r, use_flags=True, counters=None):
        xi = torch.empty_like(chi)
        xc = torch.empty_like(chi)
        self.ctx._check(lib().sfq_mlp_sample_photon_xi(self._h, chi.numel(), _ptr(chi), _ptr(r), _ptr(xi), _ptr(xc),
                                                       int(use_flags), _ptr(counters), _stream()),
                        "sfq_mlp_sample_photon_xi")
        return xi, xc

    def sample_pair_xi(self, chi, r, use_flags=True, counters=None):
        """Electron and positron energy shares for uniforms r (kind "pair")."""
        xe = torch.empty_like(chi)
        xp = torch.empty_like(chi)
        self.ctx._check(lib().sfq_mlp_sample_pair_xi(self._h, chi.numel(), _ptr(chi), _ptr(r), _ptr(xe), _ptr(xp),
                                                     int(use_flags), _ptr(counters), _stream()),
                        "sfq_mlp_sample_pair_xi")
        return xe, xp


def sort_scratch_bytes(n):
    return int(lib().sfq_sort_scratch_bytes(n))


def cascade_compact_scratch_bytes(capacity):
    return int(lib().sfq_cascade_compact_scratch_bytes(capacity))


SFQ_TABLE_NLC_RATE, SFQ_TABLE_NBW_RATE, SFQ_TABLE_NLC_INV, SFQ_TABLE_NBW_INV = 0, 1, 2, 3


def table_pieces(precision, which, basis=SFQ_EVAL_HORNER):
    """Host copy of a fitted table (sfq_table_pieces) as a flat numpy array."""
    import numpy as np
    prec = SFQ_FP64 if precision == "fp64" else SFQ_FP32
    n = C.c_size_t(0)
    st = lib().sfq_table_pieces(prec, which, basis, None, C.byref(n))
    if st != 0:
        raise SfqError(f"sfq_table_pieces: {STATUS.get(st, st)}")
    out = np.empty(n.value // (8 if prec == SFQ_FP64 else 4), dtype=np.float64 if prec == SFQ_FP64 else np.float32)
    st = lib().sfq_table_pieces(prec, which, basis, out.ctypes.data_as(C.c_void_p), C.byref(n))
    if st != 0:
        raise SfqError(f"sfq_table_pieces: {STATUS.get(st, st)}")
    return out


# --- buffers -------------------------------------------------------------------
class ParticleBuffers:
    """Structure-of-arrays particle state on the device."""

    def __init__(self, px, py, pz, tau, flags, ids=None, id_base=0, fprev=None, dfprev=None,
                 lepton_model=SFQ_LEPTON_LCFA_OD, n_dev=None):
        self.px, self.py, self.pz, self.tau, self.flags = px, py, pz, tau, flags
        self.ids, self.id_base = ids, id_base
        self.fprev, self.dfprev = fprev, dfprev
        self.lepton_model = lepton_model
        self.n_dev = n_dev          # optional int64 device tensor holding the live count
        self.n = px.numel()

    def descriptor(self, n=None):
        P = Particles()
        P.n = self.n if n is None else n
        P.px, P.py, P.pz = _ptr(self.px), _ptr(self.py), _ptr(self.pz)
        P.tau, P.flags = _ptr(self.tau), _ptr(self.flags)
        P.id = _ptr(self.ids)
        P.id_base = self.id_base
        for k in range(3):
            P.fprev[k] = _ptr(self.fprev[k]) if self.fprev is not None else None
            P.dfprev[k] = _ptr(self.dfprev[k]) if self.dfprev is not None else None
        P.lepton_model = self.lepton_model
        P.n_dev = _ptr(self.n_dev)
        return P


class FieldSource:
    def __init__(self, kind, ex=None, ey=None, ez=None, bx=None, by=None, bz=None, k0=None, amp=None, amp0=0.0,
                 table=None, k_step=0):
        self.kind = kind
        self.ex, self.ey, self.ez, self.bx, self.by, self.bz = ex, ey, ez, bx, by, bz
        self.k0, self.amp, self.amp0, self.table, self.k_step = k0, amp, amp0, table, k_step

    @staticmethod
    def soa(ex, ey, ez, bx, by, bz):
        return FieldSource(SFQ_FIELDS_SOA, ex, ey, ez, bx, by, bz)

    @staticmethod
    def plane_wave(k0, table, k_step, amp=None, amp0=0.0):
        return FieldSource(SFQ_FIELDS_PLANE_WAVE, k0=k0, table=table, k_step=k_step, amp=amp, amp0=amp0)

    def descriptor(self):
        F = Fields()
        F.kind = self.kind
        F.ex, F.ey, F.ez = _ptr(self.ex), _ptr(self.ey), _ptr(self.ez)
        F.bx, F.by, F.bz = _ptr(self.bx), _ptr(self.by), _ptr(self.bz)
        F.k0, F.amp, F.amp0 = _ptr(self.k0), _ptr(self.amp), float(self.amp0)
        F.table = _ptr(self.table)
        F.n_table = 0 if self.table is None else self.table.numel()
        F.k_step = self.k_step
        return F


class ProductBuffers:
    def __init__(self, capacity, dtype, device):
        self.capacity = capacity
        pad = max(capacity, 1)
        self.px = torch.empty(pad, dtype=dtype, device=device)
        self.py = torch.empty(pad, dtype=dtype, device=device)
        self.pz = torch.empty(pad, dtype=dtype, device=device)
        self.parent_id = torch.empty(pad, dtype=torch.int64, device=device)
        self.step = torch.empty(pad, dtype=torch.int32, device=device)
        self.meta = torch.empty(pad, dtype=torch.uint8, device=device)
        self.count = torch.zeros(2, dtype=torch.int64, device=device)

    def reset(self):
        self.count.zero_()

    def n(self):
        return int(self.count[0].item())

    def descriptor(self):
        O = Products()
        O.capacity = self.capacity
        O.px, O.py, O.pz = _ptr(self.px), _ptr(self.py), _ptr(self.pz)
        O.parent_id, O.step, O.meta = _ptr(self.parent_id), _ptr(self.step), _ptr(self.meta)
        O.count = _ptr(self.count)
        return O

    def to_numpy(self):
        k = min(self.n(), self.capacity)
        return dict(px=self.px[:k].cpu().numpy(), py=self.py[:k].cpu().numpy(), pz=self.pz[:k].cpu().numpy(),
                    parent_id=self.parent_id[:k].cpu().numpy().view("uint64"),
                    step=self.step[:k].cpu().numpy().view("uint32"), meta=self.meta[:k].cpu().numpy())


class SpawnBuffers:
    def __init__(self, particles: ParticleBuffers, k0=None, amp=None):
        self.particles, self.k0, self.amp = particles, k0, amp
        self.count = torch.zeros(2, dtype=torch.int64, device=particles.px.device)

    def descriptor(self):
        S = Spawn()
        S.p = self.particles.descriptor()
        S.k0, S.amp = _ptr(self.k0), _ptr(self.amp)
        S.count = _ptr(self.count)
        return S
