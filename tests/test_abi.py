"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/sfq.h declares, and the ctypes binding declares each with the header's number of
parameters (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sfq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sfq_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libsfq():
    from paper_2301_07684_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["sfq_init", "sfq_finalize", "sfq_photon_rate", "sfq_pair_rate", "sfq_sample_photon_xi",
                 "sfq_sample_pair_xi", "sfq_mc_step", "sfq_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(libsfq):
    missing = [n for n in declared_functions() if not hasattr(libsfq, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2301_07684_gb300 import sfq
    assert set(declared_functions()) == set(sfq.EXPORTED)


def test_init_rejects_bad_config_without_touching_a_gpu(libsfq):
    from paper_2301_07684_gb300 import sfq
    L = sfq.lib()
    h = ctypes.c_void_p()
    # both reference scales given -> argument error before any device call
    cfg = sfq.Config(ref_len_m=1e-7, ref_omega_si=1e15, dt=0.1, precision=0, device=0, seed=0)
    assert L.sfq_init(ctypes.byref(cfg), ctypes.byref(h)) == 1
    cfg = sfq.Config(ref_len_m=1e-7, ref_omega_si=0.0, dt=-1.0, precision=0, device=0, seed=0)
    assert L.sfq_init(ctypes.byref(cfg), ctypes.byref(h)) == 1
    cfg = sfq.Config(ref_len_m=1e-7, ref_omega_si=0.0, dt=0.1, precision=7, device=0, seed=0)
    assert L.sfq_init(ctypes.byref(cfg), ctypes.byref(h)) == 1
    assert h.value is None


def declared_arity():
    """Parameter count of every function include/sfq.h declares."""
    src = open(os.path.join(ROOT, "include", "sfq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for name, params in re.findall(r"\b(sfq_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S):
        params = " ".join(params.split())
        out[name] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_argument_counts_match_the_header():
    from paper_2301_07684_gb300 import build, sfq
    build.build()
    L = sfq.lib()
    arity = declared_arity()
    assert set(arity) == set(sfq.EXPORTED)
    unbound, wrong = [], []
    for name, n in sorted(arity.items()):
        at = getattr(L, name).argtypes
        if at is None:
            if n:
                unbound.append(name)
        elif len(at) != n:
            wrong.append((name, len(at), n))
    assert not wrong, wrong
    assert not unbound, unbound


def test_counters_check_maps_the_counters_to_a_status():
    """sfq_counters_check reads a host copy of the counters only (no device, no context):
    a timeout outranks dropped records, which outrank inputs outside the fitted range."""
    from paper_2301_07684_gb300 import sfq
    names = sfq.COUNTER_NAMES

    def status(**kw):
        v = [0] * 16
        for k, x in kw.items():
            v[names.index(k)] = x
        return sfq.counters_status(v)

    assert status() == "SFQ_OK"
    assert status(updates=10, events=3, emitted=3, blcfa_rejected=2, large_rdt=1, gamma_below_one=1) == "SFQ_OK"
    assert status(dropped=1) == "SFQ_ERR_CAPACITY"
    assert status(spawn_dropped=4) == "SFQ_ERR_CAPACITY"
    assert status(out_of_range=2) == "SFQ_ERR_RANGE"
    assert status(nan_input=1) == "SFQ_ERR_RANGE"
    assert status(timeouts=1) == "SFQ_ERR_TIMEOUT"
    assert status(timeouts=1, dropped=5, out_of_range=5) == "SFQ_ERR_TIMEOUT"
    assert status(dropped=5, out_of_range=5) == "SFQ_ERR_CAPACITY"
    assert sfq.STATUS[sfq.lib().sfq_counters_check(None)] == "SFQ_ERR_ARG"
