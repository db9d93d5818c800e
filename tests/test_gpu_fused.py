"""GPU tests of the fused multi-step run (sfq_mc_run_fused) for the analytic plane wave.

The fused kernel performs, per update and per event, the per-step kernels' own
arithmetic with each particle's state kept in registers across steps.  So it must
reproduce sfq_mc_step called once per step bit for bit: the same final momenta,
optical depths and flags, the same multiset of product records and the same
counters.  On top of that, sampled lineages are compared with the oracle (as for
the per-step path).  Workloads: config 2 (electrons, photon emission) and config 3
photons (pair creation, per-photon amplitude, no stepped children), at sizes of
several chunks with a ragged tail, in both precisions, with step0 != 0 and a run
split into two launches.
"""
import numpy as np
import pytest

from paper_2301_07684_gb300 import workloads as W

from mc_compare import compare_lineages
from test_gpu_mc_step import NEAR, TOL, gpu_subset, oracle_lineages

pytestmark = pytest.mark.gpu


def _ctx(precision, seed=99):
    from paper_2301_07684_gb300 import build, sfq
    build.build()
    return sfq.Context(ref_len_m=W.REF_LEN, dt=W.DT, precision=precision, seed=seed)


def _state(ctx, d):
    import torch
    from paper_2301_07684_gb300 import sfq
    dev = ctx.device
    T = lambda a, dt=None: torch.as_tensor(np.ascontiguousarray(a)).to(device=dev, dtype=dt)
    P = sfq.ParticleBuffers(T(d["px"], ctx.dtype), T(d["py"], ctx.dtype), T(d["pz"], ctx.dtype),
                            T(d["tau"], torch.float64), T(d["flags"]))
    F = sfq.FieldSource.plane_wave(T(d["k0"].view(np.int32)), T(d["table"], ctx.dtype), d["k_step"],
                                   amp=T(d["amp"], ctx.dtype) if "amp" in d else None, amp0=d.get("amp0", 0.0))
    return P, F


def _records(out):
    """Product records as a sorted structured array (order of appends is not fixed)."""
    k = min(out.n(), out.capacity)
    cols = [("pid", out.parent_id[:k].cpu().numpy().view(np.uint64)), ("step", out.step[:k].cpu().numpy()),
            ("meta", out.meta[:k].cpu().numpy()), ("px", out.px[:k].cpu().numpy()),
            ("py", out.py[:k].cpu().numpy()), ("pz", out.pz[:k].cpu().numpy())]
    rec = np.zeros(k, dtype=[(n, a.dtype) for n, a in cols])
    for n, a in cols:
        rec[n] = a
    return np.sort(rec, order=["pid", "step", "meta"])


def _bits(t):
    a = t.cpu().numpy()
    return a.view(np.uint64) if a.dtype == np.float64 else (a.view(np.uint32) if a.dtype == np.float32 else a)


def _per_step_and_fused(precision, d, step0, nsteps, splits=(None,), seed=99):
    import torch
    from paper_2301_07684_gb300 import sfq
    ctx = _ctx(precision, seed)
    n = d["px"].size
    cap = 8 * n + 64
    # reference: one sfq_mc_step per step
    Pa, Fa = _state(ctx, d)
    outa, cnta = sfq.ProductBuffers(cap, ctx.dtype, ctx.device), sfq.counters_tensor()
    for s in range(step0, step0 + nsteps):
        ctx.mc_step(Pa, Fa, s, outa, counters=cnta)
    # fused, possibly in several launches
    Pb, Fb = _state(ctx, d)
    outb, cntb = sfq.ProductBuffers(cap, ctx.dtype, ctx.device), sfq.counters_tensor()
    cuts = [step0] + [step0 + c for c in splits if c is not None] + [step0 + nsteps]
    for s0, s1 in zip(cuts[:-1], cuts[1:]):
        ctx.mc_run_fused(Pb, Fb, s0, s1 - s0, outb, counters=cntb)
    torch.cuda.synchronize()
    return ctx, (Pa, outa, cnta), (Pb, outb, cntb)


def _assert_identical(a, b):
    from paper_2301_07684_gb300 import sfq
    (Pa, outa, cnta), (Pb, outb, cntb) = a, b
    for name in ("px", "py", "pz", "tau", "flags"):
        np.testing.assert_array_equal(_bits(getattr(Pa, name)), _bits(getattr(Pb, name)), err_msg=name)
    ca, cb = sfq.counters_dict(cnta), sfq.counters_dict(cntb)
    assert ca == cb, (ca, cb)
    assert cb["timeouts"] == 0 and cb["dropped"] == 0
    ra, rb = _records(outa), _records(outb)
    assert ra.size == rb.size == outb.n()
    for name in ra.dtype.names:
        np.testing.assert_array_equal(ra[name], rb[name], err_msg=name)
    return cb


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_fused_equals_per_step_electrons(precision):
    """Config 2 electrons: 3 chunks' worth of warps and a ragged tail, 50 steps from step 7."""
    n = 3 * 8 * 128 + 45
    d = W.config2(n=n, seed=4, dtype=np.float32 if precision == "fp32" else np.float64)
    ctx, a, b = _per_step_and_fused(precision, d, step0=7, nsteps=50)
    c = _assert_identical(a, b)
    assert c["updates"] == n * 50 and c["emitted"] > n
    ctx.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_fused_equals_per_step_photons(precision):
    """Config 3 photons (per-photon amplitude, pair creation without stepped children)."""
    n = 4099
    d = W.config3(n=n, seed=6, dtype=np.float32 if precision == "fp32" else np.float64)
    ctx, a, b = _per_step_and_fused(precision, d, step0=0, nsteps=40)
    c = _assert_identical(a, b)
    assert c["pairs"] > 50 and c["emitted"] == 0
    ctx.close()


def test_fused_split_launches():
    """A run split into launches of 13 and 27 steps equals one step at a time."""
    n = 2 * 1024 + 3
    d = W.config2(n=n, seed=8)
    ctx, a, b = _per_step_and_fused("fp32", d, step0=0, nsteps=40, splits=(13,))
    _assert_identical(a, b)
    ctx.close()


def test_fused_oracle_lineages(oracle):
    """Sampled lineages of a fused config-2 run against the oracle (decisions exact except
    after a counted near-threshold decision, momenta within 1e-5)."""
    import torch
    from paper_2301_07684_gb300 import sfq
    ctx = _ctx("fp32", seed=2024)
    n, nsteps = 8192 + 77, 60
    d = W.config2(n=n, seed=0)
    P, F = _state(ctx, d)
    out, cnt = sfq.ProductBuffers(8 * n, ctx.dtype, ctx.device), sfq.counters_tensor()
    ctx.mc_run_fused(P, F, 0, nsteps, out, counters=cnt)
    torch.cuda.synchronize()
    c = sfq.counters_dict(cnt)
    assert c["updates"] == n * nsteps and c["timeouts"] == 0
    ids = np.unique(np.concatenate([W.sample_ids(n, 128, seed=3), [0, n - 1]]))
    orc = oracle_lineages(oracle, d, ids, nsteps, ctx.rho, ctx.seed, NEAR["fp32"])
    final, prod = gpu_subset(P, out, ids)
    s = compare_lineages(ids, orc, final, prod, TOL["fp32"], nsteps)
    assert s["records"] > 100 and s["near"] <= 2, s
    ctx.close()


def test_fused_rejects_unsupported():
    """Structure-of-arrays fields and beyond-LCFA leptons are refused with SFQ_ERR_ARG."""
    import torch
    from paper_2301_07684_gb300 import sfq
    ctx = _ctx("fp32")
    d = W.config2(n=256, seed=1)
    P, F = _state(ctx, d)
    out = sfq.ProductBuffers(64, ctx.dtype, ctx.device)
    z = torch.zeros(256, dtype=torch.float32, device=ctx.device)
    with pytest.raises(RuntimeError, match="plane-wave"):
        ctx.mc_run_fused(P, sfq.FieldSource.soa(z, z, z, z, z, z), 0, 3, out)
    ctx.close()
