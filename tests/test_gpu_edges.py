"""Edge cases of the Monte Carlo entry points on the GPU.

- Empty populations (n = 0) and zero steps are no-ops for sfq_mc_step, sfq_mc_run,
  sfq_mc_run_fused and sfq_push.
- Tiny and ragged populations (1, 31, 33, 1023, 1025 particles) in both step kernels and
  the fused run give the oracle's decisions and momenta (lineage comparison).
- Degenerate physics: with no field chi = 0 and nothing is emitted (W~_rad(0) chi = 0);
  photons below chi = 0.01 never convert (the pair rate is zero there, Sec. 4.2); dead
  particles are not updated.
- Capacity: records beyond the product buffer's capacity are counted as dropped, never
  written out of bounds, and the count of requested records is exact; sfq_counters_check
  reports the run as SFQ_ERR_CAPACITY.
- A decrement R dt that overflows binary32 (+inf) is an event, as its binary64 value is in
  the oracle.
- A bounded device wait that gives up is counted, reported as SFQ_ERR_TIMEOUT, and leaves
  the context usable.
"""
import numpy as np
import pytest

from paper_2301_07684_gb300 import workloads as W

from mc_compare import compare_lineages
from test_gpu_mc_step import NEAR, TOL, gpu_subset, oracle_lineages

pytestmark = pytest.mark.gpu


def _ctx(precision="fp32", seed=2024):
    from paper_2301_07684_gb300 import build, sfq
    build.build()
    return sfq.Context(ref_len_m=W.REF_LEN, dt=W.DT, precision=precision, seed=seed)


def _state(ctx, d, amp=None):
    import torch
    from paper_2301_07684_gb300 import sfq
    T = lambda a, dt=None: torch.as_tensor(np.ascontiguousarray(a)).to(device=ctx.device, dtype=dt)
    P = sfq.ParticleBuffers(T(d["px"], ctx.dtype), T(d["py"], ctx.dtype), T(d["pz"], ctx.dtype),
                            T(d["tau"], torch.float64), T(d["flags"]))
    F = sfq.FieldSource.plane_wave(T(d["k0"].view(np.int32)), T(d["table"], ctx.dtype), d["k_step"],
                                   amp=T(amp, ctx.dtype) if amp is not None else None, amp0=d.get("amp0", 0.0))
    return P, F


def test_empty_population_is_a_noop():
    import torch
    from paper_2301_07684_gb300 import sfq
    ctx = _ctx()
    d = W.config2(n=1, seed=0)
    e = torch.empty(0, dtype=ctx.dtype, device=ctx.device)
    P = sfq.ParticleBuffers(e, e.clone(), e.clone(), torch.empty(0, dtype=torch.float64, device=ctx.device),
                            torch.empty(0, dtype=torch.uint8, device=ctx.device))
    _, F = _state(ctx, d)
    z = torch.zeros(0, dtype=ctx.dtype, device=ctx.device)
    Fs = sfq.FieldSource.soa(z, z, z, z, z, z)
    out, cnt = sfq.ProductBuffers(16, ctx.dtype, ctx.device), sfq.counters_tensor()
    ctx.mc_step(P, Fs, 0, out, counters=cnt)
    ctx.mc_run(P, Fs, 0, 5, out, counters=cnt)
    ctx.mc_run_fused(P, F, 0, 5, out, counters=cnt)
    ctx.push(P, Fs, 0, W.DT)
    torch.cuda.synchronize()
    assert out.n() == 0 and int(cnt.sum().item()) == 0
    # zero steps on a real population leave it untouched
    P1, F1 = _state(ctx, W.config2(n=100, seed=1))
    before = P1.px.clone()
    ctx.mc_run_fused(P1, F1, 0, 0, out, counters=cnt)
    torch.cuda.synchronize()
    assert torch.equal(before, P1.px) and int(cnt.sum().item()) == 0
    ctx.close()


@pytest.mark.parametrize("n", [1, 31, 33, 1023, 1025])
@pytest.mark.parametrize("path", ["warp", "tma", "fused"])
def test_tiny_and_ragged_populations(oracle, n, path):
    import torch
    from paper_2301_07684_gb300 import sfq
    ctx = _ctx()
    nsteps = 40
    d = W.config2(n=n, seed=12)
    P, F = _state(ctx, d)
    out, cnt = sfq.ProductBuffers(8 * n + 64, ctx.dtype, ctx.device), sfq.counters_tensor()
    if path == "fused":
        ctx.mc_run_fused(P, F, 0, nsteps, out, counters=cnt)
    else:
        ctx.set_step_shape(1 if path == "warp" else 2, 0, 0)
        for s in range(nsteps):
            ctx.mc_step(P, F, s, out, counters=cnt)
    torch.cuda.synchronize()
    c = sfq.counters_dict(cnt)
    assert c["updates"] == n * nsteps and c["timeouts"] == 0 and c["dropped"] == 0
    ids = np.arange(n)
    orc = oracle_lineages(oracle, d, ids, nsteps, ctx.rho, ctx.seed, NEAR["fp32"])
    final, prod = gpu_subset(P, out, ids)
    compare_lineages(ids, orc, final, prod, TOL["fp32"], nsteps)
    ctx.close()


def test_no_field_no_emission_and_dead_particles():
    import torch
    from paper_2301_07684_gb300 import sfq
    ctx = _ctx()
    n = 4096
    d = W.config2(n=n, seed=3)
    d["flags"] = d["flags"].copy()
    d["flags"][::5] &= np.uint8(0xFE)                      # every fifth particle dead
    P, F = _state(ctx, d, amp=np.zeros(n, np.float32))     # a0 = 0: no field, chi = 0
    px0, tau0 = P.px.clone(), P.tau.clone()
    out, cnt = sfq.ProductBuffers(64, ctx.dtype, ctx.device), sfq.counters_tensor()
    for s in range(20):
        ctx.mc_step(P, F, s, out, counters=cnt)
    torch.cuda.synchronize()
    c = sfq.counters_dict(cnt)
    alive = (d["flags"] & 1).astype(bool)
    assert out.n() == 0 and c["events"] == 0 and c["updates"] == 20 * int(alive.sum())
    assert torch.equal(P.px, px0)
    # dead particles keep their optical depth untouched; alive ones drew theirs at step 0
    dead = torch.as_tensor(~alive, device=ctx.device)
    assert torch.equal(P.tau[dead], tau0[dead]) and bool((P.tau[~dead] > 0).all())
    ctx.close()


def test_photons_below_the_pair_domain_never_convert():
    import torch
    from paper_2301_07684_gb300 import sfq
    ctx = _ctx()
    n = 4096
    d = W.config3(n=n, seed=4)
    amp = (0.009 * W.RHO / (2.0 * d["px"].astype(np.float64) * -1.0)).astype(np.float32)   # peak chi 0.009
    P, F = _state(ctx, d, amp=amp)
    out, cnt = sfq.ProductBuffers(64, ctx.dtype, ctx.device), sfq.counters_tensor()
    for s in range(50):
        ctx.mc_step(P, F, s, out, counters=cnt)
    torch.cuda.synchronize()
    c = sfq.counters_dict(cnt)
    assert c["pairs"] == 0 and out.n() == 0 and bool((P.flags & 1).all())
    ctx.close()


def test_product_capacity_overflow_is_counted():
    import torch
    from paper_2301_07684_gb300 import sfq
    ctx = _ctx()
    n = 1 << 14
    d = W.config2(n=n, seed=5)
    P, F = _state(ctx, d)
    cap = 100
    out, cnt = sfq.ProductBuffers(cap, ctx.dtype, ctx.device), sfq.counters_tensor()
    guard = out.px.clone()
    for s in range(10):
        ctx.mc_step(P, F, s, out, counters=cnt)
    torch.cuda.synchronize()
    c = sfq.counters_dict(cnt)
    assert out.n() == c["emitted"] > cap
    assert c["dropped"] == c["emitted"] - cap
    assert out.px.numel() == guard.numel()
    assert sfq.counters_status(cnt) == "SFQ_ERR_CAPACITY"
    ctx.close()


def test_overflowing_decrement_is_an_event(oracle):
    """R dt beyond the binary32 range fires the optical-depth test in binary32 as in the
    oracle's binary64: every electron emits.  The timestep of 5e35 keeps pref dt finite in
    binary32 while R dt overflows."""
    import torch
    from paper_2301_07684_gb300 import build, sfq
    build.build()
    dt = 5e35
    ctx = sfq.Context(ref_len_m=W.REF_LEN, dt=dt, precision="fp32", seed=3)
    n = 256
    g = np.full(n, 3.0)
    pm = np.sqrt(g * g - 1)
    chi = np.full(n, 50.0)
    ey = chi * W.RHO / g                                  # p along x, E along y, B = 0: chi = gamma E / rho
    T = lambda a, t: torch.as_tensor(np.ascontiguousarray(a)).to(device=ctx.device, dtype=t)
    P = sfq.ParticleBuffers(T(pm, torch.float32), T(np.zeros(n), torch.float32), T(np.zeros(n), torch.float32),
                            T(np.ones(n), torch.float64), T(np.full(n, sfq.SFQ_ALIVE, np.uint8), torch.uint8))
    z = torch.zeros(n, dtype=torch.float32, device=ctx.device)
    F = sfq.FieldSource.soa(z, T(ey, torch.float32), z, z, z, z)
    out, cnt = sfq.ProductBuffers(4 * n, torch.float32, ctx.device), sfq.counters_tensor()
    ctx.mc_step(P, F, 0, out, counters=cnt)
    torch.cuda.synchronize()
    c = sfq.counters_dict(cnt)
    assert c["large_rdt"] == n and c["events"] == n and c["emitted"] == n, c
    E = np.zeros((n, 1, 6))
    E[:, 0, 1] = ey.astype(np.float32)                    # the field the device saw
    orc = oracle.mc_run(np.stack([pm.astype(np.float32), np.zeros(n), np.zeros(n)], 1), np.ones(n),
                        np.arange(n, dtype=np.uint64), np.full(n, 1, np.uint8), np.zeros(n, np.uint8), E,
                        rho=ctx.rho, dt=dt, seed=3, nsteps=1)
    assert np.all(orc["n_events"] == 1)
    ctx.close()


def test_bounded_wait_gives_up_and_is_reported():
    """A wait on a barrier nothing completes ends after its polls, counts one timeout,
    sfq_counters_check reports SFQ_ERR_TIMEOUT, and the context keeps working."""
    import torch
    from paper_2301_07684_gb300 import sfq
    ctx = _ctx()
    cnt = sfq.counters_tensor()
    ctx.check_bounded_wait(256, cnt)
    torch.cuda.synchronize()
    c = sfq.counters_dict(cnt)
    assert c["timeouts"] == 1 and sfq.counters_status(cnt) == "SFQ_ERR_TIMEOUT"
    # the context is still usable: a rate call right after
    g = torch.full((1024,), 1000.0, device=ctx.device)
    x = torch.full((1024,), 1.0, device=ctx.device)
    r = ctx.photon_rate(g, x)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(r).all()) and float(r[0]) > 0
    ctx.close()
