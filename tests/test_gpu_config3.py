"""GPU parity of pair creation with stepped children under the beyond-LCFA model.

Workload: config 3 (photons with peak chi log-uniform in [0.1, 100] and gamma
log-uniform in [1e2, 1e5], head-on with plane waves whose amplitude gives that
peak chi), at a size the oracle replays in seconds.  Each step runs the lepton
population (children of earlier conversions, beyond-LCFA local method, Sec. 5)
and then the photons (nonlinear Breit-Wheeler by optical depth, Sec. 2 and 4.2);
pairs are appended both as product records and as stepped children.  Lineages
(a photon, its pair and the photons the pair emits) are compared with the
oracle record by record up to their first near-threshold decision (optical depth
1e-6 tau0, local test 1e-6 r, beyond-LCFA comparisons 1e-4 relative in binary32:
the threshold of Eq. gammaLCFA comes from the second difference of Eq. condit,
which in binary32 keeps the force to ~6e-8 but its second difference, about 1/60
of it at this timestep, only to ~4e-6, and gamma_LCFA ~ delta^(3/2) for large tau/tau_C,
so gamma_LCFA carries ~6e-6; 1e-4 leaves a margin above that).  The compared
lineages must include events whose gate held and samples that Eq. rej_cond
rejected, so that the beyond-LCFA branches are exercised, and the no-emission rule
of Sec. 5 must never fire (gamma_LCFA <= 0.7 gamma_e).
"""
import numpy as np
import pytest

from paper_2301_07684_gb300 import workloads as W

from mc_compare import compare_lineages

pytestmark = pytest.mark.gpu
TOL = {"fp32": 1e-5, "fp64": 1e-10}
NEAR = {"fp32": (1e-6, 1e-6, 1e-4), "fp64": (1e-10, 1e-10, 1e-8)}


def run_config3(ctx, d, nsteps, cap_factor=4):
    import torch
    from paper_2301_07684_gb300 import sfq
    dev, dt = ctx.device, ctx.dtype
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev)
    n = d["px"].size
    P = sfq.ParticleBuffers(T(d["px"]), T(d["py"]), T(d["pz"]), T(d["tau"]), T(d["flags"]))
    table = T(d["table"])
    k0 = T(d["k0"].view(np.int32))
    amp = T(d["amp"])
    Fp = sfq.FieldSource.plane_wave(k0, table, d["k_step"], amp=amp)
    cap = 2 * n + 64
    z = lambda dtype: torch.zeros(cap, dtype=dtype, device=dev)
    spawn_count = torch.zeros(2, dtype=torch.int64, device=dev)
    Lp = sfq.ParticleBuffers(z(dt), z(dt), z(dt), z(torch.float64), z(torch.uint8), ids=z(torch.int64),
                             fprev=[z(dt) for _ in range(3)], dfprev=[z(dt) for _ in range(3)],
                             lepton_model=sfq.SFQ_LEPTON_BLCFA_LOCAL, n_dev=spawn_count)
    lk0 = z(torch.int32)
    lamp = z(dt)
    spawn = sfq.SpawnBuffers(Lp, k0=lk0, amp=lamp)
    spawn.count = spawn_count
    Fl = sfq.FieldSource.plane_wave(lk0, table, d["k_step"], amp=lamp)
    out = sfq.ProductBuffers(cap_factor * n * nsteps // 4 + 4096, dt, dev)
    cnt = sfq.counters_tensor()
    for s in range(nsteps):
        ctx.mc_step(Lp, Fl, s, out, counters=cnt)            # children created before this step
        ctx.mc_step(P, Fp, s, out, spawn=spawn, counters=cnt)
    torch.cuda.synchronize()
    return P, Lp, out, cnt, int(spawn_count[0].item())


def oracle_config3(oracle, d, ids, nsteps, rho, seed, near):
    E = np.zeros((len(ids), nsteps, 6))
    for j in range(nsteps):
        (ex, ey, ez), (bx, by, bz) = W.plane_wave_fields(d["k0"][ids], d["amp"][ids], d["table"], j)
        E[:, j, 1], E[:, j, 5] = ey, bz
    p = np.stack([d["px"][ids], d["py"][ids], d["pz"][ids]], axis=1).astype(np.float64)
    return oracle.mc_run(p, d["tau"][ids], ids.astype(np.uint64), d["flags"][ids], (d["flags"][ids] >> 2) & 3, E,
                         rho=rho, dt=W.DT, seed=seed, nsteps=nsteps, lepton_mode=oracle.MODE_BLCFA_LOCAL,
                         step_children=True, near_od=near[0], near_local=near[1], near_blcfa=near[2],
                         cap_products=64 * len(ids) * nsteps)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_config3_small(oracle, precision):
    import torch
    from paper_2301_07684_gb300 import build, sfq
    build.build()
    ctx = sfq.Context(ref_len_m=W.REF_LEN, dt=W.DT, precision=precision, seed=77)
    n, nsteps = 4096 + 13, 40
    d = W.config3(n=n, seed=0, dtype=np.float32 if precision == "fp32" else np.float64)
    P, Lp, out, cnt, nlep = run_config3(ctx, d, nsteps)
    c = sfq.counters_dict(cnt)
    assert c["dropped"] == 0 and c["spawn_dropped"] == 0 and c["timeouts"] == 0
    assert nlep == 2 * c["pairs"] and c["pairs"] > 500, c
    assert c["emitted"] > 100, c
    # every product is accounted for: pairs give two records each, emissions one
    assert out.n() == 2 * c["pairs"] + c["emitted"]
    ids = W.sample_ids(n, 96, seed=5)
    orc = oracle_config3(oracle, d, ids, nsteps, ctx.rho, ctx.seed, NEAR[precision])
    sel = torch.as_tensor(ids, device=ctx.device)
    final = dict(px=P.px[sel].cpu().numpy(), py=P.py[sel].cpu().numpy(), pz=P.pz[sel].cpu().numpy(),
                 tau=P.tau[sel].cpu().numpy(), flags=P.flags[sel].cpu().numpy())
    k = out.n()
    m = torch.isin(out.parent_id[:k], sel)
    prod = dict(px=out.px[:k][m].cpu().numpy(), py=out.py[:k][m].cpu().numpy(), pz=out.pz[:k][m].cpu().numpy(),
                parent_id=out.parent_id[:k][m].cpu().numpy().view(np.uint64),
                step=out.step[:k][m].cpu().numpy().view(np.uint32), meta=out.meta[:k][m].cpu().numpy())
    s = compare_lineages(ids, orc, final, prod, TOL[precision], nsteps)
    assert s["records"] > 60, s
    assert s["near"] <= 6, s
    assert_blcfa_exercised(orc, c)
    ctx.close()


def assert_blcfa_exercised(orc, c):
    """The compared lineages (no near-threshold decision) went through the gate and the
    rejection of Eq. rej_cond; the 0.75 gamma_e rule fired nowhere, on either side."""
    clean = orc["first_near_step"] < 0
    assert orc["n_gated"][clean].sum() > 0 and orc["n_rejected"][clean].sum() > 0, \
        (orc["n_gated"][clean].sum(), orc["n_rejected"][clean].sum())
    assert orc["n_no_emission"].sum() == 0 and c["blcfa_no_emission"] == 0
    assert c["blcfa_rejected"] > 0


@pytest.mark.slow
def test_config3_full_size(oracle):
    """Config 3 at its stated size: 2^24 photons, 100 steps, binary32 with a binary64 optical
    depth; 160 sampled photon lineages (the photon, its pair and the pair's photons)."""
    import torch
    from paper_2301_07684_gb300 import build, sfq
    build.build()
    ctx = sfq.Context(ref_len_m=W.REF_LEN, dt=W.DT, precision="fp32", seed=77)
    d = W.config3(n=1 << 24, seed=0)
    n, nsteps = d["px"].size, d["nsteps"]
    P, Lp, out, cnt, nlep = run_config3(ctx, d, nsteps, cap_factor=3)   # ~34 records per photon
    c = sfq.counters_dict(cnt)
    assert c["dropped"] == 0 and c["spawn_dropped"] == 0 and c["timeouts"] == 0, c
    assert nlep == 2 * c["pairs"] and out.n() == 2 * c["pairs"] + c["emitted"]
    ids = W.sample_ids(n, 160, seed=9)
    orc = oracle_config3(oracle, d, ids, nsteps, ctx.rho, ctx.seed, NEAR["fp32"])
    sel = torch.as_tensor(ids, device=ctx.device)
    final = dict(px=P.px[sel].cpu().numpy(), py=P.py[sel].cpu().numpy(), pz=P.pz[sel].cpu().numpy(),
                 tau=P.tau[sel].cpu().numpy(), flags=P.flags[sel].cpu().numpy())
    k = out.n()
    m = torch.isin(out.parent_id[:k], sel)
    prod = dict(px=out.px[:k][m].cpu().numpy(), py=out.py[:k][m].cpu().numpy(), pz=out.pz[:k][m].cpu().numpy(),
                parent_id=out.parent_id[:k][m].cpu().numpy().view(np.uint64),
                step=out.step[:k][m].cpu().numpy().view(np.uint32), meta=out.meta[:k][m].cpu().numpy())
    s = compare_lineages(ids, orc, final, prod, TOL["fp32"], nsteps)
    assert s["records"] > 100, s
    assert s["near"] <= 12, s
    assert_blcfa_exercised(orc, c)
    ctx.close()
