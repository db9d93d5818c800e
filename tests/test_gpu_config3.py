"""GPU parity of pair creation with stepped children under the beyond-LCFA model.

Workload: config 3 (photons with peak chi log-uniform in [0.1, 100] and gamma
log-uniform in [1e2, 1e5], head-on with plane waves whose amplitude gives that
peak chi), at a size the oracle replays in seconds.  Each step runs the lepton
population (children of earlier conversions, beyond-LCFA local method, Sec. 5)
and then the photons (nonlinear Breit-Wheeler by optical depth, Sec. 2 and 4.2);
pairs are appended both as product records and as stepped children.  Lineages
(a photon, its pair and the photons the pair emits) are compared with the
oracle record by record up to their first near-threshold decision (optical depth
1e-6 tau0, local test 1e-6 r, beyond-LCFA comparisons 1e-4 relative).
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
    ctx.close()
