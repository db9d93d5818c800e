"""GPU tests of the batched runtime: product sort, CUDA-graph run, autotuner, and
parity of a 64-beam mixed population against oracle lineages.

Workload: config 4 (64 beams, particle counts log-uniform in [1e3, 4e6] scaled
down so the oracle replays sampled lineages in seconds; species mixed
electrons/positrons/photons; a0 uniform in [10, 300] and gamma0 log-uniform in
[200, 1e4] per beam; 500 steps of dt = 0.01 period in one CUDA graph; launch
shape chosen by the autotuner; products sorted by (parent id, step, member,
parent tag)).  Photons convert by optical depth (Sec. 2, 4.2) into pairs that are
stepped as children (optical-depth photon emission, Sec. 4.1).
"""
import numpy as np
import pytest

from paper_2301_07684_gb300 import workloads as W

from mc_compare import compare_lineages

pytestmark = pytest.mark.gpu
TOL = {"fp32": 1e-5, "fp64": 1e-10}
NEAR = {"fp32": 1e-6, "fp64": 1e-10}


def _ctx(precision, seed=4242):
    from paper_2301_07684_gb300 import build, sfq
    build.build()
    return sfq.Context(ref_len_m=W.REF_LEN, dt=W.DT, precision=precision, seed=seed)


def _records(out):
    return out.to_numpy()


def _order(r):
    m = r["meta"].astype(np.int64)
    return np.lexsort(((m >> 4) & 3, (m >> 2) & 3, r["step"].astype(np.int64), r["parent_id"]))


# --- sort ------------------------------------------------------------------------
@pytest.mark.parametrize("n", [0, 1, 2, 8192, 3 * 8192 + 123])
def test_sort_matches_stable_lexsort(n):
    """Random keys with many ties and 64-bit parent ids: the sort is numpy's stable
    lexsort on (parent id, step, member, tag), applied to every column."""
    import torch
    from paper_2301_07684_gb300 import sfq
    ctx = _ctx("fp32")
    g = np.random.default_rng(n + 1)
    out = sfq.ProductBuffers(max(n, 1), torch.float32, ctx.device)
    pid = g.integers(0, 40, n).astype(np.uint64)
    pid[g.random(n) < 0.3] += np.uint64(1) << np.uint64(50)      # exercises the high digits
    step = g.integers(0, 600, n).astype(np.uint32)
    meta = g.integers(0, 256, n).astype(np.uint8)
    px = np.arange(n, dtype=np.float32)                           # original position (stability)
    py = g.standard_normal(n).astype(np.float32)
    pz = g.standard_normal(n).astype(np.float32)
    dev = ctx.device
    if n:
        out.px[:n] = torch.as_tensor(px, device=dev)
        out.py[:n] = torch.as_tensor(py, device=dev)
        out.pz[:n] = torch.as_tensor(pz, device=dev)
        out.parent_id[:n] = torch.as_tensor(pid.view(np.int64), device=dev)
        out.step[:n] = torch.as_tensor(step.view(np.int32), device=dev)
        out.meta[:n] = torch.as_tensor(meta, device=dev)
    out.count[0] = n
    ctx.sort_products(out)
    torch.cuda.synchronize()
    r = _records(out)
    ref = dict(px=px, py=py, pz=pz, parent_id=pid, step=step, meta=meta)
    o = _order(ref)
    for k in ref:
        np.testing.assert_array_equal(r[k], ref[k][o], err_msg=k)
    ctx.close()


def test_sort_rejects_small_scratch():
    import torch
    from paper_2301_07684_gb300 import sfq
    ctx = _ctx("fp32")
    out = sfq.ProductBuffers(1000, torch.float32, ctx.device)
    out.count[0] = 1000
    small = torch.empty(sfq.sort_scratch_bytes(1000) - 256, dtype=torch.uint8, device=ctx.device)
    with pytest.raises(sfq.SfqError):
        ctx.sort_products(out, scratch=small)
    with pytest.raises(sfq.SfqError):
        ctx.sort_products(out, n=1001)
    ctx.close()


# --- batched run -------------------------------------------------------------------
def _run(precision, d, nsteps, graph, autotune=True, seed=4242):
    from paper_2301_07684_gb300 import batch
    import torch
    ctx = _ctx(precision, seed)
    b = batch.BatchRun(ctx, d, products_cap=128 * d["px"].size + 4096)
    shape = b.autotune() if autotune else None
    b.run(0, nsteps, graph=graph)
    b.sort()
    torch.cuda.synchronize()
    return ctx, b, shape


def _children_sorted(b):
    k = b.n_children()
    L = b.L
    ids = L.ids[:k].cpu().numpy()
    fl = L.flags[:k].cpu().numpy()
    o = np.lexsort(((fl >> 4) & 3, ids))
    return {name: getattr(L, name)[:k].cpu().numpy()[o] for name in ("px", "py", "pz", "tau", "flags")} | \
        {"ids": ids[o]}


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_graph_run_equals_stepwise(precision):
    """sfq_mc_run (one graph) gives bit for bit the state and the sorted records of
    the same steps issued one launch at a time."""
    from paper_2301_07684_gb300 import sfq
    d = W.config4(seed=1, scale=1e-3, dtype=np.float32 if precision == "fp32" else np.float64)
    nsteps = 120
    ctx_a, a, shape = _run(precision, d, nsteps, graph=True)
    variant, ppt, ms = shape
    assert variant in (1, 2) and ms > 0
    ctx_b, b, _ = _run(precision, d, nsteps, graph=False, autotune=False)
    ca, cb = sfq.counters_dict(a.counters), sfq.counters_dict(b.counters)
    assert ca == cb, (ca, cb)
    assert ca["pairs"] > 0 and ca["emitted"] > 0 and ca["dropped"] == 0 and ca["timeouts"] == 0
    for name in ("px", "py", "pz", "tau", "flags"):
        np.testing.assert_array_equal(getattr(a.P, name).cpu().numpy(), getattr(b.P, name).cpu().numpy())
    assert a.n_children() == b.n_children() == 2 * ca["pairs"]
    la, lb = _children_sorted(a), _children_sorted(b)
    for k in la:
        np.testing.assert_array_equal(la[k], lb[k], err_msg=k)
    ra, rb = _records(a.out), _records(b.out)
    for k in ra:
        np.testing.assert_array_equal(ra[k], rb[k], err_msg=k)
    # the records come back sorted
    o = _order(ra)
    assert np.array_equal(o, np.arange(o.size))
    ctx_a.close()
    ctx_b.close()


def oracle_config4(oracle, d, ids, nsteps, rho, seed, near):
    E = np.zeros((len(ids), nsteps, 6))
    for j in range(nsteps):
        (ex, ey, ez), (bx, by, bz) = W.plane_wave_fields(d["k0"][ids], d["amp"][ids], d["table"], j)
        E[:, j, 1], E[:, j, 5] = ey, bz
    p = np.stack([d["px"][ids], d["py"][ids], d["pz"][ids]], axis=1).astype(np.float64)
    return oracle.mc_run(p, d["tau"][ids], ids.astype(np.uint64), d["flags"][ids], (d["flags"][ids] >> 2) & 3, E,
                         rho=rho, dt=W.DT, seed=seed, nsteps=nsteps, step_children=True, near_od=near,
                         cap_products=1024 * len(ids))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_config4_lineages(oracle, precision):
    """500 steps in one graph with the autotuned shape; sampled lineages of every
    species (a photon, its pair and the photons the pair emits) against the oracle."""
    import torch
    from paper_2301_07684_gb300 import sfq
    d = W.config4(seed=0, scale=2e-3, dtype=np.float32 if precision == "fp32" else np.float64)
    nsteps = d["nsteps"]
    ctx, b, shape = _run(precision, d, nsteps, graph=True)
    c = sfq.counters_dict(b.counters)
    assert c["dropped"] == 0 and c["spawn_dropped"] == 0 and c["timeouts"] == 0, c
    assert b.n_children() == 2 * c["pairs"] and c["pairs"] > 100, c
    assert b.out.n() == 2 * c["pairs"] + c["emitted"]
    r = _records(b.out)
    o = _order(r)
    assert np.array_equal(o, np.arange(o.size))
    n = d["px"].size
    sp = (d["flags"] >> 2) & 3
    ids = np.unique(np.concatenate([W.sample_ids(n, 48, seed=9)] +
                                   [np.flatnonzero(sp == s)[W.sample_ids(int((sp == s).sum()), 16, seed=10 + s)]
                                    for s in range(3)]))
    orc = oracle_config4(oracle, d, ids, nsteps, ctx.rho, ctx.seed, NEAR[precision])
    sel = torch.as_tensor(ids, device=ctx.device)
    P = b.P
    final = dict(px=P.px[sel].cpu().numpy(), py=P.py[sel].cpu().numpy(), pz=P.pz[sel].cpu().numpy(),
                 tau=P.tau[sel].cpu().numpy(), flags=P.flags[sel].cpu().numpy())
    m = np.isin(r["parent_id"], ids.astype(np.uint64))
    prod = {k: v[m] for k, v in r.items()}
    s = compare_lineages(ids, orc, final, prod, TOL[precision], nsteps)
    assert s["records"] > 500, s
    assert s["near"] <= 8, s
    ctx.close()
