"""GPU parity of the full cascade (sfq_cascade_run, sfq_cascade_compact) with the oracle's.

Workload: electrons of gamma ~ N(1e4, 5%) head-on with the plane wave of a0 = 150 (chi of
the electrons up to ~9, of their photons up to a few), so that emitted photons convert and
the created leptons emit in turn.  The run starts at the smallest capacity the stepping
policy accepts (3 n), so the population is compacted and grown on the device during the run.

Comparison, lineage by lineage (a primary and everything it creates), for the lineages the
oracle flags no near-threshold decision in: the same alive particles (by id), their state
within the precision's tolerance, and the same product records.  The lineage of a GPU
particle is found by walking the GPU's own records from child to parent (the child's id
follows from the record's parent, step, member and parent tag).  A lineage with a near
decision may legitimately branch differently and is excluded as a whole.
"""
import numpy as np
import pytest

from paper_2301_07684_gb300 import workloads as W

from mc_compare import TAU0_MAX, budget

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-10}
NEAR = {"fp32": 1e-6, "fp64": 1e-10}
SEED = 2029


def _workload(n, dtype):
    return W.config2(n=n, seed=31, dtype=dtype, a0=150.0, gamma0=1e4)


def _ctx(precision):
    from paper_2301_07684_gb300 import build, sfq
    build.build()
    return sfq.Context(ref_len_m=W.REF_LEN, dt=W.DT, precision=precision, seed=SEED)


def _oracle(oracle, d, nsteps, near):
    n = d["px"].size
    E = np.zeros((n, nsteps, 6))
    for j in range(nsteps):
        (_, ey, _), (_, _, bz) = W.plane_wave_fields(d["k0"], d["amp0"], d["table"], j)
        E[:, j, 1], E[:, j, 5] = ey, bz
    p = np.stack([d["px"], d["py"], d["pz"]], 1).astype(np.float64)
    return oracle.mc_cascade(p, d["tau"], np.arange(n, dtype=np.uint64), d["flags"], np.zeros(n, np.uint8), E,
                             rho=W.RHO, dt=W.DT, seed=SEED, nsteps=nsteps, near_od=near)


def _close(g, o, b, tol):
    """Momentum g against the oracle's o within the relative budget b (mc_compare.budget)."""
    pmag = float(np.linalg.norm(o))
    for gv, ov in zip(g, o):
        if ov == 0.0:
            assert abs(gv) <= tol * 1e-6 * max(1.0, np.abs(o).max()), (g, o)
        else:
            assert abs(float(gv) - float(ov)) < b * max(abs(float(ov)), pmag), (g, o, b)


def _compare(oracle, n, orc, gpu, rec, tol):
    """orc: oracle.mc_cascade result; gpu: alive population (CascadeRun.alive());
    rec: the GPU's product records (ProductBuffers.to_numpy())."""
    # lineage of every GPU particle from the GPU's own records
    parent = {}
    for pid, st, m in zip(rec["parent_id"].tolist(), rec["step"].tolist(), rec["meta"].tolist()):
        member, ptag = (m >> 2) & 3, (m >> 4) & 3
        parent[oracle.child_id(SEED, pid, ptag, st, member)] = pid

    def root(i):
        for _ in range(10000):
            if i < (1 << 63):
                return i
            i = parent[i]
        raise AssertionError("no root")

    clean = orc["first_near_step"] < 0
    q = orc["particles"]
    # oracle: alive particles per clean lineage, id -> (p, tau, flags)
    # (the oracle keeps the species apart from its alive / just-created bits; the GPU packs
    # them into one byte with the tag, 0 for every cascade particle)
    # error budget of a particle: its chain of creations and recoils is part of its lineage,
    # so the lineage's event count bounds the k of mc_compare.budget
    want = {}
    for j in range(n):
        if clean[j] and orc["flags"][j] & 1:
            want[j] = (orc["p"][j], orc["tau"][j], int(orc["flags"][j] & 3) | (W.SP_ELECTRON << 2),
                       int(orc["n_events"][j]))
    for k in range(len(q)):
        r = q["root"][k]
        if clean[r] and q["flags"][k] & 1:
            want[int(q["id"][k])] = (q["p"][k], q["tau"][k], int(q["flags"][k] & 3) | (int(q["species"][k]) << 2),
                                     int(orc["n_events"][r]))
    got = {}
    for k in range(len(gpu["id"])):
        i = int(gpu["id"][k])
        if gpu["flags"][k] & 1 and clean[root(i)]:
            got[i] = (np.array([gpu["px"][k], gpu["py"][k], gpu["pz"][k]], np.float64), gpu["tau"][k],
                      int(gpu["flags"][k]))
    assert set(got) == set(want), (len(set(got) - set(want)), len(set(want) - set(got)))
    for i, (po, to, fo, k) in want.items():
        pg, tg, fg = got[i]
        assert fg == fo, (i, fg, fo)
        b = budget(tol, k)
        _close(pg, po, b, tol)
        assert abs(tg - to) <= TAU0_MAX * b, (i, tg, to, k)
    # product records of the clean lineages
    o_ids = {int(i): int(r) for i, r in zip(q["id"], q["root"])}
    op = orc["products"]
    okey = sorted((int(a), int(s), int(m), int(t)) for a, s, m, t in
                  zip(op["parent_id"], op["step"], op["member"], op["parent_tag"])
                  if clean[int(a) if int(a) < n else o_ids[int(a)]])
    gsel = [k for k in range(len(rec["parent_id"])) if clean[root(int(rec["parent_id"][k]))]]
    gkey = sorted((int(rec["parent_id"][k]), int(rec["step"][k]), (int(rec["meta"][k]) >> 2) & 3,
                   (int(rec["meta"][k]) >> 4) & 3) for k in gsel)
    assert okey == gkey
    return dict(alive=len(want), records=len(okey), lineages=int(clean.sum()), excluded=int((~clean).sum()))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cascade_matches_the_oracle(oracle, precision):
    from paper_2301_07684_gb300 import cascade, sfq
    n, nsteps = 256 + 19, 60
    d = _workload(n, np.float64 if precision == "fp64" else np.float32)
    ctx = _ctx(precision)
    run = cascade.CascadeRun(ctx, d, capacity=3 * n, products_cap=64 * n)
    run.run(0, nsteps)
    c = sfq.counters_dict(run.counters)
    assert c["spawn_dropped"] == 0 and c["dropped"] == 0 and c["timeouts"] == 0, c
    assert run.compactions >= 2 and run.capacity > 3 * n       # compacted and grown on the way
    orc = _oracle(oracle, d, nsteps, NEAR[precision])
    s = _compare(oracle, n, orc, run.alive(), run.out.to_numpy(), TOL[precision])
    assert s["lineages"] >= n - 10 and s["records"] > 500, s
    # second and later generations took part
    q = orc["particles"]
    assert (q["member"] > 0).sum() > 20 and np.isin(q["parent_id"], q["id"]).sum() > 20
    # every record is one created particle
    assert c["emitted"] + 2 * c["pairs"] == run.out.n()
    ctx.close()


def test_compaction_is_invisible_to_the_physics():
    """Compacting (and growing) mid-run leaves every particle's evolution bit for bit as in a
    run that never compacts; compaction keeps the order of the alive particles."""
    import torch
    from paper_2301_07684_gb300 import cascade
    n = 1000
    d = _workload(n, np.float32)
    ctx = _ctx("fp32")
    big = cascade.CascadeRun(ctx, d, capacity=200 * n, products_cap=64 * n)
    big.run(0, 50)
    small = cascade.CascadeRun(ctx, d, capacity=200 * n, products_cap=64 * n)
    small.run(0, 25)
    before = small.alive()
    m = small.compact(capacity=300 * n)
    after = small.alive()
    alive = before["flags"] & 1 == 1
    assert m == int(alive.sum()) and small.capacity == 300 * n
    for k in before:
        assert np.array_equal(after[k], before[k][alive]), k
    small.run(25, 25)
    a, b = big.alive(), small.alive()
    ka = np.argsort(a["id"][a["flags"] & 1 == 1])
    kb = np.argsort(b["id"][b["flags"] & 1 == 1])
    for k in a:
        assert np.array_equal(a[k][a["flags"] & 1 == 1][ka], b[k][b["flags"] & 1 == 1][kb]), k
    assert int(big.counters.sum().item()) > 0
    assert torch.equal(big.counters[:4], small.counters[:4])     # updates, events, emitted, pairs
    ctx.close()
