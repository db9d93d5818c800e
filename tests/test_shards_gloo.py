"""Multi-rank sharding on the CPU (gloo, world size 2): each rank runs the oracle over its
contiguous share of the particle ids, the records and counters are gathered, and the
union equals the unsplit run record for record (the random numbers are keyed by the
particle id, so the split changes nothing).  The same holds for the full cascade, whose
created particles take ids derived from their parents' (no two ranks create the same id)."""
import os
import socket

import numpy as np
import pytest

from paper_2301_07684_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _case():
    from paper_2301_07684_gb300 import workloads as W
    d = W.config2(n=40, seed=2)
    nsteps = 30
    E = np.zeros((40, nsteps, 6))
    for j in range(nsteps):
        (ex, ey, ez), (bx, by, bz) = W.plane_wave_fields(d["k0"], d["amp0"], d["table"], j)
        E[:, j, 1], E[:, j, 5] = ey, bz
    p = np.stack([d["px"], d["py"], d["pz"]], 1).astype(np.float64)
    return d, p, E, nsteps


def _run(ids, d, p, E, nsteps):
    from oracle import oracle as O
    from paper_2301_07684_gb300 import workloads as W
    r = O.mc_run(p[ids], d["tau"][ids], ids.astype(np.uint64), d["flags"][ids], (d["flags"][ids] >> 2) & 3, E[ids],
                 rho=W.RHO, dt=W.DT, seed=99, nsteps=nsteps, near_od=1e-6)
    pr = r["products"]
    rec = dict(px=pr["p"][:, 0], py=pr["p"][:, 1], pz=pr["p"][:, 2], parent_id=pr["parent_id"],
               step=pr["step"].astype(np.uint32),
               meta=((pr["member"] << 2) | (pr["parent_tag"] << 4) | (pr["species"] << 6)).astype(np.uint8))
    return rec, {"events": int(r["n_events"].sum()), "records": len(pr)}, r


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    d, p, E, nsteps = _case()
    a, b = shard.shard_bounds(len(p), rank, world)
    rec, cnt, r = _run(np.arange(a, b), d, p, E, nsteps)
    merged, total = shard.gather(rec, cnt)
    if rank == 0:
        np.savez(os.path.join(out_dir, "merged.npz"), **merged, events=total["events"], records=total["records"])
    np.save(os.path.join(out_dir, f"final{rank}.npy"), r["p"])
    dist.barrier()
    dist.destroy_process_group()


def test_shard_bounds_cover_the_range():
    for n in (0, 1, 7, 1000):
        for world in (1, 2, 3, 8):
            edges = [shard.shard_bounds(n, r, world) for r in range(world)]
            assert edges[0][0] == 0 and edges[-1][1] == n
            assert all(edges[k][1] == edges[k + 1][0] for k in range(world - 1))
            sizes = [b - a for a, b in edges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.shard_bounds(10, 2, 2)


def test_two_gloo_ranks_equal_the_single_run(tmp_path):
    import torch.multiprocessing as mp
    from oracle import oracle as O
    O.build()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    got = np.load(tmp_path / "merged.npz")
    d, p, E, nsteps = _case()
    rec, cnt, r = _run(np.arange(len(p)), d, p, E, nsteps)
    ref = shard.merge_records([rec])
    assert int(got["records"]) == cnt["records"] > 10 and int(got["events"]) == cnt["events"]
    for k in shard.RECORD_COLUMNS:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    final = np.concatenate([np.load(tmp_path / "final0.npy"), np.load(tmp_path / "final1.npy")])
    np.testing.assert_array_equal(final, r["p"])


def _cascade_case():
    from paper_2301_07684_gb300 import workloads as W
    n, nsteps = 24, 30
    d = W.config2(n=n, seed=4, dtype=np.float64, a0=150.0, gamma0=1e4)
    E = np.zeros((n, nsteps, 6))
    for j in range(nsteps):
        (_, ey, _), (_, _, bz) = W.plane_wave_fields(d["k0"], d["amp0"], d["table"], j)
        E[:, j, 1], E[:, j, 5] = ey, bz
    p = np.stack([d["px"], d["py"], d["pz"]], 1).astype(np.float64)
    return d, p, E, nsteps


def _cascade_run(ids, d, p, E, nsteps):
    from oracle import oracle as O
    from paper_2301_07684_gb300 import workloads as W
    r = O.mc_cascade(p[ids], d["tau"][ids], ids.astype(np.uint64), d["flags"][ids], np.zeros(len(ids), np.uint8),
                     E[ids], rho=W.RHO, dt=W.DT, seed=77, nsteps=nsteps)
    pr, q = r["products"], r["particles"]
    rec = dict(px=pr["p"][:, 0], py=pr["p"][:, 1], pz=pr["p"][:, 2], parent_id=pr["parent_id"],
               step=pr["step"].astype(np.uint32),
               meta=((pr["member"] << 2) | (pr["parent_tag"] << 4) | (pr["species"] << 6)).astype(np.uint8))
    created = dict(id=q["id"], px=q["p"][:, 0], tau=q["tau"], flags=q["flags"])
    return rec, {"events": int(r["n_events"].sum()), "records": len(pr)}, created


def _cascade_worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    d, p, E, nsteps = _cascade_case()
    a, b = shard.shard_bounds(len(p), rank, world)
    rec, cnt, created = _cascade_run(np.arange(a, b), d, p, E, nsteps)
    merged, total = shard.gather(rec, cnt)
    parts = [None] * world
    dist.all_gather_object(parts, created)
    if rank == 0:
        allc = {k: np.concatenate([c[k] for c in parts]) for k in created}
        np.savez(os.path.join(out_dir, "cascade.npz"), **merged, events=total["events"], records=total["records"],
                 **{"c_" + k: v for k, v in allc.items()})
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_the_single_cascade(tmp_path):
    import torch.multiprocessing as mp
    from oracle import oracle as O
    O.build()
    port = _free_port()
    mp.start_processes(_cascade_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    got = np.load(tmp_path / "cascade.npz")
    d, p, E, nsteps = _cascade_case()
    rec, cnt, created = _cascade_run(np.arange(len(p)), d, p, E, nsteps)
    ref = shard.merge_records([rec])
    assert int(got["records"]) == cnt["records"] > 20 and int(got["events"]) == cnt["events"]
    for k in shard.RECORD_COLUMNS:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    # the created particles of both ranks: distinct ids, the single run's states
    ids = got["c_id"]
    assert len(np.unique(ids)) == len(ids) == len(created["id"])
    o1, o2 = np.argsort(ids), np.argsort(created["id"])
    for k in created:
        np.testing.assert_array_equal(got["c_" + k][o1], created[k][o2], err_msg=k)



def _synthetic_records(rank, k):
    """k random records of rank (parent ids over the whole unsigned range, so that ids with
    bit 63 set -- a cascade's created particles -- are ordered as unsigned)."""
    g = np.random.default_rng(100 + rank)
    return dict(px=g.standard_normal(k).astype(np.float32), py=g.standard_normal(k).astype(np.float32),
                pz=g.standard_normal(k).astype(np.float32),
                parent_id=g.integers(0, 2 ** 63, k, dtype=np.uint64) * np.uint64(2) + np.uint64(rank),
                step=g.integers(0, 1 << 31, k, dtype=np.uint32) * np.uint32(2),
                meta=g.integers(0, 256, k, dtype=np.uint8))


def _big_worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    k = (1 << 20) - 12345 * rank
    merged, total = shard.gather(_synthetic_records(rank, k), {"records": k, "events": 3 * k})
    if rank == 0:
        np.savez(os.path.join(out_dir, "big.npz"), **merged, records=total["records"], events=total["events"])
    dist.barrier()
    dist.destroy_process_group()


def test_gather_of_a_million_records_per_rank(tmp_path):
    """The tensor gather (counts, then padded columns) at 2^20 records per rank with unequal
    counts: the union in (parent id, step, member, tag) order, counters summed."""
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_big_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    got = np.load(tmp_path / "big.npz")
    ks = [(1 << 20) - 12345 * r for r in range(2)]
    ref = shard.merge_records([_synthetic_records(r, ks[r]) for r in range(2)])
    assert int(got["records"]) == sum(ks) and int(got["events"]) == 3 * sum(ks)
    for k in shard.RECORD_COLUMNS:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
