"""Sharding of independent particles across ranks (one process per GPU).

Particles never interact and every random number is keyed by (seed, particle id, step,
tag), so a population split into contiguous id ranges gives, rank by rank, exactly the
records and final states of the unsplit run.  The step loop needs no collective; only
the end of a run gathers: the counters are summed and the product records of all ranks
are gathered (variable size) and ordered by (parent id, step, member, parent tag).
"""
from __future__ import annotations

import numpy as np

RECORD_COLUMNS = ("px", "py", "pz", "parent_id", "step", "meta")


def shard_bounds(n: int, rank: int, world: int):
    """[start, end) of rank's contiguous share of n particles (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside [0, world)")
    return n * rank // world, n * (rank + 1) // world


def record_order(rec):
    """Indices that sort records by (parent id, step, member, parent tag)."""
    m = np.asarray(rec["meta"]).astype(np.int64)
    return np.lexsort(((m >> 4) & 3, (m >> 2) & 3, np.asarray(rec["step"]).astype(np.int64),
                       np.asarray(rec["parent_id"])))


def merge_records(parts):
    """Concatenate the record dicts of several shards and order them."""
    parts = [p for p in parts if p is not None and len(p["parent_id"])]
    if not parts:
        return {k: np.zeros(0) for k in RECORD_COLUMNS}
    rec = {k: np.concatenate([np.asarray(p[k]) for p in parts]) for k in RECORD_COLUMNS}
    o = record_order(rec)
    return {k: v[o] for k, v in rec.items()}


def merge_counters(parts):
    out = {}
    for p in parts:
        for k, v in p.items():
            out[k] = out.get(k, 0) + int(v)
    return out


def gather(records, counters, group=None):
    """All ranks: gather every rank's records and counters (torch.distributed, any backend);
    returns the merged records and summed counters on every rank."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    objs = [None] * world
    dist.all_gather_object(objs, (records, counters), group=group)
    return merge_records([o[0] for o in objs]), merge_counters([o[1] for o in objs])
