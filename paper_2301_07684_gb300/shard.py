"""Sharding of independent particles across ranks (one process per GPU).

Particles never interact and every random number is keyed by (seed, particle id, step,
tag), so a population split into contiguous id ranges gives, rank by rank, exactly the
records and final states of the unsplit run.  The step loop needs no collective; only
the end of a run gathers: the counters are summed and the product records of all ranks
are gathered (variable size: counts first, then padded columns, as tensors through
torch.distributed -- NCCL for device tensors, gloo on the CPU) and ordered by (parent id,
step, member, parent tag).
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


def order_tensors(rec):
    """Device-side record_order: indices that sort torch record columns by (parent id, step,
    member, parent tag), parent ids compared as unsigned 64-bit (stable sorts, least
    significant key first)."""
    import torch
    m = rec["meta"].to(torch.int64)
    keys = [(m >> 4) & 3, (m >> 2) & 3, rec["step"].to(torch.int64) & 0xFFFFFFFF,
            rec["parent_id"].to(torch.int64) ^ torch.iinfo(torch.int64).min]   # unsigned order
    idx = torch.arange(m.numel(), device=m.device)
    for k in keys:
        idx = idx[torch.sort(k[idx], stable=True).indices]
    return idx


def gather_tensors(records, counters, group=None):
    """All ranks: the records and counters of every rank, with no Python objects on the wire.
    `records`: dict of 1-D torch tensors (RECORD_COLUMNS, equal lengths, on this rank's device
    for NCCL, on the CPU for gloo); `counters`: an int64 tensor (sfq_counters words).  The
    counters are summed (all_reduce); the record counts are all-gathered, then every column is
    padded to the largest count and all-gathered, trimmed and ordered by (parent id, step,
    member, parent tag).  Returns (merged records, summed counters) on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    total = counters.clone()
    dist.all_reduce(total, op=dist.ReduceOp.SUM, group=group)
    dev = records["parent_id"].device
    k = torch.tensor([records["parent_id"].numel()], dtype=torch.int64, device=dev)
    ks = [torch.zeros_like(k) for _ in range(world)]
    dist.all_gather(ks, k, group=group)
    ks = [int(x.item()) for x in ks]
    kmax = max(ks) if ks else 0
    if kmax == 0:
        return {c: records[c][:0] for c in RECORD_COLUMNS}, total
    merged = {}
    for c in RECORD_COLUMNS:
        t = records[c]
        pad = torch.zeros(kmax, dtype=t.dtype, device=dev)
        pad[:t.numel()] = t
        parts = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(parts, pad, group=group)
        merged[c] = torch.cat([parts[r][:ks[r]] for r in range(world)])
    o = order_tensors(merged)
    return {c: v[o] for c, v in merged.items()}, total


def gather(records, counters, group=None):
    """All ranks: gather every rank's records (dict of numpy columns) and counters (dict of
    integers) through gather_tensors on the CPU; returns the merged records (numpy) and the
    summed counters on every rank."""
    import torch
    names = sorted(counters)
    cnt = torch.tensor([int(counters[k]) for k in names], dtype=torch.int64)
    tens = {}
    for c in RECORD_COLUMNS:
        a = np.ascontiguousarray(records[c])
        tens[c] = torch.from_numpy(a.view(np.int64) if a.dtype == np.uint64 else
                                   (a.view(np.int32) if a.dtype == np.uint32 else a))
    merged, total = gather_tensors(tens, cnt, group=group)
    out = {}
    for c in RECORD_COLUMNS:
        v = merged[c].numpy()
        dt = np.asarray(records[c]).dtype
        out[c] = v.view(dt) if dt in (np.uint64, np.uint32) else v.astype(dt, copy=False)
    return out, {k: int(v) for k, v in zip(names, total.tolist())}
