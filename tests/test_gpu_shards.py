"""Shard invariance of the GPU path: a population split into contiguous id ranges (each
shard with its own buffers and id_base, run one after another on this GPU, as ranks
would run on theirs) gives bit for bit the final states and, once merged and ordered,
the product records of the unsplit run.  No collective is involved in the steps."""
import numpy as np
import pytest

from paper_2301_07684_gb300 import shard
from paper_2301_07684_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _run(ctx, d, a, b, nsteps):
    import torch
    from paper_2301_07684_gb300 import sfq
    dev = ctx.device
    T = lambda x: torch.as_tensor(np.ascontiguousarray(x[a:b])).to(dev)
    P = sfq.ParticleBuffers(T(d["px"]), T(d["py"]), T(d["pz"]), T(d["tau"]), T(d["flags"]), id_base=a)
    table = torch.as_tensor(d["table"]).to(dev)
    F = sfq.FieldSource.plane_wave(T(d["k0"].view(np.int32)), table, d["k_step"], amp0=d["amp0"])
    out = sfq.ProductBuffers(8 * (b - a) + 1024, ctx.dtype, dev)
    cnt = sfq.counters_tensor(dev)
    for s in range(nsteps):
        ctx.mc_step(P, F, s, out, counters=cnt)
    torch.cuda.synchronize()
    final = {k: getattr(P, k).cpu().numpy() for k in ("px", "py", "pz", "tau", "flags")}
    return out.to_numpy(), sfq.counters_dict(cnt), final


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("world", [2, 3])
def test_shards_equal_single_run(precision, world):
    from paper_2301_07684_gb300 import build, sfq
    build.build()
    ctx = sfq.Context(ref_len_m=W.REF_LEN, dt=W.DT, precision=precision, seed=123)
    d = W.config2(n=20000 + 11, seed=4, dtype=np.float32 if precision == "fp32" else np.float64)
    n, nsteps = d["px"].size, 40
    rec1, cnt1, fin1 = _run(ctx, d, 0, n, nsteps)
    parts, cnts, fins = [], [], []
    for r in range(world):
        a, b = shard.shard_bounds(n, r, world)
        rec, cnt, fin = _run(ctx, d, a, b, nsteps)
        parts.append(rec)
        cnts.append(cnt)
        fins.append(fin)
    merged = shard.merge_records(parts)
    single = shard.merge_records([rec1])
    assert len(single["parent_id"]) > 1000
    for k in shard.RECORD_COLUMNS:
        np.testing.assert_array_equal(merged[k], single[k], err_msg=k)
    total = shard.merge_counters(cnts)
    for k in ("updates", "events", "emitted", "dropped"):
        assert total[k] == cnt1[k], k
    for k in fin1:
        np.testing.assert_array_equal(np.concatenate([f[k] for f in fins]), fin1[k], err_msg=k)
    ctx.close()
