"""GPU tests of the deferred event path (sfq_set_event_queue): the step kernel queues each
photon emission and an event pass samples and finishes the queue with the plain sampler.

Workload: config 2 (electrons head-on with the plane wave of a0 = 100, optical depth,
Sec. 2 and 4.1), 30 steps, at 2^18 + 77 particles (the TMA-staged kernel with a ragged
tail) and 3000 particles (the warp-streaming kernel), with the in-kernel plane wave and
with structure-of-arrays fields, and through the graph runner.  The deferred path uses
the inline path's arithmetic, so every record (sorted), the final state and the counters
must be identical bit for bit; with a queue too small for a step's emissions the excess
is finished inline and the run is still identical.
"""
import numpy as np
import pytest

from paper_2301_07684_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _ctx():
    from paper_2301_07684_gb300 import build, sfq
    build.build()
    return sfq.Context(ref_len_m=W.REF_LEN, dt=W.DT, precision="fp32", seed=99)


def _run(ctx, d, nsteps, fields, queue=None, graph=False):
    import torch
    from paper_2301_07684_gb300 import sfq
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    P = sfq.ParticleBuffers(T(d["px"]), T(d["py"]), T(d["pz"]), T(d["tau"]), T(d["flags"]))
    table, k0 = T(d["table"]), T(d["k0"].view(np.int32))
    n = d["px"].size
    if fields == "pw":
        F = sfq.FieldSource.plane_wave(k0, table, d["k_step"], amp0=d["amp0"])
        fs = lambda s: F
    else:
        k64 = T(d["k0"].astype(np.int64))
        K = d["table"].size
        z = torch.zeros(n, dtype=torch.float32, device="cuda")
        slabs = []
        for s in range(nsteps):
            f = torch.tensor(d["amp0"], dtype=torch.float32, device="cuda") * table[(k64 + (s * d["k_step"]) % K) % K]
            slabs.append(sfq.FieldSource.soa(z, f, z, z, z, f.clone()))
        fs = lambda s: slabs[s]
    out, cnt = sfq.ProductBuffers(n * nsteps // 4 + 4096, torch.float32, "cuda"), sfq.counters_tensor()
    ctx.set_event_queue(queue)
    if graph:
        ctx.mc_run(P, fs(0), 0, nsteps, out, counters=cnt)
    else:
        for s in range(nsteps):
            ctx.mc_step(P, fs(s), s, out, counters=cnt)
    torch.cuda.synchronize()
    ctx.set_event_queue(None)
    rec = out.to_numpy()
    o = np.lexsort((rec["step"], rec["parent_id"]))
    rec = {k: v[o] for k, v in rec.items()}
    state = {k: getattr(P, k).cpu().numpy() for k in ("px", "py", "pz", "tau", "flags")}
    return rec, state, sfq.counters_dict(cnt)


def _same(a, b):
    ra, sa, ca = a
    rb, sb, cb = b
    assert ca == cb, (ca, cb)
    for k in ra:
        assert np.array_equal(ra[k], rb[k]), k
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k


@pytest.mark.parametrize("n", [(1 << 18) + 77, 3000])
@pytest.mark.parametrize("fields", ["pw", "soa"])
def test_deferred_equals_inline(n, fields):
    from paper_2301_07684_gb300 import sfq
    ctx = _ctx()
    d = W.config2(n=n, seed=12)
    inline = _run(ctx, d, 30, fields)
    deferred = _run(ctx, d, 30, fields, queue=sfq.EventQueue(n // 4))
    assert inline[2]["events"] > 500 and inline[2]["dropped"] == 0
    _same(inline, deferred)
    ctx.close()


def test_deferred_in_a_graph_and_with_a_full_queue():
    from paper_2301_07684_gb300 import sfq
    ctx = _ctx()
    n = (1 << 17) + 5
    d = W.config2(n=n, seed=13)
    inline = _run(ctx, d, 20, "pw")
    _same(inline, _run(ctx, d, 20, "pw", queue=sfq.EventQueue(n // 4), graph=True))
    # a queue of 100 entries: the rest of each step's emissions are finished inline
    small = _run(ctx, d, 20, "pw", queue=sfq.EventQueue(100))
    assert small[2].pop("surrogate_fallbacks") > 0
    inline[2].pop("surrogate_fallbacks")
    _same(inline, small)
    ctx.close()
