"""sfq_sort_products_noalloc: the product sort with the library's fixed scratch array.

Collected last on purpose: it must pass on its own and after every other test has
used the device.  The GPU tests compare it with sfq_sort_products (caller scratch)
on two calls in a row of different sizes, and check its size limit.
"""
import numpy as np
import pytest


def _records(n, seed):
    g = np.random.default_rng(seed)
    pid = g.integers(0, 50, n).astype(np.uint64)
    pid[g.random(n) < 0.25] += np.uint64(3) << np.uint64(40)
    return dict(px=np.arange(n, dtype=np.float32), py=g.standard_normal(n).astype(np.float32),
                pz=g.standard_normal(n).astype(np.float32), parent_id=pid,
                step=g.integers(0, 700, n).astype(np.uint32), meta=g.integers(0, 256, n).astype(np.uint8))


def _load(sfq, torch, ctx, rec):
    n = rec["px"].size
    out = sfq.ProductBuffers(n, torch.float32, ctx.device)
    dev = ctx.device
    out.px[:n] = torch.as_tensor(rec["px"], device=dev)
    out.py[:n] = torch.as_tensor(rec["py"], device=dev)
    out.pz[:n] = torch.as_tensor(rec["pz"], device=dev)
    out.parent_id[:n] = torch.as_tensor(rec["parent_id"].view(np.int64), device=dev)
    out.step[:n] = torch.as_tensor(rec["step"].view(np.int32), device=dev)
    out.meta[:n] = torch.as_tensor(rec["meta"], device=dev)
    out.count[0] = n
    return out


def test_static_scratch_covers_the_limit():
    """The fixed array holds the sort's scratch plan at the largest allowed n (host arithmetic only)."""
    from paper_2301_07684_gb300 import build, sfq
    build.build()
    assert sfq.sort_scratch_bytes(sfq.SORT_NOALLOC_MAX_N) <= sfq.SORT_NOALLOC_SCRATCH_BYTES


@pytest.mark.gpu
def test_noalloc_sort_equals_sort_products():
    import torch
    from paper_2301_07684_gb300 import build, sfq
    build.build()
    ctx = sfq.Context(ref_len_m=0.8e-6 / (2 * np.pi), dt=0.01, precision="fp32", seed=1)
    for call, n in enumerate([200003, 3 * 8192 + 5]):          # two calls in a row, different sizes
        rec = _records(n, seed=100 + call)
        a = _load(sfq, torch, ctx, rec)
        b = _load(sfq, torch, ctx, rec)
        ctx.sort_products(a)                                     # caller scratch
        ctx.sort_products_noalloc(b)                             # library scratch
        torch.cuda.synchronize()
        ra, rb = a.to_numpy(), b.to_numpy()
        for k in ra:
            np.testing.assert_array_equal(ra[k], rb[k], err_msg=f"call {call}: {k}")
        # and both are the stable order on (parent id, step, member, tag)
        m = rec["meta"].astype(np.int64)
        o = np.lexsort(((m >> 4) & 3, (m >> 2) & 3, rec["step"].astype(np.int64), rec["parent_id"]))
        np.testing.assert_array_equal(rb["px"], rec["px"][o])
    ctx.close()


@pytest.mark.gpu
def test_noalloc_sort_rejects_more_than_the_limit():
    import torch
    from paper_2301_07684_gb300 import build, sfq
    build.build()
    ctx = sfq.Context(ref_len_m=0.8e-6 / (2 * np.pi), dt=0.01, precision="fp32", seed=1)
    n = sfq.SORT_NOALLOC_MAX_N + 1
    out = sfq.ProductBuffers(n, torch.float32, ctx.device)
    out.count[0] = n
    with pytest.raises(sfq.SfqError, match="SFQ_SORT_NOALLOC_MAX_N"):
        ctx.sort_products_noalloc(out)
    ctx.close()
