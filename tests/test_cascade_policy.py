"""Host logic of the full-cascade runtime (CascadeRun), on the CPU with a stand-in context.

The stand-in plays the device: each step multiplies the live count by a chosen factor
(at most 3, the worst case of a step: a photon leaves two leptons, a lepton one photon),
and a compaction keeps a chosen fraction.  The policy must start a run of k steps only
when 3^k times the count fits the capacity, cover every step exactly once and in order,
compact when it does not fit, and grow the capacity when compaction is not enough.
"""
import numpy as np
import pytest
import torch

from paper_2301_07684_gb300 import cascade, sfq
from paper_2301_07684_gb300 import workloads as W


class FakeCtx:
    device = "cpu"
    dtype = torch.float32

    def __init__(self, growth, alive_fraction):
        self.growth, self.alive_fraction = growth, alive_fraction
        self.runs, self.compactions = [], []

    def cascade_run(self, P, F, next_count, step0, nsteps, out, counters=None):
        n = int(P.n_dev[0])
        assert 3 ** nsteps * max(n, 1) <= P.n, (n, nsteps, P.n)
        self.runs.append((step0, nsteps, n, P.n))
        for _ in range(nsteps):
            n = min(int(np.ceil(n * self.growth)), P.n)
        P.n_dev[0] = n

    def cascade_compact(self, src, fsrc, dst, fdst, scratch):
        assert dst.n >= src.n
        n = int(src.n_dev[0])
        self.compactions.append((n, src.n, dst.n))
        dst.n_dev[0] = int(n * self.alive_fraction)


def _lib_or_skip():
    try:
        sfq.lib()
    except ImportError as e:
        pytest.skip(str(e))


def _run(growth, alive_fraction, n=100, capacity=300, nsteps=40):
    _lib_or_skip()
    ctx = FakeCtx(growth, alive_fraction)
    d = W.config2(n=n, seed=0, dtype=np.float32)
    r = cascade.CascadeRun(ctx, d, capacity=capacity, products_cap=16)
    r.run(5, nsteps)
    return ctx, r


# (growth per step, fraction alive at a compaction, steps): the population stays below ~1e6
@pytest.mark.parametrize("growth,alive,nsteps", [(1.0, 1.0, 40), (1.3, 1.0, 20), (3.0, 0.5, 8), (2.0, 0.9, 10),
                                                 (1.05, 0.3, 40)])
def test_every_step_runs_once_within_the_worst_case_bound(growth, alive, nsteps):
    ctx, r = _run(growth, alive, n=20, capacity=60, nsteps=nsteps)
    steps = [s for s0, k, _, _ in ctx.runs for s in range(s0, s0 + k)]
    assert steps == list(range(5, 5 + nsteps))
    assert all(k >= 1 for _, k, _, _ in ctx.runs)


def test_no_growth_needs_no_compaction():
    ctx, r = _run(1.0, 1.0, capacity=100 * 100)
    assert not ctx.compactions and r.capacity == 100 * 100
    assert max(k for _, k, _, _ in ctx.runs) == 4                 # 3^4 * 100 <= 10^4 < 3^5 * 100


def test_growth_compacts_then_grows_the_capacity():
    ctx, r = _run(1.5, 1.0, nsteps=12)
    assert ctx.compactions and r.capacity > 300
    # a compaction that frees nothing is followed by one into a larger buffer set
    grew = [c for c in ctx.compactions if c[2] > c[1]]
    assert grew and all(dst >= 6 * n for n, src, dst in grew if n > 0)


def test_compaction_alone_suffices_when_particles_die():
    ctx, r = _run(1.5, 0.2, capacity=3000, nsteps=30)
    assert ctx.compactions and r.capacity == 3000


def test_primary_ids_must_stay_below_two_to_the_63():
    _lib_or_skip()
    d = W.config2(n=4, seed=0, dtype=np.float32)
    with pytest.raises(ValueError):
        cascade.CascadeRun(FakeCtx(1.0, 1.0), d, capacity=64, products_cap=16,
                           ids=np.array([0, 1, 2, 1 << 63], dtype=np.uint64))
