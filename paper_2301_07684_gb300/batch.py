"""Batched runs of the Monte Carlo step: a mixed population of many beams (electrons,
positrons and photons in one structure of arrays, each particle with its own
plane-wave amplitude), the leptons its photons create by nonlinear Breit-Wheeler
conversion (Sec. 2, Eq. pp_tot_real) stepped as children in the same step loop,
and the product records, sorted at the end by (parent id, step, member, parent tag).

Every step runs the children first (those created at earlier steps), then the
primaries; a pair created at step s is appended both as two product records and as
two children, which are stepped from step s + 1 on.  The whole run is recorded once
into a CUDA graph by sfq_mc_run.  This module only allocates buffers and calls the
C ABI; all arithmetic happens in libsfq's kernels.
"""
import numpy as np
import torch

from . import sfq


class BatchRun:
    """Device buffers of one batched run.

    d: a workload dict with px, py, pz, tau, flags, k0 (uint32 phase index), amp
    (per-particle amplitude), table (cos table) and k_step; `products_cap` bounds the
    product records (records beyond it are counted as dropped)."""

    def __init__(self, ctx: "sfq.Context", d, products_cap, children_cap=None):
        dev, dt = ctx.device, ctx.dtype
        self.ctx = ctx
        T = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev)
        n = int(d["px"].size)
        self.n = n
        self.P = sfq.ParticleBuffers(T(d["px"]), T(d["py"]), T(d["pz"]), T(d["tau"]), T(d["flags"]))
        self.table = T(d["table"])
        self.k0 = T(np.asarray(d["k0"]).view(np.int32))
        self.amp = T(d["amp"])
        self.F = sfq.FieldSource.plane_wave(self.k0, self.table, d["k_step"], amp=self.amp)
        if children_cap is None:
            n_photons = int((((np.asarray(d["flags"]) >> sfq.SFQ_SPECIES_SHIFT) & 3) == sfq.SFQ_PHOTON).sum())
            children_cap = 2 * n_photons + 64          # a photon converts at most once
        cap = max(int(children_cap), 64)
        z = lambda dtype: torch.zeros(cap, dtype=dtype, device=dev)
        self.spawn_count = torch.zeros(2, dtype=torch.int64, device=dev)
        self.L = sfq.ParticleBuffers(z(dt), z(dt), z(dt), z(torch.float64), z(torch.uint8), ids=z(torch.int64),
                                     n_dev=self.spawn_count)
        self.lk0 = z(torch.int32)
        self.lamp = z(dt)
        self.spawn = sfq.SpawnBuffers(self.L, k0=self.lk0, amp=self.lamp)
        self.spawn.count = self.spawn_count
        self.FL = sfq.FieldSource.plane_wave(self.lk0, self.table, d["k_step"], amp=self.lamp)
        self.out = sfq.ProductBuffers(int(products_cap), dt, dev)
        self.counters = sfq.counters_tensor(dev)

    def autotune(self, step=0, sample_n=0):
        """Picks the launch shape of the primaries' step (kept in the context)."""
        return self.ctx.autotune_step(self.P, self.F, step, sample_n)

    def run(self, step0, nsteps, graph=True):
        if graph:
            self.ctx.mc_run(self.P, self.F, step0, nsteps, self.out, children=self.L, children_fields=self.FL,
                            spawn=self.spawn, counters=self.counters)
        else:
            for s in range(step0, step0 + nsteps):
                self.ctx.mc_step(self.L, self.FL, s, self.out, counters=self.counters)
                self.ctx.mc_step(self.P, self.F, s, self.out, spawn=self.spawn, counters=self.counters)

    def n_children(self):
        return min(int(self.spawn_count[0].item()), self.L.n)

    def sort(self, scratch=None):
        self.ctx.sort_products(self.out, scratch=scratch)
