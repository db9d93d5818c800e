"""Full cascade: a population that grows by its own products.

Every event of a step appends its products as particles of the same population (the photon
of an emission, the two leptons of a conversion), stepped from the next step on with their
own ids, in the plane wave at their primary's phase.  The live count stays on the device.
Between runs of steps the host reads it (8 bytes) and keeps room for the worst case of
the next steps: each particle creates at most two per step, so a run of k steps starts
only when 3^k times the count fits the capacity.  Otherwise the alive particles are first
compacted, in order, into the second buffer set, which is made larger when they still do
not fit.  This module only allocates buffers and calls the C ABI; the steps and the
compaction run in libsfq's kernels.
"""
import numpy as np
import torch

from . import sfq


class _Buffers:
    """One buffer set of the population (capacity `cap`)."""

    def __init__(self, ctx, cap, table, k_step, amp0, with_amp):
        dev, dt = ctx.device, ctx.dtype
        z = lambda dtype: torch.zeros(cap, dtype=dtype, device=dev)
        self.count = torch.zeros(2, dtype=torch.int64, device=dev)      # [0]: live count
        self.P = sfq.ParticleBuffers(z(dt), z(dt), z(dt), z(torch.float64), z(torch.uint8), ids=z(torch.int64),
                                     n_dev=self.count)
        self.k0 = z(torch.int32)
        self.amp = z(dt) if with_amp else None
        self.F = sfq.FieldSource.plane_wave(self.k0, table, k_step, amp=self.amp, amp0=amp0)
        self.cap = cap


class CascadeRun:
    """Device state of one full-cascade run.

    d: a workload dict with px, py, pz, tau, flags, k0 (uint32 phase index), optionally
    amp (per-particle amplitude) or amp0, table and k_step; ids default to 0 ... n-1 and
    must stay below 2^63.  `capacity` is the initial capacity (at least 3 n), and
    `products_cap` bounds the product records.  Leptons follow the optical-depth model
    (the buffers carry no beyond-LCFA state; sfq_cascade_run itself accepts populations
    that do)."""

    def __init__(self, ctx: "sfq.Context", d, capacity, products_cap, ids=None):
        dev = ctx.device
        self.ctx = ctx
        n = int(np.asarray(d["px"]).size)
        cap = max(int(capacity), 3 * n, 64)
        self.table = torch.as_tensor(np.ascontiguousarray(d["table"])).to(dev)
        self.k_step, self.amp0 = d["k_step"], float(d.get("amp0", 0.0))
        self.with_amp = d.get("amp") is not None
        self.A = _Buffers(ctx, cap, self.table, self.k_step, self.amp0, self.with_amp)
        self.B = None
        T = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev)
        P = self.A.P
        P.px[:n] = T(d["px"]).to(ctx.dtype); P.py[:n] = T(d["py"]).to(ctx.dtype); P.pz[:n] = T(d["pz"]).to(ctx.dtype)
        P.tau[:n] = T(np.asarray(d["tau"], dtype=np.float64))
        P.flags[:n] = T(np.asarray(d["flags"], dtype=np.uint8))
        ids = np.arange(n, dtype=np.uint64) if ids is None else np.asarray(ids, dtype=np.uint64)
        if n and int(ids.max()) >= 1 << 63:
            raise ValueError("primary ids must be below 2^63")
        P.ids[:n] = T(ids.view(np.int64))
        self.A.k0[:n] = T(np.asarray(d["k0"], dtype=np.uint32).view(np.int32))
        if self.with_amp:
            self.A.amp[:n] = T(d["amp"]).to(ctx.dtype)
        self.A.count[0] = n
        self.next = torch.zeros(2, dtype=torch.int64, device=dev)
        self.out = sfq.ProductBuffers(int(products_cap), ctx.dtype, dev)
        self.counters = sfq.counters_tensor(dev)
        self.scratch = None
        self.compactions = 0
        self.host_checks = 0

    # -- state ---------------------------------------------------------------------
    @property
    def P(self):
        return self.A.P

    @property
    def F(self):
        return self.A.F

    @property
    def capacity(self):
        return self.A.cap

    def count(self):
        return int(self.A.count[0].item())

    def compact(self, capacity=None):
        """Moves the alive particles, in order, into the other buffer set (of at least
        `capacity`) and makes it the current one; returns the new count."""
        cap = max(int(capacity or 0), self.A.cap)
        if self.B is None or self.B.cap < cap:
            self.B = _Buffers(self.ctx, cap, self.table, self.k_step, self.amp0, self.with_amp)
        need = sfq.cascade_compact_scratch_bytes(self.A.cap)
        if self.scratch is None or self.scratch.numel() < need:
            self.scratch = torch.empty(need, dtype=torch.uint8, device=self.ctx.device)
        self.ctx.cascade_compact(self.A.P, self.A.F, self.B.P, self.B.F, self.scratch)
        self.A, self.B = self.B, self.A
        self.compactions += 1
        return self.count()

    # -- stepping ------------------------------------------------------------------
    def run(self, step0, nsteps, max_chunk=8):
        """Steps step0 ... step0 + nsteps - 1, keeping room so that no particle is lost."""
        s, end = step0, step0 + nsteps
        while s < end:
            n = self.count()
            self.host_checks += 1
            k, m = 0, max(n, 1)
            while s + k < end and k < max_chunk and 3 * m <= self.A.cap:
                m *= 3
                k += 1
            if k == 0:
                n = self.compact()
                if 3 * max(n, 1) > self.A.cap:
                    self.compact(capacity=6 * max(n, 1))
                continue
            self.ctx.cascade_run(self.A.P, self.A.F, self.next, s, k, self.out, counters=self.counters)
            s += k

    def alive(self):
        """Host copies of the live population (in device order)."""
        n = self.count()
        P = self.A.P
        out = dict(px=P.px[:n].cpu().numpy(), py=P.py[:n].cpu().numpy(), pz=P.pz[:n].cpu().numpy(),
                   tau=P.tau[:n].cpu().numpy(), flags=P.flags[:n].cpu().numpy(),
                   id=P.ids[:n].cpu().numpy().view(np.uint64))
        return out
