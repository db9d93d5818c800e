"""Benchmark of the strong-field QED Monte Carlo step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (printed as config.workload): 2^24 electrons, gamma ~ N(2000, 5%),
head-on with a linearly polarised plane wave (a0 = 100, lambda = 0.8 um),
dt = 0.01 laser period, optical-depth LCFA photon emission; collinear photons
appended.  Fields reach the step the way a particle-in-cell code hands them
over: six structure-of-arrays field components per particle, a distinct slab
per step, resident in HBM before the timed region (inputs larger than L2).

The headline `value` is particle-updates/s of the mixed path (binary32
arithmetic, binary64 optical depth).  The plain binary64 path and the in-kernel
plane-wave field source are timed on the same GPU and reported beside it.
Under torchrun (N > 1) every rank steps its own 2^24 particles (weak scaling,
no collective on the data path); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QED particle-updates/s at 2^24 (FP32 vs FP64 path, same GPU) + % of roofline"
UNIT = "particle-updates/s"
N_PARTICLES = 1 << 24
WORKLOAD = "config2: 2^24 e-, gamma~N(2000,5%), head-on plane wave a0=100 @0.8um, dt=0.01T, LCFA NLC, optical depth"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# --- clocks -------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        """Start sampling; returns once the first sample has arrived (or after 3 s), so that
        the timed region that follows is covered from its start."""
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t_end = time.time() + 3.0
            while not self.lines and time.time() < t_end and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --- our arm ------------------------------------------------------------------
def make_state(sfq, torch, d, dtype, device):
    T = lambda a, dt=None: torch.as_tensor(np.ascontiguousarray(a)).to(device=device, dtype=dt)
    P = sfq.ParticleBuffers(T(d["px"], dtype), T(d["py"], dtype), T(d["pz"], dtype),
                            T(d["tau"], torch.float64), T(d["flags"]))
    return P


def field_slabs(torch, d, nslab, dtype, device):
    """Distinct SoA field arrays (6 per step) of the plane wave for steps 0..nslab-1."""
    table = torch.as_tensor(d["table"]).to(device=device, dtype=dtype)
    k0 = torch.as_tensor(d["k0"].astype(np.int64)).to(device)
    K = table.numel()
    amp = torch.tensor(d["amp0"], dtype=dtype, device=device)
    slabs = []
    for s in range(nslab):
        idx = (k0 + (s * d["k_step"]) % K) % K
        f = amp * table[idx]                        # E_y = B_z = a0 cos(phase), one rounding
        z = [torch.zeros_like(f) for _ in range(4)]
        slabs.append((z[0], f, z[1], z[2], z[3], f.clone()))
    return slabs


def time_mc(sfq, torch, ctx, P, fields_for_step, steps, warmup, out, counters, n, e2e=None, reset=None,
            min_repeats=1, min_total_ms=0.0):
    """W warm-up steps (0..W-1), then timed regions of exactly `steps` steps (W..W+K-1), each
    bracketed by a barrier and a device synchronisation; CUDA events around each launch and
    around each region on the launching stream.  With `reset` every region starts from the
    state after the warm-up steps (reset(capture=True) keeps it, reset() restores it, outside
    the timed region), so all regions do the same work; at least `min_repeats` regions, more
    until `min_total_ms` of timed work.
    Returns (region_ms list, launch_ms list of every launch of every region)."""
    stream = torch.cuda.current_stream()
    for s in range(warmup):
        ctx.mc_step(P, fields_for_step(s), s, out, counters=counters)
    if reset is not None:
        reset(capture=True)                         # the state after the warm-up steps
    regions, launch_ms = [], []
    n_regions = None
    while True:
        if reset is not None:
            reset()
        out.reset()
        counters.zero_()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        if torch.distributed.is_initialized():
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0.record(stream)
        if e2e is not None:
            e2e.prepare(warmup)
        for k in range(steps):
            s = warmup + k
            F = fields_for_step(s) if e2e is None else e2e.fields(s)
            if e2e is not None and k + 1 < steps:
                e2e.prepare(s + 1)                 # next step's copies overlap this step
            ev[k][0].record(stream)
            ctx.mc_step(P, F, s, out, counters=counters)
            ev[k][1].record(stream)
            if e2e is not None:
                e2e.collect(s)                     # the step's records and counters to the host
        if e2e is not None:
            e2e.finish()
        t1.record(stream)
        torch.cuda.synchronize()
        regions.append(t0.elapsed_time(t1))
        launch_ms += [a.elapsed_time(b) for a, b in ev]
        if reset is None:
            break
        if n_regions is None:
            # how many regions: decided after the first one, the same on every rank
            want = max(min_repeats, math.ceil(min_total_ms / max(regions[0], 1e-3)))
            t = torch.tensor([min(want, 2000)], device=P.px.device)
            if torch.distributed.is_initialized():
                torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            n_regions = int(t.item())
        if len(regions) >= n_regions:
            break
    return regions, launch_ms


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2301_07684_gb300 import build, sfq
    from paper_2301_07684_gb300 import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    n = args.n
    d = W.config2(n=n, seed=rank)
    hbm_peak, peak_src = peaks()
    res = {}
    ids = None

    def one_path(precision, fields_kind, steps, warmup, with_e2e, sampler_k=None, keep_final=None):
        dtype = torch.float32 if precision == "fp32" else torch.float64
        ctx = sfq.Context(ref_len_m=W.REF_LEN, dt=W.DT, precision=precision, seed=12345, device=local)
        if sampler_k:
            ctx.set_sampler_coefficients(sampler_k)
        P = make_state(sfq, torch, d, dtype, device)
        P.id_base = rank * n
        if args.event_pass and precision == "fp32" and not sampler_k:
            # the deferred event path: the step kernel queues the emissions, an event pass
            # samples and finishes them (identical results to the inline path)
            ctx.set_event_queue(sfq.EventQueue(int(0.12 * n) + 1024, device))
        nslab = steps + warmup
        out = sfq.ProductBuffers(int(0.09 * n * (steps + 1)) + 4096, dtype, device)
        cnt = sfq.counters_tensor(device)
        slabs = None
        if fields_kind == "soa":
            slabs = field_slabs(torch, d, nslab, dtype, device)
            fs = lambda s: sfq.FieldSource.soa(*slabs[s % nslab])
        else:
            table = torch.as_tensor(d["table"]).to(device=device, dtype=dtype)
            k0 = torch.as_tensor(d["k0"].view(np.int32)).to(device)
            F = sfq.FieldSource.plane_wave(k0, table, d["k_step"], amp0=d["amp0"])
            fs = lambda s: F
        # launch shape from the autotuner (timed on a copy of the population)
        if args.shape:
            v, sh, *g = (int(x) for x in args.shape.split(":"))
            ctx.set_step_shape(v, sh, g[0] if g else 0)
            tuned = (v, sh, None)
        else:
            tuned = ctx.autotune_step(P, fs(0), 0)
        init = []

        def reset(capture=False):
            if capture:
                init[:] = [t.clone() for t in (P.px, P.py, P.pz, P.tau, P.flags)]
                return
            for dst, src in zip((P.px, P.py, P.pz, P.tau, P.flags), init):
                dst.copy_(src)

        clocks = ClockSampler(local)
        clocks.start()
        regions, launch_ms = time_mc(sfq, torch, ctx, P, fs, steps, warmup, out, cnt, n, reset=reset,
                                     min_repeats=args.repeats, min_total_ms=args.min_timed_ms)
        clk = clocks.stop()
        total_ms = statistics.median(regions)
        c = sfq.counters_dict(cnt)
        final = None
        if keep_final:
            # the last region's final state and records, for the oracle's replay of sampled lineages
            final = {"ids": keep_final, "px": P.px[keep_final].cpu().numpy(), "py": P.py[keep_final].cpu().numpy(),
                     "pz": P.pz[keep_final].cpu().numpy(), "tau": P.tau[keep_final].cpu().numpy(),
                     "flags": P.flags[keep_final].cpu().numpy()}
            k = min(out.n(), out.capacity)
            sel = torch.as_tensor(keep_final, device=device) + P.id_base
            m = torch.isin(out.parent_id[:k], sel)
            final["records"] = dict(px=out.px[:k][m].cpu().numpy(), py=out.py[:k][m].cpu().numpy(),
                                    pz=out.pz[:k][m].cpu().numpy(),
                                    parent_id=(out.parent_id[:k][m] - P.id_base).cpu().numpy().view(np.uint64),
                                    step=out.step[:k][m].cpu().numpy().view(np.uint32),
                                    meta=out.meta[:k][m].cpu().numpy())
        del init
        e2e = None
        if with_e2e and fields_kind == "soa":
            # end to end through the public API: every step copies its six field arrays from
            # pinned host memory and brings the step's product records and counters back to
            # pinned host memory.  The field copies run on three copy streams into one of two
            # device buffers, so the copies of step s + 1 overlap the kernel of step s; the
            # records of step s go back on a fourth stream while step s + 1 runs.
            e2e_steps = max(3, min(steps, 20))
            host = [[a.cpu().pin_memory() for a in slabs[s % nslab]] for s in range(min(nslab, 4))]
            dev_f = [[torch.empty_like(a) for a in slabs[0]] for _ in range(2)]
            P2 = make_state(sfq, torch, d, dtype, device)
            P2.id_base = rank * n
            out2 = sfq.ProductBuffers(int(0.09 * n * (warmup + e2e_steps + 1)) + 4096, dtype, device)
            cnt2 = sfq.counters_tensor(device)
            hcap = int(0.09 * n * (e2e_steps + 1)) + 4096
            hrec = [torch.empty(hcap, dtype=t.dtype).pin_memory()
                    for t in (out2.px, out2.py, out2.pz, out2.parent_id, out2.step, out2.meta)]
            hcnt = torch.zeros((e2e_steps + warmup + 1, 16), dtype=torch.int64).pin_memory()

            class E2E:
                streams = [torch.cuda.Stream(device=device) for _ in range(3)]
                back = torch.cuda.Stream(device=device)

                def __init__(self):
                    self.done, self.counted, self.pending = {}, {}, None
                    self.base, self.h2d, self.d2h = 0, 0, 0

                def prepare(self, s):
                    main = torch.cuda.current_stream()
                    evs = []
                    for j, (dst, src) in enumerate(zip(dev_f[s % 2], host[s % len(host)])):
                        cs = self.streams[j % 3]
                        cs.wait_stream(main)          # the buffer's previous step has finished
                        with torch.cuda.stream(cs):
                            dst.copy_(src, non_blocking=True)
                        self.h2d += src.numel() * src.element_size()
                        e = torch.cuda.Event()
                        e.record(cs)
                        evs.append(e)
                    self.done[s] = evs

                def fields(self, s):
                    for e in self.done.pop(s):
                        torch.cuda.current_stream().wait_event(e)
                    return sfq.FieldSource.soa(*dev_f[s % 2])

                def _records(self, s):
                    # the counters of step s are on the host once its event completes: copy the
                    # records it appended, [base, count), while the next step runs
                    self.counted.pop(s).synchronize()
                    end = min(int(hcnt[s, 0]), out2.capacity)
                    a, b = self.base, end
                    with torch.cuda.stream(self.back):
                        for dst, src in zip(hrec, (out2.px, out2.py, out2.pz, out2.parent_id, out2.step,
                                                   out2.meta)):
                            k = min(b, hcap)
                            if k > a:
                                dst[a:k].copy_(src[a:k], non_blocking=True)
                                self.d2h += (k - a) * src.element_size()
                    self.base = end

                def collect(self, s):
                    main = torch.cuda.current_stream()
                    self.back.wait_stream(main)        # step s has written its records and counters
                    with torch.cuda.stream(self.back):
                        hcnt[s, :2].copy_(out2.count, non_blocking=True)
                        hcnt[s, 2:].copy_(cnt2[:14], non_blocking=True)
                    self.d2h += 16 * 8
                    e = torch.cuda.Event()
                    e.record(self.back)
                    self.counted[s] = e
                    if self.pending is not None:
                        self._records(self.pending)
                    self.pending = s

                def finish(self):
                    if self.pending is not None:
                        self._records(self.pending)
                        self.pending = None
                    torch.cuda.current_stream().wait_stream(self.back)

            e2e_fields = E2E()
            # warm-up steps without read-back, then one timed region with it
            regions2, _ = time_mc(sfq, torch, ctx, P2, fs, e2e_steps, warmup, out2, cnt2, n, e2e=e2e_fields)
            tot2 = regions2[0]
            got = int(hcnt[warmup + e2e_steps - 1, 0])
            e2e = {"value": n * e2e_steps / (tot2 * 1e-3), "unit": UNIT,
                   "h2d_bytes_per_step": int(e2e_fields.h2d // e2e_steps),
                   "d2h_bytes_per_step": int(e2e_fields.d2h // e2e_steps),
                   "steps": e2e_steps, "records_returned": got,
                   "note": "per step: six SoA field arrays host to device; the step's product records "
                           "(px, py, pz, parent id, step, meta) and the counters device to host"}
            del host, dev_f, P2, out2, hrec
        # algorithmic bytes per launch: reads p, tau, flags (+ six fields or the phase index);
        # writes tau; per event: p and one product record (p, parent id, step, meta)
        esz = 4 if precision == "fp32" else 8
        rd = 3 * esz + 8 + 1 + (6 * esz if fields_kind == "soa" else 4)
        wr = 8
        ev_bytes = 3 * esz + (3 * esz + 8 + 4 + 1)
        events_per_step = c["events"] / steps
        bytes_per_launch = n * (rd + wr) + events_per_step * ev_bytes
        avg_launch_s = statistics.mean(launch_ms) * 1e-3
        achieved = bytes_per_launch / avg_launch_s / 1e9
        ups = n * steps / (total_ms * 1e-3)
        out_d = dict(value=ups, ms_per_step=total_ms / steps, launch_ms=statistics.mean(launch_ms),
                     regions=len(regions), region_ms={"median": total_ms, "min": min(regions), "max": max(regions)},
                     final=final,
                     achieved_gbs=achieved, frac=achieved / hbm_peak, bytes_per_update=bytes_per_launch / n,
                     events_per_update=events_per_step / n, counters=c, clocks=clk, e2e=e2e,
                     steps=steps, shape={"variant": ["auto", "warp-streaming", "tma-staged"][tuned[0]],
                                         "shape": tuned[1]})
        slabs = None
        ctx.close()
        torch.cuda.empty_cache()
        return out_d

    def batched_leg():
        """Config 4: 64 beams of mixed species in one population, their pairs stepped as
        children, `--batched-steps` steps recorded into one CUDA graph, launch shape from
        the autotuner; products sorted afterwards (timed separately)."""
        from paper_2301_07684_gb300 import batch
        db = W.config4(seed=rank, scale=args.batched_scale)
        nb = int(db["px"].size)
        nsteps_b = args.batched_steps
        ctx = sfq.Context(ref_len_m=W.REF_LEN, dt=W.DT, precision="fp32", seed=777, device=local)
        cap = int(48 * nb) + 4096
        while True:
            b = batch.BatchRun(ctx, db, products_cap=cap)
            b.P.id_base = rank * nb
            variant, shape, tune_ms = b.autotune(sample_n=0)
            init = [t.clone() for t in (b.P.px, b.P.py, b.P.pz, b.P.tau, b.P.flags)]

            def reset():
                for dst, src in zip((b.P.px, b.P.py, b.P.pz, b.P.tau, b.P.flags), init):
                    dst.copy_(src)
                b.spawn_count.zero_()
                b.out.count.zero_()
                b.counters.zero_()

            reset()
            b.run(0, nsteps_b)                     # records the graph (cached) and warms up
            torch.cuda.synchronize()
            c = sfq.counters_dict(b.counters)
            if c["dropped"] == 0 and c["spawn_dropped"] == 0:
                break
            cap = int(1.1 * b.out.n()) + 4096      # grow the product buffer and record again
            del b, init
            torch.cuda.empty_cache()
        reset()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clocks = ClockSampler(local)
        clocks.start()
        e0.record()
        b.run(0, nsteps_b)
        e1.record()
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = e0.elapsed_time(e1)
        c = sfq.counters_dict(b.counters)
        nrec = b.out.n()
        scratch = torch.empty(sfq.sort_scratch_bytes(nrec), dtype=torch.uint8, device=device)
        e0.record()
        b.sort(scratch)
        e1.record()
        torch.cuda.synchronize()
        sort_ms = e0.elapsed_time(e1)
        out_b = {"workload": "64 beams, counts log-uniform in [1e3, 4e6], mixed e-/e+/photon, "
                             "a0 U[10, 300], gamma0 log-U[200, 1e4], plane-wave fields",
                 "particles": nb, "children": b.n_children(), "steps": nsteps_b,
                 "value": c["updates"] / (ms * 1e-3), "unit": UNIT, "ms_graph": ms, "ms_per_step": ms / nsteps_b,
                 "updates": c["updates"], "events": c["events"], "products": nrec,
                 "shape": {"variant": ["auto", "warp-streaming", "tma-staged"][variant], "shape": shape,
                           "tuned_ms_per_step": tune_ms},
                 "sort_ms": sort_ms, "sort_records_per_s": nrec / max(sort_ms, 1e-9) * 1e3,
                 "precision": "fp32-mixed", "graph": "one CUDA graph for all steps", "clocks": clk}
        del b, init, scratch
        ctx.close()
        torch.cuda.empty_cache()
        return out_b

    def config3_leg():
        """Config 3: 2^24 photons converting by nonlinear Breit-Wheeler (optical depth), the
        pairs appended as records and stepped from the next step on as beyond-LCFA leptons
        (local method with the gate, threshold and rejection of Sec. 5); `--config3-steps`
        steps of two launches each (the leptons, then the photons).  Photon and lepton
        updates are counted apart; the roofline counts the beyond-LCFA state."""
        d3 = W.config3(n=n, seed=rank)
        steps3 = args.config3_steps
        ctx = sfq.Context(ref_len_m=W.REF_LEN, dt=W.DT, precision="fp32", seed=77, device=local)
        T = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(device)
        table = T(d3["table"])
        k0 = T(d3["k0"].view(np.int32))
        amp = T(d3["amp"])
        init = [T(d3[k]) for k in ("px", "py", "pz", "tau", "flags")]
        P = sfq.ParticleBuffers(*[t.clone() for t in init])
        P.id_base = rank * n
        Fp = sfq.FieldSource.plane_wave(k0, table, d3["k_step"], amp=amp)
        cap = 2 * n + 64                                   # each photon converts at most once
        z = lambda dtype: torch.zeros(cap, dtype=dtype, device=device)
        spawn_count = torch.zeros(2, dtype=torch.int64, device=device)
        Lp = sfq.ParticleBuffers(z(torch.float32), z(torch.float32), z(torch.float32), z(torch.float64),
                                 z(torch.uint8), ids=z(torch.int64), fprev=[z(torch.float32) for _ in range(3)],
                                 dfprev=[z(torch.float32) for _ in range(3)],
                                 lepton_model=sfq.SFQ_LEPTON_BLCFA_LOCAL, n_dev=spawn_count)
        lk0, lamp = z(torch.int32), z(torch.float32)
        spawn = sfq.SpawnBuffers(Lp, k0=lk0, amp=lamp)
        spawn.count = spawn_count
        Fl = sfq.FieldSource.plane_wave(lk0, table, d3["k_step"], amp=lamp)
        out = sfq.ProductBuffers(3 * n * steps3 // 4 + 4096, torch.float32, device)   # ~34 records per photon
        cnt_l, cnt_p = sfq.counters_tensor(device), sfq.counters_tensor(device)

        def reset():
            for dst, src in zip((P.px, P.py, P.pz, P.tau, P.flags), init):
                dst.copy_(src)
            spawn_count.zero_()
            out.reset()
            cnt_l.zero_()
            cnt_p.zero_()

        for s in range(min(3, steps3)):                    # warm-up, then the run from the start
            ctx.mc_step(Lp, Fl, s, out, counters=cnt_l)
            ctx.mc_step(P, Fp, s, out, spawn=spawn, counters=cnt_p)
        reset()
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        E = lambda: torch.cuda.Event(enable_timing=True)
        evl = [(E(), E()) for _ in range(steps3)]
        evp = [(E(), E()) for _ in range(steps3)]
        t0, t1 = E(), E()
        clocks = ClockSampler(local)
        clocks.start()
        t0.record(stream)
        for s in range(steps3):
            evl[s][0].record(stream)
            ctx.mc_step(Lp, Fl, s, out, counters=cnt_l)
            evl[s][1].record(stream)
            evp[s][0].record(stream)
            ctx.mc_step(P, Fp, s, out, spawn=spawn, counters=cnt_p)
            evp[s][1].record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = t0.elapsed_time(t1)
        ms_l = sum(a.elapsed_time(b) for a, b in evl)
        ms_p = sum(a.elapsed_time(b) for a, b in evp)
        cl, cp = sfq.counters_dict(cnt_l), sfq.counters_dict(cnt_p)
        # algorithmic bytes (binary32 momenta, binary64 optical depth):
        #   photon update: p 12 + tau 8 + flags 1 + phase index 4 + amplitude 4 read, tau 8 written;
        #   conversion: flags 1 + two records (2 x 25) + two stepped leptons (2 x 61: p, tau, id,
        #   flags, force history 24, phase index, amplitude);
        #   lepton update: p 12 + flags 1 + id 8 + phase index 4 + amplitude 4 + force history 24
        #   read, force history 24 written; emission: p 12 + one record 25
        b_p = cp["updates"] * 37 + cp["pairs"] * 173
        b_l = cl["updates"] * 77 + cl["emitted"] * 37
        upd = cp["updates"] + cl["updates"]
        res3 = {"workload": "config3: 2^24 photons, chi_peak log-U[0.1,100], gamma log-U[1e2,1e5], head-on plane "
                            "wave per photon, NBW by optical depth, pairs stepped as beyond-LCFA leptons (local "
                            "method, Sec. 5), fp32 with fp64 optical depth",
                "photons": n, "steps": steps3, "value": upd / (ms * 1e-3), "unit": UNIT, "ms": ms,
                "ms_per_step": ms / steps3, "photon_updates": cp["updates"], "lepton_updates": cl["updates"],
                "photon_updates_per_s": cp["updates"] / (ms_p * 1e-3),
                "lepton_updates_per_s": cl["updates"] / max(ms_l, 1e-9) * 1e3,
                "pairs": cp["pairs"], "leptons": int(spawn_count[0].item()), "emitted": cl["emitted"],
                "blcfa_rejected": cl["blcfa_rejected"], "blcfa_no_emission": cl["blcfa_no_emission"],
                "dropped": cp["dropped"] + cl["dropped"] + cp["spawn_dropped"], "records": out.n(),
                "roofline": {"bound": "hbm", "unit": "GB/s", "peak": hbm_peak,
                             "photon_kernel": {"achieved": b_p / (ms_p * 1e-3) / 1e9,
                                               "frac": b_p / (ms_p * 1e-3) / 1e9 / hbm_peak,
                                               "bytes_per_update": b_p / max(cp["updates"], 1)},
                             "lepton_kernel": {"achieved": b_l / max(ms_l, 1e-9) / 1e6,
                                               "frac": b_l / max(ms_l, 1e-9) / 1e6 / hbm_peak,
                                               "bytes_per_update": b_l / max(cl["updates"], 1)},
                             "whole_step": {"achieved": (b_p + b_l) / (ms * 1e-3) / 1e9,
                                            "frac": (b_p + b_l) / (ms * 1e-3) / 1e9 / hbm_peak}},
                "clocks": clk}
        if rank == 0 and world == 1 and args.config3_oracle_photons > 0:
            res3["cpu_baseline"] = oracle_config3_sample(args.config3_oracle_photons, steps3)
        del P, Lp, out, init
        ctx.close()
        torch.cuda.empty_cache()
        return res3

    def cascade_leg():
        """Full cascade: 2^20 electrons of gamma ~ N(1e4, 5%) head-on with the plane wave of
        a0 = 150, `--cascade-steps` steps in which every product is appended to the population
        and stepped again.  Timed with CUDA events around the whole run, including the
        host's count checks between runs of steps and the compactions they trigger."""
        from paper_2301_07684_gb300 import cascade
        nc = 1 << 20
        dc = W.config2(n=nc, seed=rank + 11, dtype=np.float32, a0=150.0, gamma0=1e4)
        ctx = sfq.Context(ref_len_m=W.REF_LEN, dt=W.DT, precision="fp32", seed=909, device=local)
        ids = np.arange(nc, dtype=np.uint64) + np.uint64(rank * nc)
        nsteps_c = args.cascade_steps

        def fresh():
            return cascade.CascadeRun(ctx, dc, capacity=64 * nc, products_cap=16 * nc, ids=ids)

        warm = fresh()
        warm.run(0, 2)                                  # builds, loads, first launches
        warm.compact()                                  # loads the compaction kernels
        torch.cuda.synchronize()
        del warm
        r = fresh()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clocks = ClockSampler(local)
        clocks.start()
        e0.record()
        r.run(0, nsteps_c)
        e1.record()
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = e0.elapsed_time(e1)
        c = sfq.counters_dict(r.counters)
        # sfq_cascade_compact on its own: the final population (converted photons dead) into
        # the second buffer set, allocated before the timed call
        n_before = r.count()
        r.B = cascade._Buffers(ctx, r.A.cap, r.table, r.k_step, r.amp0, r.with_amp)
        r.scratch = torch.empty(sfq.cascade_compact_scratch_bytes(r.A.cap), dtype=torch.uint8, device=device)
        torch.cuda.synchronize()
        e0.record()
        ctx.cascade_compact(r.A.P, r.A.F, r.B.P, r.B.F, r.scratch)
        e1.record()
        torch.cuda.synchronize()
        ms_compact = e0.elapsed_time(e1)
        r.A, r.B = r.B, r.A
        n_after = r.count()
        # algorithmic bytes: the flags read by the count and the scatter passes (1 B each per
        # particle), and each alive particle's columns read and written (p 12, tau 8, id 8,
        # flags 1, phase index 4 = 33 B in binary32)
        cbytes = 2 * n_before + 66 * n_after
        compaction = {"particles": n_before, "alive": n_after, "ms": ms_compact,
                      "particles_per_s": n_before / (ms_compact * 1e-3),
                      "achieved_gbs": cbytes / (ms_compact * 1e-3) / 1e9,
                      "frac": cbytes / (ms_compact * 1e-3) / 1e9 / hbm_peak, "bytes": cbytes}
        out_c = {"workload": "2^20 e-, gamma0 ~ N(1e4, 5%), head-on plane wave a0 = 150, every product stepped again",
                 "compaction": compaction,
                 "particles": nc, "final_count": r.count(), "capacity": r.capacity, "steps": nsteps_c,
                 "value": c["updates"] / (ms * 1e-3), "unit": UNIT, "ms": ms, "updates": c["updates"],
                 "emitted": c["emitted"], "pairs": c["pairs"], "spawn_dropped": c["spawn_dropped"],
                 "host_checks": r.host_checks, "compactions": r.compactions, "precision": "fp32-mixed",
                 "clocks": clk}
        del r
        ctx.close()
        torch.cuda.empty_cache()
        return out_c

    def evaluator_leg():
        """The table entry points (photon rate, photon and pair samplers) over 2^24 binary32
        elements with each evaluator of the fitted tables: Horner on the monomial pieces,
        Clenshaw on the same pieces in the Chebyshev basis."""
        ne = 1 << 24
        ctx = sfq.Context(ref_len_m=W.REF_LEN, dt=W.DT, precision="fp32", seed=5, device=local)
        g = np.random.default_rng(rank + 3)
        dev = lambda a: torch.as_tensor(a.astype(np.float32)).to(device)
        chi, gam, r = dev(10.0 ** g.uniform(-3, 3, ne)), dev(10.0 ** g.uniform(1, 5, ne)), dev(g.uniform(1e-7, 1 - 1e-7, ne))
        res = {}
        for name, kind in (("horner", sfq.SFQ_EVAL_HORNER), ("clenshaw", sfq.SFQ_EVAL_CLENSHAW)):
            ctx.set_evaluator(kind)
            row = {}
            for what, fn in (("photon_rate", lambda: ctx.photon_rate(gam, chi)),
                             ("photon_xi", lambda: ctx.sample_photon_xi(chi, r)),
                             ("pair_xi", lambda: ctx.sample_pair_xi(chi, r))):
                for _ in range(3):
                    fn()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(10):
                    fn()
                e1.record()
                torch.cuda.synchronize()
                row[what] = ne * 10 / (e0.elapsed_time(e1) * 1e-3)
            res[name] = row
        ctx.close()
        torch.cuda.empty_cache()
        return {"elements": ne, "unit": "elements/s", "precision": "fp32", **res}

    def surrogate_leg():
        """Config 5: the learned inverse-CDF surrogate.  Trained on the GPU (the library's own
        forward/backward/Adam kernels) on 2^22 triples whose targets come from the plain
        fitted sampler, calibrated against it, then timed on 2^26 draws beside the plain
        sampler and the CUDA-core forward."""
        ctx = sfq.Context(ref_len_m=W.REF_LEN, dt=W.DT, precision="fp32", seed=5, device=local)
        net = sfq.Surrogate(ctx, seed=7)
        g = np.random.Generator(np.random.Philox(1000 + rank))
        nt = 1 << 22
        chi_t = torch.as_tensor(np.exp(g.uniform(np.log(1e-3), np.log(100.0), nt)).astype(np.float32)).to(device)
        u_t = torch.as_tensor(((g.integers(0, 1 << 23, nt) + 0.5) / (1 << 23)).astype(np.float32)).to(device)
        lnw_t = net.plain_targets(chi_t, u_t)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        steps_train = args.surrogate_steps
        torch.cuda.synchronize()
        e0.record()
        net.train(chi_t, u_t, lnw_t, steps=steps_train, batch=8192, lr=3e-3, quantize=True, seed=9)
        e1.record()
        torch.cuda.synchronize()
        train_ms = e0.elapsed_time(e1)
        nflag, max_err = net.calibrate(1e-3)
        nd = 1 << 26
        chi_d = torch.as_tensor(np.exp(g.uniform(np.log(1e-3), np.log(100.0), nd)).astype(np.float32)).to(device)
        u_d = torch.as_tensor(((g.integers(0, 1 << 23, nd) + 0.5) / (1 << 23)).astype(np.float32)).to(device)
        cnt = sfq.counters_tensor(device)

        def timed(fn, reps=5):
            fn()
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                e0.record()
                fn()
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            return statistics.median(ts)

        t_tc = timed(lambda: net.sample_photon_xi(chi_d, u_d, use_flags=True, counters=cnt))
        t_tc_raw = timed(lambda: net.sample_photon_xi(chi_d, u_d, use_flags=False))
        t_simt = timed(lambda: net.predict_lnw(chi_d, u_d))
        t_plain = timed(lambda: ctx.sample_photon_xi(chi_d, u_d))
        c = sfq.counters_dict(cnt)
        # algorithmic flops of the layers on the tensor cores: two 64 x 64 layers and the 64 -> 1
        # output (issued as N = 16 with 15 zero rows, which are not counted)
        flop_per_sample = 2 * (2 * 64 * 64) + 2 * 64
        tflops = nd * flop_per_sample / (t_tc_raw * 1e-3) / 1e12
        bf16_peak = None
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
                bf16_peak = float(json.load(fh)["bf16_tflops"])
        except Exception:
            pass
        out_s = {"workload": "2^22 training triples (targets from the plain sampler), 2^26 draws, "
                             "chi log-uniform in [1e-3, 100], u uniform",
                 "train_steps": steps_train, "train_batch": 8192, "train_ms": train_ms,
                 "calibration": {"tol_u": 1e-3, "flagged_cells": nflag, "cells": 4096,
                                 "max_unflagged_err_u": max_err},
                 "draws": nd, "value": nd / (t_tc * 1e-3), "unit": "samples/s", "ms": t_tc,
                 "fallback_fraction": c["surrogate_fallbacks"] / (6 * nd),
                 "network_only": {"ms": t_tc_raw, "samples_per_s": nd / (t_tc_raw * 1e-3),
                                  "tensor_tflops": tflops,
                                  "tensor_frac_of_measured_bf16": (tflops / bf16_peak) if bf16_peak else None},
                 "cuda_core_forward": {"ms": t_simt, "samples_per_s": nd / (t_simt * 1e-3)},
                 "plain_sampler": {"ms": t_plain, "samples_per_s": nd / (t_plain * 1e-3)},
                 "footprint_bytes": {"network_bf16": sfq.Surrogate.num_params() * 2,
                                     "plain_table_f32": 54027 * 4},
                 "bound": "issue and latency (SiLU epilogues: one tanh.approx per unit, 192 per draw; TMEM reads)"}
        net.close()
        # the pair-creation surrogate: trained on the plain pair sampler's ln(-ln y), timed on
        # 2^24 draws (chi log-uniform in [0.1, 100]) beside the plain pair sampler
        pnet = sfq.Surrogate(ctx, seed=17, kind="pair")
        chi_p = torch.as_tensor(np.exp(g.uniform(np.log(0.1), np.log(100.0), nt)).astype(np.float32)).to(device)
        a_p = torch.as_tensor((np.abs(2.0 * ((g.integers(0, 1 << 23, nt) + 0.5) / (1 << 23)) - 1.0))
                              .astype(np.float32)).to(device)
        tgt = pnet.plain_targets(chi_p, a_p)
        e0.record()
        pnet.train(chi_p, a_p, tgt, steps=2 * steps_train, batch=8192, lr=3e-3, quantize=True, seed=19)
        e1.record()
        torch.cuda.synchronize()
        ptrain_ms = e0.elapsed_time(e1)
        pflag, perr = pnet.calibrate(3e-3)
        npd = 1 << 24
        chi_pd = torch.as_tensor(np.exp(g.uniform(np.log(0.1), np.log(100.0), npd)).astype(np.float32)).to(device)
        r_pd = torch.as_tensor(((g.integers(0, 1 << 23, npd) + 0.5) / (1 << 23)).astype(np.float32)).to(device)
        pcnt = sfq.counters_tensor(device)
        t_pn = timed(lambda: pnet.sample_pair_xi(chi_pd, r_pd, use_flags=True, counters=pcnt))
        t_pp = timed(lambda: ctx.sample_pair_xi(chi_pd, r_pd))
        pc = sfq.counters_dict(pcnt)
        out_s["pair"] = {"workload": "2^22 training pairs (targets from the plain pair sampler), 2^24 draws, "
                                     "chi log-uniform in [0.1, 100]",
                         "train_steps": 2 * steps_train, "train_ms": ptrain_ms, "calibration": {"tol_u": 3e-3, "flagged_cells": pflag,
                                                                "max_unflagged_err_u": perr},
                         "value": npd / (t_pn * 1e-3), "unit": "samples/s", "ms": t_pn,
                         "fallback_fraction": pc["surrogate_fallbacks"] / (6 * npd),
                         "plain_sampler": {"ms": t_pp, "samples_per_s": npd / (t_pp * 1e-3)},
                         "footprint_bytes": {"network_bf16": sfq.Surrogate.num_params() * 2,
                                             "plain_table_f32": 43092 * 4}}
        pnet.close()
        ctx.close()
        del chi_t, u_t, lnw_t, chi_d, u_d, chi_p, a_p, tgt, chi_pd, r_pd
        torch.cuda.empty_cache()
        return out_s

    def fused_leg(precision):
        """The config-2 workload with the analytic plane wave, all timed steps in one launch of
        the fused kernel (each particle's state in registers across the steps)."""
        dtype = torch.float32 if precision == "fp32" else torch.float64
        ctx = sfq.Context(ref_len_m=W.REF_LEN, dt=W.DT, precision=precision, seed=12345, device=local)
        P = make_state(sfq, torch, d, dtype, device)
        P.id_base = rank * n
        table = torch.as_tensor(d["table"]).to(device=device, dtype=dtype)
        k0 = torch.as_tensor(d["k0"].view(np.int32)).to(device)
        F = sfq.FieldSource.plane_wave(k0, table, d["k_step"], amp0=d["amp0"])
        steps, warm = args.fused_steps, args.warmup
        out = sfq.ProductBuffers(int(0.09 * n * (steps + 1)) + 4096, dtype, device)
        cnt = sfq.counters_tensor(device)
        ctx.mc_run_fused(P, F, 0, warm, out, counters=cnt)            # warm-up steps
        out.reset()
        cnt.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        e0.record()
        ctx.mc_run_fused(P, F, warm, steps, out, counters=cnt)
        e1.record()
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = e0.elapsed_time(e1)
        c = sfq.counters_dict(cnt)
        esz = 4 if precision == "fp32" else 8
        # the population is read and written once per launch; every record is written
        state_bytes = n * ((3 * esz + 8 + 1 + 4) + (3 * esz + 8 + 1))
        rec_bytes = c["emitted"] * (3 * esz + 8 + 4 + 1)
        res = {"value": n * steps / (ms * 1e-3), "unit": UNIT, "ms": ms, "ms_per_step": ms / steps,
               "steps_per_launch": steps, "launches": 1, "precision": precision,
               "bytes_per_update": (state_bytes + rec_bytes) / (n * steps),
               "events_per_update": c["events"] / (n * steps), "dropped": c["dropped"], "clocks": clk,
               "bound": "issue (per-update arithmetic and event sampling; HBM traffic ~2 B/update)"}
        ctx.close()
        del P, out
        torch.cuda.empty_cache()
        return res

    def config1_leg():
        """Config 1 (FP64, no time stepping): latency of the rate and sampling entry points on
        4096 electrons and 4096 photons, one Philox draw each."""
        d1 = W.config1()
        ctx = sfq.Context(ref_len_m=W.REF_LEN, dt=W.DT, precision="fp64", seed=0, device=local)
        T = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(device=device, dtype=torch.float64)
        ge, xe, gg, xg = T(d1["gamma_e"]), T(d1["chi_e"]), T(d1["gamma_g"]), T(d1["chi_g"])
        ids = torch.as_tensor(d1["id_e"].astype(np.int64)).to(device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        def calls():
            r = ctx.uniforms(ids, step=0, tag=0)[:, 1].contiguous()
            ctx.photon_rate(ge, xe)
            ctx.pair_rate(gg, xg)
            ctx.sample_photon_xi(xe, r)
            ctx.sample_pair_xi(xg, r)

        for _ in range(3):
            calls()
        torch.cuda.synchronize()
        ts = []
        for _ in range(10):
            e0.record()
            calls()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ctx.close()
        return {"workload": "config 1: 4096 e- and 4096 photons, both rates and one energy sample each, FP64",
                "ms": statistics.median(ts), "calls": 5}

    legs = set(args.legs.split(","))
    config1 = config1_leg() if "config1" in legs else None
    replay_ids = (W.sample_ids(n, args.oracle_particles, seed=17).tolist()
                  if world == 1 and args.oracle_particles > 0 else None)
    main = one_path("fp32", "soa", args.steps, args.warmup, with_e2e=True, keep_final=replay_ids)
    fused = fused_leg("fp32") if "fused" in legs and args.fused else None
    fused64 = fused_leg("fp64") if "fused64" in legs and args.fused else None
    pw = one_path("fp32", "pw", args.steps, args.warmup, with_e2e=False) if "pw" in legs else None
    f64_steps = max(2, args.steps // 10)
    f64 = one_path("fp64", "soa", f64_steps, max(3, min(args.warmup, 3)), with_e2e=False) if "fp64" in legs else None
    trunc = one_path("fp32", "soa", args.steps, args.warmup, with_e2e=False, sampler_k=8) if "trunc" in legs else None
    batched = batched_leg() if "batched" in legs and args.batched_steps > 0 else None
    casc = cascade_leg() if "cascade" in legs and args.cascade_steps > 0 else None
    config3 = config3_leg() if "config3" in legs and args.config3_steps > 0 else None
    evaluators = evaluator_leg() if "evaluators" in legs else None
    surrogate = surrogate_leg() if "surrogate" in legs and args.surrogate_steps > 0 else None

    def fp64_entry(f64, sms):
        """The binary64 path against its own roofline: FP64-pipe instructions per second (the
        per-update count from the ncu capture times the measured update rate) over the nominal
        FP64 peak of 1.25 TFLOP/s dense, i.e. 1.25e12 / 2 flops per DFMA / (152 SMs x 2.07 GHz)
        = 1.99 FP64 instructions per clock per SM, at the SM clock sampled during the region."""
        mhz = (f64["clocks"] or {}).get("sm_mhz") or 2070.0
        peak = 1.25e12 / 2 / (152 * 2.07e9) * sms * mhz * 1e6
        ach = f64["value"] * args.fp64_inst_per_update
        return {"value": f64["value"], "unit": UNIT, "ms_per_step": f64["ms_per_step"],
                "achieved_gbs": f64["achieved_gbs"], "hbm_frac": f64["frac"], "steps": f64["steps"],
                "regions": f64["regions"],
                "roofline": {"bound": "alu", "unit": "FP64 instructions/s", "achieved": ach, "peak": peak,
                             "frac": ach / peak, "fp64_inst_per_update": args.fp64_inst_per_update,
                             "peak_source": "nominal 1.25 TFLOP/s dense FP64 = 1.99 DFMA/clk/SM at the sampled clock",
                             "pipe_busy_ncu": args.fp64_pipe_busy,
                             "source": "FP64-pipe instructions per update from the ncu capture of the 2^22 case"}}

    # max over ranks of the headline time
    t = torch.tensor([main["ms_per_step"]], device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    total_updates = n * world
    value = total_updates / (ms * 1e-3)
    if rank == 0:
        replay = None
        if main["final"] is not None:
            replay = dict(d=d, final=main["final"], warmup=args.warmup, steps=args.steps, seed=12345)
        cpu = cpu_baseline(args, replay) if world == 1 and args.oracle_particles > 0 else None
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        dev_name = torch.cuda.get_device_name(local)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (f64 optical depth)", "data": "synthetic",
            "config": {"workload": WORKLOAD, "particles": n, "fields": "SoA, distinct slab per step",
                       "precision": "fp32-mixed", "l2": "inputs larger than L2 (~760 MB read per step)",
                       "event_path": "deferred (step kernel, then an event pass)" if args.event_pass else "inline",
                       "launch_shape": main["shape"],
                       "parallelism": f"dp{world} (independent particles, no collective)"},
            "roofline": {"bound": "hbm", "achieved": main["achieved_gbs"], "peak": hbm_peak, "unit": "GB/s",
                         "frac": main["frac"],
                         "traffic": (args.traffic_per_update * n if args.traffic_per_update else None),
                         "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per update, "
                                           "4,194,304-particle capture scaled to n",
                         "peak_source": peak_src,
                         "bytes_per_update": main["bytes_per_update"]},
            "cpu_baseline": cpu,
            "e2e": main["e2e"],
            "gpu_launches": args.steps,
            "clocks": main["clocks"],
            "regions": {"count": main["regions"], "ms": main["region_ms"]},
            "parity_sample": (cpu or {}).get("parity_sample"),
            "fp64_path": None if f64 is None else fp64_entry(f64, sms),
            "plane_wave_fields": None if pw is None else {"value": pw["value"], "unit": UNIT, "ms_per_step": pw["ms_per_step"],
                                  "achieved_gbs": pw["achieved_gbs"], "frac": pw["frac"],
                                  "bytes_per_update": pw["bytes_per_update"]},
            "sampler_8x8": None if trunc is None else {
                "value": trunc["value"], "unit": UNIT, "ms_per_step": trunc["ms_per_step"], "frac": trunc["frac"],
                "note": "headline workload with the inverse-CDF pieces cut to 8 x 8 Chebyshev coefficients "
                        "(sfq_set_sampler_coefficients; worst w-bar error 6.3e-7)"},
            "config1_latency": config1,
            "fused_plane_wave": fused,
            "fused_plane_wave_fp64": fused64,
            "batched": batched,
            "cascade": casc,
            "config3": config3,
            "evaluators": evaluators,
            "surrogate": surrogate,
            "events_per_update": main["events_per_update"],
            "device": dev_name,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# --- CPU oracle -----------------------------------------------------------------
def oracle_sample_run(n_sample, nsteps, step0=0):
    """Run the FP64 oracle over a bounded sample of the workload; returns (updates, seconds, threads)."""
    from oracle import oracle as O
    from paper_2301_07684_gb300 import workloads as W
    O.build()
    d = W.config2(n=max(n_sample, 1024), seed=0, dtype=np.float32)
    ids = np.arange(n_sample)
    E = np.zeros((n_sample, nsteps, 6))
    for j in range(nsteps):
        (ex, ey, ez), (bx, by, bz) = W.plane_wave_fields(d["k0"][ids], d["amp0"], d["table"], step0 + j)
        E[:, j, 1] = ey
        E[:, j, 5] = bz
    p = np.stack([d["px"][ids], d["py"][ids], d["pz"][ids]], 1).astype(np.float64)
    t = time.perf_counter()
    O.mc_run(p, d["tau"][ids], ids.astype(np.uint64), d["flags"][ids], np.zeros(n_sample, np.uint8), E,
             rho=W.RHO, dt=W.DT, seed=12345, step0=step0, nsteps=nsteps)
    dt = time.perf_counter() - t
    return n_sample * nsteps, dt, O.num_threads()


def oracle_config1(n_sample=1024):
    """The oracle on config 1: the first n_sample of its 4096 electrons and 4096 photons, both
    rates and one energy sample each (quadrature and Brent roots).  Returns the seconds it
    took and the time scaled to the full config."""
    from oracle import oracle as O
    from paper_2301_07684_gb300 import workloads as W
    O.build()
    d = W.config1()
    k = slice(0, n_sample)
    r = O.uniforms_from_words(O.philox(d["id_e"][k], 0, 0, 0))[:, 1]
    pref = O.rate_prefactor(W.RHO)
    t = time.perf_counter()
    O.photon_rate(d["gamma_e"][k], d["chi_e"][k], pref)
    O.pair_rate(d["gamma_g"][k], d["chi_g"][k], pref)
    O.photon_s(r, d["chi_e"][k])
    O.pair_shares(r, d["chi_g"][k])
    sec = time.perf_counter() - t
    return {"sample": f"{n_sample} electrons and {n_sample} photons of config 1", "s": sec,
            "full_config_s": sec * d["chi_e"].size / n_sample}


def oracle_config3_sample(n_photons, nsteps):
    """The oracle on config 3: n_photons photon lineages (the photon, its pair and the pair's
    photons) over all steps.  Updates are counted from the records: a photon converted at
    step s made s + 1 updates and each of its leptons nsteps - 1 - s; an unconverted photon
    made nsteps."""
    from oracle import oracle as O
    from paper_2301_07684_gb300 import workloads as W
    O.build()
    d = W.config3(n=max(n_photons, 1024), seed=0)
    ids = np.arange(n_photons)
    E = np.zeros((n_photons, nsteps, 6))
    for j in range(nsteps):
        (_, ey, _), (_, _, bz) = W.plane_wave_fields(d["k0"][ids], d["amp"][ids], d["table"], j)
        E[:, j, 1], E[:, j, 5] = ey, bz
    p = np.stack([d["px"][ids], d["py"][ids], d["pz"][ids]], 1).astype(np.float64)
    t = time.perf_counter()
    r = O.mc_run(p, d["tau"][ids], ids.astype(np.uint64), d["flags"][ids], (d["flags"][ids] >> 2) & 3, E,
                 rho=W.RHO, dt=W.DT, seed=77, nsteps=nsteps, lepton_mode=O.MODE_BLCFA_LOCAL, step_children=True,
                 cap_products=64 * n_photons * nsteps)
    sec = time.perf_counter() - t
    conv = r["products"][r["products"]["member"] == 1]["step"].astype(np.int64)
    upd = int((n_photons - conv.size) * nsteps + (conv + 1).sum() + 2 * (nsteps - 1 - conv).sum())
    return {"value": upd / sec, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": f"{n_photons} photon lineages x {nsteps} steps of config 3 ({upd} updates in {sec:.1f} s)"}


def oracle_replay(rep):
    """The oracle replays sampled lineages of the timed run: the same particles from the same
    initial state over the warm-up and timed steps (0 .. W+K-1), fields and Philox key, and
    compares the timed steps W .. W+K-1.  Returns
    (updates, seconds, threads, parity), parity comparing the oracle's decisions (the steps
    at which each lineage emitted) with the records the GPU wrote in its last timed region:
    lineages whose decisions match, lineages cut at a near-threshold decision (|tau_d| <=
    1e-6 tau0, counted, compared up to that step), mismatches elsewhere, and the largest
    relative difference of a record's momentum."""
    from oracle import oracle as O
    from paper_2301_07684_gb300 import workloads as W
    O.build()
    d, fin, K, s0 = rep["d"], rep["final"], rep["steps"], rep["warmup"]
    ids = np.asarray(fin["ids"], np.int64)
    E = np.zeros((ids.size, s0 + K, 6))
    for j in range(s0 + K):
        (_, ey, _), (_, _, bz) = W.plane_wave_fields(d["k0"][ids], d["amp0"], d["table"], j)
        E[:, j, 1], E[:, j, 5] = ey, bz
    p = np.stack([d["px"][ids], d["py"][ids], d["pz"][ids]], 1).astype(np.float64)
    t = time.perf_counter()
    orc = O.mc_run(p, d["tau"][ids], ids.astype(np.uint64), d["flags"][ids], np.zeros(ids.size, np.uint8), E,
                   rho=W.RHO, dt=W.DT, seed=rep["seed"], step0=0, nsteps=s0 + K, near_od=1e-6)
    sec = time.perf_counter() - t
    op, gr = orc["products"], fin["records"]
    near = mism = 0
    worst = 0.0
    for j, pid in enumerate(ids.tolist()):
        cut = orc["first_near_step"][j] if orc["first_near_step"][j] >= 0 else s0 + K
        near += orc["first_near_step"][j] >= 0
        # the timed region's records are those of steps W ... W+K-1
        mo = np.nonzero((op["parent_id"] == pid) & (op["step"] >= s0) & (op["step"] < cut))[0]
        mg = np.nonzero((gr["parent_id"] == pid) & (gr["step"] < cut))[0]
        so, sg = np.sort(op["step"][mo]), np.sort(gr["step"][mg])
        if not np.array_equal(so, sg):
            mism += 1
            continue
        mo, mg = mo[np.argsort(op["step"][mo])], mg[np.argsort(gr["step"][mg])]
        for a, b in zip(mo, mg):
            po = op["p"][a]
            pg = np.array([gr["px"][b], gr["py"][b], gr["pz"][b]], np.float64)
            worst = max(worst, float(np.linalg.norm(pg - po) / np.linalg.norm(po)))
    parity = {"lineages": int(ids.size), "steps": K, "events": int(orc["n_events"].sum()),
              "near_threshold_lineages": int(near), "decision_mismatches": int(mism),
              "max_record_rel_diff": worst,
              "protocol": "decisions compared up to the first near-threshold one (|tau_d| <= 1e-6 tau0)"}
    return ids.size * (s0 + K), sec, O.num_threads(), parity


def cpu_baseline(args, replay=None):
    if replay is not None:
        upd, sec, thr, parity = oracle_replay(replay)
        sample = (f"{len(replay['final']['ids'])} sampled particles of the timed run over its "
                  f"{replay['warmup']} + {replay['steps']} steps, replayed from the initial state "
                  f"({upd} updates in {sec:.1f} s)")
    else:
        upd, sec, thr = oracle_sample_run(args.oracle_particles, args.oracle_steps)
        parity = None
        sample = (f"{args.oracle_particles} particles x {args.oracle_steps} steps of the same workload "
                  f"({upd} updates in {sec:.1f} s)")
    c1 = oracle_config1() if args.oracle_config1 else None
    return {"value": upd / sec, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": sample,
            "parity_sample": parity, "config1": c1}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per_step = max(16, args.oracle_particles // 8)
    for s in range(args.warmup):
        oracle_sample_run(per_step, 1, step0=s)
    tot_upd, tot_sec, thr = 0, 0.0, 1
    for s in range(args.steps):
        upd, sec, thr = oracle_sample_run(per_step, 1, step0=args.warmup + s)
        tot_upd += upd
        tot_sec += sec
    value = tot_upd / tot_sec
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_sec / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "particles": N_PARTICLES, "precision": "fp64 oracle"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle",
                             "sample": f"{per_step} particles of the workload per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_PARTICLES)
    ap.add_argument("--batched-steps", type=int, default=500,
                    help="steps of the 64-beam batched run in one CUDA graph (0 skips it)")
    ap.add_argument("--batched-scale", type=float, default=1.0,
                    help="scale of the 64-beam particle counts")
    ap.add_argument("--surrogate-steps", type=int, default=30000,
                    help="training steps of the surrogate leg (0 skips it)")
    ap.add_argument("--fused", type=int, default=1, help="time the fused multi-step plane-wave run (0: skip)")
    ap.add_argument("--fused-steps", type=int, default=200,
                    help="steps in the one timed launch of the fused run (the run it stands for is long)")
    ap.add_argument("--cascade-steps", type=int, default=100, help="steps of the full-cascade leg")
    ap.add_argument("--config3-steps", type=int, default=100, help="steps of the config-3 leg (0 skips it)")
    ap.add_argument("--config3-oracle-photons", type=int, default=32,
                    help="photon lineages of config 3 the oracle replays for its CPU baseline")
    ap.add_argument("--legs", default="config1,pw,fp64,trunc,fused,fused64,batched,cascade,config3,evaluators,surrogate",
                    help="legs timed beside the headline step (comma list; the headline always runs)")
    ap.add_argument("--shape", default="",
                    help="fixed launch shape 'variant:shape[:grid]' of the per-step legs (e.g. 2:16) instead of the autotuner")
    ap.add_argument("--oracle-config1", type=int, default=1, help="also time the oracle on config 1 (0: skip)")
    ap.add_argument("--oracle-particles", type=int, default=512,
                    help="sampled particles of the timed run the oracle replays (CPU baseline and parity sample)")
    ap.add_argument("--event-pass", type=int, default=0,
                    help="1: binary32 per-step legs run the deferred event path (measured slower on GB300: "
                         "0.229 against 0.200 ms per 2^24 step)")
    ap.add_argument("--repeats", type=int, default=10,
                    help="timed regions of --steps steps each (at least); the line reports the median")
    ap.add_argument("--min-timed-ms", type=float, default=1500.0,
                    help="add regions until this much timed work (so the clock sampler sees the region)")
    ap.add_argument("--oracle-steps", type=int, default=50)
    # DRAM bytes (read + write) per update of mc_step_tma_kernel<float, SoA, 16 warps>, from the
    # ncu capture summarised in profiles/mc_step_tma_fp32_soa_4M.md (4,194,304 particles;
    # the per-particle streams scale in proportion to n).  Re-measure whenever that kernel
    # changes, and pass --traffic-per-update 0 to report null meanwhile.
    ap.add_argument("--fp64-inst-per-update", type=float, default=69.86,
                    help="FP64-pipe instructions per update of the binary64 step kernel (ncu capture)")
    ap.add_argument("--fp64-pipe-busy", type=float, default=0.874,
                    help="sm__pipe_fp64_cycles_active of the binary64 step kernel (ncu capture)")
    ap.add_argument("--traffic-per-update", type=float, default=51.46,
                    help="DRAM bytes per update of the step kernel from an ncu capture (for roofline.traffic)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
