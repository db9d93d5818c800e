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
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "10"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
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


def time_mc(sfq, torch, ctx, P, fields_for_step, steps, warmup, out, counters, n, e2e=None):
    """Run warmup + steps MC steps; CUDA events around each launch on the launching stream."""
    stream = torch.cuda.current_stream()
    for s in range(warmup):
        ctx.mc_step(P, fields_for_step(s), s, out, counters=counters)
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
            e2e.prepare(s + 1)                     # next step's copies overlap this step
        ev[k][0].record(stream)
        ctx.mc_step(P, F, s, out, counters=counters)
        ev[k][1].record(stream)
        if e2e is not None:
            _ = counters[:2].cpu()                 # the step's result read back to the host
    t1.record(stream)
    torch.cuda.synchronize()
    total_ms = t0.elapsed_time(t1)
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    return total_ms, launch_ms


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

    def one_path(precision, fields_kind, steps, warmup, with_e2e, sampler_k=None):
        dtype = torch.float32 if precision == "fp32" else torch.float64
        ctx = sfq.Context(ref_len_m=W.REF_LEN, dt=W.DT, precision=precision, seed=12345, device=local)
        if sampler_k:
            ctx.set_sampler_coefficients(sampler_k)
        P = make_state(sfq, torch, d, dtype, device)
        P.id_base = rank * n
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
            v, sh = (int(x) for x in args.shape.split(":"))
            ctx.set_step_shape(v, sh, 0)
            tuned = (v, sh, None)
        else:
            tuned = ctx.autotune_step(P, fs(0), 0)
        clocks = ClockSampler(local)
        clocks.start()
        total_ms, launch_ms = time_mc(sfq, torch, ctx, P, fs, steps, warmup, out, cnt, n)
        clk = clocks.stop()
        c = sfq.counters_dict(cnt)
        e2e = None
        if with_e2e and fields_kind == "soa":
            # end to end through the public API: every step copies its six field arrays
            # from pinned host memory and reads the step's counters back.  The copies run
            # on three copy streams into one of two device buffers, so the copies of step
            # s + 1 overlap the kernel of step s.
            host = [[a.cpu().pin_memory() for a in slabs[s % nslab]] for s in range(min(nslab, 4))]
            dev_f = [[torch.empty_like(a) for a in slabs[0]] for _ in range(2)]

            class E2E:
                streams = [torch.cuda.Stream(device=device) for _ in range(3)]

                def __init__(self):
                    self.done = {}

                def prepare(self, s):
                    main = torch.cuda.current_stream()
                    evs = []
                    for j, (dst, src) in enumerate(zip(dev_f[s % 2], host[s % len(host)])):
                        cs = self.streams[j % 3]
                        cs.wait_stream(main)          # the buffer's previous step has finished
                        with torch.cuda.stream(cs):
                            dst.copy_(src, non_blocking=True)
                        e = torch.cuda.Event()
                        e.record(cs)
                        evs.append(e)
                    self.done[s] = evs

                def fields(self, s):
                    for e in self.done.pop(s):
                        torch.cuda.current_stream().wait_event(e)
                    return sfq.FieldSource.soa(*dev_f[s % 2])

            e2e_fields = E2E()

            P2 = make_state(sfq, torch, d, dtype, device)
            out2 = sfq.ProductBuffers(out.capacity, dtype, device)
            cnt2 = sfq.counters_tensor(device)
            e2e_steps = max(3, min(steps, 20))
            tot2, _ = time_mc(sfq, torch, ctx, P2, fs, e2e_steps, warmup, out2, cnt2, n, e2e=e2e_fields)
            e2e = {"value": n * e2e_steps / (tot2 * 1e-3), "unit": UNIT,
                   "h2d_bytes_per_step": int(sum(a.numel() * a.element_size() for a in dev_f[0])),
                   "d2h_bytes_per_step": 16}
            del host, dev_f, P2, out2
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
        out_c = {"workload": "2^20 e-, gamma0 ~ N(1e4, 5%), head-on plane wave a0 = 150, every product stepped again",
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
        flop_per_sample = 2 * (2 * 64 * 64)            # the two 64 x 64 layers on the tensor cores
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
                 "bound": "alu (SFU: two exponential/reciprocal per SiLU, 192 SiLU per draw)"}
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
        steps, warm = args.steps, args.warmup
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
    main = one_path("fp32", "soa", args.steps, args.warmup, with_e2e=True)
    fused = fused_leg("fp32") if "fused" in legs and args.fused else None
    fused64 = fused_leg("fp64") if "fused64" in legs and args.fused else None
    pw = one_path("fp32", "pw", args.steps, args.warmup, with_e2e=False) if "pw" in legs else None
    f64_steps = max(2, args.steps // 10)
    f64 = one_path("fp64", "soa", f64_steps, max(3, min(args.warmup, 3)), with_e2e=False) if "fp64" in legs else None
    trunc = one_path("fp32", "soa", args.steps, args.warmup, with_e2e=False, sampler_k=8) if "trunc" in legs else None
    batched = batched_leg() if "batched" in legs and args.batched_steps > 0 else None
    casc = cascade_leg() if "cascade" in legs and args.cascade_steps > 0 else None
    evaluators = evaluator_leg() if "evaluators" in legs else None
    surrogate = surrogate_leg() if "surrogate" in legs and args.surrogate_steps > 0 else None

    # max over ranks of the headline time
    t = torch.tensor([main["ms_per_step"]], device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    total_updates = n * world
    value = total_updates / (ms * 1e-3)
    if rank == 0:
        cpu = cpu_baseline(args) if world == 1 else None
        dev_name = torch.cuda.get_device_name(local)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (f64 optical depth)", "data": "synthetic",
            "config": {"workload": WORKLOAD, "particles": n, "fields": "SoA, distinct slab per step",
                       "precision": "fp32-mixed", "l2": "inputs larger than L2 (~760 MB read per step)",
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
            "fp64_path": None if f64 is None else {"value": f64["value"], "unit": UNIT, "ms_per_step": f64["ms_per_step"],
                          "achieved_gbs": f64["achieved_gbs"], "hbm_frac": f64["frac"],
                          "steps": f64["steps"], "bound": "alu (fp64 pipe)",
                          "roofline": {"bound": "alu", "unit": "FP64 instructions/s",
                                       "achieved": f64["value"] * args.fp64_inst_per_update,
                                       "fp64_inst_per_update": args.fp64_inst_per_update,
                                       "frac": args.fp64_pipe_busy,
                                       "source": "ncu of the 2^22 capture: FP64-pipe instructions per update "
                                                 "and sm__pipe_fp64_cycles_active (the pipe's busy fraction)"}},
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


def cpu_baseline(args):
    upd, sec, thr = oracle_sample_run(args.oracle_particles, args.oracle_steps)
    c1 = oracle_config1() if args.oracle_config1 else None
    return {"value": upd / sec, "unit": UNIT, "cores": thr, "kind": "oracle",
            "sample": f"{args.oracle_particles} particles x {args.oracle_steps} steps of the same workload "
                      f"({upd} updates in {sec:.1f} s)",
            "config1": c1}


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
    ap.add_argument("--cascade-steps", type=int, default=100, help="steps of the full-cascade leg")
    ap.add_argument("--legs", default="config1,pw,fp64,trunc,fused,fused64,batched,cascade,evaluators,surrogate",
                    help="legs timed beside the headline step (comma list; the headline always runs)")
    ap.add_argument("--shape", default="",
                    help="fixed launch shape 'variant:shape' of the per-step legs (e.g. 2:16) instead of the autotuner")
    ap.add_argument("--oracle-config1", type=int, default=1, help="also time the oracle on config 1 (0: skip)")
    ap.add_argument("--oracle-particles", type=int, default=512)
    ap.add_argument("--oracle-steps", type=int, default=50)
    # DRAM bytes (read + write) per update of mc_step_tma_kernel<float, SoA, 16 warps>, from the
    # ncu capture summarised in profiles/mc_step_tma_fp32_soa_4M.md (4,194,304 particles;
    # the per-particle streams scale in proportion to n).  Re-measure whenever that kernel
    # changes, and pass --traffic-per-update 0 to report null meanwhile.
    ap.add_argument("--fp64-inst-per-update", type=float, default=69.86,
                    help="FP64-pipe instructions per update of the binary64 step kernel (ncu capture)")
    ap.add_argument("--fp64-pipe-busy", type=float, default=0.874,
                    help="sm__pipe_fp64_cycles_active of the binary64 step kernel (ncu capture)")
    ap.add_argument("--traffic-per-update", type=float, default=51.87,
                    help="DRAM bytes per update of the step kernel from an ncu capture (for roofline.traffic)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
