// sfq_launch.cuh -- launchers of one precision; included by sfq_launch_f32.cu and
// sfq_launch_f64.cu with SFQ_T set to float or double.
#pragma once
#include "sfq_internal.h"
#include "sfq_fused.cuh"
#include "sfq_push.cuh"
#include "sfq_step_tma.cuh"

namespace sfq {

template <typename T>
static Tables<T> tables_of(const sfq_ctx *ctx) {
    Tables<T> t;
    t.nlc_rate = static_cast<const T *>(ctx->d_nlc_rate);
    t.nbw_rate = static_cast<const T *>(ctx->d_nbw_rate);
    t.nlc_inv = static_cast<const T *>(ctx->d_nlc_inv);
    t.nbw_inv = static_cast<const T *>(ctx->d_nbw_inv);
    t.k23 = static_cast<const T *>(ctx->d_k23);
    t.ki13 = static_cast<const T *>(ctx->d_ki13);
    t.nlc_inv_r = static_cast<const T *>(ctx->d_nlc_inv_r);
    t.nbw_inv_r = static_cast<const T *>(ctx->d_nbw_inv_r);
    t.tr = ctx->inv_tr;
    return t;
}

template <typename T>
static cudaError_t launch_rate_t(const RateLaunch &L, bool pair) {
    if (L.n == 0) return cudaSuccess;
    const T *g = static_cast<const T *>(L.gamma), *x = static_cast<const T *>(L.chi);
    T *out = static_cast<T *>(L.rate);
    const T *tab = static_cast<const T *>(L.table);
    auto kern = pair ? (L.cheb ? rate_kernel<T, true, true> : rate_kernel<T, true, false>)
                     : (L.cheb ? rate_kernel<T, false, true> : rate_kernel<T, false, false>);
    kern<<<L.grid, 256, 0, L.stream>>>(L.n, g, x, out, tab, (T)L.pref, L.counters, (T)L.pair_chi_min);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_sample_t(const SampleLaunch &L, bool pair) {
    if (L.n == 0) return cudaSuccess;
    const T *x = static_cast<const T *>(L.chi), *r = static_cast<const T *>(L.r);
    T *a = static_cast<T *>(L.a), *b = static_cast<T *>(L.b);
    Tables<T> tab = tables_of<T>(L.ctx);
    if (L.ctx->eval == SFQ_EVAL_CLENSHAW) {
        // the comparison evaluator: Chebyshev pieces of the full tables, Clenshaw's recurrence
        tab.nlc_inv = static_cast<const T *>(L.ctx->d_nlc_inv_ch);
        tab.nbw_inv = static_cast<const T *>(L.ctx->d_nbw_inv_ch);
        if (pair)
            sample_kernel<T, true, false, true><<<L.grid, 256, 0, L.stream>>>(L.n, x, r, a, b, tab, L.counters);
        else
            sample_kernel<T, false, false, true><<<L.grid, 256, 0, L.stream>>>(L.n, x, r, a, b, tab, L.counters);
        return cudaGetLastError();
    }
    const bool tr = tab.tr > 0;
    if (pair && tr)
        sample_kernel<T, true, true><<<L.grid, 256, 0, L.stream>>>(L.n, x, r, a, b, tab, L.counters);
    else if (pair)
        sample_kernel<T, true, false><<<L.grid, 256, 0, L.stream>>>(L.n, x, r, a, b, tab, L.counters);
    else if (tr)
        sample_kernel<T, false, true><<<L.grid, 256, 0, L.stream>>>(L.n, x, r, a, b, tab, L.counters);
    else
        sample_kernel<T, false, false><<<L.grid, 256, 0, L.stream>>>(L.n, x, r, a, b, tab, L.counters);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_uniforms_t(int64_t n, const uint64_t *id, uint32_t step, uint32_t tag, uint64_t seed,
                                     void *u, cudaStream_t s, int grid) {
    if (n == 0) return cudaSuccess;
    uniforms_kernel<T><<<grid, 256, 0, s>>>(n, id, step, tag, seed, static_cast<T *>(u));
    return cudaGetLastError();
}

// Dynamic shared-memory limits of the TMA-staged kernels, set once per process (and before
// any stream capture, where the launch itself is recorded).
// The TMA-staged shapes compiled with the truncated samplers (TRUNC) are limited to 16
// consumer warps; the warp-streaming ones to 2 particles per lane.
constexpr int TRUNC_CW = 16, TRUNC_PPT = 2;

template <typename T, bool TRUNC>
static cudaError_t prepare_step_t() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaSuccess;
#define SFQ_PREP(CWV)                                                                                         \
    if (e == cudaSuccess)                                                                                     \
        e = cudaFuncSetAttribute(mc_step_tma_kernel<T, FK_SOA, CWV, TRUNC>,                                  \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma_smem_bytes<T, FK_SOA, CWV>()); \
    if (e == cudaSuccess)                                                                                     \
        e = cudaFuncSetAttribute(mc_step_tma_kernel<T, FK_PW, CWV, TRUNC>,                                   \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma_smem_bytes<T, FK_PW, CWV>());
    if constexpr (TRUNC) {
        SFQ_PREP(TRUNC_CW)
    } else {
        SFQ_PREP(8)
        SFQ_PREP(16)
        SFQ_PREP(20)
    }
#undef SFQ_PREP
    if (e == cudaSuccess) done = true;
    return e;
}

// Kernel arguments of one step (or of the first step of a fused run) from the C descriptors.
template <typename T>
static StepArgs<T> make_step_args(const StepLaunch &L) {
    const sfq_particles &p = *L.p;
    const sfq_fields &f = *L.f;
    const sfq_ctx *ctx = L.ctx;
    StepArgs<T> a{};
    a.n = p.n;
    a.n_dev = p.n_dev;
    a.px = static_cast<T *>(p.px); a.py = static_cast<T *>(p.py); a.pz = static_cast<T *>(p.pz);
    for (int k = 0; k < 3; ++k) {
        a.fprev[k] = static_cast<T *>(p.fprev[k]);
        a.dfprev[k] = static_cast<T *>(p.dfprev[k]);
    }
    a.lepton_model = p.lepton_model;
    a.tau = p.tau;
    a.id = p.id;
    a.id_base = p.id_base;
    a.flags = p.flags;
    a.ex = static_cast<const T *>(f.ex); a.ey = static_cast<const T *>(f.ey); a.ez = static_cast<const T *>(f.ez);
    a.bx = static_cast<const T *>(f.bx); a.by = static_cast<const T *>(f.by); a.bz = static_cast<const T *>(f.bz);
    a.k0 = f.k0;
    a.amp = static_cast<const T *>(f.amp);
    a.amp0 = (T)f.amp0;
    a.pw_table = static_cast<const T *>(f.table);
    a.n_table = f.n_table;
    a.pw_offset = f.kind == SFQ_FIELDS_PLANE_WAVE
                      ? (uint32_t)(((uint64_t)L.step * (uint64_t)f.k_step) % (uint64_t)f.n_table)
                      : 0u;
    a.cap = L.out->capacity;
    a.opx = static_cast<T *>(L.out->px); a.opy = static_cast<T *>(L.out->py); a.opz = static_cast<T *>(L.out->pz);
    a.opid = L.out->parent_id;
    a.ostep = L.out->step;
    a.ometa = L.out->meta;
    a.ocount = L.out->count;
    if (L.spawn) {
        const sfq_spawn &s = *L.spawn;
        a.scap = s.p.n;
        a.spx = static_cast<T *>(s.p.px); a.spy = static_cast<T *>(s.p.py); a.spz = static_cast<T *>(s.p.pz);
        a.stau = s.p.tau;
        a.sid = const_cast<uint64_t *>(s.p.id);
        a.sflags = s.p.flags;
        for (int k = 0; k < 3; ++k) {
            a.sfp[k] = static_cast<T *>(s.p.fprev[k]);
            a.sdf[k] = static_cast<T *>(s.p.dfprev[k]);
        }
        a.sk0 = s.k0;
        a.samp = static_cast<T *>(s.amp);
        a.scount = s.count;
    }
    a.step = L.step;
    a.seed = ctx->cfg.seed;
    a.prefdt = (T)(ctx->pref * ctx->cfg.dt);
    a.inv_rho = (T)(1.0 / ctx->rho);
    a.rho = (T)ctx->rho;
    a.inv_dt = (T)(1.0 / ctx->cfg.dt);
    a.dt = (T)ctx->cfg.dt;
    a.inv_dt2 = (T)(1.0 / (ctx->cfg.dt * ctx->cfg.dt));
    a.pair_chi_min = (T)ctx->pair_chi_min;
    a.tab = tables_of<T>(ctx);
    a.counters = L.counters;
    if (ctx->surr || ctx->defer_q.count) {
        const sfq_event_queue &q = ctx->surr ? ctx->surr_q : ctx->defer_q;
        a.qcap = q.capacity;
        a.qidx = q.index;
        a.qchi = q.chi; a.qr = q.r; a.qg = q.gamma;
        a.qpx = q.px; a.qpy = q.py; a.qpz = q.pz;
        a.qcount = q.count;
    }
    return a;
}

template <typename T, bool TRUNC>
static cudaError_t launch_step_t(const StepLaunch &L) {
    const sfq_particles &p = *L.p;
    const sfq_fields &f = *L.f;
    const sfq_ctx *ctx = L.ctx;
    if (p.n == 0) return cudaSuccess;
    const StepArgs<T> a = make_step_args<T>(L);
    const bool pw = f.kind == SFQ_FIELDS_PLANE_WAVE;
    // TMA-staged kernel: one persistent block per SM; chosen automatically when every
    // SM gets at least one full tile.  `ppt` selects the consumer warps per block.
    const int cw = TRUNC ? TRUNC_CW : ((L.ppt == 8 || L.ppt == 16 || L.ppt == 20) ? L.ppt : 16);
    const int tile = cw * (sizeof(T) == 4 ? 64 : 32);
    // the beyond-LCFA model runs on the warp-streaming kernel (its state is read directly)
    const bool tma = !L.cascade && p.lepton_model == SFQ_LEPTON_LCFA_OD &&
                     (L.variant == 2 || (L.variant == 0 && p.n >= (int64_t)tile * ctx->num_sms));
    if (tma) {
        void (*kern)(const StepArgs<T>) = nullptr;
        size_t smem = 0;
#define SFQ_TMA_CASE(CWV)                                                                             \
    case CWV:                                                                                         \
        kern = pw ? mc_step_tma_kernel<T, FK_PW, CWV, TRUNC> : mc_step_tma_kernel<T, FK_SOA, CWV, TRUNC>; \
        smem = pw ? tma_smem_bytes<T, FK_PW, CWV>() : tma_smem_bytes<T, FK_SOA, CWV>();                 \
        break;
        if constexpr (TRUNC) {
            switch (cw) {
                default:
                SFQ_TMA_CASE(TRUNC_CW)
            }
        } else {
            switch (cw) {
                SFQ_TMA_CASE(8)
                SFQ_TMA_CASE(20)
                default:
                SFQ_TMA_CASE(16)
            }
        }
#undef SFQ_TMA_CASE
        cudaError_t e = prepare_step_t<T, TRUNC>();
        if (e != cudaSuccess) return e;
        (void)smem;
        const int64_t ntiles = (p.n + tile - 1) / tile;
        int grid = L.grid > 0 ? L.grid : ctx->num_sms;
        if (ntiles < grid) grid = (int)ntiles;
        kern<<<grid, 32 * (cw + 1), smem, L.stream>>>(a);
        return cudaGetLastError();
    }
    void (*kern)(const StepArgs<T>) = nullptr;
    if (L.cascade) {
        // the full cascade (plane-wave fields only) runs its own instance of this kernel
        kern = mc_step_kernel<T, FK_PW, TRUNC ? TRUNC_PPT : 2, TRUNC, true, false, SFQ_LEPTON_MINB>;
    } else if constexpr (TRUNC) {
        kern = pw ? mc_step_kernel<T, FK_PW, TRUNC_PPT, true> : mc_step_kernel<T, FK_SOA, TRUNC_PPT, true>;
    } else if (p.lepton_model != SFQ_LEPTON_LCFA_OD) {
        // beyond-LCFA leptons: their own instance
        kern = pw ? mc_step_kernel<T, FK_PW, 2, false, false, false, SFQ_LEPTON_MINB>
                 : mc_step_kernel<T, FK_SOA, 2, false, false, false, SFQ_LEPTON_MINB>;
    } else {
        switch ((pw ? 10 : 0) + L.ppt) {
            case 1: kern = mc_step_kernel<T, FK_SOA, 1>; break;
            case 4: kern = mc_step_kernel<T, FK_SOA, 4>; break;
            case 11: kern = mc_step_kernel<T, FK_PW, 1>; break;
            case 12: kern = mc_step_kernel<T, FK_PW, 2>; break;
            case 14: kern = mc_step_kernel<T, FK_PW, 4>; break;
            default: kern = mc_step_kernel<T, FK_SOA, 2>; break;
        }
    }
    const int ppt = TRUNC ? TRUNC_PPT : ((L.cascade || p.lepton_model != SFQ_LEPTON_LCFA_OD) ? 2 : L.ppt);
    int grid = L.grid;
    if (grid <= 0) {
        // one wave of resident blocks: a multiple of the SM count
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, STEP_BS, 0);
        if (e != cudaSuccess || per_sm < 1) per_sm = 1;
        grid = per_sm * ctx->num_sms;
        const int64_t chunks = (p.n + 32 * ppt - 1) / (32 * ppt);
        const int64_t need = (chunks + STEP_BS / 32 - 1) / (STEP_BS / 32);
        if (need < grid) grid = (int)(need > 0 ? need : 1);
    }
    kern<<<grid, STEP_BS, 0, L.stream>>>(a);
    return cudaGetLastError();
}

// nsteps steps from L.step on in one launch of the fused plane-wave kernel (sfq_fused.cuh).
template <typename T, bool TRUNC>
static cudaError_t launch_fused_t(const StepLaunch &L, uint32_t nsteps) {
    constexpr int PPL = sizeof(T) == 4 ? 4 : 2;
    using CFG = FusedCfg<T, PPL>;
    const sfq_particles &p = *L.p;
    const sfq_fields &f = *L.f;
    if (p.n == 0 || nsteps == 0) return cudaSuccess;
    const StepArgs<T> a = make_step_args<T>(L);
    auto kern = mc_fused_kernel<T, PPL, TRUNC>;
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)CFG::smem(FUSED_TABLE_MAX));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const size_t smem = CFG::smem(f.n_table);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, FUSED_BS, smem);
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    int grid = L.grid > 0 ? L.grid : per_sm * L.ctx->num_sms;
    const int64_t chunks = (p.n + 32 * PPL - 1) / (32 * PPL);
    const int64_t need = (chunks + CFG::WARPS - 1) / CFG::WARPS;
    if (need < grid) grid = (int)need;
    const uint32_t K = f.n_table;
    const uint32_t kstep = f.k_step % K;
    const uint32_t off0 = (uint32_t)(((uint64_t)L.step * (uint64_t)f.k_step) % (uint64_t)K);
    kern<<<grid, FUSED_BS, smem, L.stream>>>(a, L.step, nsteps, off0, kstep);
    return cudaGetLastError();
}

// One Boris push of the population at L.step (sfq_push.cuh).
template <typename T>
static cudaError_t launch_push_t(const StepLaunch &L, double dt) {
    if (L.p->n == 0) return cudaSuccess;
    const StepArgs<T> a = make_step_args<T>(L);
    const int64_t blocks = (L.p->n + 255) / 256;
    const int grid = (int)(blocks < (int64_t)L.ctx->num_sms * 8 ? blocks : (int64_t)L.ctx->num_sms * 8);
    if (L.f->kind == SFQ_FIELDS_PLANE_WAVE)
        push_kernel<T, FK_PW><<<grid, 256, 0, L.stream>>>(a, (T)dt);
    else
        push_kernel<T, FK_SOA><<<grid, 256, 0, L.stream>>>(a, (T)dt);
    return cudaGetLastError();
}

}  // namespace sfq
