// sfq_launch.cuh -- launchers of one precision; included by sfq_launch_f32.cu and
// sfq_launch_f64.cu with SFQ_T set to float or double.
#pragma once
#include "sfq_internal.h"
#include "sfq_step_tma.cuh"

namespace sfq {

template <typename T>
static Tables<T> tables_of(const sfq_ctx *ctx) {
    Tables<T> t;
    t.nlc_rate = static_cast<const T *>(ctx->d_nlc_rate);
    t.nbw_rate = static_cast<const T *>(ctx->d_nbw_rate);
    t.nlc_inv = static_cast<const T *>(ctx->d_nlc_inv);
    t.nbw_inv = static_cast<const T *>(ctx->d_nbw_inv);
    return t;
}

template <typename T>
static cudaError_t launch_rate_t(const RateLaunch &L, bool pair) {
    if (L.n == 0) return cudaSuccess;
    const T *g = static_cast<const T *>(L.gamma), *x = static_cast<const T *>(L.chi);
    T *out = static_cast<T *>(L.rate);
    const T *tab = static_cast<const T *>(L.table);
    if (pair)
        rate_kernel<T, true><<<L.grid, 256, 0, L.stream>>>(L.n, g, x, out, tab, (T)L.pref, L.counters);
    else
        rate_kernel<T, false><<<L.grid, 256, 0, L.stream>>>(L.n, g, x, out, tab, (T)L.pref, L.counters);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_sample_t(const SampleLaunch &L, bool pair) {
    if (L.n == 0) return cudaSuccess;
    const T *x = static_cast<const T *>(L.chi), *r = static_cast<const T *>(L.r);
    T *a = static_cast<T *>(L.a), *b = static_cast<T *>(L.b);
    const T *inv = static_cast<const T *>(L.inv);
    if (pair)
        sample_kernel<T, true><<<L.grid, 256, 0, L.stream>>>(L.n, x, r, a, b, inv, L.counters);
    else
        sample_kernel<T, false><<<L.grid, 256, 0, L.stream>>>(L.n, x, r, a, b, inv, L.counters);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_uniforms_t(int64_t n, const uint64_t *id, uint32_t step, uint32_t tag, uint64_t seed,
                                     void *u, cudaStream_t s, int grid) {
    if (n == 0) return cudaSuccess;
    uniforms_kernel<T><<<grid, 256, 0, s>>>(n, id, step, tag, seed, static_cast<T *>(u));
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_step_t(const StepLaunch &L) {
    const sfq_particles &p = *L.p;
    const sfq_fields &f = *L.f;
    const sfq_ctx *ctx = L.ctx;
    if (p.n == 0) return cudaSuccess;
    StepArgs<T> a{};
    a.n = p.n;
    a.px = static_cast<T *>(p.px); a.py = static_cast<T *>(p.py); a.pz = static_cast<T *>(p.pz);
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
    a.tab = tables_of<T>(ctx);
    a.counters = L.counters;
    const bool pw = f.kind == SFQ_FIELDS_PLANE_WAVE;
    // TMA-staged kernel: one persistent block per SM; chosen automatically when every
    // SM gets at least one full tile
    constexpr int TILE = TmaStage<T, FK_SOA>::TILE;
    const bool tma = L.variant == 2 || (L.variant == 0 && p.n >= (int64_t)TILE * ctx->num_sms);
    if (tma) {
        // 16 consumer warps with 1024/16 particles each, or 8 warps with twice as many per lane (ppt = 4)
        const bool w8 = L.ppt == 4;
        void (*kern)(const StepArgs<T>) =
            pw ? (w8 ? mc_step_tma_kernel<T, FK_PW, 8> : mc_step_tma_kernel<T, FK_PW, 16>)
               : (w8 ? mc_step_tma_kernel<T, FK_SOA, 8> : mc_step_tma_kernel<T, FK_SOA, 16>);
        const int threads = 32 * ((w8 ? 8 : 16) + 1);
        const size_t smem = pw ? tma_smem_bytes<T, FK_PW>() : tma_smem_bytes<T, FK_SOA>();
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        const int64_t ntiles = (p.n + TILE - 1) / TILE;
        int grid = L.grid > 0 ? L.grid : ctx->num_sms;
        if (ntiles < grid) grid = (int)ntiles;
        kern<<<grid, threads, smem, L.stream>>>(a);
        return cudaGetLastError();
    }
    void (*kern)(const StepArgs<T>) = nullptr;
    switch ((pw ? 10 : 0) + L.ppt) {
        case 1: kern = mc_step_kernel<T, FK_SOA, 1>; break;
        case 4: kern = mc_step_kernel<T, FK_SOA, 4>; break;
        case 11: kern = mc_step_kernel<T, FK_PW, 1>; break;
        case 12: kern = mc_step_kernel<T, FK_PW, 2>; break;
        case 14: kern = mc_step_kernel<T, FK_PW, 4>; break;
        default: kern = mc_step_kernel<T, FK_SOA, 2>; break;
    }
    int grid = L.grid;
    if (grid <= 0) {
        // one wave of resident blocks: a multiple of the SM count
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, STEP_BS, 0);
        if (e != cudaSuccess || per_sm < 1) per_sm = 1;
        grid = per_sm * ctx->num_sms;
        const int64_t chunks = (p.n + 32 * L.ppt - 1) / (32 * L.ppt);
        const int64_t need = (chunks + STEP_BS / 32 - 1) / (STEP_BS / 32);
        if (need < grid) grid = (int)(need > 0 ? need : 1);
    }
    kern<<<grid, STEP_BS, 0, L.stream>>>(a);
    return cudaGetLastError();
}

}  // namespace sfq
