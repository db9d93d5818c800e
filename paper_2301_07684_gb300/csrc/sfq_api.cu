// sfq_api.cu -- the C ABI of libsfq (declared in include/sfq.h): configuration,
// table upload, argument validation and kernel launches.  No computation of the
// method happens on the host.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "sfq_device.cuh"
#include "sfq_internal.h"
#include "sfq_tables_layout.h"

namespace {

// CODATA 2018
constexpr double ALPHA = 7.2973525693e-3;          // fine-structure constant
constexpr double LAMBDA_C = 3.8615926796e-13;      // reduced Compton length [m]
constexpr double C_LIGHT = 299792458.0;            // [m/s]
constexpr double PI = 3.14159265358979323846;

sfq_status fail(sfq_ctx *ctx, sfq_status st, const char *msg) {
    if (ctx) ctx->err = msg;
    return st;
}

sfq_status cuda_fail(sfq_ctx *ctx, cudaError_t e, const char *where) {
    if (ctx) {
        ctx->err = std::string(where) + ": " + cudaGetErrorString(e);
    }
    return SFQ_ERR_CUDA;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }
bool aligned8(const void *p) { return ((uintptr_t)p & 7u) == 0; }

int grid_for(const sfq_ctx *ctx, int64_t n, int per_block) {
    // a multiple of the SM count, no more blocks than needed
    const int64_t blocks = (n + per_block - 1) / per_block;
    const int64_t cap = (int64_t)ctx->num_sms * 8;
    return (int)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

bool is_fp64(const sfq_ctx *ctx) { return ctx->cfg.precision == SFQ_FP64; }

}  // namespace

namespace sfq {

sfq_status validate_step(sfq_ctx *ctx, const sfq_particles *p, const sfq_fields *f, const sfq_products *out,
                         const sfq_spawn *spawn, const sfq_counters *counters) {
    if (!p || !f || !out) return fail(ctx, SFQ_ERR_ARG, "null descriptor");
    if (p->n < 0 || out->capacity < 0) return fail(ctx, SFQ_ERR_ARG, "negative size");
    if (p->lepton_model != SFQ_LEPTON_LCFA_OD && p->lepton_model != SFQ_LEPTON_BLCFA_LOCAL &&
        p->lepton_model != SFQ_LEPTON_BLCFA_PUSHED)
        return fail(ctx, SFQ_ERR_ARG, "unknown lepton model");
    if (p->n == 0) return SFQ_OK;
    if (p->lepton_model != SFQ_LEPTON_LCFA_OD) {
        for (int k = 0; k < 3; ++k)
            if (!p->fprev[k] || !p->dfprev[k] || !aligned16(p->fprev[k]) || !aligned16(p->dfprev[k]))
                return fail(ctx, SFQ_ERR_ARG, "beyond-LCFA state arrays null or misaligned");
    }
    if (p->n_dev && !aligned8(p->n_dev)) return fail(ctx, SFQ_ERR_ARG, "n_dev misaligned");
    const void *need16[] = {p->px, p->py, p->pz, p->tau, p->flags};
    for (const void *q : need16)
        if (!q || !aligned16(q)) return fail(ctx, SFQ_ERR_ARG, "particle buffer null or misaligned");
    if (p->id && !aligned16(p->id)) return fail(ctx, SFQ_ERR_ARG, "id misaligned");
    if (f->kind == SFQ_FIELDS_SOA) {
        const void *fl[] = {f->ex, f->ey, f->ez, f->bx, f->by, f->bz};
        for (const void *q : fl)
            if (!q || !aligned16(q)) return fail(ctx, SFQ_ERR_ARG, "field buffer null or misaligned");
    } else if (f->kind == SFQ_FIELDS_PLANE_WAVE) {
        if (!f->k0 || !f->table || f->n_table == 0 || !aligned16(f->k0) || !aligned16(f->table) ||
            (f->amp && !aligned16(f->amp)))
            return fail(ctx, SFQ_ERR_ARG, "plane-wave description null or misaligned");
    } else {
        return fail(ctx, SFQ_ERR_ARG, "unknown field kind");
    }
    if (!out->count || !aligned8(out->count)) return fail(ctx, SFQ_ERR_ARG, "product counter null or misaligned");
    if (out->capacity > 0) {
        const void *ob[] = {out->px, out->py, out->pz, out->parent_id, out->step, out->meta};
        for (const void *q : ob)
            if (!q || !aligned16(q)) return fail(ctx, SFQ_ERR_ARG, "product buffer null or misaligned");
    }
    if (spawn) {
        if (!spawn->count || spawn->p.n < 0) return fail(ctx, SFQ_ERR_ARG, "spawn counter null or negative capacity");
        if (spawn->p.n > 0) {
            const void *sb[] = {spawn->p.px, spawn->p.py, spawn->p.pz, spawn->p.tau, spawn->p.id, spawn->p.flags};
            for (const void *q : sb)
                if (!q || !aligned16(q)) return fail(ctx, SFQ_ERR_ARG, "spawn buffer null or misaligned");
            if (f->kind == SFQ_FIELDS_PLANE_WAVE && !spawn->k0)
                return fail(ctx, SFQ_ERR_ARG, "spawn needs k0 for plane-wave fields");
        }
    }
    if (counters && !aligned8(counters)) return fail(ctx, SFQ_ERR_ARG, "counters misaligned");
    return SFQ_OK;
}

cudaError_t launch_step(const sfq_ctx *ctx, const sfq_particles *p, const sfq_fields *f, uint32_t step,
                        const sfq_products *out, const sfq_spawn *spawn, sfq_counters *counters, cudaStream_t stream,
                        int cascade) {
    if (p->n == 0) return cudaSuccess;
    const int ppt = ctx->step_ppt ? ctx->step_ppt : (ctx->cfg.precision == SFQ_FP64 ? 1 : 2);
    StepLaunch L{ctx, p, f, step, out, spawn, counters, stream, ctx->step_grid, ppt, ctx->step_variant, cascade};
    if ((ctx->surr || ctx->defer_q.count) && !cascade && ctx->cfg.precision == SFQ_FP32 &&
        p->lepton_model == SFQ_LEPTON_LCFA_OD) {
        // photon emissions deferred to a queue, then sampled and finished in a pass of their
        // own: by the surrogate (sfq_set_surrogate) or by the plain sampler (sfq_set_event_queue)
        const sfq_event_queue &q = ctx->surr ? ctx->surr_q : ctx->defer_q;
        cudaError_t e = cudaMemsetAsync(q.count, 0, sizeof(unsigned long long), stream);
        if (e == cudaSuccess) e = launch_step_surr_f32(L);
        if (e == cudaSuccess)
            e = ctx->surr ? launch_surrogate_apply(ctx, p, step, out, counters, stream) : launch_event_pass_f32(L);
        return e;
    }
    return ctx->cfg.precision == SFQ_FP64 ? launch_step_f64(L) : launch_step_f32(L);
}

}  // namespace sfq

extern "C" {

const char *sfq_version(void) { return "libsfq 0.1 (sm_103a)"; }

sfq_status sfq_init(const sfq_config *cfg, sfq_ctx **out) {
    if (!out) return SFQ_ERR_ARG;
    *out = nullptr;
    if (!cfg) return SFQ_ERR_ARG;
    const bool by_len = cfg->ref_len_m > 0.0, by_freq = cfg->ref_omega_si > 0.0;
    if (by_len == by_freq) return SFQ_ERR_ARG;                    // exactly one of the two
    if (!(cfg->dt > 0.0) || !std::isfinite(cfg->dt)) return SFQ_ERR_ARG;
    if (cfg->precision != SFQ_FP32 && cfg->precision != SFQ_FP64) return SFQ_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
        cudaGetLastError();
        return SFQ_ERR_CUDA;
    }
    sfq_ctx *ctx = new (std::nothrow) sfq_ctx();
    if (!ctx) return SFQ_ERR_ARG;
    ctx->cfg = *cfg;
    ctx->device = cfg->device;
    const double ref_len = by_len ? cfg->ref_len_m : C_LIGHT / cfg->ref_omega_si;
    ctx->rho = ref_len / LAMBDA_C;                                // lambda_r / lambda_C
    ctx->pref = ALPHA / (std::sqrt(3.0) * PI) * ctx->rho;        // Eq. pe_rate_3, Eq. pp_tot_real
    DeviceGuard g(ctx->device);
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, ctx->device);
    if (e != cudaSuccess) { delete ctx; return SFQ_ERR_CUDA; }
    ctx->num_sms = prop.multiProcessorCount;
    const sfq::HostTables t = sfq::host_tables(cfg->precision);
    const void *src[6] = {t.nlc_rate, t.nbw_rate, t.nlc_inv, t.nbw_inv, t.k23, t.ki13};
    const size_t bytes[6] = {t.nlc_rate_bytes, t.nbw_rate_bytes, t.nlc_inv_bytes, t.nbw_inv_bytes, t.k23_bytes,
                             t.ki13_bytes};
    void **dst[6] = {&ctx->d_nlc_rate, &ctx->d_nbw_rate, &ctx->d_nlc_inv, &ctx->d_nbw_inv, &ctx->d_k23,
                     &ctx->d_ki13};
    // the 2-D inverse-CDF tables (k = 2, 3) go to the device with every row of a piece
    // padded to 16 bytes, the layout the kernels read with vector loads
    const bool f64 = cfg->precision == SFQ_FP64;
    const size_t esz = f64 ? 8 : 4;
    const int row[6] = {0, 0, (f64 ? NLC_INV_F64_DY : NLC_INV_F32_DY) + 1, (f64 ? NBW_INV_F64_DY : NBW_INV_F32_DY) + 1,
                        0, 0};
    for (int k = 0; k < 6; ++k) {
        if (!src[k] || bytes[k] == 0 || bytes[k] % esz) { sfq_finalize(ctx); return SFQ_ERR_TABLE; }
        // every coefficient of a fitted table is finite
        for (size_t j = 0; j < bytes[k] / esz; ++j) {
            const unsigned char *q = static_cast<const unsigned char *>(src[k]) + j * esz;
            double v;
            if (f64) {
                std::memcpy(&v, q, 8);
            } else {
                float w;
                std::memcpy(&w, q, 4);
                v = w;
            }
            if (!std::isfinite(v)) {
                ctx->err = "fitted table has a non-finite coefficient";
                sfq_finalize(ctx);
                return SFQ_ERR_TABLE;
            }
        }
        std::vector<unsigned char> padded;
        const void *h = src[k];
        size_t nb = bytes[k];
        if (row[k] > 0) {
            const size_t rb = row[k] * esz, pb = sfq::padded_row(row[k], (int)esz) * esz;
            if (bytes[k] % rb) { sfq_finalize(ctx); return SFQ_ERR_TABLE; }
            const size_t rows = bytes[k] / rb;
            padded.assign(rows * pb, 0);
            for (size_t r = 0; r < rows; ++r)
                std::memcpy(padded.data() + r * pb, static_cast<const unsigned char *>(src[k]) + r * rb, rb);
            h = padded.data();
            nb = padded.size();
        }
        e = cudaMalloc(dst[k], nb);
        if (e == cudaSuccess) e = cudaMemcpy(*dst[k], h, nb, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { sfq_finalize(ctx); return SFQ_ERR_CUDA; }
    }
    *out = ctx;
    return SFQ_OK;
}

void sfq_finalize(sfq_ctx *ctx) {
    if (!ctx) return;
    {
        DeviceGuard g(ctx->device);
        sfq::release_graphs(ctx);
        void *ptrs[12] = {ctx->d_nlc_rate, ctx->d_nbw_rate, ctx->d_nlc_inv, ctx->d_nbw_inv, ctx->d_k23, ctx->d_ki13,
                          ctx->d_nlc_inv_r, ctx->d_nbw_inv_r, ctx->d_nlc_rate_ch, ctx->d_nbw_rate_ch,
                          ctx->d_nlc_inv_ch, ctx->d_nbw_inv_ch};
        for (void *p : ptrs)
            if (p) cudaFree(p);
    }
    delete ctx;
}

const char *sfq_last_error(const sfq_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

sfq_status sfq_constants(const sfq_ctx *ctx, double *rho, double *pref) {
    if (!ctx) return SFQ_ERR_ARG;
    if (rho) *rho = ctx->rho;
    if (pref) *pref = ctx->pref;
    return SFQ_OK;
}

static sfq_status rate_common(sfq_ctx *ctx, int64_t n, const void *gamma, const void *chi, void *rate,
                              sfq_counters *counters, void *stream, bool pair) {
    if (!ctx) return SFQ_ERR_ARG;
    if (n < 0) return fail(ctx, SFQ_ERR_ARG, "n < 0");
    if (n == 0) return SFQ_OK;
    if (!gamma || !chi || !rate) return fail(ctx, SFQ_ERR_ARG, "null buffer");
    if (!aligned16(gamma) || !aligned16(chi) || !aligned16(rate) || (counters && !aligned8(counters)))
        return fail(ctx, SFQ_ERR_ARG, "misaligned buffer (16 bytes required)");
    DeviceGuard g(ctx->device);
    const bool ch = ctx->eval == SFQ_EVAL_CLENSHAW;
    const void *table = ch ? (pair ? ctx->d_nbw_rate_ch : ctx->d_nlc_rate_ch)
                           : (pair ? ctx->d_nbw_rate : ctx->d_nlc_rate);
    sfq::RateLaunch L{n, gamma, chi, rate, table, ctx->pref, counters, (cudaStream_t)stream,
                      grid_for(ctx, n, 256 * 4), ctx->pair_chi_min, ch ? 1 : 0};
    const cudaError_t e = is_fp64(ctx) ? sfq::launch_rate_f64(L, pair) : sfq::launch_rate_f32(L, pair);
    return e == cudaSuccess ? SFQ_OK : cuda_fail(ctx, e, pair ? "sfq_pair_rate" : "sfq_photon_rate");
}

sfq_status sfq_photon_rate(sfq_ctx *ctx, int64_t n, const void *gamma, const void *chi, void *rate,
                           sfq_counters *counters, void *stream) {
    return rate_common(ctx, n, gamma, chi, rate, counters, stream, false);
}

sfq_status sfq_pair_rate(sfq_ctx *ctx, int64_t n, const void *gamma, const void *chi, void *rate,
                         sfq_counters *counters, void *stream) {
    return rate_common(ctx, n, gamma, chi, rate, counters, stream, true);
}

sfq_status sfq_uniforms(sfq_ctx *ctx, int64_t n, const uint64_t *id, uint32_t step, uint32_t tag, void *u,
                        void *stream) {
    if (!ctx) return SFQ_ERR_ARG;
    if (n < 0) return fail(ctx, SFQ_ERR_ARG, "n < 0");
    if (n == 0) return SFQ_OK;
    if (!id || !u) return fail(ctx, SFQ_ERR_ARG, "null buffer");
    if (!aligned16(id) || !aligned16(u)) return fail(ctx, SFQ_ERR_ARG, "misaligned buffer (16 bytes required)");
    DeviceGuard g(ctx->device);
    const int grid = grid_for(ctx, n, 256 * 4);
    const cudaError_t e = is_fp64(ctx)
                              ? sfq::launch_uniforms_f64(n, id, step, tag, ctx->cfg.seed, u, (cudaStream_t)stream, grid)
                              : sfq::launch_uniforms_f32(n, id, step, tag, ctx->cfg.seed, u, (cudaStream_t)stream, grid);
    return e == cudaSuccess ? SFQ_OK : cuda_fail(ctx, e, "sfq_uniforms");
}

static sfq_status sample_common(sfq_ctx *ctx, int64_t n, const void *chi, const void *r, void *a, void *b,
                                sfq_counters *counters, void *stream, bool pair) {
    if (!ctx) return SFQ_ERR_ARG;
    if (n < 0) return fail(ctx, SFQ_ERR_ARG, "n < 0");
    if (n == 0) return SFQ_OK;
    if (!chi || !r || !a) return fail(ctx, SFQ_ERR_ARG, "null buffer");
    if (!aligned16(chi) || !aligned16(r) || !aligned16(a) || (b && !aligned16(b)) ||
        (counters && !aligned8(counters)))
        return fail(ctx, SFQ_ERR_ARG, "misaligned buffer (16 bytes required)");
    DeviceGuard g(ctx->device);
    sfq::SampleLaunch L{n, chi, r, a, b, ctx, counters, (cudaStream_t)stream, grid_for(ctx, n, 256 * 4)};
    const cudaError_t e = is_fp64(ctx) ? sfq::launch_sample_f64(L, pair) : sfq::launch_sample_f32(L, pair);
    return e == cudaSuccess ? SFQ_OK : cuda_fail(ctx, e, pair ? "sfq_sample_pair_xi" : "sfq_sample_photon_xi");
}

sfq_status sfq_sample_photon_xi(sfq_ctx *ctx, int64_t n, const void *chi, const void *r, void *xi, void *xi_c,
                                sfq_counters *counters, void *stream) {
    return sample_common(ctx, n, chi, r, xi, xi_c, counters, stream, false);
}

sfq_status sfq_sample_pair_xi(sfq_ctx *ctx, int64_t n, const void *chi, const void *r, void *xi_e, void *xi_p,
                              sfq_counters *counters, void *stream) {
    return sample_common(ctx, n, chi, r, xi_e, xi_p, counters, stream, true);
}

sfq_status sfq_mc_step(sfq_ctx *ctx, const sfq_particles *p, const sfq_fields *f, uint32_t step,
                       const sfq_products *out, const sfq_spawn *spawn, sfq_counters *counters, void *stream) {
    if (!ctx) return SFQ_ERR_ARG;
    const sfq_status st = sfq::validate_step(ctx, p, f, out, spawn, counters);
    if (st != SFQ_OK) return st;
    if (p->n == 0) return SFQ_OK;
    DeviceGuard g(ctx->device);
    const cudaError_t e = sfq::launch_step(ctx, p, f, step, out, spawn, counters, (cudaStream_t)stream);
    return e == cudaSuccess ? SFQ_OK : cuda_fail(ctx, e, "sfq_mc_step");
}

sfq_status sfq_mc_run_fused(sfq_ctx *ctx, const sfq_particles *p, const sfq_fields *f, uint32_t step0,
                            uint32_t nsteps, const sfq_products *out, sfq_counters *counters, void *stream) {
    if (!ctx) return SFQ_ERR_ARG;
    const sfq_status st = sfq::validate_step(ctx, p, f, out, nullptr, counters);
    if (st != SFQ_OK) return st;
    if (f->kind != SFQ_FIELDS_PLANE_WAVE) return fail(ctx, SFQ_ERR_ARG, "fused run: plane-wave fields only");
    if (p->lepton_model != SFQ_LEPTON_LCFA_OD) return fail(ctx, SFQ_ERR_ARG, "fused run: optical-depth leptons only");
    if (f->n_table > (uint32_t)SFQ_FUSED_TABLE_MAX)
        return fail(ctx, SFQ_ERR_ARG, "fused run: cosine table longer than SFQ_FUSED_TABLE_MAX");
    if ((uint64_t)step0 + nsteps > 0xFFFFFFFFull) return fail(ctx, SFQ_ERR_ARG, "step0 + nsteps exceeds 2^32 - 1");
    if (p->n == 0 || nsteps == 0) return SFQ_OK;
    DeviceGuard g(ctx->device);
    sfq::StepLaunch L{ctx, p, f, step0, out, nullptr, counters, (cudaStream_t)stream, 0, 0, 0};
    const cudaError_t e = ctx->cfg.precision == SFQ_FP64 ? sfq::launch_fused_f64(L, nsteps)
                                                         : sfq::launch_fused_f32(L, nsteps);
    return e == cudaSuccess ? SFQ_OK : cuda_fail(ctx, e, "sfq_mc_run_fused");
}

sfq_status sfq_cascade_run(sfq_ctx *ctx, const sfq_particles *p, const sfq_fields *f, unsigned long long *next,
                           uint32_t step0, uint32_t nsteps, const sfq_products *out, sfq_counters *counters,
                           void *stream) {
    if (!ctx) return SFQ_ERR_ARG;
    if (!p || !f) return fail(ctx, SFQ_ERR_ARG, "null descriptor");
    if (f->kind != SFQ_FIELDS_PLANE_WAVE) return fail(ctx, SFQ_ERR_ARG, "cascade: plane-wave fields only");
    if (!p->n_dev || !aligned8(p->n_dev) || !next || !aligned8(next))
        return fail(ctx, SFQ_ERR_ARG, "cascade: device count or append counter null or misaligned");
    if (p->n > 0 && !p->id) return fail(ctx, SFQ_ERR_ARG, "cascade: particle ids required");
    // the population is its own spawn target
    sfq_spawn sp{};
    sp.p = *p;
    sp.p.n_dev = nullptr;
    sp.k0 = const_cast<uint32_t *>(f->k0);
    sp.amp = const_cast<void *>(f->amp);
    sp.count = next;
    const sfq_status st = sfq::validate_step(ctx, p, f, out, &sp, counters);
    if (st != SFQ_OK) return st;
    if ((uint64_t)step0 + nsteps > 0xFFFFFFFFull) return fail(ctx, SFQ_ERR_ARG, "step0 + nsteps exceeds 2^32 - 1");
    if (p->n == 0 || nsteps == 0) return SFQ_OK;
    DeviceGuard g(ctx->device);
    const cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *count = const_cast<unsigned long long *>(p->n_dev);
    cudaError_t e = sfq::launch_cascade_sync(count, next, p->n, true, s);
    for (uint32_t j = 0; j < nsteps && e == cudaSuccess; ++j) {
        e = sfq::launch_step(ctx, p, f, step0 + j, out, &sp, counters, s, 1);
        if (e == cudaSuccess) e = sfq::launch_cascade_sync(count, next, p->n, false, s);
    }
    return e == cudaSuccess ? SFQ_OK : cuda_fail(ctx, e, "sfq_cascade_run");
}

size_t sfq_cascade_compact_scratch_bytes(int64_t capacity) { return sfq::compact_scratch_bytes(capacity); }

sfq_status sfq_table_pieces(int32_t precision, int32_t which, int32_t basis, void *out, size_t *bytes) {
    if (!bytes || (precision != SFQ_FP32 && precision != SFQ_FP64) || which < SFQ_TABLE_NLC_RATE ||
        which > SFQ_TABLE_NBW_INV || (basis != SFQ_EVAL_HORNER && basis != SFQ_EVAL_CLENSHAW))
        return SFQ_ERR_ARG;
    const bool pair = which == SFQ_TABLE_NBW_RATE || which == SFQ_TABLE_NBW_INV;
    const bool inv = which >= SFQ_TABLE_NLC_INV;
    const std::vector<unsigned char> t =
        basis == SFQ_EVAL_HORNER ? sfq::monomial_table(precision, which)
                                 : (inv ? sfq::chebyshev_inv_table(precision, pair)
                                        : sfq::chebyshev_rate_table(precision, pair));
    const size_t cap = *bytes;
    *bytes = t.size();
    if (out) {
        if (cap < t.size()) return SFQ_ERR_CAPACITY;
        std::memcpy(out, t.data(), t.size());
    }
    return SFQ_OK;
}

sfq_status sfq_cascade_compact(sfq_ctx *ctx, const sfq_particles *src, const sfq_fields *fsrc,
                               const sfq_particles *dst, const sfq_fields *fdst, void *scratch, size_t scratch_bytes,
                               void *stream) {
    if (!ctx) return SFQ_ERR_ARG;
    if (!src || !fsrc || !dst || !fdst) return fail(ctx, SFQ_ERR_ARG, "null descriptor");
    if (src->n < 0 || dst->n < src->n) return fail(ctx, SFQ_ERR_ARG, "compaction: dst capacity below src capacity");
    if (fsrc->kind != SFQ_FIELDS_PLANE_WAVE || fdst->kind != SFQ_FIELDS_PLANE_WAVE)
        return fail(ctx, SFQ_ERR_ARG, "compaction: plane-wave fields only");
    if (!src->n_dev || !dst->n_dev || !aligned8(src->n_dev) || !aligned8(dst->n_dev))
        return fail(ctx, SFQ_ERR_ARG, "compaction: device counts null or misaligned");
    if (src->lepton_model != dst->lepton_model) return fail(ctx, SFQ_ERR_ARG, "compaction: lepton models differ");
    if (src->n > 0) {
        const void *b[] = {src->px, src->py, src->pz, src->tau, src->id, src->flags, fsrc->k0,
                           dst->px, dst->py, dst->pz, dst->tau, dst->id, dst->flags, fdst->k0};
        for (const void *q : b)
            if (!q || !aligned16(q)) return fail(ctx, SFQ_ERR_ARG, "compaction: buffer null or misaligned");
        if (!fsrc->amp != !fdst->amp) return fail(ctx, SFQ_ERR_ARG, "compaction: amp given on one side only");
        if (src->lepton_model != SFQ_LEPTON_LCFA_OD)
            for (int k = 0; k < 3; ++k)
                if (!src->fprev[k] || !src->dfprev[k] || !dst->fprev[k] || !dst->dfprev[k])
                    return fail(ctx, SFQ_ERR_ARG, "compaction: beyond-LCFA state arrays null");
    }
    if (!scratch || !aligned16(scratch) || scratch_bytes < sfq::compact_scratch_bytes(src->n))
        return fail(ctx, SFQ_ERR_ARG, "compaction: scratch null, misaligned or too small");
    DeviceGuard g(ctx->device);
    const cudaError_t e = sfq::launch_compact(ctx->cfg.precision, *src, *fsrc, *dst, *fdst, scratch,
                                              (cudaStream_t)stream, ctx->num_sms);
    return e == cudaSuccess ? SFQ_OK : cuda_fail(ctx, e, "sfq_cascade_compact");
}

sfq_status sfq_push(sfq_ctx *ctx, const sfq_particles *p, const sfq_fields *f, uint32_t step, double dt,
                    void *stream) {
    if (!ctx) return SFQ_ERR_ARG;
    sfq_products none{};
    unsigned long long *dummy = nullptr;
    none.count = reinterpret_cast<unsigned long long *>(&dummy);   // only validated, never written
    const sfq_status st = sfq::validate_step(ctx, p, f, &none, nullptr, nullptr);
    if (st != SFQ_OK) return st;
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, SFQ_ERR_ARG, "dt must be positive and finite");
    if (p->n == 0) return SFQ_OK;
    DeviceGuard g(ctx->device);
    sfq::StepLaunch L{ctx, p, f, step, &none, nullptr, nullptr, (cudaStream_t)stream, 0, 0, 0};
    const cudaError_t e = ctx->cfg.precision == SFQ_FP64 ? sfq::launch_push_f64(L, dt) : sfq::launch_push_f32(L, dt);
    return e == cudaSuccess ? SFQ_OK : cuda_fail(ctx, e, "sfq_push");
}

sfq_status sfq_set_pair_rate_cutoff(sfq_ctx *ctx, double chi_min) {
    if (!ctx) return SFQ_ERR_ARG;
    if (!(chi_min >= 0.01) || !(chi_min <= 2000.0))
        return fail(ctx, SFQ_ERR_ARG, "pair-rate cutoff outside [0.01, 2000]");
    ctx->pair_chi_min = chi_min;
    return SFQ_OK;
}

sfq_status sfq_set_evaluator(sfq_ctx *ctx, int32_t kind) {
    if (!ctx) return SFQ_ERR_ARG;
    if (kind != SFQ_EVAL_HORNER && kind != SFQ_EVAL_CLENSHAW) return fail(ctx, SFQ_ERR_ARG, "unknown evaluator");
    if (kind == SFQ_EVAL_CLENSHAW && ctx->inv_tr > 0)
        return fail(ctx, SFQ_ERR_ARG, "the Clenshaw evaluator reads the full tables: set n coefficients first");
    if (kind == SFQ_EVAL_CLENSHAW && !ctx->d_nlc_rate_ch) {
        DeviceGuard g(ctx->device);
        const int prec = ctx->cfg.precision;
        const std::vector<unsigned char> h[4] = {sfq::chebyshev_rate_table(prec, false),
                                                 sfq::chebyshev_rate_table(prec, true),
                                                 sfq::chebyshev_inv_table(prec, false),
                                                 sfq::chebyshev_inv_table(prec, true)};
        void *d[4] = {nullptr, nullptr, nullptr, nullptr};
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
            e = cudaMalloc(&d[k], h[k].size());
            if (e == cudaSuccess) e = cudaMemcpy(d[k], h[k].data(), h[k].size(), cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) {
            for (void *q : d)
                if (q) cudaFree(q);
            return cuda_fail(ctx, e, "sfq_set_evaluator");
        }
        ctx->d_nlc_rate_ch = d[0];
        ctx->d_nbw_rate_ch = d[1];
        ctx->d_nlc_inv_ch = d[2];
        ctx->d_nbw_inv_ch = d[3];
    }
    ctx->eval = kind;
    return SFQ_OK;
}

sfq_status sfq_set_sampler_coefficients(sfq_ctx *ctx, int32_t k) {
    if (!ctx) return SFQ_ERR_ARG;
    const int n = sfq::inv_coefficients(ctx->cfg.precision);
    if (k < n - 2 || k > n) return fail(ctx, SFQ_ERR_ARG, "coefficients per variable must be n, n - 1 or n - 2");
    if (k < n && (ctx->surr || ctx->defer_q.count))
        return fail(ctx, SFQ_ERR_ARG, "truncated samplers with a deferred event path or a surrogate attached");
    if (k < n && ctx->eval == SFQ_EVAL_CLENSHAW)
        return fail(ctx, SFQ_ERR_ARG, "truncated samplers need the Horner evaluator");
    const int tr = n - k;
    DeviceGuard g(ctx->device);
    void *nlc = nullptr, *nbw = nullptr;
    if (tr > 0) {
        const std::vector<unsigned char> hn = sfq::truncated_inv_table(ctx->cfg.precision, false, tr);
        const std::vector<unsigned char> hb = sfq::truncated_inv_table(ctx->cfg.precision, true, tr);
        cudaError_t e = cudaMalloc(&nlc, hn.size());
        if (e == cudaSuccess) e = cudaMalloc(&nbw, hb.size());
        if (e == cudaSuccess) e = cudaMemcpy(nlc, hn.data(), hn.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(nbw, hb.data(), hb.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            if (nlc) cudaFree(nlc);
            if (nbw) cudaFree(nbw);
            return cuda_fail(ctx, e, "sfq_set_sampler_coefficients");
        }
    }
    // work queued with the previous tables finishes before they are freed
    cudaDeviceSynchronize();
    if (ctx->d_nlc_inv_r) cudaFree(ctx->d_nlc_inv_r);
    if (ctx->d_nbw_inv_r) cudaFree(ctx->d_nbw_inv_r);
    ctx->d_nlc_inv_r = nlc;
    ctx->d_nbw_inv_r = nbw;
    ctx->inv_tr = tr;
    return SFQ_OK;
}

sfq_status sfq_sampler_coefficients(const sfq_ctx *ctx, int32_t *n, int32_t *k) {
    if (!ctx) return SFQ_ERR_ARG;
    const int nn = sfq::inv_coefficients(ctx->cfg.precision);
    if (n) *n = nn;
    if (k) *k = nn - ctx->inv_tr;
    return SFQ_OK;
}

sfq_status sfq_set_step_shape(sfq_ctx *ctx, int32_t variant, int32_t ppt, int32_t grid_blocks) {
    if (!ctx) return SFQ_ERR_ARG;
    if (variant < 0 || variant > 2) return fail(ctx, SFQ_ERR_ARG, "variant must be 0, 1 or 2");
    const bool ok = variant == 2 ? (ppt == 0 || ppt == 8 || ppt == 16 || ppt == 20)
                                 : (ppt == 0 || ppt == 1 || ppt == 2 || ppt == 4);
    if (!ok) return fail(ctx, SFQ_ERR_ARG, "shape: 1, 2 or 4 particles per lane (variant 1), 8/16/20 warps (variant 2)");
    if (grid_blocks < 0) return fail(ctx, SFQ_ERR_ARG, "grid_blocks < 0");
    ctx->step_variant = variant;
    ctx->step_ppt = ppt;
    ctx->step_grid = grid_blocks;
    return SFQ_OK;
}

sfq_status sfq_set_event_queue(sfq_ctx *ctx, const sfq_event_queue *queue) {
    if (!ctx) return SFQ_ERR_ARG;
    if (!queue) {
        ctx->defer_q = sfq_event_queue{};
        return SFQ_OK;
    }
    if (ctx->cfg.precision != SFQ_FP32) return fail(ctx, SFQ_ERR_ARG, "the deferred event path needs a binary32 context");
    if (ctx->inv_tr > 0) return fail(ctx, SFQ_ERR_ARG, "truncated samplers are set: restore the full coefficients");
    if (queue->capacity < 0 || !queue->count || !aligned8(queue->count))
        return fail(ctx, SFQ_ERR_ARG, "queue capacity or counter invalid");
    if (queue->capacity > 0) {
        const void *b[7] = {queue->index, queue->chi, queue->r, queue->gamma, queue->px, queue->py, queue->pz};
        for (const void *q : b)
            if (!q || !aligned16(q)) return fail(ctx, SFQ_ERR_ARG, "queue buffer null or misaligned (16 bytes)");
    }
    DeviceGuard g(ctx->device);
    const cudaError_t e = sfq::prepare_step_surr_f32();    // kernel attributes, outside any capture
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sfq_set_event_queue: attributes");
    ctx->defer_q = *queue;
    return SFQ_OK;
}

sfq_status sfq_counters_check(const sfq_counters *c) {
    if (!c) return SFQ_ERR_ARG;
    if (c->timeouts) return SFQ_ERR_TIMEOUT;
    if (c->dropped || c->spawn_dropped) return SFQ_ERR_CAPACITY;
    if (c->out_of_range || c->nan_input) return SFQ_ERR_RANGE;
    return SFQ_OK;
}

sfq_status sfq_check_bounded_wait(sfq_ctx *ctx, uint32_t polls, sfq_counters *counters, void *stream) {
    if (!ctx) return SFQ_ERR_ARG;
    if (!counters || !aligned8(counters)) return fail(ctx, SFQ_ERR_ARG, "counters null or misaligned");
    if (polls < 1 || polls > 65536) return fail(ctx, SFQ_ERR_ARG, "polls must be in [1, 65536]");
    DeviceGuard g(ctx->device);
    const cudaError_t e = sfq::launch_wait_check(polls, counters, (cudaStream_t)stream);
    return e == cudaSuccess ? SFQ_OK : cuda_fail(ctx, e, "bounded-wait check");
}

sfq_status sfq_check_sqrt(sfq_ctx *ctx, int64_t n, const float *x, float *sqrt_out, float *rsqrt_out, void *stream) {
    if (!ctx) return SFQ_ERR_ARG;
    if (n < 0) return fail(ctx, SFQ_ERR_ARG, "n < 0");
    if (n > 0 && (!x || !sqrt_out || !rsqrt_out)) return fail(ctx, SFQ_ERR_ARG, "null buffer");
    DeviceGuard g(ctx->device);
    const cudaError_t e = sfq::launch_sqrt_check(n, x, sqrt_out, rsqrt_out, ctx->num_sms, (cudaStream_t)stream);
    return e == cudaSuccess ? SFQ_OK : cuda_fail(ctx, e, "square-root check");
}

}  // extern "C"
