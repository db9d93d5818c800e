// sfq_runtime.cu -- the batched runtime around the Monte Carlo step: many steps recorded
// into one CUDA graph (sfq_mc_run), the launch-shape autotuner (sfq_autotune_step) and
// the product sort (sfq_sort_products).  All arithmetic of the method stays in the step
// kernels; this file only records, times and orders launches.
#include <cstring>
#include <string>

#include "sfq_internal.h"

namespace {

constexpr size_t GRAPH_CACHE = 8;   // graphs kept per context (oldest evicted first)

sfq_status fail(sfq_ctx *ctx, sfq_status st, const char *msg) {
    if (ctx) ctx->err = msg;
    return st;
}

sfq_status cuda_fail(sfq_ctx *ctx, cudaError_t e, const char *where) {
    if (ctx) ctx->err = std::string(where) + ": " + cudaGetErrorString(e);
    return SFQ_ERR_CUDA;
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

template <typename S>
void put(std::string &k, const S *s) {
    const char flag = s ? 1 : 0;
    k.append(&flag, 1);
    if (s) k.append(reinterpret_cast<const char *>(s), sizeof(S));
}

// Everything a recorded graph depends on: descriptors (pointers, sizes, kinds), the
// step range and the launch shape.
std::string graph_key(const sfq_ctx *ctx, const sfq_particles *p, const sfq_fields *f, const sfq_particles *c,
                      const sfq_fields *cf, uint32_t step0, uint32_t nsteps, const sfq_products *out,
                      const sfq_spawn *spawn, const sfq_counters *counters) {
    std::string k;
    put(k, p); put(k, f); put(k, c); put(k, cf); put(k, out); put(k, spawn);
    const uintptr_t cp = reinterpret_cast<uintptr_t>(counters);
    const int32_t shape[3] = {ctx->step_variant, ctx->step_ppt, ctx->step_grid};
    k.append(reinterpret_cast<const char *>(&cp), sizeof(cp));
    k.append(reinterpret_cast<const char *>(&step0), sizeof(step0));
    k.append(reinterpret_cast<const char *>(&nsteps), sizeof(nsteps));
    k.append(reinterpret_cast<const char *>(shape), sizeof(shape));
    // options baked into the recorded kernel arguments
    const double cut = ctx->pair_chi_min;
    const void *inv_r[3] = {ctx->d_nlc_inv_r, ctx->d_nbw_inv_r, reinterpret_cast<const void *>((intptr_t)ctx->inv_tr)};
    k.append(reinterpret_cast<const char *>(&cut), sizeof(cut));
    k.append(reinterpret_cast<const char *>(inv_r), sizeof(inv_r));
    // the surrogate on the event path (network, queue, fallback flags)
    const void *surr = ctx->surr;
    k.append(reinterpret_cast<const char *>(&surr), sizeof(surr));
    if (ctx->surr) {
        k.append(reinterpret_cast<const char *>(&ctx->surr_q), sizeof(ctx->surr_q));
        k.append(reinterpret_cast<const char *>(&ctx->surr_flags), sizeof(ctx->surr_flags));
    }
    k.append(reinterpret_cast<const char *>(&ctx->defer_q), sizeof(ctx->defer_q));   // the deferred event path
    return k;
}

}  // namespace

namespace sfq {

void release_graphs(sfq_ctx *ctx) {
    for (auto &g : ctx->graphs)
        if (g.second) cudaGraphExecDestroy(g.second);
    ctx->graphs.clear();
}

}  // namespace sfq

extern "C" {

sfq_status sfq_mc_run(sfq_ctx *ctx, const sfq_particles *p, const sfq_fields *f, const sfq_particles *children,
                      const sfq_fields *children_fields, uint32_t step0, uint32_t nsteps, const sfq_products *out,
                      const sfq_spawn *spawn, sfq_counters *counters, void *stream) {
    if (!ctx) return SFQ_ERR_ARG;
    sfq_status st = sfq::validate_step(ctx, p, f, out, spawn, counters);
    if (st != SFQ_OK) return st;
    if (children) {
        if (!children_fields) return fail(ctx, SFQ_ERR_ARG, "children without a field source");
        st = sfq::validate_step(ctx, children, children_fields, out, nullptr, counters);
        if (st != SFQ_OK) return st;
    }
    if (nsteps == 0) return SFQ_OK;
    if ((uint64_t)step0 + nsteps > 0xFFFFFFFFull) return fail(ctx, SFQ_ERR_ARG, "step range exceeds 32 bits");
    DeviceGuard g(ctx->device);
    const cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sfq_mc_run");
    if (cap != cudaStreamCaptureStatusNone) return fail(ctx, SFQ_ERR_ARG, "stream is being captured");

    const std::string key = graph_key(ctx, p, f, children, children_fields, step0, nsteps, out, spawn, counters);
    cudaGraphExec_t exec = nullptr;
    for (auto &it : ctx->graphs)
        if (it.first == key) exec = it.second;
    if (!exec) {
        // Kernel attributes are set outside the capture; the launches are recorded on a
        // private stream in thread-local mode, so other threads' work is not affected.
        e = ctx->cfg.precision == SFQ_FP64 ? sfq::prepare_step_f64() : sfq::prepare_step_f32();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "sfq_mc_run: kernel attributes");
        cudaStream_t cs = nullptr;
        e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "sfq_mc_run: capture stream");
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        cudaError_t el = cudaSuccess;
        if (e == cudaSuccess) {
            for (uint32_t k = 0; k < nsteps && el == cudaSuccess; ++k) {
                const uint32_t step = step0 + k;
                if (children && children->n > 0)
                    el = sfq::launch_step(ctx, children, children_fields, step, out, nullptr, counters, cs);
                if (el == cudaSuccess) el = sfq::launch_step(ctx, p, f, step, out, spawn, counters, cs);
            }
            cudaGraph_t graph = nullptr;
            e = cudaStreamEndCapture(cs, &graph);
            if (e == cudaSuccess && el == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
        }
        cudaStreamDestroy(cs);
        if (el != cudaSuccess) return cuda_fail(ctx, el, "sfq_mc_run: recording");
        if (e != cudaSuccess) return cuda_fail(ctx, e, "sfq_mc_run: capture");
        if (ctx->graphs.size() >= GRAPH_CACHE) {
            cudaGraphExecDestroy(ctx->graphs.front().second);
            ctx->graphs.erase(ctx->graphs.begin());
        }
        ctx->graphs.emplace_back(key, exec);
    }
    e = cudaGraphLaunch(exec, s);
    return e == cudaSuccess ? SFQ_OK : cuda_fail(ctx, e, "sfq_mc_run: launch");
}

sfq_status sfq_autotune_step(sfq_ctx *ctx, const sfq_particles *p, const sfq_fields *f, uint32_t step,
                             int64_t sample_n, int32_t *variant, int32_t *shape, double *ms_per_step, void *stream) {
    if (!ctx) return SFQ_ERR_ARG;
    if (!p || !f) return fail(ctx, SFQ_ERR_ARG, "null descriptor");
    DeviceGuard g(ctx->device);
    const cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    int64_t n = p->n;
    if (p->n_dev && n > 0) {
        long long nd = 0;
        e = cudaMemcpyAsync(&nd, p->n_dev, sizeof(nd), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "sfq_autotune_step: n_dev");
        if (nd < n) n = nd < 0 ? 0 : nd;
    }
    if (sample_n > 0 && sample_n < n) n = sample_n;
    if (n <= 0) return fail(ctx, SFQ_ERR_ARG, "no particles to time");
    const bool fp64 = ctx->cfg.precision == SFQ_FP64;
    const size_t es = fp64 ? 8 : 4;
    const bool blcfa = p->lepton_model != SFQ_LEPTON_LCFA_OD;
    const int64_t pcap = 2 * n + 1024;
    // one allocation: particle copy, pristine copy of the mutable state, products, counters
    auto a256 = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t state_cols = 3 + (blcfa ? 6 : 0);     // px,py,pz (+ fprev, dfprev)
    const size_t state_bytes = a256(n * es) * state_cols + a256(n * 8) + a256(n);   // + tau, flags
    const size_t prod_bytes = a256(pcap * es) * 3 + a256(pcap * 8) + a256(pcap * 4) + a256(pcap) + 256;
    const size_t total = 2 * state_bytes + a256(n * 8) + prod_bytes + a256(sizeof(sfq_counters));
    char *buf = nullptr;
    e = cudaMalloc(&buf, total);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sfq_autotune_step: temporary memory");
    char *cur = buf;
    auto take = [&](size_t b) { char *r = cur; cur += a256(b); return r; };
    // working copy
    sfq_particles w = *p;
    w.n = n;
    w.n_dev = nullptr;
    void **wcols[9] = {&w.px, &w.py, &w.pz, &w.fprev[0], &w.fprev[1], &w.fprev[2], &w.dfprev[0], &w.dfprev[1],
                       &w.dfprev[2]};
    const void *scols[9] = {p->px, p->py, p->pz, p->fprev[0], p->fprev[1], p->fprev[2], p->dfprev[0], p->dfprev[1],
                            p->dfprev[2]};
    char *pristine[11] = {};
    for (size_t k = 0; k < state_cols; ++k) *wcols[k] = take(n * es);
    w.tau = reinterpret_cast<double *>(take(n * 8));
    w.flags = reinterpret_cast<uint8_t *>(take(n));
    for (size_t k = 0; k < state_cols; ++k) pristine[k] = take(n * es);
    pristine[9] = take(n * 8);
    pristine[10] = take(n);
    uint64_t *ids = reinterpret_cast<uint64_t *>(take(n * 8));
    if (p->id) {
        w.id = ids;
        e = cudaMemcpyAsync(ids, p->id, n * 8, cudaMemcpyDeviceToDevice, s);
    }
    sfq_products o{};
    o.capacity = pcap;
    o.px = take(pcap * es); o.py = take(pcap * es); o.pz = take(pcap * es);
    o.parent_id = reinterpret_cast<uint64_t *>(take(pcap * 8));
    o.step = reinterpret_cast<uint32_t *>(take(pcap * 4));
    o.meta = reinterpret_cast<uint8_t *>(take(pcap));
    o.count = reinterpret_cast<unsigned long long *>(take(256));
    sfq_counters *cnt = reinterpret_cast<sfq_counters *>(take(sizeof(sfq_counters)));
    for (size_t k = 0; k < state_cols && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(pristine[k], scols[k], n * es, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pristine[9], p->tau, n * 8, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pristine[10], p->flags, n, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s);
        cudaFree(buf);
        return cuda_fail(ctx, e, "sfq_autotune_step: copies");
    }
    sfq_status st = sfq::validate_step(ctx, &w, f, &o, nullptr, cnt);
    if (st != SFQ_OK) {
        cudaStreamSynchronize(s);
        cudaFree(buf);
        return st;
    }
    struct Shape { int variant, ppt; };
    const Shape shapes[6] = {{1, 1}, {1, 2}, {1, 4}, {2, 8}, {2, 16}, {2, 20}};
    const int nshapes = blcfa ? 3 : 6;           // the beyond-LCFA model runs on the warp-streaming kernel
    const int saved[3] = {ctx->step_variant, ctx->step_ppt, ctx->step_grid};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    e = cudaEventCreate(&ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ev1);
    float best = -1.0f;
    int best_k = -1;
    constexpr int REPS = 3;
    for (int k = 0; k < nshapes && e == cudaSuccess; ++k) {
        ctx->step_variant = shapes[k].variant;
        ctx->step_ppt = shapes[k].ppt;
        ctx->step_grid = 0;
        // restore the sampled state, then one untimed and REPS timed steps
        for (size_t c = 0; c < state_cols && e == cudaSuccess; ++c)
            e = cudaMemcpyAsync(*wcols[c], pristine[c], n * es, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(w.tau, pristine[9], n * 8, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(w.flags, pristine[10], n, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(o.count, 0, 8, s);
        if (e == cudaSuccess) e = sfq::launch_step(ctx, &w, f, step, &o, nullptr, cnt, s);
        if (e == cudaSuccess) e = cudaEventRecord(ev0, s);
        for (int r = 0; r < REPS && e == cudaSuccess; ++r) {
            e = cudaMemsetAsync(o.count, 0, 8, s);
            if (e == cudaSuccess) e = sfq::launch_step(ctx, &w, f, step + 1 + r, &o, nullptr, cnt, s);
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
        if (e == cudaSuccess && (best < 0.0f || ms < best)) {
            best = ms;
            best_k = k;
        }
    }
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    cudaStreamSynchronize(s);
    cudaFree(buf);
    if (e != cudaSuccess || best_k < 0) {
        ctx->step_variant = saved[0]; ctx->step_ppt = saved[1]; ctx->step_grid = saved[2];
        return cuda_fail(ctx, e, "sfq_autotune_step: trial steps");
    }
    ctx->step_variant = shapes[best_k].variant;
    ctx->step_ppt = shapes[best_k].ppt;
    ctx->step_grid = 0;
    if (variant) *variant = shapes[best_k].variant;
    if (shape) *shape = shapes[best_k].ppt;
    if (ms_per_step) *ms_per_step = best / REPS;
    return SFQ_OK;
}

size_t sfq_sort_scratch_bytes(int64_t n) { return sfq::sort_scratch_bytes(n < 0 ? 0 : n, 8); }

sfq_status sfq_sort_products(sfq_ctx *ctx, const sfq_products *out, int64_t n, void *scratch, size_t scratch_bytes,
                             void *stream) {
    if (!ctx) return SFQ_ERR_ARG;
    if (!out) return fail(ctx, SFQ_ERR_ARG, "null descriptor");
    if (n < 0 || n > out->capacity) return fail(ctx, SFQ_ERR_ARG, "n outside [0, capacity]");
    if (n > 0xFFFFFFFFll) return fail(ctx, SFQ_ERR_ARG, "more than 2^32 records");
    if (n <= 1) return SFQ_OK;
    if (!scratch || ((uintptr_t)scratch & 255u) != 0) return fail(ctx, SFQ_ERR_ARG, "scratch null or not 256-byte aligned");
    if (scratch_bytes < sfq::sort_scratch_bytes(n, 8)) return fail(ctx, SFQ_ERR_ARG, "scratch smaller than sfq_sort_scratch_bytes(n)");
    const void *cols[6] = {out->px, out->py, out->pz, out->parent_id, out->step, out->meta};
    for (const void *c : cols)
        if (!c) return fail(ctx, SFQ_ERR_ARG, "null product column");
    DeviceGuard g(ctx->device);
    const cudaError_t e = sfq::sort_products(*out, n, ctx->cfg.precision == SFQ_FP64 ? 8 : 4, scratch,
                                             (cudaStream_t)stream, ctx->num_sms);
    return e == cudaSuccess ? SFQ_OK : cuda_fail(ctx, e, "sfq_sort_products");
}

}  // extern "C"
