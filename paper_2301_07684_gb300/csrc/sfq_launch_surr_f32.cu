// Launchers of the mixed-path step kernels whose photon emissions go to a queue (contexts
// with sfq_set_event_queue or sfq_set_surrogate) and the event pass that finishes the queue
// with the plain fitted sampler, in a translation unit of their own so that the build
// compiles them beside the default kernels; the default instances carry no code for the
// queue.
#include "sfq_launch.cuh"

namespace sfq {

namespace {
constexpr int SURR_CW = 16;     // consumer warps of the TMA-staged instance
}

cudaError_t prepare_step_surr_f32() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(mc_step_tma_kernel<float, FK_SOA, SURR_CW, false, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tma_smem_bytes<float, FK_SOA, SURR_CW>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mc_step_tma_kernel<float, FK_PW, SURR_CW, false, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma_smem_bytes<float, FK_PW, SURR_CW>());
    if (e == cudaSuccess) done = true;
    return e;
}

// As launch_step_t<float, false>, with the SURR instances: the TMA-staged kernel when every
// SM gets a full tile (or variant 2), else the warp-streaming kernel with 2 particles per lane.
cudaError_t launch_step_surr_f32(const StepLaunch &L) {
    const sfq_particles &p = *L.p;
    const sfq_ctx *ctx = L.ctx;
    if (p.n == 0) return cudaSuccess;
    const StepArgs<float> a = make_step_args<float>(L);
    const bool pw = L.f->kind == SFQ_FIELDS_PLANE_WAVE;
    constexpr int TILE = SURR_CW * 64;
    const bool tma = p.lepton_model == SFQ_LEPTON_LCFA_OD &&
                     (L.variant == 2 || (L.variant == 0 && p.n >= (int64_t)TILE * ctx->num_sms));
    if (tma) {
        cudaError_t e = prepare_step_surr_f32();
        if (e != cudaSuccess) return e;
        auto kern = pw ? mc_step_tma_kernel<float, FK_PW, SURR_CW, false, true>
                       : mc_step_tma_kernel<float, FK_SOA, SURR_CW, false, true>;
        const size_t smem = pw ? tma_smem_bytes<float, FK_PW, SURR_CW>() : tma_smem_bytes<float, FK_SOA, SURR_CW>();
        const int64_t ntiles = (p.n + TILE - 1) / TILE;
        int grid = L.grid > 0 ? L.grid : ctx->num_sms;
        if (ntiles < grid) grid = (int)ntiles;
        kern<<<grid, 32 * (SURR_CW + 1), smem, L.stream>>>(a);
        return cudaGetLastError();
    }
    auto kern = pw ? mc_step_kernel<float, FK_PW, 2, false, false, true> : mc_step_kernel<float, FK_SOA, 2, false, false, true>;
    int grid = L.grid;
    if (grid <= 0) {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, STEP_BS, 0);
        if (e != cudaSuccess || per_sm < 1) per_sm = 1;
        grid = per_sm * ctx->num_sms;
        const int64_t chunks = (p.n + 63) / 64;
        const int64_t need = (chunks + STEP_BS / 32 - 1) / (STEP_BS / 32);
        if (need < grid) grid = (int)(need > 0 ? need : 1);
    }
    kern<<<grid, STEP_BS, 0, L.stream>>>(a);
    return cudaGetLastError();
}

// The event pass of a deferred step (sfq_set_event_queue): one queued photon emission per
// thread.  Inverse-transform sampling of s (Eq. again, Eq. subs_altri, the plain fitted
// sampler), the recoil of the emitter to gamma / (1 + s) along its direction and the
// collinear photon's record (Sec. 3), with the arithmetic of the step kernels' own event
// path, so that a deferred step gives the records (in another order) and the state of an
// inline one bit for bit.
__global__ void __launch_bounds__(256) event_pass_kernel(const StepArgs<float> a, const float *__restrict__ qxi_out) {
    (void)qxi_out;
    Cnt c;
    c.zero();
    const int64_t cap = a.qcap, q = (int64_t)*a.qcount;
    const int64_t n = q < cap ? q : cap;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // every lane of a warp runs the same number of rounds (the record reservation is warp-wide)
    const int64_t rounds = (n + stride - 1) / stride;
    for (int64_t k = 0; k < rounds; ++k) {
        const int64_t j = k * stride + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        const bool valid = j < n;
        unsigned long long bp = 0, bs = 0;
        reserve_records(a.ocount, nullptr, valid ? 1 : 0, 0, bp, bs);
        if (!valid) continue;
        const int64_t ei = a.qidx[j];
        const float eg = a.qg[j], echi = a.qchi[j], r1 = a.qr[j];
        const float px = a.qpx[j], py = a.qpy[j], pz = a.qpz[j];
        bool oor = false;
        const float s = photon_s_sel<float, false>(a.tab, echi, r1, oor);
        c.v[C_OOR] += oor;
        ++c.v[C_EMIT];
        const uint8_t fl = a.flags[ei];
        const uint64_t id = a.id ? a.id[ei] : a.id_base + (uint64_t)ei;
        const uint32_t tag = (fl >> SFQ_TAG_SHIFT) & 3u;
        const float pm = sqrtf(fmaf(px, px, fmaf(py, py, pz * pz)));
        const float inv_pm = pm > 0.0f ? 1.0f / pm : 0.0f;
        const float nx = px * inv_pm, ny = py * inv_pm, nz = pz * inv_pm;
        const float inv1s = 1.0f / (1.0f + s);
        const float gph = eg * s * inv1s;
        const float pnew = lepton_pmag(eg * inv1s, c);
        if (bp < (unsigned long long)a.cap) {
            a.opx[bp] = nx * gph; a.opy[bp] = ny * gph; a.opz[bp] = nz * gph;
            a.opid[bp] = id;
            a.ostep[bp] = a.step;
            a.ometa[bp] = (uint8_t)(SFQ_PHOTON | (tag << 4));
        } else {
            ++c.v[C_DROP];
        }
        a.px[ei] = nx * pnew; a.py[ei] = ny * pnew; a.pz[ei] = nz * pnew;
        // a lepton left without momentum leaves the step (as in the step kernels)
        if (!(pnew > 0.0f)) a.flags[ei] = (uint8_t)(fl & ~SFQ_ALIVE);
    }
    flush_counters(c, a.counters);
}

cudaError_t launch_event_pass_f32(const StepLaunch &L) {
    const sfq_ctx *ctx = L.ctx;
    if (ctx->defer_q.capacity <= 0) return cudaSuccess;
    const StepArgs<float> a = make_step_args<float>(L);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, event_pass_kernel, 256, 0);
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    const int64_t need = (ctx->defer_q.capacity + 255) / 256;
    int64_t grid = (int64_t)per_sm * ctx->num_sms;
    if (need < grid) grid = need;
    event_pass_kernel<<<(unsigned)grid, 256, 0, L.stream>>>(a, nullptr);
    return cudaGetLastError();
}

}  // namespace sfq
