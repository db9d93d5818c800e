// Launchers of the mixed-path step kernels whose photon emissions go to the surrogate's
// queue (contexts with sfq_set_surrogate), in a translation unit of their own so that the
// build compiles them beside the default kernels; the default instances carry no code for
// the queue.
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

}  // namespace sfq
