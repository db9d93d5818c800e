// Launchers of the mixed path (binary32 arithmetic, binary64 optical depth).
#include "sfq_launch.cuh"

namespace sfq {
cudaError_t launch_rate_f32(const RateLaunch &L, bool pair) { return launch_rate_t<float>(L, pair); }
cudaError_t launch_sample_f32(const SampleLaunch &L, bool pair) { return launch_sample_t<float>(L, pair); }
cudaError_t launch_uniforms_f32(int64_t n, const uint64_t *id, uint32_t step, uint32_t tag, uint64_t seed, void *u,
                                cudaStream_t s, int grid) {
    return launch_uniforms_t<float>(n, id, step, tag, seed, u, s, grid);
}
cudaError_t launch_step_f32(const StepLaunch &L) { return launch_step_t<float>(L); }
cudaError_t prepare_step_f32() { return prepare_step_t<float>(); }
cudaError_t launch_fused_f32(const StepLaunch &L, uint32_t nsteps) { return launch_fused_t<float>(L, nsteps); }
}  // namespace sfq
