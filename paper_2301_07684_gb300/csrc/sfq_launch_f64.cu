// Launchers of the plain binary64 path.
#include "sfq_launch.cuh"

namespace sfq {
cudaError_t launch_rate_f64(const RateLaunch &L, bool pair) { return launch_rate_t<double>(L, pair); }
cudaError_t launch_sample_f64(const SampleLaunch &L, bool pair) { return launch_sample_t<double>(L, pair); }
cudaError_t launch_uniforms_f64(int64_t n, const uint64_t *id, uint32_t step, uint32_t tag, uint64_t seed, void *u,
                                cudaStream_t s, int grid) {
    return launch_uniforms_t<double>(n, id, step, tag, seed, u, s, grid);
}
cudaError_t launch_step_f64(const StepLaunch &L) { return launch_step_t<double>(L); }
cudaError_t prepare_step_f64() { return prepare_step_t<double>(); }
cudaError_t launch_fused_f64(const StepLaunch &L, uint32_t nsteps) { return launch_fused_t<double>(L, nsteps); }
}  // namespace sfq
