// Launchers of the mixed path compiled with the truncated inverse-CDF samplers
// (contexts that set sfq_set_sampler_coefficients below the full count), in a translation
// unit of their own so that the build compiles them beside the default kernels.
#include "sfq_launch.cuh"

namespace sfq {
cudaError_t launch_step_trunc_f32(const StepLaunch &L) { return launch_step_t<float, true>(L); }
cudaError_t prepare_step_trunc_f32() { return prepare_step_t<float, true>(); }
cudaError_t launch_fused_trunc_f32(const StepLaunch &L, uint32_t nsteps) { return launch_fused_t<float, true>(L, nsteps); }
}  // namespace sfq
