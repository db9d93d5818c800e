// Launchers of the binary64 path compiled with the truncated inverse-CDF samplers
// (contexts that set sfq_set_sampler_coefficients below the full count), in a translation
// unit of their own so that the build compiles them beside the default kernels.
#include "sfq_launch.cuh"

namespace sfq {
cudaError_t launch_step_trunc_f64(const StepLaunch &L) { return launch_step_t<double, true>(L); }
cudaError_t prepare_step_trunc_f64() { return prepare_step_t<double, true>(); }
cudaError_t launch_fused_trunc_f64(const StepLaunch &L, uint32_t nsteps) { return launch_fused_t<double, true>(L, nsteps); }
}  // namespace sfq
