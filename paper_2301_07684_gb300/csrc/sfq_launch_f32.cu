// Launchers of the mixed path (binary32 arithmetic, binary64 optical depth).
#include "sfq_launch.cuh"

namespace sfq {
cudaError_t launch_rate_f32(const RateLaunch &L, bool pair) { return launch_rate_t<float>(L, pair); }
cudaError_t launch_sample_f32(const SampleLaunch &L, bool pair) { return launch_sample_t<float>(L, pair); }
cudaError_t launch_uniforms_f32(int64_t n, const uint64_t *id, uint32_t step, uint32_t tag, uint64_t seed, void *u,
                                cudaStream_t s, int grid) {
    return launch_uniforms_t<float>(n, id, step, tag, seed, u, s, grid);
}
cudaError_t launch_step_f32(const StepLaunch &L) {
    return L.ctx->inv_tr > 0 ? launch_step_trunc_f32(L) : launch_step_t<float, false>(L);
}
cudaError_t prepare_step_f32() {
    const cudaError_t e = prepare_step_t<float, false>();
    return e == cudaSuccess ? prepare_step_trunc_f32() : e;
}
cudaError_t launch_fused_f32(const StepLaunch &L, uint32_t nsteps) {
    return L.ctx->inv_tr > 0 ? launch_fused_trunc_f32(L, nsteps) : launch_fused_t<float, false>(L, nsteps);
}
cudaError_t launch_push_f32(const StepLaunch &L, double dt) { return launch_push_t<float>(L, dt); }
cudaError_t launch_wait_check(uint32_t polls, sfq_counters *c, cudaStream_t s) {
    wait_check_kernel<0><<<1, 32, 0, s>>>(polls, c);
    return cudaGetLastError();
}

// The kernels' binary32 square roots on n values (sfq_check_sqrt).
__global__ void sqrt_check_kernel(int64_t n, const float *__restrict__ x, float *__restrict__ so,
                                  float *__restrict__ ro) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = x[i];
        so[i] = sqrt_nr(v);
        ro[i] = rsqrt_nr(v);
    }
}
cudaError_t launch_sqrt_check(int64_t n, const float *x, float *so, float *ro, int num_sms, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = (n + 255) / 256;
    const int grid = (int)(blocks < (int64_t)num_sms * 8 ? blocks : (int64_t)num_sms * 8);
    sqrt_check_kernel<<<grid, 256, 0, s>>>(n, x, so, ro);
    return cudaGetLastError();
}
}  // namespace sfq
