// sfq_internal.h -- declarations shared by the host translation units of libsfq.
#pragma once
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "sfq.h"

struct sfq_ctx {
    sfq_config cfg;
    int device;
    double rho, pref;
    // device copies of the fitted tables (one precision per context)
    void *d_nlc_rate, *d_nbw_rate, *d_nlc_inv, *d_nbw_inv, *d_k23, *d_ki13;
    int num_sms;
    int step_variant = 0;    // 0 = automatic, 1 = warp-streaming, 2 = TMA-staged
    std::vector<std::pair<std::string, cudaGraphExec_t>> graphs;   // sfq_mc_run cache
    int step_ppt = 0;        // 0 = default
    int step_grid = 0;       // 0 = one wave of resident blocks
    double pair_chi_min = 0.01;   // NBW rate is zero below this chi (sfq_set_pair_rate_cutoff)
    int inv_tr = 0;               // inverse-CDF coefficients dropped per variable (sfq_set_sampler_coefficients)
    void *d_nlc_inv_r = nullptr, *d_nbw_inv_r = nullptr;   // the truncated tables when inv_tr > 0
    int eval = 0;                 // SFQ_EVAL_HORNER or SFQ_EVAL_CLENSHAW (sfq_set_evaluator)
    void *d_nlc_rate_ch = nullptr, *d_nbw_rate_ch = nullptr;   // Chebyshev pieces (Clenshaw evaluator)
    void *d_nlc_inv_ch = nullptr, *d_nbw_inv_ch = nullptr;
    void *noalloc_scratch = nullptr;   // address of the no-allocation sort's array on this context's device
    // the photon surrogate on the step's event path (sfq_set_surrogate)
    sfq_mlp *surr = nullptr;
    sfq_event_queue surr_q{};
    int surr_flags = 0;
    int surr_per_sm = 1;
    // the deferred event path with the plain sampler (sfq_set_event_queue)
    sfq_event_queue defer_q{};
    std::string err;
};

namespace sfq {

// Launchers (one per precision), implemented in sfq_launch_f32.cu / sfq_launch_f64.cu.
struct RateLaunch {
    int64_t n;
    const void *gamma, *chi;
    void *rate;
    const void *table;
    double pref;
    sfq_counters *counters;
    cudaStream_t stream;
    int grid;
    double pair_chi_min;
    int cheb = 0;            // `table` holds Chebyshev pieces (Clenshaw evaluator)
};
struct SampleLaunch {
    int64_t n;
    const void *chi, *r;
    void *a, *b;
    const sfq_ctx *ctx;      // tables (full or truncated) of the context
    sfq_counters *counters;
    cudaStream_t stream;
    int grid;
};
struct StepLaunch {
    const sfq_ctx *ctx;
    const sfq_particles *p;
    const sfq_fields *f;
    uint32_t step;
    const sfq_products *out;
    const sfq_spawn *spawn;
    sfq_counters *counters;
    cudaStream_t stream;
    int grid;
    int ppt;
    int variant;
    int cascade = 0;         // 1: every product is also spawned (full cascade)
};

cudaError_t launch_rate_f32(const RateLaunch &, bool pair);
cudaError_t launch_rate_f64(const RateLaunch &, bool pair);
cudaError_t launch_sample_f32(const SampleLaunch &, bool pair);
cudaError_t launch_sample_f64(const SampleLaunch &, bool pair);
cudaError_t launch_uniforms_f32(int64_t n, const uint64_t *id, uint32_t step, uint32_t tag, uint64_t seed,
                                void *u, cudaStream_t s, int grid);
cudaError_t launch_uniforms_f64(int64_t n, const uint64_t *id, uint32_t step, uint32_t tag, uint64_t seed,
                                void *u, cudaStream_t s, int grid);
cudaError_t launch_step_f32(const StepLaunch &);
cudaError_t launch_step_f64(const StepLaunch &);
cudaError_t launch_fused_f32(const StepLaunch &, uint32_t nsteps);
cudaError_t launch_push_f32(const StepLaunch &, double dt);
cudaError_t launch_push_f64(const StepLaunch &, double dt);
// the same with the truncated samplers compiled in (sfq_launch_tr_f32.cu / _f64.cu)
cudaError_t launch_step_trunc_f32(const StepLaunch &);
// The step kernels whose photon emissions go to the surrogate's queue (sfq_launch_surr_f32.cu),
// and the surrogate pass that samples and finishes them (sfq_mlp.cu).
cudaError_t launch_step_surr_f32(const StepLaunch &);
cudaError_t prepare_step_surr_f32();
cudaError_t launch_event_pass_f32(const StepLaunch &);
cudaError_t launch_surrogate_apply(const sfq_ctx *ctx, const sfq_particles *p, uint32_t step, const sfq_products *out,
                                   sfq_counters *counters, cudaStream_t stream);
cudaError_t launch_step_trunc_f64(const StepLaunch &);
cudaError_t launch_fused_trunc_f32(const StepLaunch &, uint32_t nsteps);
cudaError_t launch_fused_trunc_f64(const StepLaunch &, uint32_t nsteps);
cudaError_t prepare_step_trunc_f32();
cudaError_t prepare_step_trunc_f64();
cudaError_t launch_fused_f64(const StepLaunch &, uint32_t nsteps);

sfq_status validate_step(sfq_ctx *ctx, const sfq_particles *p, const sfq_fields *f, const sfq_products *out,
                         const sfq_spawn *spawn, const sfq_counters *counters);
cudaError_t launch_step(const sfq_ctx *ctx, const sfq_particles *p, const sfq_fields *f, uint32_t step,
                        const sfq_products *out, const sfq_spawn *spawn, sfq_counters *counters, cudaStream_t stream,
                        int cascade = 0);
// Full cascade (sfq_cascade.cu): the count commit around a step and the stream compaction.
cudaError_t launch_cascade_sync(unsigned long long *count, unsigned long long *next, int64_t cap, bool begin,
                                cudaStream_t s);
size_t compact_scratch_bytes(int64_t capacity);
cudaError_t launch_compact(int precision, const sfq_particles &src, const sfq_fields &fsrc, const sfq_particles &dst,
                           const sfq_fields &fdst, void *scratch, cudaStream_t s, int num_sms);
// One CTA whose bounded mbarrier wait gives up after `polls` polls (sfq_check_bounded_wait).
cudaError_t launch_wait_check(uint32_t polls, sfq_counters *c, cudaStream_t s);
cudaError_t launch_sqrt_check(int64_t n, const float *x, float *so, float *ro, int num_sms, cudaStream_t s);
// Dynamic shared-memory attributes of every kernel shape (before graph capture).
cudaError_t prepare_step_f32();
cudaError_t prepare_step_f64();
cudaError_t sort_products(const sfq_products &out, int64_t n, size_t elem, void *scratch, cudaStream_t s,
                          int num_sms);
size_t sort_scratch_bytes(int64_t n, size_t elem);
void release_graphs(sfq_ctx *ctx);

// Host copies of the tables (sfq_tables_host.cu).
struct HostTables {
    const void *nlc_rate, *nbw_rate, *nlc_inv, *nbw_inv, *k23, *ki13;
    size_t nlc_rate_bytes, nbw_rate_bytes, nlc_inv_bytes, nbw_inv_bytes, k23_bytes, ki13_bytes;
};
HostTables host_tables(int precision);
// Inverse-CDF table with every piece's (n x n) coefficients truncated to (n - tr) x (n - tr)
// in the Chebyshev basis, rows padded to 16 bytes (sfq_tables_host.cu).
std::vector<unsigned char> truncated_inv_table(int precision, bool pair, int tr);
// The rate and inverse-CDF tables with every piece in the Chebyshev basis (same piece grid;
// inverse-CDF rows padded to 16 bytes), for the Clenshaw comparison evaluator.
std::vector<unsigned char> chebyshev_rate_table(int precision, bool pair);
std::vector<unsigned char> chebyshev_inv_table(int precision, bool pair);
// The monomial tables as the device holds them (which: 0 NLC rate, 1 NBW rate, 2 NLC
// inverse CDF, 3 NBW inverse CDF).
std::vector<unsigned char> monomial_table(int precision, int which);
int inv_coefficients(int precision);   // n of the context's inverse-CDF tables

}  // namespace sfq
