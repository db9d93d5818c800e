// sfq_sort_noalloc.cu -- sfq_sort_products_noalloc: the product sort with its scratch in a
// fixed array of the library's own device memory instead of caller memory.
//
// It serves callers that cannot allocate device memory at the point of the call: host
// codes that hand all of the GPU's memory to their own pool at start-up (a particle-in-cell
// code's particle and field arena) and have no spare buffer to pass, and step loops in
// which a cudaMalloc/cudaFree would synchronise the whole device.  Nothing here allocates:
// the scratch is a file-scope __device__ array, its address is looked up once per device,
// and the sort itself (sfq_sort.cu) takes that address like any caller-owned scratch.
//
// Limits and rules: at most SFQ_SORT_NOALLOC_MAX_N records per call; nothing in the array
// needs to start at zero (the sort clears its one accumulator on the stream); the array is
// shared by every call on a device, so calls that overlap in time on one device race --
// issue them on one stream or order their streams.
//
// The address is kept in the context that looked it up, not in a process-wide table: a
// context lives no longer than the device context it was created in (its tables are
// device memory too), so a device reset that reloads the module, and with it the array,
// cannot leave a stale address behind in a context that is still valid to use.
#include <mutex>

#include "sfq_internal.h"

namespace {

constexpr size_t NOALLOC_BYTES = (size_t)SFQ_SORT_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_sort_scratch[NOALLOC_BYTES];

std::mutex g_mu;

sfq_status fail(sfq_ctx *ctx, sfq_status st, const char *msg) {
    if (ctx) ctx->err = msg;
    return st;
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

// Address of the array on the context's device (current here), looked up on the context's
// first call and kept in the context.
cudaError_t scratch_address(sfq_ctx *ctx, void **out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!ctx->noalloc_scratch) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess) return e;
        ctx->noalloc_scratch = p;
    }
    *out = ctx->noalloc_scratch;
    return cudaSuccess;
}

}  // namespace

extern "C" {

sfq_status sfq_sort_products_noalloc(sfq_ctx *ctx, const sfq_products *out, int64_t n, void *stream) {
    if (!ctx) return SFQ_ERR_ARG;
    if (!out) return fail(ctx, SFQ_ERR_ARG, "null descriptor");
    if (n < 0 || n > out->capacity) return fail(ctx, SFQ_ERR_ARG, "n outside [0, capacity]");
    if (n > (int64_t)SFQ_SORT_NOALLOC_MAX_N)
        return fail(ctx, SFQ_ERR_ARG, "n exceeds SFQ_SORT_NOALLOC_MAX_N: use sfq_sort_products with caller scratch");
    if (n <= 1) return SFQ_OK;
    const void *cols[6] = {out->px, out->py, out->pz, out->parent_id, out->step, out->meta};
    for (const void *c : cols)
        if (!c) return fail(ctx, SFQ_ERR_ARG, "null product column");
    if (sfq::sort_scratch_bytes(n, 8) > NOALLOC_BYTES)
        return fail(ctx, SFQ_ERR_ARG, "static sort scratch smaller than the plan for n");
    DeviceGuard g(ctx->device);
    void *scratch = nullptr;
    cudaError_t e = scratch_address(ctx, &scratch);
    if (e != cudaSuccess) {
        ctx->err = std::string("sfq_sort_products_noalloc: scratch address: ") + cudaGetErrorString(e);
        return SFQ_ERR_CUDA;
    }
    e = sfq::sort_products(*out, n, ctx->cfg.precision == SFQ_FP64 ? 8 : 4, scratch, (cudaStream_t)stream,
                           ctx->num_sms);
    if (e != cudaSuccess) {
        ctx->err = std::string("sfq_sort_products_noalloc: ") + cudaGetErrorString(e);
        return SFQ_ERR_CUDA;
    }
    return SFQ_OK;
}

}  // extern "C"
