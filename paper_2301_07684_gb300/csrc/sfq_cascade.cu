// sfq_cascade.cu -- device side of the full cascade: the count commit between steps and the
// stable stream compaction of a population (count, scan, scatter into a second buffer set).
#include <cstdint>

#include "sfq_internal.h"

namespace sfq {
namespace {

constexpr int CB = 256;              // threads per block of the compaction
constexpr int CG_PER_SM = 8;         // compaction blocks per SM (the grid)
constexpr int CG_MAX = 4096;         // largest compaction grid (bounds the scratch)
constexpr int SCAN_BS = 1024;        // the single block of the scan

// begin: clamp the live count to the capacity and start the append counter there; after a
// step: the appended total (clamped) becomes the live count of the next step.
__global__ void cascade_sync_kernel(unsigned long long *count, unsigned long long *next, unsigned long long cap,
                                    int begin) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        unsigned long long c = begin ? *count : *next;
        c = c < cap ? c : cap;
        *count = c;
        *next = c;
    }
}

__device__ __forceinline__ int64_t live_count(const unsigned long long *count, int64_t n) {
    const int64_t m = (int64_t)*count;
    return m < n ? m : n;
}

// The contiguous share [lo, hi) of the live range [0, m) that block b of g takes, in whole
// chunks of CB particles, so that the blocks' shares keep the particles' order.
__device__ __forceinline__ void block_share(int64_t m, int b, int g, int64_t &lo, int64_t &hi) {
    const int64_t chunks = (m + CB - 1) / CB;
    const int64_t per = (chunks + g - 1) / g;
    lo = (int64_t)b * per * CB;
    hi = lo + per * CB;
    lo = lo < m ? lo : m;
    hi = hi < m ? hi : m;
}

// Alive particles of each block's share of the live range.
__global__ void __launch_bounds__(CB) compact_count_kernel(const uint8_t *flags, const unsigned long long *count,
                                                           int64_t n, uint32_t *block_alive) {
    __shared__ int ws[CB / 32];
    int64_t lo, hi;
    block_share(live_count(count, n), blockIdx.x, gridDim.x, lo, hi);
    int k = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += CB) k += (flags[i] & SFQ_ALIVE) ? 1 : 0;
    k = __reduce_add_sync(0xFFFFFFFFu, k);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = k;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
#pragma unroll
        for (int w = 0; w < CB / 32; ++w) t += ws[w];
        block_alive[blockIdx.x] = (uint32_t)t;
    }
}

// Exclusive scan of the block counts in one block (chunks of SCAN_BS); the total is the
// compacted population's count.
__global__ void __launch_bounds__(SCAN_BS) compact_scan_kernel(const uint32_t *block_alive, int64_t nb,
                                                               unsigned long long *block_off,
                                                               unsigned long long *total) {
    __shared__ unsigned long long ws[SCAN_BS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += SCAN_BS) {
        const int64_t b = b0 + threadIdx.x;
        const unsigned long long v = b < nb ? block_alive[b] : 0ull;
        unsigned long long x = v;                              // inclusive scan in the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) ws[warp] = x;
        __syncthreads();
        if (warp == 0) {                                        // inclusive scan of the warp totals
            unsigned long long w = ws[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, w, o);
                if (lane >= o) w += y;
            }
            ws[lane] = w;
        }
        __syncthreads();
        const unsigned long long before = warp ? ws[warp - 1] : 0ull;
        if (b < nb) block_off[b] = carry + before + x - v;
        carry += ws[SCAN_BS / 32 - 1];
        __syncthreads();                                        // ws is rewritten by the next chunk
    }
    if (threadIdx.x == 0) *total = carry;
}

template <typename T>
struct CompactArgs {
    int64_t n;
    const unsigned long long *count;
    const unsigned long long *block_off;
    const T *px, *py, *pz;
    const double *tau;
    const uint64_t *id;
    const uint8_t *flags;
    const uint32_t *k0;
    const T *amp;
    const T *fp[3], *df[3];
    T *dpx, *dpy, *dpz;
    double *dtau;
    uint64_t *did;
    uint8_t *dflags;
    uint32_t *dk0;
    T *damp;
    T *dfp[3], *ddf[3];
};

// Each alive particle goes to its block's offset plus the alive particles before it in the
// block's share: chunk by chunk, warp ballots and the warps' counts in shared memory.
template <typename T>
__global__ void __launch_bounds__(CB) compact_scatter_kernel(const CompactArgs<T> a) {
    __shared__ int ws[CB / 32];
    int64_t lo, hi;
    block_share(live_count(a.count, a.n), blockIdx.x, gridDim.x, lo, hi);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long off = a.block_off[blockIdx.x];
    for (int64_t c0 = lo; c0 < hi; c0 += CB) {                 // block-uniform trip count
        const int64_t i = c0 + threadIdx.x;
        const bool in = i < hi;
        // the particle's columns are loaded before the ranking, so that their latency
        // overlaps the ballot and the block's count exchange
        const uint8_t fl = in ? a.flags[i] : (uint8_t)0;
        T px = (T)0, py = (T)0, pz = (T)0, am = (T)0;
        double ta = 0.0;
        uint64_t idv = 0;
        uint32_t kv = 0;
        if (in) {
            px = a.px[i]; py = a.py[i]; pz = a.pz[i];
            ta = a.tau[i];
            idv = a.id[i];
            kv = a.k0[i];
            if (a.amp) am = a.amp[i];
        }
        const bool alive = in && (fl & SFQ_ALIVE);
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, alive);
        if (lane == 0) ws[warp] = __popc(bal);
        __syncthreads();
        int before = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < CB / 32; ++w) {
            const int c = ws[w];
            before += w < warp ? c : 0;
            tot += c;
        }
        if (alive) {
            const unsigned long long j = off + (unsigned long long)(before + __popc(bal & ((1u << lane) - 1u)));
            a.dpx[j] = px; a.dpy[j] = py; a.dpz[j] = pz;
            a.dtau[j] = ta;
            a.did[j] = idv;
            a.dflags[j] = fl;
            a.dk0[j] = kv;
            if (a.amp) a.damp[j] = am;
            if (a.fp[0]) {
#pragma unroll
                for (int d3 = 0; d3 < 3; ++d3) { a.dfp[d3][j] = a.fp[d3][i]; a.ddf[d3][j] = a.df[d3][i]; }
            }
        }
        off += (unsigned long long)tot;
        __syncthreads();                                        // ws is rewritten by the next chunk
    }
}

// Compaction grid: CG_PER_SM blocks per SM, no more blocks than chunks of the capacity.
int64_t grid_of(int64_t capacity, int num_sms) {
    const int64_t chunks = (capacity + CB - 1) / CB;
    int64_t g = (int64_t)CG_PER_SM * (num_sms > 0 ? num_sms : 1);
    g = g < CG_MAX ? g : CG_MAX;
    return chunks < g ? chunks : g;
}

template <typename T>
cudaError_t compact_t(const sfq_particles &src, const sfq_fields &fsrc, const sfq_particles &dst,
                      const sfq_fields &fdst, void *scratch, cudaStream_t s, int num_sms) {
    const int64_t nb = grid_of(src.n, num_sms);
    if (nb == 0) {
        return cudaMemsetAsync(const_cast<unsigned long long *>(dst.n_dev), 0, sizeof(unsigned long long), s);
    }
    unsigned long long *block_off = static_cast<unsigned long long *>(scratch);
    uint32_t *block_alive = reinterpret_cast<uint32_t *>(block_off + nb);
    compact_count_kernel<<<(unsigned)nb, CB, 0, s>>>(src.flags, src.n_dev, src.n, block_alive);
    compact_scan_kernel<<<1, SCAN_BS, 0, s>>>(block_alive, nb, block_off,
                                              const_cast<unsigned long long *>(dst.n_dev));
    CompactArgs<T> a{};
    a.n = src.n;
    a.count = src.n_dev;
    a.block_off = block_off;
    a.px = static_cast<const T *>(src.px); a.py = static_cast<const T *>(src.py); a.pz = static_cast<const T *>(src.pz);
    a.tau = src.tau;
    a.id = src.id;
    a.flags = src.flags;
    a.k0 = fsrc.k0;
    a.amp = static_cast<const T *>(fsrc.amp);
    a.dpx = static_cast<T *>(dst.px); a.dpy = static_cast<T *>(dst.py); a.dpz = static_cast<T *>(dst.pz);
    a.dtau = dst.tau;
    a.did = const_cast<uint64_t *>(dst.id);
    a.dflags = dst.flags;
    a.dk0 = const_cast<uint32_t *>(fdst.k0);
    a.damp = static_cast<T *>(const_cast<void *>(fdst.amp));
    if (src.lepton_model != SFQ_LEPTON_LCFA_OD) {
        for (int k = 0; k < 3; ++k) {
            a.fp[k] = static_cast<const T *>(src.fprev[k]);
            a.df[k] = static_cast<const T *>(src.dfprev[k]);
            a.dfp[k] = static_cast<T *>(dst.fprev[k]);
            a.ddf[k] = static_cast<T *>(dst.dfprev[k]);
        }
    }
    compact_scatter_kernel<T><<<(unsigned)nb, CB, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_cascade_sync(unsigned long long *count, unsigned long long *next, int64_t cap, bool begin,
                                cudaStream_t s) {
    cascade_sync_kernel<<<1, 32, 0, s>>>(count, next, (unsigned long long)cap, begin ? 1 : 0);
    return cudaGetLastError();
}

size_t compact_scratch_bytes(int64_t capacity) {
    // the largest grid any device gets (CG_MAX blocks), so the size needs no device
    const int64_t chunks = ((capacity < 0 ? 0 : capacity) + CB - 1) / CB;
    const int64_t nb = chunks < CG_MAX ? chunks : CG_MAX;
    return (size_t)(nb * (int64_t)(sizeof(unsigned long long) + sizeof(uint32_t)) + 16);
}

cudaError_t launch_compact(int precision, const sfq_particles &src, const sfq_fields &fsrc, const sfq_particles &dst,
                           const sfq_fields &fdst, void *scratch, cudaStream_t s, int num_sms) {
    return precision == SFQ_FP64 ? compact_t<double>(src, fsrc, dst, fdst, scratch, s, num_sms)
                                 : compact_t<float>(src, fsrc, dst, fdst, scratch, s, num_sms);
}

}  // namespace sfq
