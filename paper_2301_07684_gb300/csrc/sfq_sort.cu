// sfq_sort.cu -- stable LSD radix sort of product records by (parent id, step, member,
// parent tag), so that runs can be compared with the oracle record by record.
//
// Keys are sorted in two stable stages: first the secondary key (step << 4 | member << 2 |
// tag), then the parent id; digits are 8 bits and passes whose digit is zero for every
// record are skipped.  One pass = a per-block digit histogram, a digit-major exclusive scan
// over (digit, block) (reduce, then scan), and a stable scatter in which one warp ranks its tile 32 records at
// a time (__match_any_sync).  The records are then gathered into sorted order through the
// caller's scratch memory.
#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

#include "sfq_internal.h"

namespace sfq {
namespace {

constexpr int SORT_TILE = 32 * 64;       // records per block (one warp, 64 rounds)
constexpr int RADIX = 256;

__global__ void keys_kernel(int64_t n, const uint64_t *__restrict__ pid, const uint32_t *__restrict__ step,
                            const uint8_t *__restrict__ meta, uint64_t *__restrict__ k_secondary,
                            uint64_t *__restrict__ k_primary, uint32_t *__restrict__ idx,
                            unsigned long long *__restrict__ or_bits) {
    uint64_t acc_s = 0, acc_p = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t m = meta[i];
        // member (bits 2-3) ranks before the parent tag (bits 4-5)
        const uint64_t ks = ((uint64_t)step[i] << 4) | (((m >> 2) & 3u) << 2) | ((m >> 4) & 3u);
        k_secondary[i] = ks;
        k_primary[i] = pid[i];
        idx[i] = (uint32_t)i;
        acc_s |= ks;
        acc_p |= pid[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc_s |= __shfl_xor_sync(0xFFFFFFFFu, acc_s, o);
        acc_p |= __shfl_xor_sync(0xFFFFFFFFu, acc_p, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicOr(&or_bits[0], (unsigned long long)acc_s);
        atomicOr(&or_bits[1], (unsigned long long)acc_p);
    }
}

// Histogram of one digit per block tile (digit-major counts[d * nblocks + b]).
__global__ void hist_kernel(int64_t n, const uint64_t *__restrict__ key, int shift, uint32_t *__restrict__ counts,
                            int nblocks) {
    __shared__ uint32_t h[RADIX];
    for (int d = threadIdx.x; d < RADIX; d += blockDim.x) h[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE;
    for (int k = threadIdx.x; k < SORT_TILE; k += blockDim.x) {
        const int64_t i = base + k;
        if (i < n) atomicAdd(&h[(key[i] >> shift) & 0xFF], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RADIX; d += blockDim.x) counts[(int64_t)d * nblocks + blockIdx.x] = h[d];
}

// Exclusive scan of m 32-bit counts (the total fits in 32 bits) in three kernels: sums of
// SCAN_CHUNK-element chunks, a single-block scan of those sums, and a scan of every chunk
// from its offset.
constexpr int SCAN_BS = 1024;
constexpr int SCAN_PT = 4;                               // consecutive elements per thread
constexpr int SCAN_CHUNK = SCAN_BS * SCAN_PT;

// Block-wide exclusive scan of one value per thread; returns the block total in *total.
__device__ __forceinline__ uint32_t block_exclusive(uint32_t v, uint32_t *wsum, uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t y = lane < nw ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, y, o);
            if (lane >= o) y += t;
        }
        if (lane < nw) wsum[lane] = y;
    }
    __syncthreads();
    const uint32_t before = (warp ? wsum[warp - 1] : 0u) + x - v;
    *total = wsum[nw - 1];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(SCAN_BS) chunk_sum_kernel(const uint32_t *__restrict__ c, int64_t m,
                                                            uint32_t *__restrict__ sums) {
    __shared__ uint32_t wsum[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_PT;
    uint32_t v = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PT; ++k)
        if (base + k < m) v += c[base + k];
    uint32_t total;
    block_exclusive(v, wsum, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Single block over the chunk sums (in place).
__global__ void __launch_bounds__(SCAN_BS) scan_sums_kernel(uint32_t *__restrict__ c, int64_t m) {
    __shared__ uint32_t wsum[32];
    uint32_t carry = 0;
    for (int64_t base = 0; base < m; base += SCAN_BS) {
        const int64_t i = base + threadIdx.x;
        const uint32_t v = i < m ? c[i] : 0u;
        uint32_t total;
        const uint32_t before = block_exclusive(v, wsum, &total);
        if (i < m) c[i] = carry + before;
        carry += total;
    }
}

__global__ void __launch_bounds__(SCAN_BS) chunk_scan_kernel(uint32_t *__restrict__ c, int64_t m,
                                                             const uint32_t *__restrict__ offsets) {
    __shared__ uint32_t wsum[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_PT;
    uint32_t v[SCAN_PT];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PT; ++k) {
        v[k] = base + k < m ? c[base + k] : 0u;
        sum += v[k];
    }
    uint32_t total;
    uint32_t run = offsets[blockIdx.x] + block_exclusive(sum, wsum, &total);
#pragma unroll
    for (int k = 0; k < SCAN_PT; ++k) {
        if (base + k < m) c[base + k] = run;
        run += v[k];
    }
}

// Stable scatter of (key, index) pairs: one warp per block ranks its tile in order.
__global__ void scatter_kernel(int64_t n, const uint64_t *__restrict__ key_in, const uint32_t *__restrict__ idx_in,
                               uint64_t *__restrict__ key_out, uint32_t *__restrict__ idx_out, int shift,
                               const uint32_t *__restrict__ offsets, int nblocks) {
    __shared__ uint32_t run[RADIX];
    const int lane = threadIdx.x;
    for (int d = lane; d < RADIX; d += 32) run[d] = offsets[(int64_t)d * nblocks + blockIdx.x];
    __syncwarp();
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE;
    for (int r = 0; r < SORT_TILE / 32; ++r) {
        const int64_t i = base + r * 32 + lane;
        const bool valid = i < n;
        const uint64_t k = valid ? key_in[i] : 0ull;
        const uint32_t d = valid ? (uint32_t)((k >> shift) & 0xFF) : 0x100u + lane;   // invalid lanes: unique
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
        const unsigned lt = peers & ((1u << lane) - 1u);
        const uint32_t pos = valid ? run[d] + __popc(lt) : 0u;
        if (valid && pos < n) {                               // pos < n holds for a correct scan
            key_out[pos] = k;
            idx_out[pos] = idx_in[i];
        }
        __syncwarp();
        if (valid && lt == 0) run[d] += __popc(peers);       // the lowest peer advances the digit
        __syncwarp();
    }
}

__global__ void gather_keys_kernel(int64_t n, const uint32_t *__restrict__ perm, const uint64_t *__restrict__ src,
                                   uint64_t *__restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    {
        const uint32_t j = perm[i];
        dst[i] = j < n ? src[j] : 0ull;                       // perm is a permutation of [0, n)
    }
}

template <typename T>
__global__ void gather_kernel(int64_t n, const uint32_t *__restrict__ perm, const T *__restrict__ src,
                              T *__restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    {
        const uint32_t j = perm[i];
        dst[i] = j < n ? src[j] : T(0);
    }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Plan {
    size_t o_ks, o_kp, o_k1, o_i0, o_i1, o_cnt, o_sums, o_or, o_tmp, total;
    int nblocks;
    int64_t ncnt, nchunks;
};

Plan plan(int64_t n, size_t elem) {
    Plan p{};
    p.nblocks = (int)((n + SORT_TILE - 1) / SORT_TILE);
    size_t o = 0;
    p.o_ks = o; o += align256(n * 8);
    p.o_kp = o; o += align256(n * 8);
    p.o_k1 = o; o += align256(n * 8);
    p.o_i0 = o; o += align256(n * 4);
    p.o_i1 = o; o += align256(n * 4);
    p.ncnt = (int64_t)p.nblocks * RADIX;
    p.nchunks = (p.ncnt + SCAN_CHUNK - 1) / SCAN_CHUNK;
    p.o_cnt = o; o += align256((size_t)p.ncnt * 4);
    p.o_sums = o; o += align256((size_t)p.nchunks * 4);
    p.o_or = o; o += 256;
    p.o_tmp = o; o += align256(n * (elem > 8 ? elem : 8));     // one record column at a time
    p.total = o;
    return p;
}

int bits_of(uint64_t v) { return v ? 64 - __builtin_clzll(v) : 0; }

}  // namespace

cudaError_t sort_products(const sfq_products &out, int64_t n, size_t elem, void *scratch, cudaStream_t s,
                          int num_sms) {
    if (n <= 1) return cudaSuccess;
    const Plan P = plan(n, elem);
    char *sc = static_cast<char *>(scratch);
    uint64_t *ks = reinterpret_cast<uint64_t *>(sc + P.o_ks), *kp = reinterpret_cast<uint64_t *>(sc + P.o_kp);
    uint32_t *i0 = reinterpret_cast<uint32_t *>(sc + P.o_i0), *i1 = reinterpret_cast<uint32_t *>(sc + P.o_i1);
    uint32_t *cnt = reinterpret_cast<uint32_t *>(sc + P.o_cnt);
    uint32_t *sums = reinterpret_cast<uint32_t *>(sc + P.o_sums);
    unsigned long long *orb = reinterpret_cast<unsigned long long *>(sc + P.o_or);
    const int grid = num_sms * 8;
    cudaError_t e = cudaMemsetAsync(orb, 0, 16, s);
    if (e != cudaSuccess) return e;
    keys_kernel<<<grid, 256, 0, s>>>(n, out.parent_id, out.step, out.meta, ks, kp, i0, orb);
    unsigned long long h_or[2];
    e = cudaMemcpyAsync(h_or, orb, 16, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    uint64_t *k1 = reinterpret_cast<uint64_t *>(sc + P.o_k1);
    uint64_t *kcur = ks, *knxt = k1;
    uint32_t *cur = i0, *nxt = i1;
    for (int stage = 0; stage < 2; ++stage) {
        if (stage == 1) {
            // primary keys in the order of the stage-0 permutation
            gather_keys_kernel<<<grid, 256, 0, s>>>(n, cur, kp, knxt);
            uint64_t *t = kcur; kcur = knxt; knxt = t;
        }
        const int nb = bits_of(h_or[stage]);
        for (int shift = 0; shift < nb; shift += 8) {
            hist_kernel<<<P.nblocks, 256, 0, s>>>(n, kcur, shift, cnt, P.nblocks);
            chunk_sum_kernel<<<(unsigned)P.nchunks, SCAN_BS, 0, s>>>(cnt, P.ncnt, sums);
            scan_sums_kernel<<<1, SCAN_BS, 0, s>>>(sums, P.nchunks);
            chunk_scan_kernel<<<(unsigned)P.nchunks, SCAN_BS, 0, s>>>(cnt, P.ncnt, sums);
            scatter_kernel<<<P.nblocks, 32, 0, s>>>(n, kcur, cur, knxt, nxt, shift, cnt, P.nblocks);
            uint64_t *tk = kcur; kcur = knxt; knxt = tk;
            uint32_t *ti = cur; cur = nxt; nxt = ti;
        }
    }
    // apply the permutation to every record column
    void *tmp = sc + P.o_tmp;
#define SFQ_GATHER(T, ptr)                                                                          \
    gather_kernel<T><<<grid, 256, 0, s>>>(n, cur, static_cast<const T *>(ptr), static_cast<T *>(tmp)); \
    e = cudaMemcpyAsync(ptr, tmp, (size_t)n * sizeof(T), cudaMemcpyDeviceToDevice, s);                 \
    if (e != cudaSuccess) return e;
    if (elem == 4) {
        SFQ_GATHER(float, out.px) SFQ_GATHER(float, out.py) SFQ_GATHER(float, out.pz)
    } else {
        SFQ_GATHER(double, out.px) SFQ_GATHER(double, out.py) SFQ_GATHER(double, out.pz)
    }
    SFQ_GATHER(uint64_t, out.parent_id)
    SFQ_GATHER(uint32_t, out.step)
    SFQ_GATHER(uint8_t, out.meta)
#undef SFQ_GATHER
    return cudaGetLastError();
}

size_t sort_scratch_bytes(int64_t n, size_t elem) { return n <= 1 ? 256 : plan(n, elem).total; }

}  // namespace sfq
