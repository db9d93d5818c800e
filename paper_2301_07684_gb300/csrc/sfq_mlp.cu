// sfq_mlp.cu -- the learned inverse-CDF surrogate for photon emission: a 2 -> 64 -> 64 ->
// 64 -> 1 SiLU network that maps (ln chi, u) to the paper's inverse-CDF variable w-bar
// (Eq. again), and from it xi = s / (1 + s) with s = 3 chi w-bar^3 / 2 (Eq. subs_altri).
//
//   features  x1 = (ln chi - C_CHI) / S_CHI,  x2 = L / 8 - 1,  L = -ln(1 - u)
//   output    y  = network(x1, x2),  ln w-bar = y + ln u
//
// Training runs on the GPU in binary32 (SIMT kernels written here: forward, backward with
// per-block gradient partials reduced in a fixed order, Adam).  With `quantize`, the
// forward pass rounds the weights and the inputs of layers 2-4 to bfloat16 exactly as the
// inference kernel does (the rounding is passed straight through in the backward pass).
// Inference runs layers 2-4 on the tensor cores (tcgen05.mma, bfloat16 operands staged in
// shared memory, binary32 accumulators in tensor memory, read back with tcgen05.ld); layer
// 1 and the SiLU epilogues run on the CUDA cores.  Cells
// of (ln chi, u) where the network disagrees with the plain fitted sampler by more than a
// tolerance in u (a bound on its contribution to the KS distance of the sampled energies)
// are flagged by sfq_mlp_calibrate; draws in flagged cells, and chi outside the training
// range [1e-3, 100], use the plain sampler.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "sfq_internal.h"
#include "sfq_kernels.cuh"

struct sfq_mlp {
    sfq_ctx *ctx;
    int kind;                         // 0: photon emission (Eq. again), 1: pair creation (Eq. again_pp)
    float *params, *m, *v, *grad;     // binary32 master parameters, Adam moments, gradient
    uint8_t *flags;                   // fallback cells (NCELL bytes)
    float *cell_err;                  // per-cell calibration error (NCELL floats)
    int64_t adam_t;
    int calibrated;
};

namespace sfq {
namespace mlp {

constexpr int H = 64;
constexpr int NP = 8577;
constexpr int O_W1 = 0, O_B1 = 128, O_W2 = 192, O_B2 = 4288, O_W3 = 4352, O_B3 = 8448, O_W4 = 8512, O_B4 = 8576;
constexpr float C_CHI = -1.1512925464970229f;    // (ln 1e-3 + ln 100) / 2
constexpr float S_CHI = 5.7564627324851140f;     // (ln 100 - ln 1e-3) / 2
constexpr float L_SCALE = 0.125f;
constexpr float CHI_LO = 1e-3f, CHI_HI = 100.0f;
constexpr int NCX = 64, NCU = 64, NCELL = NCX * NCU;   // calibration cells in (ln chi, u)

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float qz(float x, bool q) { return q ? bf16r(x) : x; }
__device__ __forceinline__ float silu(float z) { return __fdividef(z, 1.0f + __expf(-z)); }
// SiLU of the inference paths (tensor-core kernel, SIMT reference and calibration) with one
// special-function instruction: z sigma(z) = h (1 + tanh h), h = z / 2, from
// sigma(z) = (1 + tanh(z/2)) / 2.  tanh.approx.f32 has a relative error below 2^-10.987
// (PTX ISA), which is below the bfloat16 rounding the activations then get (2^-9).
// `h` is passed in: the callers form it as 0.5 z + 0.5 b in one fma from halved biases.
__device__ __forceinline__ float silu_h(float h) {
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(h));
    return fmaf(h, t, h);
}
__device__ __forceinline__ float dsilu(float z) {
    const float s = __fdividef(1.0f, 1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}
// What distinguishes the two samplers the network can stand for.  Photon emission: input
// u = r, chi in [1e-3, 100], sampler variable ln w-bar.  Pair creation: input u = |r'| =
// |2r - 1|, chi in [0.1, 100], sampler variable ln(-ln y) with y = 1 - v-bar (Eq.
// again_pp): -ln y ~ v-bar ~ u as u -> 0, so both variables minus ln u stay smooth at
// u -> 0, and y = exp(-u e^network) never exceeds 1.  The network output is always the
// sampler variable minus ln u.
struct Kind {
    float c_chi, inv_s_chi, chi_lo, chi_hi;
    int pair;
};
constexpr float P_C_CHI = 1.1512925464970229f;      // (ln 0.1 + ln 100) / 2
constexpr float P_S_CHI = 3.4538776394910684f;      // (ln 100 - ln 0.1) / 2
constexpr float P_CHI_LO = 0.1f, P_CHI_HI = 100.0f;
inline Kind kind_of(int pair) {
    return pair ? Kind{P_C_CHI, 1.0f / P_S_CHI, P_CHI_LO, P_CHI_HI, 1} : Kind{C_CHI, 1.0f / S_CHI, CHI_LO, CHI_HI, 0};
}
__device__ __forceinline__ void features(const Kind &K, float chi, float u, float &x1, float &x2) {
    x1 = (logf(chi) - K.c_chi) * K.inv_s_chi;
    x2 = -log1pf(-u) * L_SCALE - 1.0f;
}
// network output + offset = the sampler's variable (ln w-bar or ln(-ln y))
__device__ __forceinline__ float out_offset(const Kind &, float u) { return logf(u); }
__device__ __forceinline__ int cell_of(const Kind &K, float chi, float u) {
    const float t = (logf(chi) - logf(K.chi_lo)) * (float)NCX / (logf(K.chi_hi) - logf(K.chi_lo));
    int cx = (int)t, cu = (int)(u * (float)NCU);
    cx = cx < 0 ? 0 : (cx >= NCX ? NCX - 1 : cx);
    cu = cu < 0 ? 0 : (cu >= NCU ? NCU - 1 : cu);
    return cx * NCU + cu;
}

// ---------------------------------------------------------------------------------------
// Initialisation: U(-1/sqrt(fan_in), 1/sqrt(fan_in)) for weights and biases (Philox).
__global__ void init_kernel(float *p, uint64_t seed) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NP) return;
    const float fan = i < O_W2 ? 2.0f : 64.0f;
    const u4 w = draws(seed, (uint64_t)i, 0, 7);
    p[i] = (2.0f * uniform<float>(w.w[0]) - 1.0f) * rsqrtf(fan);
}

// ---------------------------------------------------------------------------------------
// Training: forward and backward of TS samples per block, gradient partial per block.
constexpr int TS = 64, TB = 256, LD = 65;
struct TrainSmem {
    float w2[H * LD], w3[H * LD];
    float w1[H * 2], b1[H], b2[H], b3[H], w4[H], b4;
    float x[TS * 2], yt[TS], dy[TS];
    int valid[TS];
    float z1[TS * LD], a1[TS * LD], z2[TS * LD], a2[TS * LD], z3[TS * LD], a3[TS * LD], t[TS * LD];
    float red[TB];
};

struct TrainArgs {
    const float *params;
    int64_t n;
    const float *chi, *u, *lnw;
    int64_t base;          // sequential mode: first sample of block 0
    int random;            // 1: minibatch indices drawn by Philox(seed, k, step)
    uint64_t seed;
    uint32_t step;
    int quantize;
    float scale;           // d loss / d y = scale * r  (2 / batch)
    float *partial;        // [gridDim.x][NP]
    float *partial_loss;   // [gridDim.x]
    Kind K;
};

// Z[s][j] = sum_k A[s][k] W[j][k] + b[j] over the block's samples (K = 64).
__device__ __forceinline__ void layer_fwd(const float *A, const float *W, const float *b, float *Z, float *Aout,
                                          bool q) {
    const int j = threadIdx.x & 63, s0 = threadIdx.x >> 6;
    float acc[TS / 4];
#pragma unroll
    for (int k = 0; k < TS / 4; ++k) acc[k] = b[j];
    for (int k = 0; k < H; ++k) {
        const float w = W[j * LD + k];
#pragma unroll
        for (int r = 0; r < TS / 4; ++r) acc[r] = fmaf(A[(s0 + 4 * r) * LD + k], w, acc[r]);
    }
#pragma unroll
    for (int r = 0; r < TS / 4; ++r) {
        const int s = s0 + 4 * r;
        Z[s * LD + j] = acc[r];
        Aout[s * LD + j] = qz(silu(acc[r]), q);
    }
}
// gW[j][k] = sum_s dZ[s][j] A[s][k]  (written to g[j * 64 + k]),  gb[j] = sum_s dZ[s][j].
// Lanes run over k, so the partial-gradient rows are written coalesced.
__device__ __forceinline__ void layer_gw(const float *dZ, const float *A, float *g, float *gb) {
    const int k = threadIdx.x & 63, j0 = threadIdx.x >> 6;
    float acc[H / 4];
#pragma unroll
    for (int r = 0; r < H / 4; ++r) acc[r] = 0.0f;
    for (int s = 0; s < TS; ++s) {
        const float av = A[s * LD + k];
#pragma unroll
        for (int r = 0; r < H / 4; ++r) acc[r] = fmaf(dZ[s * LD + j0 + 4 * r], av, acc[r]);
    }
#pragma unroll
    for (int r = 0; r < H / 4; ++r) g[(j0 + 4 * r) * H + k] = acc[r];
    if (threadIdx.x < H) {
        float sb = 0.0f;
        for (int s = 0; s < TS; ++s) sb += dZ[s * LD + threadIdx.x];
        gb[threadIdx.x] = sb;
    }
}
// dA[s][k] = sum_j dZ[s][j] W[j][k]; then dZprev[s][k] = dA[s][k] * silu'(Zprev[s][k]) in place.
__device__ __forceinline__ void layer_bwd_input(const float *dZ, const float *W, float *T, float *Zprev) {
    const int k = threadIdx.x & 63, s0 = threadIdx.x >> 6;
    float acc[TS / 4];
#pragma unroll
    for (int r = 0; r < TS / 4; ++r) acc[r] = 0.0f;
    for (int j = 0; j < H; ++j) {
        const float w = W[j * LD + k];
#pragma unroll
        for (int r = 0; r < TS / 4; ++r) acc[r] = fmaf(dZ[(s0 + 4 * r) * LD + j], w, acc[r]);
    }
#pragma unroll
    for (int r = 0; r < TS / 4; ++r) {
        const int s = s0 + 4 * r;
        T[s * LD + k] = acc[r];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < TS / 4; ++r) {
        const int s = s0 + 4 * r;
        Zprev[s * LD + k] = T[s * LD + k] * dsilu(Zprev[s * LD + k]);
    }
}

__global__ void __launch_bounds__(TB) train_kernel(const TrainArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    TrainSmem &S = *reinterpret_cast<TrainSmem *>(smraw);
    const bool q = a.quantize != 0;
    const int tid = threadIdx.x;
    const float *P = a.params;
    for (int e = tid; e < H * H; e += TB) {
        const int j = e >> 6, k = e & 63;
        S.w2[j * LD + k] = qz(P[O_W2 + e], q);
        S.w3[j * LD + k] = qz(P[O_W3 + e], q);
    }
    if (tid < H) {
        S.w1[2 * tid] = qz(P[O_W1 + 2 * tid], q);
        S.w1[2 * tid + 1] = qz(P[O_W1 + 2 * tid + 1], q);
        S.b1[tid] = P[O_B1 + tid];
        S.b2[tid] = P[O_B2 + tid];
        S.b3[tid] = P[O_B3 + tid];
        S.w4[tid] = qz(P[O_W4 + tid], q);
    }
    if (tid == 0) S.b4 = P[O_B4];
    if (tid < TS) {
        int64_t idx;
        bool ok;
        if (a.random) {
            const u4 w = draws(a.seed, (uint64_t)blockIdx.x * TS + tid, a.step, 5);
            idx = (int64_t)(((uint64_t)w.w[0] * (uint64_t)a.n) >> 32);
            ok = true;
        } else {
            idx = a.base + (int64_t)blockIdx.x * TS + tid;
            ok = idx < a.n;
        }
        float chi = 1.0f, u = 0.5f, lw = 0.0f;
        if (ok) {
            chi = a.chi[idx];
            u = a.u[idx];
            lw = a.lnw[idx];
            ok = isfinite(lw);            // samples without a target (NaN) do not enter the loss
            if (!ok) { chi = 1.0f; u = 0.5f; lw = 0.0f; }
        }
        float x1, x2;
        features(a.K, chi, u, x1, x2);
        S.x[2 * tid] = x1;
        S.x[2 * tid + 1] = x2;
        S.yt[tid] = lw - out_offset(a.K, u);
        S.valid[tid] = ok;
    }
    __syncthreads();
    // layer 1 (2 -> 64)
    {
        const int j = tid & 63, s0 = tid >> 6;
#pragma unroll
        for (int r = 0; r < TS / 4; ++r) {
            const int s = s0 + 4 * r;
            const float z = fmaf(S.w1[2 * j], S.x[2 * s], fmaf(S.w1[2 * j + 1], S.x[2 * s + 1], S.b1[j]));
            S.z1[s * LD + j] = z;
            S.a1[s * LD + j] = qz(silu(z), q);
        }
    }
    __syncthreads();
    layer_fwd(S.a1, S.w2, S.b2, S.z2, S.a2, q);
    __syncthreads();
    layer_fwd(S.a2, S.w3, S.b3, S.z3, S.a3, q);
    __syncthreads();
    // layer 4 (64 -> 1): four threads per sample
    {
        const int s = tid >> 2, part = tid & 3;
        float acc = 0.0f;
        for (int k = part * 16; k < part * 16 + 16; ++k) acc = fmaf(S.a3[s * LD + k], S.w4[k], acc);
        acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 1);
        acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 2);
        if (part == 0) {
            const float y = acc + S.b4;
            const float r = S.valid[s] ? y - S.yt[s] : 0.0f;
            S.dy[s] = a.scale * r;
            S.red[s] = r * r;
        }
    }
    __syncthreads();
    float *G = a.partial + (size_t)blockIdx.x * NP;
    if (tid == 0) {
        float l = 0.0f, gb = 0.0f;
        for (int s = 0; s < TS; ++s) {
            l += S.red[s];
            gb += S.dy[s];
        }
        a.partial_loss[blockIdx.x] = l;
        G[O_B4] = gb;
    }
    // layer 4 backward: gW4, and dZ3 = (dy w4) * silu'(z3) in place
    if (tid < H) {
        float g = 0.0f;
        for (int s = 0; s < TS; ++s) g = fmaf(S.dy[s], S.a3[s * LD + tid], g);
        G[O_W4 + tid] = g;
    }
    __syncthreads();
    {
        const int k = tid & 63, s0 = tid >> 6;
#pragma unroll
        for (int r = 0; r < TS / 4; ++r) {
            const int s = s0 + 4 * r;
            S.z3[s * LD + k] = S.dy[s] * S.w4[k] * dsilu(S.z3[s * LD + k]);
        }
    }
    __syncthreads();
    layer_gw(S.z3, S.a2, G + O_W3, G + O_B3);
    layer_bwd_input(S.z3, S.w3, S.t, S.z2);          // z2 <- dZ2
    __syncthreads();
    layer_gw(S.z2, S.a1, G + O_W2, G + O_B2);
    layer_bwd_input(S.z2, S.w2, S.t, S.z1);          // z1 <- dZ1
    __syncthreads();
    if (tid < H) {
        float g0 = 0.0f, g1 = 0.0f, gb = 0.0f;
        for (int s = 0; s < TS; ++s) {
            const float d = S.z1[s * LD + tid];
            g0 = fmaf(d, S.x[2 * s], g0);
            g1 = fmaf(d, S.x[2 * s + 1], g1);
            gb += d;
        }
        G[O_W1 + 2 * tid] = g0;
        G[O_W1 + 2 * tid + 1] = g1;
        G[O_B1 + tid] = gb;
    }
}

// Sum of the per-block partials in a fixed order (deterministic).
__global__ void reduce_kernel(const float *__restrict__ partial, const float *__restrict__ partial_loss, int nb,
                              float *__restrict__ grad, float *__restrict__ loss, float loss_scale) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NP) {
        float g = 0.0f;
        for (int b = 0; b < nb; ++b) g += partial[(size_t)b * NP + p];
        grad[p] = g;
    }
    if (p == 0 && loss) {
        double l = 0.0;
        for (int b = 0; b < nb; ++b) l += partial_loss[b];
        *loss = (float)(l * loss_scale);
    }
}

__global__ void adam_kernel(float *p, float *m, float *v, const float *g, float lr, float b1t, float b2t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NP) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.0f - b1t), vh = vi / (1.0f - b2t);
    p[i] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

// ---------------------------------------------------------------------------------------
// SIMT forward of one sample with the weights in shared memory (calibration and the
// reference inference path).  Same rounding as the tensor-core kernel.
struct SimtW {
    float w1[H * 2], b1[H], w2[H * H], b2[H], w3[H * H], b3[H], w4[H], b4;
};
__device__ __forceinline__ void stage_simt(SimtW &W, const float *P) {
    for (int e = threadIdx.x; e < H * H; e += blockDim.x) {
        W.w2[e] = bf16r(P[O_W2 + e]);
        W.w3[e] = bf16r(P[O_W3 + e]);
    }
    for (int e = threadIdx.x; e < H; e += blockDim.x) {
        W.w1[2 * e] = bf16r(P[O_W1 + 2 * e]);
        W.w1[2 * e + 1] = bf16r(P[O_W1 + 2 * e + 1]);
        W.b1[e] = P[O_B1 + e];
        W.b2[e] = P[O_B2 + e];
        W.b3[e] = P[O_B3 + e];
        W.w4[e] = bf16r(P[O_W4 + e]);
    }
    if (threadIdx.x == 0) W.b4 = P[O_B4];
}
__device__ __forceinline__ float forward_simt(const SimtW &W, const Kind &K, float chi, float u) {
    float x1, x2;
    features(K, chi, u, x1, x2);
    float a[H], b[H];
#pragma unroll
    for (int j = 0; j < H; ++j)
        a[j] = bf16r(silu_h(0.5f * fmaf(W.w1[2 * j], x1, fmaf(W.w1[2 * j + 1], x2, W.b1[j]))));
    // layers 2 and 3: the products summed in binary32 (the tensor cores' order differs), then
    // h = (sum + b) / 2 as the tensor-core epilogue forms it
#pragma unroll
    for (int j = 0; j < H; ++j) {
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < H; ++k) acc = fmaf(a[k], W.w2[j * H + k], acc);
        b[j] = bf16r(silu_h(fmaf(0.5f, acc, 0.5f * W.b2[j])));
    }
#pragma unroll
    for (int j = 0; j < H; ++j) {
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < H; ++k) acc = fmaf(b[k], W.w3[j * H + k], acc);
        a[j] = bf16r(silu_h(fmaf(0.5f, acc, 0.5f * W.b3[j])));
    }
    float y = W.b4;
#pragma unroll
    for (int k = 0; k < H; ++k) y = fmaf(a[k], W.w4[k], y);
    return y;
}

__global__ void __launch_bounds__(128) predict_kernel(const float *__restrict__ P, const Kind K, int64_t n,
                                                      const float *__restrict__ chi, const float *__restrict__ u,
                                                      float *__restrict__ lnw) {
    __shared__ SimtW W;
    stage_simt(W, P);
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float uu = u[i];
        lnw[i] = forward_simt(W, K, chi[i], uu) + out_offset(K, uu);
    }
}

// ---------------------------------------------------------------------------------------
// Calibration: per cell, the largest |u_net - u| implied by the network's ln w-bar against
// the plain sampler's, |d ln w| / (d ln w / du), over 8 x 8 points of the cell.
// The plain fitted sampler's variable: ln w-bar (photon) or ln(-ln y) (pair, u = |r'|).
__device__ __forceinline__ float plain_lnw(const Kind &K, const float *inv, float chi, float u) {
    bool oor = false;
    if (K.pair) {
        // -ln y from v-bar = 1 - y where y is near 1; where 1 - y falls below the binary32
        // table's resolution (|r'| below about 1e-5) the variable is unresolved: NaN
        const float y = pair_y<float>(inv, chi, u, oor);
        const float v = 1.0f - y;
        if (!(v >= 1.52587890625e-05f)) return __int_as_float(0x7fffffff);    // 2^-16
        return logf(y < 0.5f ? -logf(y) : -log1pf(-v));
    }
    const float s = photon_s<float>(inv, chi, u, oor);
    return (logf(2.0f * s) - logf(3.0f * chi)) * (1.0f / 3.0f);
}
__global__ void __launch_bounds__(64) calibrate_kernel(const float *__restrict__ P, const Kind K,
                                                       const float *__restrict__ inv, float tol_u,
                                                       uint8_t *__restrict__ flags, float *__restrict__ cell_err) {
    __shared__ SimtW W;
    __shared__ float red[64];
    stage_simt(W, P);
    __syncthreads();
    const int cell = blockIdx.x, cx = cell / NCU, cu = cell % NCU;
    const int pa = threadIdx.x >> 3, pb = threadIdx.x & 7;
    const float lo = logf(K.chi_lo), span = logf(K.chi_hi) - logf(K.chi_lo);
    const float chi = expf(lo + span * ((float)cx + ((float)pa + 0.5f) * 0.125f) / (float)NCX);
    const float u = ((float)cu + ((float)pb + 0.5f) * 0.125f) / (float)NCU;
    const float ln_net = forward_simt(W, K, chi, u) + out_offset(K, u);
    const float ln_p = plain_lnw(K, inv, chi, u);
    const float h = 1.0f / (float)(NCU * 64);
    // |d ln w / du| (both sampler variables rise with u)
    const float dlnw_du = fabsf(plain_lnw(K, inv, chi, u + h) - plain_lnw(K, inv, chi, u - h)) / (2.0f * h);
    float e = fabsf(ln_net - ln_p) / fmaxf(dlnw_du, 1e-30f);
    if (!(e == e)) e = 1e30f;
    red[threadIdx.x] = e;
    __syncthreads();
    for (int o = 32; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        cell_err[cell] = red[0];
        flags[cell] = red[0] > tol_u ? 1 : 0;
    }
}

// ln w-bar of the plain fitted sampler (training targets without the oracle).
__global__ void plain_targets_kernel(const float *__restrict__ inv, const Kind K, int64_t n,
                                     const float *__restrict__ chi, const float *__restrict__ u,
                                     float *__restrict__ lnw) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        lnw[i] = plain_lnw(K, inv, chi[i], u[i]);
}

// ---------------------------------------------------------------------------------------
// Tensor-core inference.  One block of 128 threads handles tiles of 128 samples (one
// sample per thread, one row of the 128 x 64 activation tile).  Layers 2 and 3 are
//   D[128 x 64] (fp32, tensor memory) = A[128 x 64] (bf16, smem) * W^T (W: 64 x 64 bf16, smem)
// issued as four K = 16 steps of tcgen05.mma.kind::f16 by one thread; the output layer is
// the same with a 16 x 64 W whose row 0 is w4 (column 0 of D is the output).  Operands use the
// no-swizzle K-major layout: 8-row x 16-byte core matrices, core matrix (row group g, K
// chunk j) at ((g * 8) + j) * 128 bytes, i.e. K-adjacent core matrices 128 bytes apart
// (leading byte offset) and row groups 1024 bytes apart (stride byte offset).
constexpr uint32_t MMA_WAIT_LIMIT = 1u << 22;
constexpr int IT = 128;                       // samples per tile
constexpr uint32_t TMEM_COLS = 64;
// kind::f16 instruction descriptor: D f32 (bit 4), A bf16 (bits 7-9 = 1), B bf16 (bits
// 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
// the output layer: N = 16 (row 0 of its B operand holds w4, rows 1-15 are zero)
constexpr uint32_t IDESC4 = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t s_u32(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    const uint64_t lbo = 128, sbo = 1024;
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) | (1ull << 46);
}
__device__ __forceinline__ void mbar_init1(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    const uint32_t ad = s_u32(bar);
    for (uint32_t it = 0; it < MMA_WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(ad), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mma_k16(uint32_t d_tmem, uint64_t ad, uint64_t bd, uint32_t accumulate,
                                        uint32_t idesc = IDESC) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_u32(bar))
                 : "memory");
}
// 32 consecutive fp32 columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}
// Column 0 of this thread's lane.
__device__ __forceinline__ float tmem_ld1(uint32_t taddr) {
    uint32_t r;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr) : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    return __uint_as_float(r);
}
// Row m of a 128 x 64 (or 64 x 64) K-major operand: 8 chunks of 8 bf16 (16 bytes).
__device__ __forceinline__ uint32_t row_chunk_offset(int m, int j) { return (uint32_t)((((m >> 3) * 8) + j) * 128 + (m & 7) * 16); }
// The finishing of queued photon emissions (APPLY): the emitter's state before the event,
// its population, and the product records (sfq_set_surrogate).
struct ApplyOut {
    const int64_t *idx;
    const float *g, *px, *py, *pz;
    float *ppx, *ppy, *ppz;
    uint8_t *flags;
    const uint64_t *id;
    uint64_t id_base;
    int64_t cap;
    float *opx, *opy, *opz;
    uint64_t *opid;
    uint32_t *ostep;
    uint8_t *ometa;
    unsigned long long *ocount;
    uint32_t step;
};

struct InferArgs {
    const float *params;
    const uint8_t *flags;     // NULL: no calibration (every in-range draw uses the network)
    const float *inv;         // plain inverse-CDF table (fallback)
    int64_t n;
    const float *chi, *r;
    float *xi, *xi_c;
    sfq_counters *counters;
    int *status;              // set to 1 when a bounded wait gave up
    Kind K;                   // photon: xi, xi_c = 1 - xi; pair: xi = electron share, xi_c = positron share
    const unsigned long long *n_dev;   // APPLY: device count of queued samples (min with n)
    ApplyOut ap;
};

// Warp-wide reservation of one slot per lane that wants one: one atomic per warp.
__device__ __forceinline__ unsigned long long warp_reserve(unsigned long long *ctr, bool want) {
    const unsigned m = __ballot_sync(0xFFFFFFFFu, want);
    const int lane = threadIdx.x & 31;
    const int leader = m ? __ffs(m) - 1 : 0;
    unsigned long long base = 0;
    if (m && lane == leader) base = atomicAdd(ctr, (unsigned long long)__popc(m));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    return base + (unsigned long long)__popc(m & ((1u << lane) - 1u));
}

// Operands (no-swizzle K-major, 16-byte aligned): A 128 x 64, W2 and W3 64 x 64, W4 16 x 64;
// then layer 1's weights, the halved biases of layers 2 and 3, b4 and the fallback flags.
constexpr uint32_t SM_A = 0, SM_B2 = 16384, SM_B3 = 24576, SM_B4 = 32768, SM_SMALL = 34816;
constexpr uint32_t SM_FLAGS = SM_SMALL + ((H * 2 + 3 * H + 1) * 4 + 15) / 16 * 16;
constexpr uint32_t SM_BYTES = SM_FLAGS + NCELL / 8;    // the fallback flags as one bit per cell
constexpr uint32_t INFER_SMEM = SM_BYTES + 128;      // + alignment slack
#ifndef SFQ_INFER_MINB
#define SFQ_INFER_MINB 6
#endif
constexpr int INFER_MINB = SFQ_INFER_MINB;            // resident blocks per SM (registers, 36 KB of shared memory each)

// Eight bfloat16 (one 16-byte K chunk of an operand row) from eight binary32 values.
__device__ __forceinline__ uint4 pack8_bf16(const float *a) {
    uint4 v;
    __nv_bfloat162 p0 = __floats2bfloat162_rn(a[0], a[1]);
    __nv_bfloat162 p1 = __floats2bfloat162_rn(a[2], a[3]);
    __nv_bfloat162 p2 = __floats2bfloat162_rn(a[4], a[5]);
    __nv_bfloat162 p3 = __floats2bfloat162_rn(a[6], a[7]);
    v.x = *reinterpret_cast<uint32_t *>(&p0);
    v.y = *reinterpret_cast<uint32_t *>(&p1);
    v.z = *reinterpret_cast<uint32_t *>(&p2);
    v.w = *reinterpret_cast<uint32_t *>(&p3);
    return v;
}

// The epilogue of a hidden tensor-core layer for this thread's row, 32 accumulator columns
// at a time (so that no more than 32 accumulators are live): h = (d + b) / 2 from the
// halved biases hb, SiLU, and the bfloat16 row of the next layer's operand A.
__device__ __forceinline__ void epilogue(uint32_t t_row, const float *hb, unsigned char *a_base, int row) {
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        float d[32];
        tmem_ld32(t_row + 32 * half, d);
#pragma unroll
        for (int j = 0; j < 32; ++j) d[j] = silu_h(fmaf(0.5f, d[j], hb[32 * half + j]));
#pragma unroll
        for (int c = 0; c < 4; ++c)
            *reinterpret_cast<uint4 *>(a_base + row_chunk_offset(row, 4 * half + c)) = pack8_bf16(d + 8 * c);
    }
}

// One block of 128 threads walks over tiles of 128 samples (one sample per thread, one
// row of the 128 x 64 activation tile); INFER_MINB blocks share an SM, so that the tensor
// cores of one block's layer run while the others compute their SiLU epilogues.
// APPLY (photon kind): the samples are the queued emissions of a Monte Carlo step; each
// sampled xi also recoils its emitter (Sec. 3: the lepton keeps (1 - xi) gamma along its
// direction) and appends the collinear photon's record.
template <bool APPLY>
__global__ void __launch_bounds__(IT, INFER_MINB) infer_tc_kernel(const InferArgs a) {
    extern __shared__ unsigned char sraw[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_err;
    __shared__ unsigned long long s_cnt[6];
    // 128-byte aligned operand area (the no-swizzle layout needs 16-byte alignment)
    const uint32_t raw = s_u32(sraw);
    unsigned char *sm = sraw + ((128u - (raw & 127u)) & 127u);
    const uint32_t sbase = s_u32(sm);
    float *w1 = reinterpret_cast<float *>(sm + SM_SMALL);
    float *b1 = w1 + 2 * H, *hb2 = b1 + H, *hb3 = hb2 + H, *b4 = hb3 + H;
    uint32_t *fl = reinterpret_cast<uint32_t *>(sm + SM_FLAGS);
    const int tid = threadIdx.x, warp = tid >> 5;
    const float *P = a.params;

    // weights: W2, W3 and W4 (row 0 of a 16-row operand, the other rows zero) as bf16 in the
    // K-major core-matrix layout; layer 1 binary32 (bf16-rounded weights); the biases of
    // layers 2 and 3 halved for the SiLU form
    for (int e = tid; e < H * H; e += IT) {
        const int n_ = e >> 6, k = e & 63;
        const uint32_t off = row_chunk_offset(n_, k >> 3) + (k & 7) * 2;
        *reinterpret_cast<__nv_bfloat16 *>(sm + SM_B2 + off) = __float2bfloat16_rn(P[O_W2 + e]);
        *reinterpret_cast<__nv_bfloat16 *>(sm + SM_B3 + off) = __float2bfloat16_rn(P[O_W3 + e]);
    }
    for (int e = tid; e < 16 * H; e += IT) {
        const int n_ = e >> 6, k = e & 63;
        const uint32_t off = row_chunk_offset(n_, k >> 3) + (k & 7) * 2;
        *reinterpret_cast<__nv_bfloat16 *>(sm + SM_B4 + off) = __float2bfloat16_rn(n_ == 0 ? P[O_W4 + k] : 0.0f);
    }
    for (int e = tid; e < H; e += IT) {
        // layer 1 halved as well (exact: a power of two), so that h = z / 2 comes out of its fmas
        w1[2 * e] = 0.5f * bf16r(P[O_W1 + 2 * e]);
        w1[2 * e + 1] = 0.5f * bf16r(P[O_W1 + 2 * e + 1]);
        b1[e] = 0.5f * P[O_B1 + e];
        hb2[e] = 0.5f * P[O_B2 + e];
        hb3[e] = 0.5f * P[O_B3 + e];
    }
    if (tid == 0) *b4 = P[O_B4];
    for (int e = tid; e < NCELL / 32; e += IT) {
        uint32_t w = 0;
        if (a.flags)
            for (int b = 0; b < 32; ++b) w |= (a.flags[32 * e + b] ? 1u : 0u) << b;
        fl[e] = w;
    }
    if (tid < 6) s_cnt[tid] = 0;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_u32(&tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init1(&mbar);
        s_err = 0;
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = tmem_base;
    const uint32_t t_row = taddr + ((uint32_t)(warp * 32) << 16);
    uint32_t phase = 0;
    uint32_t n_nan = 0, n_oor = 0, n_fb = 0, n_emit = 0, n_drop = 0, n_g1 = 0;
    int64_t n_all = a.n;
    if (APPLY) {
        const int64_t q = (int64_t)*a.n_dev;
        n_all = q < n_all ? q : n_all;
    }
    const int64_t ntiles = (n_all + IT - 1) / IT;
    int pending = 0;                              // an MMA group issued and not yet waited for

    // the inputs of the block's next tile are loaded a tile ahead, so that their latency falls
    // in the current tile's work
    float chi_n = 1.0f, r_n = 0.5f;
    {
        const int64_t i0 = (int64_t)blockIdx.x * IT + tid;
        if (i0 < n_all) { chi_n = a.chi[i0]; r_n = a.r[i0]; }
    }
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t i = tile * IT + tid;
        const bool valid = i < n_all;
        const float chi = chi_n, r = r_n;
        {
            const int64_t inext = (tile + gridDim.x) * IT + tid;
            chi_n = 1.0f;
            r_n = 0.5f;
            if (inext < n_all) { chi_n = a.chi[inext]; r_n = a.r[inext]; }
        }
        const bool bad = !(chi >= 0.0f) || !(r > 0.0f) || !(r < 1.0f);
        const float rp = 2.0f * r - 1.0f;                 // pair creation: r' (exact for r in (0, 1))
        const float u = a.K.pair ? fabsf(rp) : r;
        const bool in_range = chi >= a.K.chi_lo && chi <= a.K.chi_hi;
        const int cell = cell_of(a.K, chi, u);
        const bool fallback = !bad && (!in_range || ((fl[cell >> 5] >> (cell & 31)) & 1u));
        // layer 1 on the CUDA cores (binary32 features, bf16-rounded weights), 8 columns at a time
        float x1, x2;
        features(a.K, in_range ? chi : 1.0f, bad ? 0.5f : u, x1, x2);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int j = 8 * c + q;
                v[q] = silu_h(fmaf(w1[2 * j], x1, fmaf(w1[2 * j + 1], x2, b1[j])));
            }
            *reinterpret_cast<uint4 *>(sm + SM_A + row_chunk_offset(tid, c)) = pack8_bf16(v);
        }
        float y = 0.0f;
#pragma unroll 1
        for (int layer = 0; layer < 3; ++layer) {
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                const uint32_t bw = layer == 0 ? SM_B2 : (layer == 1 ? SM_B3 : SM_B4);
                const uint32_t idesc = layer == 2 ? IDESC4 : IDESC;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    mma_k16(taddr, smem_desc(sbase + SM_A + 256 * kk), smem_desc(sbase + bw + 256 * kk), kk > 0,
                            idesc);
                mma_commit(&mbar);
            }
            pending = 1;
            if (!mbar_wait_bounded(&mbar, phase)) s_err = 1;
            __syncthreads();
            if (s_err) break;
            pending = 0;
            phase ^= 1;
            tc_fence_after();
            // layers 2 and 3: the SiLU row goes to A (the MMA that read A has completed); the
            // output layer: column 0 plus b4
            if (layer < 2) epilogue(t_row, layer == 0 ? hb2 : hb3, sm + SM_A, tid);
            else y = tmem_ld1(t_row) + *b4;
            tc_fence_before();
        }
        if (s_err) break;
        float xi_v = 0.0f, xc_v = 0.0f;
        if (valid) {
            float xi, xc;
            if (bad) {
                ++n_nan;
                xi = 0.0f;
                xc = 0.0f;
            } else if (a.K.pair) {
                bool oor = false;
                if (fallback) {
                    pair_shares<float>(a.inv, chi, r, xi, xc, oor);
                    n_oor += oor;
                    ++n_fb;
                } else {
                    // 1 - v-bar = exp(-u e^y): at most 1 for any network output
                    const float small = 0.5f * expf(-expf(y + logf(u))), big = 1.0f - small;
                    xi = rp >= 0.0f ? big : small;
                    xc = rp >= 0.0f ? small : big;
                }
            } else {
                float s;
                if (fallback) {
                    bool oor = false;
                    s = photon_s<float>(a.inv, chi, u, oor);
                    n_oor += oor;
                    ++n_fb;
                } else {
                    s = 1.5f * chi * expf(3.0f * (y + logf(u)));
                }
                xc = 1.0f / (1.0f + s);
                xi = s < 1e30f ? s * xc : 1.0f;
            }
            a.xi[i] = xi;
            if (a.xi_c) a.xi_c[i] = xc;
            xi_v = xi;
            xc_v = xc;
        }
        if (APPLY) {
            // recoil of the emitter and the photon's record (every lane takes part in the
            // warp-wide reservation)
            const ApplyOut &o = a.ap;
            const bool emit = valid && !bad;
            const unsigned long long slot = warp_reserve(o.ocount, emit);
            if (emit) {
                // xi and 1 - xi = 1/(1 + s), the latter with relative precision (hard photons)
                const float xi = xi_v, xc = xc_v;
                const int64_t e = o.idx[i];
                const float g = o.g[i], px = o.px[i], py = o.py[i], pz = o.pz[i];
                const float pm = sqrtf(fmaf(px, px, fmaf(py, py, pz * pz)));
                const float inv_pm = pm > 0.0f ? 1.0f / pm : 0.0f;
                const float nx = px * inv_pm, ny = py * inv_pm, nz = pz * inv_pm;
                const float gph = g * xi, gnew = g * xc;
                const float q2 = fmaf(gnew, gnew, -1.0f);
                const float pnew = q2 > 0.0f ? sqrtf(q2) : 0.0f;
                n_g1 += !(q2 > 0.0f);
                const uint8_t fl = o.flags[e];
                if (slot < (unsigned long long)o.cap) {
                    o.opx[slot] = nx * gph; o.opy[slot] = ny * gph; o.opz[slot] = nz * gph;
                    o.opid[slot] = o.id ? o.id[e] : o.id_base + (uint64_t)e;
                    o.ostep[slot] = o.step;
                    o.ometa[slot] = (uint8_t)(SFQ_PHOTON | (((fl >> SFQ_TAG_SHIFT) & 3u) << 4));
                } else {
                    ++n_drop;
                }
                o.ppx[e] = nx * pnew; o.ppy[e] = ny * pnew; o.ppz[e] = nz * pnew;
                // a lepton left without momentum leaves the step (as in the step kernels)
                if (!(pnew > 0.0f)) o.flags[e] = (uint8_t)(fl & ~SFQ_ALIVE);
                ++n_emit;
            }
        }
    }
    // a group whose wait gave up: wait once more (bounded) before the tensor memory is freed
    if (pending && tid == 0) {
        if (!mbar_wait_bounded(&mbar, phase) && a.status) atomicExch(a.status, 1);
    }
    if (s_err && tid == 0 && a.counters) atomicAdd(&a.counters->timeouts, 1ull);
    atomicAdd(&s_cnt[0], (unsigned long long)n_nan);
    atomicAdd(&s_cnt[1], (unsigned long long)n_oor);
    atomicAdd(&s_cnt[2], (unsigned long long)n_fb);
    if (APPLY) {
        atomicAdd(&s_cnt[3], (unsigned long long)n_emit);
        atomicAdd(&s_cnt[4], (unsigned long long)n_drop);
        atomicAdd(&s_cnt[5], (unsigned long long)n_g1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TMEM_COLS) : "memory");
    }
    if (tid == 0 && a.counters) {
        if (s_cnt[0]) atomicAdd(&a.counters->nan_input, s_cnt[0]);
        if (s_cnt[1]) atomicAdd(&a.counters->out_of_range, s_cnt[1]);
        if (s_cnt[2]) atomicAdd(&a.counters->surrogate_fallbacks, s_cnt[2]);
        if (APPLY) {
            if (s_cnt[3]) atomicAdd(&a.counters->emitted, s_cnt[3]);
            if (s_cnt[4]) atomicAdd(&a.counters->dropped, s_cnt[4]);
            if (s_cnt[5]) atomicAdd(&a.counters->gamma_below_one, s_cnt[5]);
        }
    }
    if (s_err && tid == 0 && a.status) atomicExch(a.status, 1);
}

}  // namespace mlp

// The surrogate pass of a step: sample the queued emissions and finish them (recoil and
// records), one persistent grid over the queue's capacity (the count is read on the device).
cudaError_t launch_surrogate_apply(const sfq_ctx *ctx, const sfq_particles *p, uint32_t step, const sfq_products *out,
                                   sfq_counters *counters, cudaStream_t stream) {
    using namespace mlp;
    const sfq_mlp *m = ctx->surr;
    const sfq_event_queue &q = ctx->surr_q;
    if (q.capacity <= 0) return cudaSuccess;
    const int64_t ntiles = (q.capacity + IT - 1) / IT;
    int64_t grid = (int64_t)ctx->surr_per_sm * ctx->num_sms;
    if (ntiles < grid) grid = ntiles;
    InferArgs a{};
    a.params = m->params;
    a.flags = ctx->surr_flags ? m->flags : nullptr;
    a.inv = static_cast<const float *>(ctx->d_nlc_inv);
    a.n = q.capacity;
    a.chi = q.chi;
    a.r = q.r;
    a.xi = q.xi;
    a.xi_c = nullptr;
    a.counters = counters;
    a.status = nullptr;
    a.K = kind_of(0);
    a.n_dev = q.count;
    ApplyOut &o = a.ap;
    o.idx = q.index;
    o.g = q.gamma; o.px = q.px; o.py = q.py; o.pz = q.pz;
    o.ppx = static_cast<float *>(p->px); o.ppy = static_cast<float *>(p->py); o.ppz = static_cast<float *>(p->pz);
    o.flags = p->flags;
    o.id = p->id;
    o.id_base = p->id_base;
    o.cap = out->capacity;
    o.opx = static_cast<float *>(out->px); o.opy = static_cast<float *>(out->py); o.opz = static_cast<float *>(out->pz);
    o.opid = out->parent_id;
    o.ostep = out->step;
    o.ometa = out->meta;
    o.ocount = out->count;
    o.step = step;
    infer_tc_kernel<true><<<(unsigned)grid, IT, INFER_SMEM, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace sfq

// ---------------------------------------------------------------------------------------
// C ABI
namespace {

using namespace sfq::mlp;

sfq_status fail(sfq_ctx *ctx, sfq_status st, const char *msg) {
    if (ctx) ctx->err = msg;
    return st;
}
sfq_status cuda_fail(sfq_ctx *ctx, cudaError_t e, const char *where) {
    if (ctx) ctx->err = std::string(where) + ": " + cudaGetErrorString(e);
    return SFQ_ERR_CUDA;
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
bool a16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Attributes of an inference kernel instance: its dynamic shared memory, and the largest
// shared-memory carveout, so that INFER_MINB blocks (6 x 36 KB) are resident on an SM.  The
// grid is then INFER_MINB blocks per SM: registers (at most 85 a thread by the launch
// bounds), shared memory and tensor memory (6 x 64 of the 512 columns) all admit them.
template <typename K>
cudaError_t set_infer_attributes(K kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)INFER_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    return e;
}

// The plain fitted sampler the surrogate stands for (training targets, calibration, fallback).
const float *inv_table(const sfq_mlp *m) {
    return static_cast<const float *>(m->kind ? m->ctx->d_nbw_inv : m->ctx->d_nlc_inv);
}

}  // namespace

extern "C" {

static sfq_status mlp_create(sfq_ctx *ctx, uint64_t seed, int kind, sfq_mlp **out) {
    if (!ctx || !out) return SFQ_ERR_ARG;
    *out = nullptr;
    if (ctx->cfg.precision != SFQ_FP32) return fail(ctx, SFQ_ERR_ARG, "the surrogate serves binary32 contexts");
    DeviceGuard g(ctx->device);
    sfq_mlp *m = new sfq_mlp();
    m->ctx = ctx;
    m->kind = kind;
    float **bufs[4] = {&m->params, &m->m, &m->v, &m->grad};
    cudaError_t e = cudaSuccess;
    for (auto b : bufs)
        if (e == cudaSuccess) e = cudaMalloc(b, NP * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->flags, NCELL);
    if (e == cudaSuccess) e = cudaMalloc(&m->cell_err, NCELL * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(m->m, 0, NP * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(m->v, 0, NP * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(m->flags, 0, NCELL);
    if (e == cudaSuccess) {
        init_kernel<<<(NP + 255) / 256, 256>>>(m->params, seed);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        sfq_mlp_destroy(m);
        return cuda_fail(ctx, e, "sfq_mlp_create");
    }
    *out = m;
    return SFQ_OK;
}

sfq_status sfq_mlp_create(sfq_ctx *ctx, uint64_t seed, sfq_mlp **out) { return mlp_create(ctx, seed, 0, out); }
sfq_status sfq_mlp_create_pair(sfq_ctx *ctx, uint64_t seed, sfq_mlp **out) { return mlp_create(ctx, seed, 1, out); }

void sfq_mlp_destroy(sfq_mlp *m) {
    if (!m) return;
    if (m->ctx->surr == m) m->ctx->surr = nullptr;     // detach from the context's step
    DeviceGuard g(m->ctx->device);
    void *p[6] = {m->params, m->m, m->v, m->grad, m->flags, m->cell_err};
    for (void *q : p)
        if (q) cudaFree(q);
    delete m;
}

int32_t sfq_mlp_num_params(void) { return NP; }

sfq_status sfq_mlp_get_params(sfq_mlp *m, float *host) {
    if (!m || !host) return SFQ_ERR_ARG;
    DeviceGuard g(m->ctx->device);
    const cudaError_t e = cudaMemcpy(host, m->params, NP * sizeof(float), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? SFQ_OK : cuda_fail(m->ctx, e, "sfq_mlp_get_params");
}

sfq_status sfq_mlp_set_params(sfq_mlp *m, const float *host) {
    if (!m || !host) return SFQ_ERR_ARG;
    DeviceGuard g(m->ctx->device);
    cudaError_t e = cudaMemcpy(m->params, host, NP * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->m, 0, NP * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(m->v, 0, NP * sizeof(float));
    m->adam_t = 0;
    m->calibrated = 0;
    return e == cudaSuccess ? SFQ_OK : cuda_fail(m->ctx, e, "sfq_mlp_set_params");
}

static sfq_status check_data(sfq_mlp *m, int64_t n, const float *chi, const float *u, const float *lnw) {
    if (n <= 0) return fail(m->ctx, SFQ_ERR_ARG, "n must be positive");
    if (n > 0xFFFFFFFFll) return fail(m->ctx, SFQ_ERR_ARG, "n above 2^32");
    if (!chi || !u || !lnw) return fail(m->ctx, SFQ_ERR_ARG, "null data buffer");
    return SFQ_OK;
}

static cudaError_t set_train_smem() {
    static bool done = false;
    if (done) return cudaSuccess;
    const cudaError_t e =
        cudaFuncSetAttribute(train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainSmem));
    if (e == cudaSuccess) done = true;
    return e;
}

sfq_status sfq_mlp_loss_grad(sfq_mlp *m, int64_t n, const float *chi, const float *u, const float *lnw,
                             int32_t quantize, float *grad, float *loss, void *stream) {
    if (!m) return SFQ_ERR_ARG;
    sfq_status st = check_data(m, n, chi, u, lnw);
    if (st != SFQ_OK) return st;
    if (!grad) return fail(m->ctx, SFQ_ERR_ARG, "null gradient buffer");
    DeviceGuard g(m->ctx->device);
    const cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = set_train_smem();
    const int nb = (int)((n + TS - 1) / TS);
    float *part = nullptr;
    if (e == cudaSuccess) e = cudaMallocAsync(&part, ((size_t)nb * NP + nb) * sizeof(float), s);
    if (e != cudaSuccess) return cuda_fail(m->ctx, e, "sfq_mlp_loss_grad");
    TrainArgs a{m->params, n, chi, u, lnw, 0, 0, 0, 0, quantize, 2.0f / (float)n, part, part + (size_t)nb * NP,
                kind_of(m->kind)};
    train_kernel<<<nb, TB, sizeof(TrainSmem), s>>>(a);
    reduce_kernel<<<(NP + 255) / 256, 256, 0, s>>>(part, part + (size_t)nb * NP, nb, grad, loss, 1.0f / (float)n);
    e = cudaGetLastError();
    cudaFreeAsync(part, s);
    return e == cudaSuccess ? SFQ_OK : cuda_fail(m->ctx, e, "sfq_mlp_loss_grad");
}

sfq_status sfq_mlp_train(sfq_mlp *m, int64_t n, const float *chi, const float *u, const float *lnw, int64_t steps,
                         int32_t batch, float lr, int32_t quantize, uint64_t seed, float *loss_history, void *stream) {
    if (!m) return SFQ_ERR_ARG;
    sfq_status st = check_data(m, n, chi, u, lnw);
    if (st != SFQ_OK) return st;
    if (steps <= 0 || batch < TS || batch % TS != 0) return fail(m->ctx, SFQ_ERR_ARG, "steps > 0 and batch a multiple of 64");
    if (!(lr > 0.0f)) return fail(m->ctx, SFQ_ERR_ARG, "lr must be positive");
    DeviceGuard g(m->ctx->device);
    const cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = set_train_smem();
    const int nb = batch / TS;
    float *part = nullptr;
    if (e == cudaSuccess) e = cudaMallocAsync(&part, ((size_t)nb * NP + nb) * sizeof(float), s);
    if (e != cudaSuccess) return cuda_fail(m->ctx, e, "sfq_mlp_train");
    for (int64_t t = 0; t < steps && e == cudaSuccess; ++t) {
        TrainArgs a{m->params, n, chi, u, lnw, 0, 1, seed, (uint32_t)(m->adam_t + 1), quantize,
                    2.0f / (float)batch, part, part + (size_t)nb * NP, kind_of(m->kind)};
        train_kernel<<<nb, TB, sizeof(TrainSmem), s>>>(a);
        reduce_kernel<<<(NP + 255) / 256, 256, 0, s>>>(part, part + (size_t)nb * NP, nb, m->grad,
                                                        loss_history ? loss_history + t : nullptr,
                                                        1.0f / (float)batch);
        m->adam_t += 1;
        // cosine schedule from lr to 0
        const float lrt = 0.5f * lr * (1.0f + cosf(3.14159265f * (float)t / (float)steps));
        const float b1t = powf(0.9f, (float)m->adam_t), b2t = powf(0.999f, (float)m->adam_t);
        adam_kernel<<<(NP + 255) / 256, 256, 0, s>>>(m->params, m->m, m->v, m->grad, lrt, b1t, b2t);
        e = cudaGetLastError();
    }
    cudaFreeAsync(part, s);
    m->calibrated = 0;
    return e == cudaSuccess ? SFQ_OK : cuda_fail(m->ctx, e, "sfq_mlp_train");
}

sfq_status sfq_mlp_predict_lnw(sfq_mlp *m, int64_t n, const float *chi, const float *u, float *lnw, void *stream) {
    if (!m) return SFQ_ERR_ARG;
    if (n < 0) return fail(m->ctx, SFQ_ERR_ARG, "n < 0");
    if (n == 0) return SFQ_OK;
    if (!chi || !u || !lnw) return fail(m->ctx, SFQ_ERR_ARG, "null buffer");
    DeviceGuard g(m->ctx->device);
    const int64_t blocks = (n + 127) / 128;
    const int grid = (int)(blocks < (int64_t)m->ctx->num_sms * 8 ? blocks : (int64_t)m->ctx->num_sms * 8);
    predict_kernel<<<grid, 128, 0, (cudaStream_t)stream>>>(m->params, kind_of(m->kind), n, chi, u, lnw);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SFQ_OK : cuda_fail(m->ctx, e, "sfq_mlp_predict_lnw");
}

sfq_status sfq_mlp_plain_targets(sfq_mlp *m, int64_t n, const float *chi, const float *u, float *lnw, void *stream) {
    if (!m) return SFQ_ERR_ARG;
    if (n < 0) return fail(m->ctx, SFQ_ERR_ARG, "n < 0");
    if (n == 0) return SFQ_OK;
    if (!chi || !u || !lnw) return fail(m->ctx, SFQ_ERR_ARG, "null buffer");
    DeviceGuard g(m->ctx->device);
    const int64_t blocks = (n + 255) / 256;
    const int grid = (int)(blocks < (int64_t)m->ctx->num_sms * 8 ? blocks : (int64_t)m->ctx->num_sms * 8);
    plain_targets_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(inv_table(m), kind_of(m->kind), n, chi, u, lnw);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SFQ_OK : cuda_fail(m->ctx, e, "sfq_mlp_plain_targets");
}

sfq_status sfq_mlp_calibrate(sfq_mlp *m, float tol_u, int32_t *n_flagged, float *max_err, void *stream) {
    if (!m) return SFQ_ERR_ARG;
    if (!(tol_u > 0.0f)) return fail(m->ctx, SFQ_ERR_ARG, "tol_u must be positive");
    DeviceGuard g(m->ctx->device);
    const cudaStream_t s = (cudaStream_t)stream;
    calibrate_kernel<<<NCELL, 64, 0, s>>>(m->params, kind_of(m->kind), inv_table(m), tol_u, m->flags, m->cell_err);
    cudaError_t e = cudaGetLastError();
    std::vector<uint8_t> f(NCELL);
    std::vector<float> ce(NCELL);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f.data(), m->flags, NCELL, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ce.data(), m->cell_err, NCELL * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(m->ctx, e, "sfq_mlp_calibrate");
    int32_t nf = 0;
    float mx = 0.0f;
    for (int c = 0; c < NCELL; ++c) {
        nf += f[c];
        if (!f[c] && ce[c] > mx) mx = ce[c];
    }
    if (n_flagged) *n_flagged = nf;
    if (max_err) *max_err = mx;
    m->calibrated = 1;
    return SFQ_OK;
}

static sfq_status mlp_sample(sfq_mlp *m, int64_t n, const void *chi, const void *r, void *xi, void *xi_c,
                             int32_t use_flags, sfq_counters *counters, void *stream) {
    if (!m) return SFQ_ERR_ARG;
    if (n < 0) return fail(m->ctx, SFQ_ERR_ARG, "n < 0");
    if (n == 0) return SFQ_OK;
    if (!chi || !r || !xi) return fail(m->ctx, SFQ_ERR_ARG, "null buffer");
    if (!a16(chi) || !a16(r) || !a16(xi) || (xi_c && !a16(xi_c)) || (counters && ((uintptr_t)counters & 7u)))
        return fail(m->ctx, SFQ_ERR_ARG, "misaligned buffer (16 bytes required)");
    if (use_flags && !m->calibrated) return fail(m->ctx, SFQ_ERR_ARG, "use_flags before sfq_mlp_calibrate");
    DeviceGuard g(m->ctx->device);
    static bool attr = false;
    cudaError_t e = cudaSuccess;
    if (!attr) {
        e = set_infer_attributes(infer_tc_kernel<false>);
        if (e != cudaSuccess) return cuda_fail(m->ctx, e, "sfq_mlp_sample_photon_xi: attributes");
        attr = true;
    }
    const int per_sm = INFER_MINB;
    const int64_t ntiles = (n + IT - 1) / IT;
    int64_t grid = (int64_t)per_sm * m->ctx->num_sms;
    if (ntiles < grid) grid = ntiles;
    InferArgs a{m->params, use_flags ? m->flags : nullptr, inv_table(m), n,
                static_cast<const float *>(chi), static_cast<const float *>(r), static_cast<float *>(xi),
                static_cast<float *>(xi_c), counters, nullptr, kind_of(m->kind), nullptr, ApplyOut{}};
    infer_tc_kernel<false><<<(unsigned)grid, IT, INFER_SMEM, (cudaStream_t)stream>>>(a);
    e = cudaGetLastError();
    return e == cudaSuccess ? SFQ_OK : cuda_fail(m->ctx, e, "sfq_mlp_sample_*_xi");
}

sfq_status sfq_mlp_sample_photon_xi(sfq_mlp *m, int64_t n, const void *chi, const void *r, void *xi, void *xi_c,
                                    int32_t use_flags, sfq_counters *counters, void *stream) {
    if (m && m->kind != 0) return fail(m->ctx, SFQ_ERR_ARG, "a pair-creation surrogate: use sfq_mlp_sample_pair_xi");
    return mlp_sample(m, n, chi, r, xi, xi_c, use_flags, counters, stream);
}

sfq_status sfq_mlp_sample_pair_xi(sfq_mlp *m, int64_t n, const void *chi, const void *r, void *xi_e, void *xi_p,
                                  int32_t use_flags, sfq_counters *counters, void *stream) {
    if (m && m->kind != 1) return fail(m->ctx, SFQ_ERR_ARG, "a photon-emission surrogate: use sfq_mlp_sample_photon_xi");
    return mlp_sample(m, n, chi, r, xi_e, xi_p, use_flags, counters, stream);
}

sfq_status sfq_set_surrogate(sfq_ctx *ctx, sfq_mlp *net, const sfq_event_queue *queue, int32_t use_flags) {
    if (!ctx) return SFQ_ERR_ARG;
    if (!net) {
        ctx->surr = nullptr;
        ctx->surr_q = sfq_event_queue{};
        ctx->surr_flags = 0;
        return SFQ_OK;
    }
    if (ctx->cfg.precision != SFQ_FP32) return fail(ctx, SFQ_ERR_ARG, "the surrogate needs a binary32 context");
    if (net->ctx != ctx) return fail(ctx, SFQ_ERR_ARG, "a surrogate of another context");
    if (net->kind != 0) return fail(ctx, SFQ_ERR_ARG, "a pair-creation surrogate: the step takes the photon one");
    if (use_flags && !net->calibrated) return fail(ctx, SFQ_ERR_ARG, "use_flags before sfq_mlp_calibrate");
    if (ctx->inv_tr > 0) return fail(ctx, SFQ_ERR_ARG, "truncated samplers are set: restore the full coefficients");
    if (!queue || queue->capacity < 0 || !queue->count || ((uintptr_t)queue->count & 7u))
        return fail(ctx, SFQ_ERR_ARG, "queue descriptor, capacity or counter invalid");
    if (queue->capacity > 0) {
        const void *b[8] = {queue->index, queue->chi, queue->r, queue->gamma, queue->px, queue->py, queue->pz, queue->xi};
        for (const void *q : b)
            if (!q || !a16(q)) return fail(ctx, SFQ_ERR_ARG, "queue buffer null or misaligned (16 bytes)");
    }
    DeviceGuard g(ctx->device);
    // kernel attributes and the grid of the surrogate pass, set here (outside any capture)
    cudaError_t e = sfq::prepare_step_surr_f32();
    if (e == cudaSuccess) e = set_infer_attributes(infer_tc_kernel<true>);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sfq_set_surrogate: attributes");
    const int per_sm = INFER_MINB;
    ctx->surr = net;
    ctx->surr_q = *queue;
    ctx->surr_flags = use_flags ? 1 : 0;
    ctx->surr_per_sm = per_sm;
    return SFQ_OK;
}

}  // extern "C"
