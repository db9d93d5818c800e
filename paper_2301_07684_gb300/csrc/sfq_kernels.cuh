// sfq_kernels.cuh -- the Monte Carlo step and the batched rate / sampling kernels.
//
// One template serves both precisions: T = float is the mixed path (binary32
// arithmetic, binary64 optical depth updated on the integer pipe), T = double
// the plain binary64 path.  Equations are those of Montefiori & Tamburini,
// "SFQEDtoolkit" (arXiv:2301.07684).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "sfq.h"
#include "sfq_device.cuh"

namespace sfq {

// ---------------------------------------------------------------------------
// Table layouts per precision (from the generated sfq_tables.inc).
template <typename T> struct L;
#define SFQ_LAYOUT(T, P)                                                                          \
    template <> struct L<T> {                                                                     \
        static constexpr int RATE_NLC_N = NLC_RATE_##P##_COUNT, RATE_NBW_N = NBW_RATE_##P##_COUNT; \
        static constexpr int NLC_DEG = NLC_RATE_##P##_DEG, NBW_DEG = NBW_RATE_##P##_DEG;          \
        static constexpr int NLC_ELO = NLC_RATE_##P##_X_ELO, NLC_EHI = NLC_RATE_##P##_X_EHI,      \
                             NLC_SUB = NLC_RATE_##P##_X_SUB, NLC_LOW = NLC_RATE_##P##_X_LOW,      \
                             NLC_SUBLOW = NLC_RATE_##P##_X_SUBLOW;                                 \
        static constexpr int NBW_ELO = NBW_RATE_##P##_X_ELO, NBW_EHI = NBW_RATE_##P##_X_EHI,      \
                             NBW_SUB = NBW_RATE_##P##_X_SUB, NBW_LOW = NBW_RATE_##P##_X_LOW,      \
                             NBW_SUBLOW = NBW_RATE_##P##_X_SUBLOW;                                 \
        static constexpr int PI_DX = NLC_INV_##P##_DX, PI_DY = NLC_INV_##P##_DY;                  \
        static constexpr int PI_XELO = NLC_INV_##P##_X_ELO, PI_XEHI = NLC_INV_##P##_X_EHI,        \
                             PI_XSUB = NLC_INV_##P##_X_SUB, PI_XLOW = NLC_INV_##P##_X_LOW,        \
                             PI_XSUBLOW = NLC_INV_##P##_X_SUBLOW;                                  \
        static constexpr int PI_YE0 = NLC_INV_##P##_Y_ELO, PI_YSUB = NLC_INV_##P##_Y_SUB,         \
                             PI_YSUBLOW = NLC_INV_##P##_Y_SUBLOW, PI_YQLO = NLC_INV_##P##_Y_QLO,  \
                             PI_YSUBQ = NLC_INV_##P##_Y_SUBQ, PI_NY = NLC_INV_##P##_Y_NPIECES;    \
        static constexpr int PP_DX = NBW_INV_##P##_DX, PP_DY = NBW_INV_##P##_DY;                  \
        static constexpr int PP_XELO = NBW_INV_##P##_X_ELO, PP_XEHI = NBW_INV_##P##_X_EHI,        \
                             PP_XSUB = NBW_INV_##P##_X_SUB, PP_XLOW = NBW_INV_##P##_X_LOW,        \
                             PP_XSUBLOW = NBW_INV_##P##_X_SUBLOW;                                  \
        static constexpr int PP_YE0 = NBW_INV_##P##_Y_ELO, PP_YSUB = NBW_INV_##P##_Y_SUB,         \
                             PP_YSUBLOW = NBW_INV_##P##_Y_SUBLOW, PP_YQLO = NBW_INV_##P##_Y_QLO,  \
                             PP_YSUBQ = NBW_INV_##P##_Y_SUBQ, PP_NY = NBW_INV_##P##_Y_NPIECES;    \
        static constexpr int K23_DEG = K23_##P##_DEG, K23_ELO = K23_##P##_X_ELO, K23_EHI = K23_##P##_X_EHI, \
                             K23_SUB = K23_##P##_X_SUB;                                            \
        static constexpr int KI13_DEG = KI13_##P##_DEG, KI13_ELO = KI13_##P##_X_ELO,             \
                             KI13_EHI = KI13_##P##_X_EHI, KI13_SUB = KI13_##P##_X_SUB;            \
    };
SFQ_LAYOUT(float, F32)
SFQ_LAYOUT(double, F64)
#undef SFQ_LAYOUT

template <typename T>
struct Tables {
    const T *nlc_rate, *nbw_rate, *nlc_inv, *nbw_inv, *k23, *ki13;
    // inverse-CDF tables truncated to (n - tr) x (n - tr) coefficients per piece (tr = 1 or 2),
    // used by the samplers when tr > 0 (the coefficient-count knob of Sec. 4.5)
    const T *nlc_inv_r, *nbw_inv_r;
    int tr;
};

// Rate tables in shared memory: each piece padded to a multiple of 16 bytes so that
// its coefficients are read with vector loads.
template <typename T, int DEG>
struct Padded {
    static constexpr int V = 16 / (int)sizeof(T);
    static constexpr int STRIDE = ((DEG + 1) + V - 1) / V * V;
};
template <typename T>
struct RateSmem {
    using Q = L<T>;
    static constexpr int NLC_STRIDE = Padded<T, Q::NLC_DEG>::STRIDE;
    static constexpr int NBW_STRIDE = Padded<T, Q::NBW_DEG>::STRIDE;
    static constexpr int NLC_N = Q::RATE_NLC_N / (Q::NLC_DEG + 1) * NLC_STRIDE;
    static constexpr int NBW_N = Q::RATE_NBW_N / (Q::NBW_DEG + 1) * NBW_STRIDE;
};
// Copy a rate table into padded shared memory (all threads of the block take part).
template <typename T, int DEG, int STRIDE>
__device__ __forceinline__ void stage_rate_table(T *dst, const T *src, int npieces, int tid, int nthreads) {
    for (int k = tid; k < npieces * STRIDE; k += nthreads) {
        const int p = k / STRIDE, c = k - p * STRIDE;
        dst[k] = c <= DEG ? src[p * (DEG + 1) + c] : (T)0;
    }
}
template <int DEG, int STRIDE>
__device__ __forceinline__ float horner_smem(const float *c, float x) {
    float co[STRIDE];
#pragma unroll
    for (int k = 0; k < STRIDE / 4; ++k) {
        const float4 v = reinterpret_cast<const float4 *>(c)[k];
        co[4 * k] = v.x; co[4 * k + 1] = v.y; co[4 * k + 2] = v.z; co[4 * k + 3] = v.w;
    }
    float acc = co[DEG];
#pragma unroll
    for (int k = DEG - 1; k >= 0; --k) acc = fmaf(acc, x, co[k]);
    return acc;
}
template <int DEG, int STRIDE>
__device__ __forceinline__ double horner_smem(const double *c, double x) {
    double co[STRIDE];
#pragma unroll
    for (int k = 0; k < STRIDE / 2; ++k) {
        const double2 v = reinterpret_cast<const double2 *>(c)[k];
        co[2 * k] = v.x; co[2 * k + 1] = v.y;
    }
    double acc = co[DEG];
#pragma unroll
    for (int k = DEG - 1; k >= 0; --k) acc = fma(acc, x, co[k]);
    return acc;
}

// Clenshaw's recurrence for sum_a c_a T_a(x), the Chebyshev series of a piece on [-1, 1]:
// b_a = c_a + 2x b_(a+1) - b_(a+2) from a = DEG down to 1, then c_0 + x b_1 - b_2.  The
// comparison evaluator of the tables in the Chebyshev basis (two operations per
// coefficient against Horner's one on the same piece in the monomial basis).
template <int DEG, int STRIDE, typename T>
__device__ __forceinline__ T clenshaw_smem(const T *c, T x) {
    T co[STRIDE];
#pragma unroll
    for (int k = 0; k < STRIDE; ++k) co[k] = c[k];
    const T x2 = x + x;
    T b1 = (T)0, b2 = (T)0;
#pragma unroll
    for (int a = DEG; a >= 1; --a) {
        const T b0 = fma(x2, b1, co[a] - b2);
        b2 = b1;
        b1 = b0;
    }
    return fma(x, b1, co[0] - b2);
}

// ---------------------------------------------------------------------------
// Fitted functions.  CH = true evaluates tables that hold every piece in the Chebyshev
// basis by Clenshaw's recurrence (the comparison evaluator); the default is Horner on the
// monomial pieces.
// W~_rad(chi) (Eq. wtilde); `c` is the rate table (shared memory in the step kernel).
template <typename T, bool CH = false>
__device__ __forceinline__ T wtilde_rad(const T *c, T chi, bool &oor) {
    using Q = L<T>;
    constexpr int ST = RateSmem<T>::NLC_STRIDE;
    T x;
    const int p = octave_piece<T, Q::NLC_ELO, Q::NLC_EHI, Q::NLC_SUB, Q::NLC_LOW, Q::NLC_SUBLOW>(chi, x, oor);
    if (CH) return clenshaw_smem<Q::NLC_DEG, ST>(c + p * ST, x);
    return horner_smem<Q::NLC_DEG, ST>(c + p * ST, x);
}

// exp(-8/(3 chi)): binary32 with the argument carried to ~2^-48 (the argument
// reaches 267 at chi = 0.01, where one rounding of it would cost ~1.6e-5).
__device__ __forceinline__ float exp_m83(float chi) {
    const float hi = 2.66666674613952636719f;                  // binary32(8/3)
    const float lo = -7.94728632e-08f;                         // 8/3 - hi
    const float t = hi / chi;
    const float rem = fmaf(-t, chi, hi) + lo;                  // hi + lo - t chi (exact fma)
    const float tl = rem / chi;
    return expf(-t) * (1.0f - tl);
}
__device__ __forceinline__ double exp_m83(double chi) { return exp(-(8.0 / 3.0) / chi); }

// W~_pair(chi) = chi h(chi) exp(-8/(3 chi)) (Eq. wtilde_pair); zero below chi_min, which is
// 0.01, the lower end of the fitted domain (Sec. 4.2), or larger for the "fast" rate that
// neglects pair creation below e.g. chi = 0.3 (Sec. 4.2).
template <typename T, bool CH = false>
__device__ __forceinline__ T wtilde_pair(const T *c, T chi, bool &oor, T chi_min = (T)0.01) {
    using Q = L<T>;
    if (!(chi >= chi_min)) return (T)0;
    T x;
    constexpr int ST = RateSmem<T>::NBW_STRIDE;
    const int p = octave_piece<T, Q::NBW_ELO, Q::NBW_EHI, Q::NBW_SUB, Q::NBW_LOW, Q::NBW_SUBLOW>(chi, x, oor);
    const T h = CH ? clenshaw_smem<Q::NBW_DEG, ST>(c + p * ST, x) : horner_smem<Q::NBW_DEG, ST>(c + p * ST, x);
    return chi * h * exp_m83(chi);
}

// s = 3 chi w^3 / 2 for w-bar = G~_pe(r, chi) (Eq. again, Eq. subs_altri).  TR > 0 reads the
// table truncated by TR degrees in each variable.
template <typename T, int TR = 0, bool CH = false>
__device__ __forceinline__ T photon_s(const T *__restrict__ inv, T chi, T r, bool &oor) {
    using Q = L<T>;
    constexpr int DX = Q::PI_DX - TR, DY = Q::PI_DY - TR;
    T xc, xr;
    bool low;
    const int ic = octave_piece<T, Q::PI_XELO, Q::PI_XEHI, Q::PI_XSUB, Q::PI_XLOW, Q::PI_XSUBLOW>(chi, xc, oor);
    const int ir = prob_piece<T, Q::PI_YE0, Q::PI_YSUB, Q::PI_YSUBLOW, Q::PI_YQLO, Q::PI_YSUBQ>(r, xr, low, oor);
    const T *c = inv + ((size_t)ic * Q::PI_NY + ir) * ((DX + 1) * padded_row(DY + 1, sizeof(T)));
    T w = CH ? clenshaw2<DX, DY>(c, xc, xr) : horner2<DX, DY>(c, xc, xr);
    if (low) w *= r;                          // the low-r block holds w-bar / r
    const T chi_eff = chi > (T)4096 ? (T)4096 : chi;
    return (T)1.5 * chi_eff * w * w * w;
}

// Electron and positron shares for r (Eq. again_pp, Eq. return_to_nrg): the table
// holds y = 1 - v-bar as a function of (chi, |r'|).
// y = 1 - v-bar at a = |r'| (Eq. again_pp): the table's value.
template <typename T, int TR = 0, bool CH = false>
__device__ __forceinline__ T pair_y(const T *__restrict__ inv, T chi, T a, bool &oor) {
    using Q = L<T>;
    constexpr int DX = Q::PP_DX - TR, DY = Q::PP_DY - TR;
    T xc, xr;
    bool low;
    const int ic = octave_piece<T, Q::PP_XELO, Q::PP_XEHI, Q::PP_XSUB, Q::PP_XLOW, Q::PP_XSUBLOW>(chi, xc, oor);
    const int ir = prob_piece<T, Q::PP_YE0, Q::PP_YSUB, Q::PP_YSUBLOW, Q::PP_YQLO, Q::PP_YSUBQ>(a, xr, low, oor);
    const T *c = inv + ((size_t)ic * Q::PP_NY + ir) * ((DX + 1) * padded_row(DY + 1, sizeof(T)));
    return CH ? clenshaw2<DX, DY>(c, xc, xr) : horner2<DX, DY>(c, xc, xr);
}

template <typename T, int TR = 0, bool CH = false>
__device__ __forceinline__ void pair_shares(const T *__restrict__ inv, T chi, T r, T &xe, T &xp, bool &oor) {
    const T rp = (T)2 * r - (T)1;
    const T y = pair_y<T, TR, CH>(inv, chi, fabs(rp), oor);
    const T small = (T)0.5 * y, big = (T)1 - small;
    if (rp >= (T)0) { xe = big; xp = small; }
    else { xe = small; xp = big; }
}

// The samplers with the coefficient count compiled into the kernel.  TRUNC = false reads the
// full tables.  TRUNC = true reads the tables truncated by t.tr = 1 or 2 degrees in each
// variable.  Kernels are instantiated with TRUNC = true only for contexts that use the
// knob, so the default kernels carry no code for it.
template <typename T, bool TRUNC>
__device__ __forceinline__ T photon_s_sel(const Tables<T> &t, T chi, T r, bool &oor) {
    if (TRUNC) {
        if (t.tr == 2) return photon_s<T, 2>(t.nlc_inv_r, chi, r, oor);
        return photon_s<T, 1>(t.nlc_inv_r, chi, r, oor);
    }
    return photon_s<T, 0>(t.nlc_inv, chi, r, oor);
}
template <typename T, bool TRUNC>
__device__ __forceinline__ void pair_shares_sel(const Tables<T> &t, T chi, T r, T &xe, T &xp, bool &oor) {
    if (TRUNC) {
        if (t.tr == 2) pair_shares<T, 2>(t.nbw_inv_r, chi, r, xe, xp, oor);
        else pair_shares<T, 1>(t.nbw_inv_r, chi, r, xe, xp, oor);
        return;
    }
    pair_shares<T, 0>(t.nbw_inv, chi, r, xe, xp, oor);
}

// ln of the photon spectrum Eq. pe_dp at u = eps_gamma/(eps_e - eps_gamma), without the
// factor common to both sides of Eq. rej_cond:
//   S(u) = ((1 + (1+u)^2)/(1+u)) K_2/3(x) - Ki_1/3(x),  x = 2u/(3 chi),
// with K_2/3(x) = g1(x) x^{-2/3} e^{-x} and Ki_1/3(x) = g2(x) e^{-x} from the fitted g1, g2.
__device__ __forceinline__ float pow_m23(float x) { return exp2f(-0.666666686534881591796875f * log2f(x)); }
__device__ __forceinline__ double pow_m23(double x) { return exp2(-(2.0 / 3.0) * log2(x)); }
template <typename T>
__device__ __forceinline__ T ln_spectrum(const T *__restrict__ k23, const T *__restrict__ ki13, T u, T chi,
                                         bool &oor) {
    using Q = L<T>;
    const T x = (T)2 * u / ((T)3 * chi);
    T xl;
    int p = octave_piece<T, Q::K23_ELO, Q::K23_EHI, Q::K23_SUB, 0, 0>(x, xl, oor);
    T c1[Q::K23_DEG + 1];
#pragma unroll
    for (int k = 0; k <= Q::K23_DEG; ++k) c1[k] = __ldg(k23 + p * (Q::K23_DEG + 1) + k);
    const T g1 = horner1<Q::K23_DEG>(c1, xl);
    p = octave_piece<T, Q::KI13_ELO, Q::KI13_EHI, Q::KI13_SUB, 0, 0>(x, xl, oor);
    T c2[Q::KI13_DEG + 1];
#pragma unroll
    for (int k = 0; k <= Q::KI13_DEG; ++k) c2[k] = __ldg(ki13 + p * (Q::KI13_DEG + 1) + k);
    const T g2 = horner1<Q::KI13_DEG>(c2, xl);
    const T opu = (T)1 + u;
    const T g = ((T)1 + opu * opu) / opu * g1 * pow_m23(x) - g2;
    return log(g) - x;
}

// ---------------------------------------------------------------------------
// Boris push of a momentum (Boris 1970) in the normalised units of the step:
// du/dt = q (E + u x B / gamma), q in units of |e|.
//   u- = u + q E dt/2;  t = q B dt / (2 gamma(u-));  s = 2 t / (1 + t.t);
//   u' = u- + u- x t;  u+ = u- + u' x s;  u_new = u+ + q E dt/2.
template <typename T>
__device__ __forceinline__ void boris(T u[3], const T E[3], const T B[3], T q, T dt) {
    const T h = (T)0.5 * q * dt;
    T um[3], t[3], s[3], up[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) um[k] = fma(h, E[k], u[k]);
    const T gm = sqrt(fma(um[0], um[0], fma(um[1], um[1], fma(um[2], um[2], (T)1))));
    const T hg = h / gm;
#pragma unroll
    for (int k = 0; k < 3; ++k) t[k] = hg * B[k];
    const T f = (T)2 / fma(t[0], t[0], fma(t[1], t[1], fma(t[2], t[2], (T)1)));
#pragma unroll
    for (int k = 0; k < 3; ++k) s[k] = f * t[k];
    const T c0 = um[1] * t[2] - um[2] * t[1], c1 = um[2] * t[0] - um[0] * t[2], c2 = um[0] * t[1] - um[1] * t[0];
    const T v0 = um[0] + c0, v1 = um[1] + c1, v2 = um[2] + c2;
    up[0] = um[0] + (v1 * s[2] - v2 * s[1]);
    up[1] = um[1] + (v2 * s[0] - v0 * s[2]);
    up[2] = um[2] + (v0 * s[1] - v1 * s[0]);
#pragma unroll
    for (int k = 0; k < 3; ++k) u[k] = fma(h, E[k], up[k]);
}

// ---------------------------------------------------------------------------
// Counters: per-thread registers, reduced per block, one atomic per counter.
struct Cnt {
    uint32_t v[13];     // per-thread counts of one launch (fit in 32 bits); widened when flushed
    __device__ void zero() {
#pragma unroll
        for (int k = 0; k < 13; ++k) v[k] = 0;
    }
};
// v[k] goes to word k of sfq_counters for k < 12; C_SURR (surrogate fallbacks) to word 13
enum { C_UPD, C_EV, C_EMIT, C_PAIR, C_DROP, C_SDROP, C_OOR, C_NAN, C_G1, C_RDT, C_NOEM, C_REJ, C_SURR };

__device__ __forceinline__ void flush_counters(Cnt &c, sfq_counters *out) {
    if (!out) return;
    __shared__ unsigned long long red[13];
    if (threadIdx.x < 13) red[threadIdx.x] = 0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 13; ++k) {
        unsigned long long s = (unsigned long long)c.v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
        if ((threadIdx.x & 31) == 0 && s) atomicAdd(&red[k], s);
    }
    __syncthreads();
    if (threadIdx.x < 13 && red[threadIdx.x])
        atomicAdd(reinterpret_cast<unsigned long long *>(out) + (threadIdx.x < 12 ? threadIdx.x : 13),
                  red[threadIdx.x]);
}

// ---------------------------------------------------------------------------
// Batched rate kernels (App. A functions 5, 6).
// CH: the tables hold Chebyshev pieces, evaluated by Clenshaw's recurrence.
template <typename T, bool PAIR, bool CH = false>
__global__ void __launch_bounds__(256) rate_kernel(int64_t n, const T *__restrict__ gamma,
                                                   const T *__restrict__ chi, T *__restrict__ rate,
                                                   const T *__restrict__ table, T pref,
                                                   sfq_counters *counters, T pair_chi_min) {
    using RS = RateSmem<T>;
    constexpr int N = PAIR ? RS::NBW_N : RS::NLC_N;
    __shared__ __align__(16) T tab[N];
    if (PAIR)
        stage_rate_table<T, L<T>::NBW_DEG, RS::NBW_STRIDE>(tab, table, L<T>::RATE_NBW_N / (L<T>::NBW_DEG + 1),
                                                            threadIdx.x, blockDim.x);
    else
        stage_rate_table<T, L<T>::NLC_DEG, RS::NLC_STRIDE>(tab, table, L<T>::RATE_NLC_N / (L<T>::NLC_DEG + 1),
                                                            threadIdx.x, blockDim.x);
    __syncthreads();
    Cnt c;
    c.zero();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const T g = gamma[i], x = chi[i];
        bool oor = false;
        T r;
        if (!(x >= (T)0) || !(g > (T)0)) {   // NaN or invalid
            ++c.v[C_NAN];
            r = (T)0;
        } else if (PAIR) {
            r = pref * wtilde_pair<T, CH>(tab, x, oor, pair_chi_min) / g;
        } else {
            r = pref * (x / g) * wtilde_rad<T, CH>(tab, x, oor);
        }
        c.v[C_OOR] += oor;
        rate[i] = r;
    }
    flush_counters(c, counters);
}

// Batched samplers (App. A functions 9 and 11, Eqs. again, again_pp).
// CH: tab.nlc_inv / tab.nbw_inv hold Chebyshev pieces, evaluated by Clenshaw's recurrence.
template <typename T, bool PAIR, bool TRUNC, bool CH = false>
__global__ void __launch_bounds__(256) sample_kernel(int64_t n, const T *__restrict__ chi,
                                                     const T *__restrict__ r, T *__restrict__ out_a,
                                                     T *__restrict__ out_b, const Tables<T> tab,
                                                     sfq_counters *counters) {
    Cnt c;
    c.zero();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const T x = chi[i], u = r[i];
        bool oor = false;
        if (!(x >= (T)0) || !(u > (T)0) || !(u < (T)1)) {
            ++c.v[C_NAN];
            out_a[i] = (T)0;
            if (out_b) out_b[i] = (T)0;
            continue;
        }
        if (PAIR) {
            T xe, xp;
            if (CH) pair_shares<T, 0, true>(tab.nbw_inv, x, u, xe, xp, oor);
            else pair_shares_sel<T, TRUNC>(tab, x, u, xe, xp, oor);
            out_a[i] = xe;
            if (out_b) out_b[i] = xp;
        } else {
            const T s = CH ? photon_s<T, 0, true>(tab.nlc_inv, x, u, oor) : photon_s_sel<T, TRUNC>(tab, x, u, oor);
            const T inv1s = (T)1 / ((T)1 + s);
            out_a[i] = s * inv1s;          // xi = s/(1+s)
            if (out_b) out_b[i] = inv1s;   // 1 - xi
        }
        c.v[C_OOR] += oor;
    }
    flush_counters(c, counters);
}

// Philox uniforms (4 per particle).
template <typename T>
__global__ void __launch_bounds__(256) uniforms_kernel(int64_t n, const uint64_t *__restrict__ id, uint32_t step,
                                                       uint32_t tag, uint64_t seed, T *__restrict__ u) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const u4 w = draws(seed, id[i], step, tag);
#pragma unroll
        for (int k = 0; k < 4; ++k) u[4 * i + k] = uniform<T>(w.w[k]);
    }
}

}  // namespace sfq
