// sfq_device.cuh -- device building blocks of the Monte Carlo step.
//
// Philox4x32-10 (Salmon et al., SC'11), the uniform map of the step, exact piece
// selection for the fitted tables (binary exponent + top mantissa bits), Horner
// evaluation, and the exact widening of a binary32 decrement for the binary64 optical
// depth.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "sfq_tables_layout.h"

namespace sfq {

// ---------------------------------------------------------------------------
// Philox4x32-10, keyed by the 64-bit seed; counter (id_lo, id_hi, step, tag).
struct u4 { uint32_t w[4]; };

__device__ __forceinline__ u4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    u4 r;
    r.w[0] = c0; r.w[1] = c1; r.w[2] = c2; r.w[3] = c3;
    return r;
}

__device__ __forceinline__ u4 draws(uint64_t seed, uint64_t id, uint32_t step, uint32_t tag) {
    return philox4x32_10((uint32_t)id, (uint32_t)(id >> 32), step, tag, (uint32_t)seed,
                         (uint32_t)(seed >> 32));
}

// Id of a particle created in a full cascade: bit 63 over the first two words of the
// counter (parent id lo, hi, step, 0x100 | parent tag << 2 | member) under the run's key.
// The counter's last word is outside the 0 ... 3 of the step draws; the set bit keeps
// descendants apart from primaries (ids below 2^63).
__device__ __forceinline__ uint64_t child_id(uint64_t seed, uint64_t parent, uint32_t parent_tag, uint32_t step,
                                             uint32_t member) {
    const u4 w = philox4x32_10((uint32_t)parent, (uint32_t)(parent >> 32), step,
                               0x100u | ((parent_tag & 3u) << 2) | member, (uint32_t)seed, (uint32_t)(seed >> 32));
    return (1ull << 63) | ((uint64_t)(w.w[1] & 0x7FFFFFFFu) << 32) | (uint64_t)w.w[0];
}

// u = (floor(w / 2^9) + 1/2) 2^-23: exact in binary32 and binary64, in [2^-24, 1 - 2^-24].
template <typename T>
__device__ __forceinline__ T uniform(uint32_t w) {
    return ((T)(w >> 9) + (T)0.5) * (T)1.1920928955078125e-07;   // 2^-23
}

// ---------------------------------------------------------------------------
// Floating-point bit access.
template <typename T> struct fp;
template <> struct fp<float> {
    using U = uint32_t;
    static constexpr int MANT = 23, BIAS = 127;
    static __device__ __forceinline__ U bits(float v) { return __float_as_uint(v); }
    static __device__ __forceinline__ float from(U b) { return __uint_as_float(b); }
    static __device__ __forceinline__ int expo(float v) { return (int)(bits(v) >> 23) - 127; }
    static __device__ __forceinline__ float mant(float v) {     // in [1, 2)
        return from((bits(v) & 0x7FFFFFu) | 0x3F800000u);
    }
};
template <> struct fp<double> {
    using U = uint64_t;
    static constexpr int MANT = 52, BIAS = 1023;
    static __device__ __forceinline__ U bits(double v) { return (U)__double_as_longlong(v); }
    static __device__ __forceinline__ double from(U b) { return __longlong_as_double((long long)b); }
    static __device__ __forceinline__ int expo(double v) { return (int)(bits(v) >> 52) - 1023; }
    static __device__ __forceinline__ double mant(double v) {
        return from((bits(v) & 0xFFFFFFFFFFFFFull) | 0x3FF0000000000000ull);
    }
};

// 2^k as a constant of type T (|k| small).
template <typename T>
__host__ __device__ constexpr T pow2(int k) {
    return k >= 0 ? (k == 0 ? (T)1 : (T)2 * pow2<T>(k - 1)) : (T)0.5 * pow2<T>(k + 1);
}

// ---------------------------------------------------------------------------
// Piece selection.  Layouts (written by the table generator):
//   octave axis: [low block of 2^SUBLOW pieces over [0, 2^ELO) if LOW]
//                + octaves [2^e, 2^(e+1)), e in [ELO, EHI), 2^SUB pieces each;
//   prob axis:   low block [0, 2^E0) of 2^SUBLOW pieces
//                + octaves of r in [2^E0, 1/2), 2^SUB each
//                + octaves of q = 1 - r, e = -2 down to QLO, 2^SUBQ each (q = 1/2 closes the first).
// Each returns the piece index and the local variable x in [-1, 1]; all steps are
// exact (scaling by powers of two and Sterbenz subtractions).
// Sub-piece j (top SUB mantissa bits) and local variable x in [-1, 1) of a value with
// mantissa m in [1, 2): x = 2 (frac(2^SUB (m - 1))) - 1, formed from the bits.
template <typename T, int SUB>
__device__ __forceinline__ int mant_split(T v, T &x) {
    using U = typename fp<T>::U;
    constexpr int M = fp<T>::MANT;
    const U b = fp<T>::bits(v);
    const U frac = b & ((((U)1) << M) - 1);
    const int j = SUB ? (int)(frac >> (M - SUB)) : 0;
    const U rest = SUB ? ((frac << SUB) & ((((U)1) << M) - 1)) : frac;
    const T one_plus = fp<T>::from(fp<T>::bits((T)1) | rest);          // 1 + fractional part
    x = (T)2 * one_plus - (T)3;
    return j;
}

template <typename T, int ELO, int EHI, int SUB, int LOW, int SUBLOW>
__device__ __forceinline__ int octave_piece(T v, T &x, bool &oor) {
    constexpr int NLOW = LOW ? (1 << SUBLOW) : 0;
    constexpr int NPIECES = NLOW + (EHI - ELO) * (1 << SUB);
    const int e = fp<T>::expo(v);
    if (e < ELO) {                     // zero, subnormal or below the first octave
        if (LOW) {
            const T t = v * pow2<T>(SUBLOW - ELO);
            int j = SUBLOW ? (int)t : 0;
            j = j > NLOW - 1 ? NLOW - 1 : j;
            x = (T)2 * (t - (T)j) - (T)1;
            return j;
        }
        oor = true;
        x = (T)-1;
        return 0;
    }
    if (e >= EHI) {
        oor = true;
        x = (T)1;
        return NPIECES - 1;
    }
    const int j = mant_split<T, SUB>(v, x);
    return NLOW + (e - ELO) * (1 << SUB) + j;
}

template <typename T, int E0, int SUB, int SUBLOW, int QLO, int SUBQ>
__device__ __forceinline__ int prob_piece(T r, T &x, bool &low, bool &oor) {
    constexpr int NLOW = 1 << SUBLOW;
    constexpr int NROCT = (-1 - E0) * (1 << SUB);
    low = false;
    if (r < (T)0.5) {
        const int e = fp<T>::expo(r);
        if (e < E0) {
            const T t = r * pow2<T>(SUBLOW - E0);
            int j = SUBLOW ? (int)t : 0;
            j = j > NLOW - 1 ? NLOW - 1 : j;
            x = (T)2 * (t - (T)j) - (T)1;
            low = true;
            return j;
        }
        const int j = mant_split<T, SUB>(r, x);
        return NLOW + (e - E0) * (1 << SUB) + j;
    }
    const T q = (T)1 - r;              // exact for r >= 1/2
    int e = fp<T>::expo(q);
    int j;
    if (e >= -1) {                     // q = 1/2: right end of the first q-octave
        e = -2;
        j = (1 << SUBQ) - 1;
        x = (T)1;
    } else if (e < QLO) {              // beyond the fitted tail (binary64 inputs only)
        oor = true;
        e = QLO;
        j = 0;
        x = (T)-1;
    } else {
        j = mant_split<T, SUBQ>(q, x);
    }
    return NLOW + NROCT + (-2 - e) * (1 << SUBQ) + j;
}

// ---------------------------------------------------------------------------
// Horner evaluation of the monomial pieces.
template <int DEG, typename T>
__device__ __forceinline__ T horner1(const T *c, T x) {
    T acc = c[DEG];
#pragma unroll
    for (int k = DEG - 1; k >= 0; --k) acc = fma(acc, x, c[k]);
    return acc;
}

// Row length, in elements, of a 2-D table piece whose rows of n coefficients are padded
// to a multiple of 16 bytes (so that a row is read with vector loads).
__host__ __device__ constexpr int padded_row(int n, int esz) { return (n * esz + 15) / 16 * 16 / esz; }

// Vector load of V = 16/sizeof(T) consecutive coefficients through the read-only cache.
__device__ __forceinline__ void ldg_vec(const float *p, float *d) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
}
__device__ __forceinline__ void ldg_vec(const double *p, double *d) {
    const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
    d[0] = v.x; d[1] = v.y;
}

// sum_ij c[i*ROW+j] x^i y^j, i <= DX, j <= DY: Horner in y for each row i, then in x.
// Rows are ROW = padded_row(DY + 1) elements apart (16-byte aligned) and each is read
// with ROW / V vector loads.
template <int DX, int DY, typename T>
__device__ __forceinline__ T horner2(const T *__restrict__ c, T x, T y) {
    constexpr int ROW = padded_row(DY + 1, (int)sizeof(T));
    constexpr int V = 16 / (int)sizeof(T);
    T acc = (T)0;
#pragma unroll
    for (int i = DX; i >= 0; --i) {
        T co[ROW];
#pragma unroll
        for (int k = 0; k < ROW / V; ++k) ldg_vec(c + i * ROW + k * V, co + k * V);
        T b = co[DY];
#pragma unroll
        for (int j = DY - 1; j >= 0; --j) b = fma(b, y, co[j]);
        acc = (i == DX) ? b : fma(acc, x, b);
    }
    return acc;
}

// sum_ab c[a*ROW+b] T_a(x) T_b(y), a <= DX, b <= DY (Chebyshev pieces): Clenshaw's
// recurrence in y for each row a, then in x over the rows' values.  Same row layout as
// horner2.
template <int DX, int DY, typename T>
__device__ __forceinline__ T clenshaw2(const T *__restrict__ c, T x, T y) {
    constexpr int ROW = padded_row(DY + 1, (int)sizeof(T));
    constexpr int V = 16 / (int)sizeof(T);
    const T x2 = x + x, y2 = y + y;
    T ob1 = (T)0, ob2 = (T)0;                 // the recurrence in x
#pragma unroll
    for (int a = DX; a >= 0; --a) {
        T co[ROW];
#pragma unroll
        for (int k = 0; k < ROW / V; ++k) ldg_vec(c + a * ROW + k * V, co + k * V);
        T b1 = (T)0, b2 = (T)0;
#pragma unroll
        for (int b = DY; b >= 1; --b) {
            const T b0 = fma(y2, b1, co[b] - b2);
            b2 = b1;
            b1 = b0;
        }
        const T ra = fma(y, b1, co[0] - b2);     // the row's series at y
        if (a >= 1) {
            const T o0 = fma(x2, ob1, ra - ob2);
            ob2 = ob1;
            ob1 = o0;
        } else {
            return fma(x, ob1, ra - ob2);
        }
    }
    return (T)0;
}

// ---------------------------------------------------------------------------
// Square root and reciprocal square root from the hardware estimate plus one Newton
// step (about 1 ulp in binary32; the binary64 versions use the library functions).
__device__ __forceinline__ float sqrt_nr(float q) {
    if (!(q > 0.0f)) return 0.0f;
    const float r = rsqrtf(q);
    const float s = q * r;
    return fmaf(0.5f * r, fmaf(-s, s, q), s);
}
__device__ __forceinline__ double sqrt_nr(double q) { return q > 0.0 ? sqrt(q) : 0.0; }
__device__ __forceinline__ float rsqrt_nr(float q) {
    const float r = rsqrtf(q);
    return fmaf(0.5f * r, fmaf(-q * r, r, 1.0f), r);
}
__device__ __forceinline__ double rsqrt_nr(double q) { return rsqrt(q); }

// ---------------------------------------------------------------------------
// binary32 -> binary64 bits for a finite positive normal value (exact), on 32-bit halves:
// the high word is the binary32 pattern shifted right by 3 with the exponent rebiased by
// 1023 - 127 = 896; the low word holds the last 3 mantissa bits.
__device__ __forceinline__ uint64_t f32_to_f64_bits(float v) {
    const uint32_t b = __float_as_uint(v);
    const uint32_t hi = (b >> 3) + (896u << 20);
    const uint32_t lo = b << 29;
    return ((uint64_t)hi << 32) | lo;
}

}  // namespace sfq
