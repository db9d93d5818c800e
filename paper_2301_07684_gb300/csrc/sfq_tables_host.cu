// Host copies of the fitted tables (generated by fitgen/generate.py), uploaded to the
// device by sfq_init.
#include <cstring>
#include <vector>

#include "sfq_internal.h"
#include "sfq_tables_layout.h"
#include "sfq_tables.inc"

namespace sfq {
HostTables host_tables(int precision) {
    HostTables t;
    if (precision == SFQ_FP64) {
        t.nlc_rate = nlc_rate_f64; t.nlc_rate_bytes = sizeof(nlc_rate_f64);
        t.nbw_rate = nbw_rate_f64; t.nbw_rate_bytes = sizeof(nbw_rate_f64);
        t.nlc_inv = nlc_inv_f64; t.nlc_inv_bytes = sizeof(nlc_inv_f64);
        t.nbw_inv = nbw_inv_f64; t.nbw_inv_bytes = sizeof(nbw_inv_f64);
        t.k23 = k23_f64; t.k23_bytes = sizeof(k23_f64);
        t.ki13 = ki13_f64; t.ki13_bytes = sizeof(ki13_f64);
    } else {
        t.nlc_rate = nlc_rate_f32; t.nlc_rate_bytes = sizeof(nlc_rate_f32);
        t.nbw_rate = nbw_rate_f32; t.nbw_rate_bytes = sizeof(nbw_rate_f32);
        t.nlc_inv = nlc_inv_f32; t.nlc_inv_bytes = sizeof(nlc_inv_f32);
        t.nbw_inv = nbw_inv_f32; t.nbw_inv_bytes = sizeof(nbw_inv_f32);
        t.k23 = k23_f32; t.k23_bytes = sizeof(k23_f32);
        t.ki13 = ki13_f32; t.ki13_bytes = sizeof(ki13_f32);
    }
    return t;
}

int inv_coefficients(int precision) {
    static_assert(NLC_INV_F32_DX == NLC_INV_F32_DY && NBW_INV_F32_DX == NLC_INV_F32_DX &&
                      NBW_INV_F32_DY == NLC_INV_F32_DY, "square binary32 inverse-CDF pieces");
    static_assert(NLC_INV_F64_DX == NLC_INV_F64_DY && NBW_INV_F64_DX == NLC_INV_F64_DX &&
                      NBW_INV_F64_DY == NLC_INV_F64_DY, "square binary64 inverse-CDF pieces");
    return precision == SFQ_FP64 ? NLC_INV_F64_DX + 1 : NLC_INV_F32_DX + 1;
}

namespace {

// Monomial <-> Chebyshev bases of degree < n on [-1, 1] (row-major n x n):
//   c2m[a n + k]: coefficient of x^k in T_a (T_0 = 1, T_1 = x, T_{a+1} = 2x T_a - T_{a-1});
//   m2c[k n + a]: coefficient of T_a in x^k (x T_0 = T_1, x T_a = (T_{a+1} + T_{a-1})/2).
void cheb_bases(int n, std::vector<double> &c2m, std::vector<double> &m2c) {
    c2m.assign((size_t)n * n, 0.0);
    m2c.assign((size_t)n * n, 0.0);
    c2m[0] = 1.0;
    if (n > 1) c2m[n + 1] = 1.0;
    for (int a = 1; a + 1 < n; ++a)
        for (int k = 0; k < n; ++k)
            c2m[(a + 1) * n + k] = (k > 0 ? 2.0 * c2m[a * n + k - 1] : 0.0) - c2m[(a - 1) * n + k];
    m2c[0] = 1.0;
    for (int k = 0; k + 1 < n; ++k)
        for (int a = 0; a < n; ++a) {
            const double v = m2c[k * n + a];
            if (v == 0.0) continue;
            if (a == 0) {
                m2c[(k + 1) * n + 1] += v;
            } else {
                if (a + 1 < n) m2c[(k + 1) * n + a + 1] += 0.5 * v;
                m2c[(k + 1) * n + a - 1] += 0.5 * v;
            }
        }
}

// Every 1-D piece (n monomial coefficients) in the Chebyshev basis, same layout.
template <typename T>
std::vector<unsigned char> cheb_pieces_1d(const T *src, size_t count, int n) {
    std::vector<double> c2m, m2c;
    cheb_bases(n, c2m, m2c);
    std::vector<unsigned char> out(count * sizeof(T), 0);
    T *dst = reinterpret_cast<T *>(out.data());
    for (size_t p = 0; p < count / (size_t)n; ++p)
        for (int a = 0; a < n; ++a) {
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc += m2c[k * n + a] * (double)src[p * n + k];
            dst[p * n + a] = (T)acc;
        }
    return out;
}

// Every 2-D piece (n x n monomial coefficients x^i y^j) in the tensor Chebyshev basis
// T_a(x) T_b(y), rows padded to 16 bytes as on the device.
template <typename T>
std::vector<unsigned char> cheb_pieces_2d(const T *src, size_t count, int n) {
    const int row = (n * (int)sizeof(T) + 15) / 16 * 16 / (int)sizeof(T);
    const size_t pieces = count / ((size_t)n * n);
    std::vector<double> c2m, m2c;
    cheb_bases(n, c2m, m2c);
    std::vector<unsigned char> out(pieces * (size_t)n * row * sizeof(T), 0);
    T *dst = reinterpret_cast<T *>(out.data());
    std::vector<double> Q((size_t)n * n);
    for (size_t p = 0; p < pieces; ++p) {
        const T *P = src + p * (size_t)n * n;
        for (int a = 0; a < n; ++a)
            for (int j = 0; j < n; ++j) {
                double acc = 0.0;
                for (int i = 0; i < n; ++i) acc += m2c[i * n + a] * (double)P[i * n + j];
                Q[a * n + j] = acc;
            }
        T *D = dst + p * (size_t)n * row;
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) {
                double acc = 0.0;
                for (int j = 0; j < n; ++j) acc += Q[a * n + j] * m2c[j * n + b];
                D[a * row + b] = (T)acc;
            }
    }
    return out;
}

template <typename T>
std::vector<unsigned char> truncate_pieces(const T *src, size_t count, int n, int tr) {
    const int m = n - tr;                                   // kept coefficients per variable
    const int row = (m * (int)sizeof(T) + 15) / 16 * 16 / (int)sizeof(T);
    const size_t pieces = count / ((size_t)n * n);
    std::vector<double> c2m, m2c;
    cheb_bases(n, c2m, m2c);
    std::vector<unsigned char> out(pieces * (size_t)m * row * sizeof(T), 0);
    T *dst = reinterpret_cast<T *>(out.data());
    std::vector<double> C((size_t)n * n), Q((size_t)n * n);
    for (size_t p = 0; p < pieces; ++p) {
        const T *P = src + p * (size_t)n * n;               // P[i n + j]: x^i y^j
        // C = M P M^T in the Chebyshev basis, M[a][i] = m2c[i][a]
        for (int a = 0; a < n; ++a)
            for (int j = 0; j < n; ++j) {
                double acc = 0.0;
                for (int i = 0; i < n; ++i) acc += m2c[i * n + a] * (double)P[i * n + j];
                Q[a * n + j] = acc;
            }
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) {
                double acc = 0.0;
                for (int j = 0; j < n; ++j) acc += Q[a * n + j] * m2c[j * n + b];
                C[a * n + b] = acc;
            }
        // keep T_a(x) T_b(y) with a, b < m and return to monomials: P' = N C' N^T, N[i][a] = c2m[a][i]
        for (int i = 0; i < m; ++i)
            for (int b = 0; b < m; ++b) {
                double acc = 0.0;
                for (int a = 0; a < m; ++a) acc += c2m[a * n + i] * C[a * n + b];
                Q[i * n + b] = acc;
            }
        T *D = dst + p * (size_t)m * row;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                double acc = 0.0;
                for (int b = 0; b < m; ++b) acc += Q[i * n + b] * c2m[b * n + j];
                D[i * row + j] = (T)acc;
            }
    }
    return out;
}

}  // namespace

std::vector<unsigned char> truncated_inv_table(int precision, bool pair, int tr) {
    const int n = inv_coefficients(precision);
    if (precision == SFQ_FP64)
        return pair ? truncate_pieces(nbw_inv_f64, sizeof(nbw_inv_f64) / sizeof(double), n, tr)
                    : truncate_pieces(nlc_inv_f64, sizeof(nlc_inv_f64) / sizeof(double), n, tr);
    return pair ? truncate_pieces(nbw_inv_f32, sizeof(nbw_inv_f32) / sizeof(float), n, tr)
                : truncate_pieces(nlc_inv_f32, sizeof(nlc_inv_f32) / sizeof(float), n, tr);
}

std::vector<unsigned char> chebyshev_rate_table(int precision, bool pair) {
    if (precision == SFQ_FP64)
        return pair ? cheb_pieces_1d(nbw_rate_f64, sizeof(nbw_rate_f64) / sizeof(double), NBW_RATE_F64_DEG + 1)
                    : cheb_pieces_1d(nlc_rate_f64, sizeof(nlc_rate_f64) / sizeof(double), NLC_RATE_F64_DEG + 1);
    return pair ? cheb_pieces_1d(nbw_rate_f32, sizeof(nbw_rate_f32) / sizeof(float), NBW_RATE_F32_DEG + 1)
                : cheb_pieces_1d(nlc_rate_f32, sizeof(nlc_rate_f32) / sizeof(float), NLC_RATE_F32_DEG + 1);
}

std::vector<unsigned char> chebyshev_inv_table(int precision, bool pair) {
    const int n = inv_coefficients(precision);
    if (precision == SFQ_FP64)
        return pair ? cheb_pieces_2d(nbw_inv_f64, sizeof(nbw_inv_f64) / sizeof(double), n)
                    : cheb_pieces_2d(nlc_inv_f64, sizeof(nlc_inv_f64) / sizeof(double), n);
    return pair ? cheb_pieces_2d(nbw_inv_f32, sizeof(nbw_inv_f32) / sizeof(float), n)
                : cheb_pieces_2d(nlc_inv_f32, sizeof(nlc_inv_f32) / sizeof(float), n);
}

std::vector<unsigned char> monomial_table(int precision, int which) {
    const HostTables t = host_tables(precision);
    const void *src[4] = {t.nlc_rate, t.nbw_rate, t.nlc_inv, t.nbw_inv};
    const size_t bytes[4] = {t.nlc_rate_bytes, t.nbw_rate_bytes, t.nlc_inv_bytes, t.nbw_inv_bytes};
    const unsigned char *b = static_cast<const unsigned char *>(src[which]);
    if (which < 2) return std::vector<unsigned char>(b, b + bytes[which]);
    // inverse-CDF pieces: rows padded to 16 bytes, as on the device
    const size_t esz = precision == SFQ_FP64 ? 8 : 4;
    const size_t n = (size_t)inv_coefficients(precision), rb = n * esz, pb = (rb + 15) / 16 * 16;
    const size_t rows = bytes[which] / rb;
    std::vector<unsigned char> out(rows * pb, 0);
    for (size_t r = 0; r < rows; ++r) std::memcpy(out.data() + r * pb, b + r * rb, rb);
    return out;
}

}  // namespace sfq

