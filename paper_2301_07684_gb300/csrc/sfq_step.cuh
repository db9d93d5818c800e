// sfq_step.cuh -- the per-particle, per-timestep Monte Carlo step (Sec. 2, 3, 4 of
// Montefiori & Tamburini, arXiv:2301.07684).
//
// A CTA walks over tiles of BS*PPT particles.  Phase A (every particle of the tile):
// coalesced structure-of-arrays loads, chi (Eq. chi_exact), the rate from the fitted
// table staged in shared memory (Eq. pe_rate_3 / Eq. pp_tot_real), the optical-depth
// decrement and event test (Sec. 2), and a push of event particles onto a
// shared-memory queue.  Phase B (queue only, so that the rare sampling work runs on
// compacted threads): Philox draws, inverse-transform sampling (Eq. again /
// Eq. again_pp), recoil or removal of the parent, and the product records, written
// after one global atomic reservation per tile.
#pragma once
#include "sfq_kernels.cuh"

namespace sfq {

template <typename T>
struct StepArgs {
    // particles
    int64_t n;
    T *px, *py, *pz;
    double *tau;
    const uint64_t *id;
    uint64_t id_base;
    uint8_t *flags;
    // fields
    const T *ex, *ey, *ez, *bx, *by, *bz;
    const uint32_t *k0;
    const T *amp;
    T amp0;
    const T *pw_table;
    uint32_t n_table, pw_offset;        // offset = (step * k_step) mod n_table
    // products
    int64_t cap;
    T *opx, *opy, *opz;
    uint64_t *opid;
    uint32_t *ostep;
    uint8_t *ometa;
    unsigned long long *ocount;
    // children (pair creation)
    int64_t scap;
    T *spx, *spy, *spz;
    double *stau;
    uint64_t *sid;
    uint8_t *sflags;
    T *sfp[3], *sdf[3];
    uint32_t *sk0;
    T *samp;
    unsigned long long *scount;
    // step constants
    uint32_t step;
    uint64_t seed;
    T prefdt;        // pref * dt
    T inv_rho;       // 1 / rho
    Tables<T> tab;
    sfq_counters *counters;
};

template <typename T>
struct QEntry {
    int lidx;           // index within the tile
    uint16_t o_prod, o_spawn;
    T g;                // energy of the particle
    T a;                // chi in phase A; then s (emission) or xi_e (pair)
    T b;                // xi_p (pair)
};

constexpr int STEP_BS = 256;

enum { FK_SOA = 0, FK_PW = 1 };

template <typename T, int FK>
__device__ __forceinline__ void load_fields(const StepArgs<T> &a, int64_t i, T E[3], T B[3]) {
    if (FK == FK_SOA) {
        E[0] = a.ex[i]; E[1] = a.ey[i]; E[2] = a.ez[i];
        B[0] = a.bx[i]; B[1] = a.by[i]; B[2] = a.bz[i];
    } else {
        uint32_t k = a.k0[i] + a.pw_offset;
        k -= (k >= a.n_table) ? a.n_table : 0u;
        k = k < a.n_table ? k : a.n_table - 1u;         // in bounds for any k0
        const T amp = a.amp ? a.amp[i] : a.amp0;
        const T f = amp * __ldg(a.pw_table + k);
        E[0] = (T)0; E[1] = f; E[2] = (T)0;
        B[0] = (T)0; B[1] = (T)0; B[2] = f;
    }
}

// chi rho = sqrt((gamma E + p x B)^2 - (p.E)^2): Eq. chi_exact multiplied through by gamma.
template <typename T>
__device__ __forceinline__ T chi_of(T g, T px, T py, T pz, const T E[3], const T B[3], T inv_rho) {
    const T fx = fma(g, E[0], py * B[2] - pz * B[1]);
    const T fy = fma(g, E[1], pz * B[0] - px * B[2]);
    const T fz = fma(g, E[2], px * B[1] - py * B[0]);
    const T pe = fma(px, E[0], fma(py, E[1], pz * E[2]));
    const T q = fma(fx, fx, fma(fy, fy, fz * fz)) - pe * pe;
    return sqrt(q > (T)0 ? q : (T)0) * inv_rho;
}

// Optical-depth decrement (Sec. 2).  Returns true on an event; otherwise stores
// the new tau.  `draw0` holds -ln(u3) when the particle arrived without one.
__device__ __forceinline__ bool od_update(double *tau_ptr, float d, uint64_t seed, uint64_t id,
                                          uint32_t step, uint32_t tag) {
    uint64_t b = (uint64_t)__double_as_longlong(*tau_ptr);
    uint64_t q;
    if (b >> 63) {                                  // no optical depth yet: draw it (word 3)
        const u4 w = draws(seed, id, step, tag);
        const float t0 = -logf(uniform<float>(w.w[3]));
        b = f32_to_f64_bits(t0);
    }
    if (!tau_to_fixed(b, q)) {                      // tau >= 32: plain binary64
        const double t = __longlong_as_double((long long)b) - (double)d;
        if (t < 0.0) return true;
        *tau_ptr = t;
        return false;
    }
    const uint64_t D = dec_to_fixed(d);
    if (D > q) return true;
    *tau_ptr = __longlong_as_double((long long)fixed_to_tau(q - D));
    return false;
}
__device__ __forceinline__ bool od_update(double *tau_ptr, double d, uint64_t seed, uint64_t id,
                                          uint32_t step, uint32_t tag) {
    double t = *tau_ptr;
    if (t < 0.0 || signbit(t)) {
        const u4 w = draws(seed, id, step, tag);
        t = -log(uniform<double>(w.w[3]));
    }
    t = t - d;
    if (t < 0.0) return true;
    *tau_ptr = t;
    return false;
}

__device__ __forceinline__ float fresh_tau(float u) { return -logf(u); }
__device__ __forceinline__ double fresh_tau(double u) { return -log(u); }

template <typename T>
__device__ __forceinline__ double to_tau(T v) { return (double)v; }
template <>
__device__ __forceinline__ double to_tau<float>(float v) {
    return __longlong_as_double((long long)f32_to_f64_bits(v));
}

template <typename T>
__device__ __forceinline__ T lepton_pmag(T g, Cnt &c) {
    const T q = g * g - (T)1;
    if (!(q > (T)0)) { ++c.v[C_G1]; return (T)0; }
    return sqrt(q);
}

// T: float (mixed) or double; FK: field source; PPT: particles per thread per tile.
template <typename T, int FK, int PPT>
__global__ void __launch_bounds__(STEP_BS) mc_step_kernel(const StepArgs<T> a) {
    constexpr int TILE = STEP_BS * PPT;
    using Q = L<T>;
    __shared__ T s_nlc[Q::RATE_NLC_N];
    __shared__ T s_nbw[Q::RATE_NBW_N];
    __shared__ QEntry<T> q[TILE];
    __shared__ int q_n, q_prod, q_spawn;
    __shared__ unsigned long long q_pbase, q_sbase;

    for (int k = threadIdx.x; k < Q::RATE_NLC_N; k += STEP_BS) s_nlc[k] = a.tab.nlc_rate[k];
    for (int k = threadIdx.x; k < Q::RATE_NBW_N; k += STEP_BS) s_nbw[k] = a.tab.nbw_rate[k];

    Cnt c;
    c.zero();
    const int64_t ntiles = (a.n + TILE - 1) / TILE;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        if (threadIdx.x == 0) { q_n = 0; q_prod = 0; q_spawn = 0; }
        __syncthreads();
        const int64_t base = tile * TILE;

        // ---------------- phase A: rate and event test for every particle
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const int lidx = k * STEP_BS + threadIdx.x;
            const int64_t i = base + lidx;
            if (i >= a.n) continue;
            const uint8_t fl = a.flags[i];
            if (!(fl & SFQ_ALIVE)) continue;
            const T px = a.px[i], py = a.py[i], pz = a.pz[i];
            T E[3], B[3];
            load_fields<T, FK>(a, i, E, B);
            const bool photon = ((fl >> SFQ_SPECIES_SHIFT) & 3) == SFQ_PHOTON;
            const T p2 = fma(px, px, fma(py, py, pz * pz));
            const T g = photon ? sqrt(p2) : sqrt((T)1 + p2);
            const T chi = chi_of<T>(g, px, py, pz, E, B, a.inv_rho);
            ++c.v[C_UPD];
            bool oor = false;
            T d;
            if (!(chi >= (T)0) || !(g > (T)0)) {
                ++c.v[C_NAN];
                d = (T)0;
            } else if (photon) {
                d = a.prefdt * wtilde_pair<T>(s_nbw, chi, oor) / g;
            } else {
                d = a.prefdt * (chi / g) * wtilde_rad<T>(s_nlc, chi, oor);
            }
            c.v[C_OOR] += oor;
            c.v[C_RDT] += d > (T)0.1;
            const uint64_t id = a.id ? a.id[i] : a.id_base + (uint64_t)i;
            const uint32_t tag = (fl >> SFQ_TAG_SHIFT) & 3u;
            if (od_update(a.tau + i, d, a.seed, id, a.step, tag)) {
                const int slot = atomicAdd(&q_n, 1);
                QEntry<T> e;
                e.lidx = lidx;
                e.g = g;
                e.a = chi;
                e.b = (T)0;
                q[slot] = e;
            }
        }
        __syncthreads();

        // ---------------- phase B1: sampling on the compacted queue
        const int nq = q_n;
        for (int k = threadIdx.x; k < nq; k += STEP_BS) {
            QEntry<T> e = q[k];
            const int64_t i = base + e.lidx;
            const uint8_t fl = a.flags[i];
            const uint64_t id = a.id ? a.id[i] : a.id_base + (uint64_t)i;
            const u4 w = draws(a.seed, id, a.step, (fl >> SFQ_TAG_SHIFT) & 3u);
            const T r1 = uniform<T>(w.w[1]);
            bool oor = false;
            ++c.v[C_EV];
            if (((fl >> SFQ_SPECIES_SHIFT) & 3) == SFQ_PHOTON) {
                T xe, xp;
                pair_shares<T>(a.tab.nbw_inv, e.a, r1, xe, xp, oor);
                e.a = xe;
                e.b = xp;
                e.o_prod = (uint16_t)atomicAdd(&q_prod, 2);
                e.o_spawn = a.scount ? (uint16_t)atomicAdd(&q_spawn, 2) : (uint16_t)0;
                ++c.v[C_PAIR];
            } else {
                e.a = photon_s<T>(a.tab.nlc_inv, e.a, r1, oor);
                e.o_prod = (uint16_t)atomicAdd(&q_prod, 1);
                ++c.v[C_EMIT];
            }
            c.v[C_OOR] += oor;
            q[k] = e;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            q_pbase = q_prod ? atomicAdd(a.ocount, (unsigned long long)q_prod) : 0ull;
            q_sbase = (q_spawn && a.scount) ? atomicAdd(a.scount, (unsigned long long)q_spawn) : 0ull;
        }
        __syncthreads();

        // ---------------- phase B2: parents and product records
        for (int k = threadIdx.x; k < nq; k += STEP_BS) {
            const QEntry<T> e = q[k];
            const int64_t i = base + e.lidx;
            const uint8_t fl = a.flags[i];
            const uint64_t id = a.id ? a.id[i] : a.id_base + (uint64_t)i;
            const uint32_t tag = (fl >> SFQ_TAG_SHIFT) & 3u;
            const T px = a.px[i], py = a.py[i], pz = a.pz[i];
            const T pm = sqrt(fma(px, px, fma(py, py, pz * pz)));
            const T inv_pm = pm > (T)0 ? (T)1 / pm : (T)0;
            const T nx = px * inv_pm, ny = py * inv_pm, nz = pz * inv_pm;
            if (((fl >> SFQ_SPECIES_SHIFT) & 3) == SFQ_PHOTON) {
                // pair creation: the photon is removed, two leptons along its direction
                const T ge = e.a * e.g, gp = e.b * e.g;
                const T pme = lepton_pmag(ge, c), pmp = lepton_pmag(gp, c);
                for (int m = 0; m < 2; ++m) {
                    const unsigned long long j = q_pbase + e.o_prod + m;
                    const T pmag = m == 0 ? pme : pmp;
                    if (j < (unsigned long long)a.cap) {
                        a.opx[j] = nx * pmag; a.opy[j] = ny * pmag; a.opz[j] = nz * pmag;
                        a.opid[j] = id;
                        a.ostep[j] = a.step;
                        a.ometa[j] = (uint8_t)((m == 0 ? SFQ_ELECTRON : SFQ_POSITRON) | ((m + 1) << 2) | (tag << 4));
                    } else {
                        ++c.v[C_DROP];
                    }
                    if (a.scount) {
                        const unsigned long long s = q_sbase + e.o_spawn + m;
                        if (s < (unsigned long long)a.scap) {
                            a.spx[s] = nx * pmag; a.spy[s] = ny * pmag; a.spz[s] = nz * pmag;
                            a.stau[s] = -1.0;
                            a.sid[s] = id;
                            a.sflags[s] = (uint8_t)(SFQ_ALIVE | SFQ_JUST_CREATED |
                                                    ((m == 0 ? SFQ_ELECTRON : SFQ_POSITRON) << SFQ_SPECIES_SHIFT) |
                                                    ((m + 1) << SFQ_TAG_SHIFT));
                            if (a.sfp[0]) {
#pragma unroll
                                for (int d3 = 0; d3 < 3; ++d3) { a.sfp[d3][s] = (T)0; a.sdf[d3][s] = (T)0; }
                            }
                            if (a.sk0) a.sk0[s] = a.k0[i];
                            if (a.samp) a.samp[s] = a.amp ? a.amp[i] : a.amp0;
                        } else {
                            ++c.v[C_SDROP];
                        }
                    }
                }
                a.flags[i] = (uint8_t)(fl & ~SFQ_ALIVE);
            } else {
                // photon emission: xi = s/(1+s) to the photon, the lepton keeps gamma/(1+s)
                const T s = e.a;
                const T inv1s = (T)1 / ((T)1 + s);
                const T gph = e.g * s * inv1s;
                const T pnew = lepton_pmag(e.g * inv1s, c);
                const unsigned long long j = q_pbase + e.o_prod;
                if (j < (unsigned long long)a.cap) {
                    a.opx[j] = nx * gph; a.opy[j] = ny * gph; a.opz[j] = nz * gph;
                    a.opid[j] = id;
                    a.ostep[j] = a.step;
                    a.ometa[j] = (uint8_t)(SFQ_PHOTON | (tag << 4));
                } else {
                    ++c.v[C_DROP];
                }
                a.px[i] = nx * pnew; a.py[i] = ny * pnew; a.pz[i] = nz * pnew;
                // fresh optical depth from word 0 (Sec. 2)
                const u4 w = draws(a.seed, id, a.step, tag);
                a.tau[i] = to_tau<T>(fresh_tau(uniform<T>(w.w[0])));
            }
        }
        __syncthreads();
    }
    flush_counters(c, a.counters);
}

}  // namespace sfq
