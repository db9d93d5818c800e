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
    const unsigned long long *n_dev;    // optional device count (min with n)
    T *px, *py, *pz;
    double *tau;
    const uint64_t *id;
    uint64_t id_base;
    uint8_t *flags;
    T *fprev[3], *dfprev[3];            // beyond-LCFA state
    int lepton_model;
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
    T rho;
    T inv_dt, inv_dt2;
    T dt;            // timestep (the pusher of the BLCFA_PUSHED model)
    T pair_chi_min;  // NBW rate is zero below this chi (0.01, or the "fast" cutoff)
    Tables<T> tab;
    sfq_counters *counters;
    // queue of photon emissions for the surrogate pass (the SURR kernel instances only)
    int64_t qcap;
    int64_t *qidx;
    float *qchi, *qr, *qg, *qpx, *qpy, *qpz;
    unsigned long long *qcount;
};

// Entry of the TMA-staged kernel's event queue: the particle's state as the step read it,
// so that the event path re-reads nothing from global memory.
template <typename T>
struct QEntry {
    int64_t i;          // particle index
    T g;                // energy of the particle
    T chi;              // quantum parameter at the event
    T px, py, pz;       // momentum before the event
    uint32_t fl;        // flags
};
// Entry of the warp-streaming kernel, which also serves beyond-LCFA leptons.
template <typename T>
struct QEntryX {
    int64_t i;
    T g, chi;
    T aux;              // -1: optical-depth event; beyond-LCFA: gamma_LCFA (> 0) or 0 (no rejection)
};

template <typename T>
__device__ __forceinline__ int64_t effective_n(const StepArgs<T> &a) {
    if (!a.n_dev) return a.n;
    const int64_t m = (int64_t)*a.n_dev;
    return m < a.n ? m : a.n;
}

constexpr int STEP_BS = 256;
#ifndef SFQ_STEP_MINB
#define SFQ_STEP_MINB 4   // resident blocks per SM the register allocation aims for (measured best)
#endif
#ifndef SFQ_LEPTON_MINB
#define SFQ_LEPTON_MINB 4 // the same for the beyond-LCFA lepton and full-cascade instances
#endif

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
    return sqrt_nr(q) * inv_rho;
}

// chi in the linearly polarised plane wave E = (0, f, 0), B = (0, 0, f): Eq. chi_exact with
// the vanishing components dropped (gamma E + p x B = (py f, gamma f - px f, 0), p.E = py f).
// Every operation is rounded explicitly, so all kernels form the same bits.
__device__ __forceinline__ float mul_rn(float x, float y) { return __fmul_rn(x, y); }
__device__ __forceinline__ double mul_rn(double x, double y) { return __dmul_rn(x, y); }
__device__ __forceinline__ float sub_rn(float x, float y) { return __fsub_rn(x, y); }
__device__ __forceinline__ double sub_rn(double x, double y) { return __dsub_rn(x, y); }
template <typename T>
__device__ __forceinline__ T chi_pw(T g, T px, T py, T f, T inv_rho) {
    const T fx = mul_rn(py, f);
    const T fy = fma(g, f, -mul_rn(px, f));
    const T q = sub_rn(fma(fx, fx, mul_rn(fy, fy)), mul_rn(fx, fx));
    return sqrt_nr(q) * inv_rho;
}

// Optical-depth decrement (Sec. 2).  od_update returns true on an event; otherwise it
// stores the new tau.  It is od_fill followed by od_sub.
// The optical depth a particle starts from: its stored bits, or a fresh draw -ln(u3) when
// it arrived without one (sign bit set).
template <typename IdF>
__device__ __forceinline__ uint64_t od_fill(uint64_t b, uint64_t seed, IdF id_of, uint32_t step, uint32_t tag) {
    if (b >> 63) {                                  // no optical depth yet: draw it (word 3)
        const u4 w = draws(seed, id_of(), step, tag);
        const float t0 = -logf(uniform<float>(w.w[3]));
        b = f32_to_f64_bits(t0);
    }
    return b;
}
// tau_d - R dt in binary64: the binary32 decrement is widened exactly with integer
// operations and the subtraction is the only binary64 instruction of the update.  A
// decrement that overflowed binary32 (+inf) is an event, as the binary64 one would be;
// zero, subnormal and NaN decrements subtract nothing.
__device__ __forceinline__ bool od_sub(double *tau_ptr, uint64_t b, float d) {
    const uint32_t db = __float_as_uint(d);
    const uint64_t dd = ((db >> 23) - 1u < 254u) ? f32_to_f64_bits(d)                    // normal d > 0
                                                 : (db == 0x7F800000u ? 0x7FF0000000000000ull : 0ull);
    const double t = __dsub_rn(__longlong_as_double((long long)b), __longlong_as_double((long long)dd));
    // the difference of two non-negative binary64 values is negative exactly when its sign
    // bit is set (it is never -0), so the test runs on the integer pipe
    if (__double_as_longlong(t) < 0) return true;
    *tau_ptr = t;
    return false;
}
template <typename IdF>
__device__ __forceinline__ bool od_update(double *tau_ptr, float d, uint64_t seed, IdF id_of,
                                          uint32_t step, uint32_t tag) {
    const uint64_t b = od_fill((uint64_t)__double_as_longlong(*tau_ptr), seed, id_of, step, tag);
    return od_sub(tau_ptr, b, d);
}
template <typename IdF>
__device__ __forceinline__ bool od_update(double *tau_ptr, double d, uint64_t seed, IdF id_of,
                                          uint32_t step, uint32_t tag) {
    double t = *tau_ptr;
    if (t < 0.0 || signbit(t)) {
        const u4 w = draws(seed, id_of(), step, tag);
        t = -log(uniform<double>(w.w[3]));
    }
    t = t - d;
    if (__double_as_longlong(t) < 0) return true;   // t < 0 (never -0: tau, d >= 0)
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

// Beyond-LCFA lepton (Sec. 5): force history (Eqs. fl ... condit; no pusher: F_L = E + beta x B,
// p_L = p), local test R dt > r (Sec. 2, word 0) and the threshold gamma_LCFA (Eq. gammaLCFA,
// with sinh(3 asinh z) = 3z + 4z^3).  Returns true when an emission is to be sampled; aux is
// gamma_LCFA when the rejection of Eq. rej_cond applies, 0 when the LCFA spectrum applies.
template <typename T>
__device__ __forceinline__ bool blcfa_phase_a(const StepArgs<T> &a, const T *s_nlc, int64_t i, uint8_t fl, T px,
                                              T py, T pz, const T E[3], const T B[3], T &g, T &chi, T &aux,
                                              Cnt &c) {
    T FL[3];
    if (a.lepton_model == SFQ_LEPTON_BLCFA_PUSHED) {
        // the pusher advances p^(n-1/2) to p_L^(n+1/2); F_L = (p_L^(n+1/2) - p^(n-1/2)) / dt and
        // p_L^(n) = (p_L^(n+1/2) + p^(n-1/2)) / 2 (Eqs. fl); the particle keeps the pushed momentum
        T u[3] = {px, py, pz};
        const int sp = (fl >> SFQ_SPECIES_SHIFT) & 3;
        boris<T>(u, E, B, sp == SFQ_ELECTRON ? (T)-1 : (T)1, a.dt);
#pragma unroll
        for (int k = 0; k < 3; ++k) FL[k] = (u[k] - (k == 0 ? px : k == 1 ? py : pz)) * a.inv_dt;
        a.px[i] = u[0]; a.py[i] = u[1]; a.pz[i] = u[2];
        px = (T)0.5 * (u[0] + px); py = (T)0.5 * (u[1] + py); pz = (T)0.5 * (u[2] + pz);
    }
    const T g2 = fma(px, px, fma(py, py, fma(pz, pz, (T)1)));
    const T inv_g = rsqrt_nr(g2);
    g = sqrt_nr(g2);
    if (a.lepton_model != SFQ_LEPTON_BLCFA_PUSHED) {
        // without a pusher: F_L = E + beta x B at the particle, p_L = p (reading R9)
        const T bx = px * inv_g, by = py * inv_g, bz = pz * inv_g;
        FL[0] = E[0] + (by * B[2] - bz * B[1]);
        FL[1] = E[1] + (bz * B[0] - bx * B[2]);
        FL[2] = E[2] + (bx * B[1] - by * B[0]);
    }
    const T fp = (FL[0] * px + FL[1] * py + FL[2] * pz) * inv_g * inv_g;
    const T F[3] = {FL[0] - fp * px, FL[1] - fp * py, FL[2] - fp * pz};      // Eq. fl_perp
    const T F2 = F[0] * F[0] + F[1] * F[1] + F[2] * F[2];
    chi = g * sqrt_nr(F2) * a.inv_rho;                                       // Eq. chi_p
    ++c.v[C_UPD];
    if (fl & SFQ_JUST_CREATED) {
        // first update after creation: F^(n-2) = F^(n-1) = F^(n), no emission
#pragma unroll
        for (int k = 0; k < 3; ++k) { a.fprev[k][i] = F[k]; a.dfprev[k][i] = (T)0; }
        a.flags[i] = (uint8_t)(fl & ~SFQ_JUST_CREATED);
        return false;
    }
    // the stored history first, all six loads together (the stores below could alias them)
    T fpv[3], dfv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) { fpv[k] = a.fprev[k][i]; dfv[k] = a.dfprev[k][i]; }
    const uint64_t id = a.id ? a.id[i] : a.id_base + (uint64_t)i;
    T d1[3], Fd2 = (T)0, FFdd = (T)0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        d1[k] = F[k] - fpv[k];
        const T fd = d1[k] * a.inv_dt;
        const T fdd = (d1[k] - dfv[k]) * a.inv_dt2;
        Fd2 = fma(fd, fd, Fd2);
        FFdd = fma(F[k], fdd, FFdd);
        a.fprev[k][i] = F[k];
        a.dfprev[k][i] = d1[k];
    }
    const T D = Fd2 + fabs(FFdd);                                            // delta / tau_C^2, Eq. condit
    // gamma^2 delta/zeta^2 > chi^2 F^2 divided by gamma^2 tau_C^2 > 0, zeta = 2^-52
    const T zeta = (T)2.220446049250313080847263336181640625e-16;
    const T zeta2 = (T)4.930380657631323783823303533017413935457540219431393779648e-32;
    const bool gate = (D > zeta2 * F2 * F2) && (chi > zeta);
    const u4 w = draws(a.seed, id, a.step, (fl >> SFQ_TAG_SHIFT) & 3u);
    const T r0 = uniform<T>(w.w[0]);
    // Acceptance-rejection of the local method (Sec. 2): W~_rad(chi) <= W~_rad(0) = 5 pi / 2,
    // so the same product with that bound (a margin above the fit's and Horner's rounding)
    // majorises R dt.  Unless the majorant exceeds r (or 0.1, the threshold of the large-R dt
    // counter), no event can occur and the fitted rate is not evaluated.
    const T wmax = sizeof(T) == 4 ? (T)(7.8539816339744830962 * (1.0 + 1.52587890625e-05))
                                  : (T)(7.8539816339744830962 * (1.0 + 9.094947017729282e-13));
    const T dmax = a.prefdt * (chi * inv_g) * wmax;
    if (!(dmax > r0) && !(dmax > (T)0.1)) {
        c.v[C_OOR] += !(chi < pow2<T>(L<T>::NLC_EHI));                      // as the table would count it
        return false;
    }
    bool oor = false;
    const T d = a.prefdt * (chi * inv_g) * wtilde_rad<T>(s_nlc, chi, oor);
    c.v[C_OOR] += oor;
    c.v[C_RDT] += d > (T)0.1;
    if (!(d > r0)) return false;                                            // local test
    ++c.v[C_EV];
    aux = (T)0;
    if (gate) {
        const T tau_ratio = (T)6.283185307179586476925286766559 * a.rho * sqrt_nr(F2 / D);   // tau / tau_C
        const T z = chi / ((T)8 * g) * tau_ratio;
        const T gL = (T)0.7 * g / ((T)1 + (T)4 / ((T)3 * (T)3.1415926535897932384626433832795 * chi) *
                                              (z * fma((T)4 * z, z, (T)3)));
        if (!(gL < (T)0.75 * g)) {                                          // no emission (Sec. 5)
            ++c.v[C_NOEM];
            return false;
        }
        aux = gL;
    }
    return true;
}

// New state of an event's parent, returned by process_events_core: bit 0 of `what` =
// momentum replaced, bit 1 = fresh optical depth, bit 2 = flags replaced.
template <typename T>
struct EvOut {
    T px, py, pz;
    double tau;
    uint8_t fl;
    uint8_t what;
};

// Warp-collective reservation of nprod product records and nspawn children per lane:
// one atomic per counter for the warp; returns each lane's first index.
__device__ __forceinline__ void reserve_records(unsigned long long *ocount, unsigned long long *scount, int nprod,
                                                int nspawn, unsigned long long &bp, unsigned long long &bs) {
    const int lane = threadIdx.x & 31;
    int pre_p = nprod, pre_s = nspawn;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int tp = __shfl_up_sync(0xFFFFFFFFu, pre_p, o);
        const int ts = __shfl_up_sync(0xFFFFFFFFu, pre_s, o);
        if (lane >= o) { pre_p += tp; pre_s += ts; }
    }
    const int tot_p = __shfl_sync(0xFFFFFFFFu, pre_p, 31);
    const int tot_s = __shfl_sync(0xFFFFFFFFu, pre_s, 31);
    unsigned long long b0 = 0, b1 = 0;
    if (lane == 31) {
        if (tot_p) b0 = atomicAdd(ocount, (unsigned long long)tot_p);
        if (tot_s) b1 = atomicAdd(scount, (unsigned long long)tot_s);
    }
    bp = __shfl_sync(0xFFFFFFFFu, b0, 31) + (unsigned long long)(pre_p - nprod);
    bs = __shfl_sync(0xFFFFFFFFu, b1, 31) + (unsigned long long)(pre_s - nspawn);
}

// One batch of up to 32 queued events, one per lane (lanes with valid = false idle); all
// 32 lanes execute it (warp shuffles).  The lane receives the particle's index i, its
// energy g, chi at the event, aux (-1 for an optical-depth event; for beyond-LCFA,
// gamma_LCFA or 0), and the momentum and flags the step read.  Sampling (Eq. again /
// Eq. again_pp), parent update and product records.  The records are reserved with one
// global atomic per batch, before the sampling when every record count is known up
// front (no beyond-LCFA lane, whose emission may be rejected), so that the atomic's
// latency overlaps the sampling.
template <typename T, bool TRUNC = false, bool CASC = false, bool SURR = false>
__device__ __forceinline__ void process_events_core(const StepArgs<T> &a, uint32_t step, int64_t ei, T eg, T echi,
                                                    T e_aux, T px, T py, T pz, uint8_t fl, bool valid, Cnt &c,
                                                    EvOut<T> &o) {
    o.what = 0;
    const bool photon = valid && ((fl >> SFQ_SPECIES_SHIFT) & 3) == SFQ_PHOTON;
    const bool maybe = valid && !photon && !(e_aux < (T)0);        // beyond-LCFA: may be rejected
    const bool late = __any_sync(0xFFFFFFFFu, maybe);
    // SURR: photon emissions by the optical-depth method go to the surrogate's queue (one
    // entry each, reserved warp-wide); an event the queue cannot take is sampled here
    bool queued = false;
    unsigned long long qslot = 0;
    if constexpr (SURR) {
        const bool want = valid && !photon && e_aux < (T)0;
        unsigned long long dummy = 0;
        reserve_records(a.qcount, nullptr, want ? 1 : 0, 0, qslot, dummy);
        queued = want && qslot < (unsigned long long)a.qcap;
        c.v[C_SURR] += want && !queued;
    }
    int nprod = valid && !queued ? (photon ? 2 : 1) : 0;
    // spawned particles: the pair of a converted photon; in a cascade also the emitted photon
    int nspawn = a.scount ? (photon ? 2 : (CASC ? nprod : 0)) : 0;
    unsigned long long bp = 0, bs = 0;
    if (!late) reserve_records(a.ocount, a.scount, nprod, nspawn, bp, bs);
    T xa = 0, xb = 0;
    uint64_t id = 0;
    uint32_t tag = 0;
    bool oor = false;
    if (valid) {
        id = a.id ? a.id[ei] : a.id_base + (uint64_t)ei;
        tag = (fl >> SFQ_TAG_SHIFT) & 3u;
        const u4 w = draws(a.seed, id, step, tag);
        const T r1 = uniform<T>(w.w[1]);
        if (photon) {
            ++c.v[C_EV];
            pair_shares_sel<T, TRUNC>(a.tab, echi, r1, xa, xb, oor);
            ++c.v[C_PAIR];
        } else if (e_aux < (T)0) {
            ++c.v[C_EV];
            xb = uniform<T>(w.w[0]);                               // for the fresh optical depth
            if (queued) {
                // the surrogate pass samples this emission, applies the recoil and writes the record
                a.qidx[qslot] = ei;
                a.qchi[qslot] = (float)echi;
                a.qr[qslot] = (float)r1;
                a.qg[qslot] = (float)eg;
                a.qpx[qslot] = (float)px; a.qpy[qslot] = (float)py; a.qpz[qslot] = (float)pz;
            } else {
                xa = photon_s_sel<T, TRUNC>(a.tab, echi, r1, oor);  // s
                ++c.v[C_EMIT];
            }
        } else {
            // beyond-LCFA: LCFA sample, then the rejection of Eq. rej_cond below gamma_LCFA
            xa = photon_s_sel<T, TRUNC>(a.tab, echi, r1, oor);
            xb = (T)-1;                                            // marks: no optical depth
            bool accept = true;
            const T gbar = eg * xa / ((T)1 + xa);
            if (e_aux > (T)0 && !(gbar > e_aux)) {
                const T uL = e_aux / (eg - e_aux);
                const T lhs = log(uniform<T>(w.w[2])) + ln_spectrum<T>(a.tab.k23, a.tab.ki13, xa, echi, oor);
                const T rhs = ln_spectrum<T>(a.tab.k23, a.tab.ki13, uL, echi, oor);
                accept = lhs <= rhs;
            }
            if (accept) {
                ++c.v[C_EMIT];
            } else {
                nprod = 0;
                nspawn = 0;
                ++c.v[C_REJ];
            }
        }
        c.v[C_OOR] += oor;
    }
    if (late) reserve_records(a.ocount, a.scount, nprod, nspawn, bp, bs);
    if (!valid) return;
    if (queued) {
        o.tau = to_tau<T>(fresh_tau(xb));                        // fresh optical depth, word 0 (Sec. 2)
        o.what = 2;
        return;
    }
    const T pm = sqrt(fma(px, px, fma(py, py, pz * pz)));
    const T inv_pm = pm > (T)0 ? (T)1 / pm : (T)0;
    const T nx = px * inv_pm, ny = py * inv_pm, nz = pz * inv_pm;
    if (photon) {
        // pair creation: the photon is removed, two leptons along its direction
        const T pme = lepton_pmag(xa * eg, c), pmp = lepton_pmag(xb * eg, c);
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const unsigned long long j = bp + m;
            const T pmag = m == 0 ? pme : pmp;
            if (j < (unsigned long long)a.cap) {
                a.opx[j] = nx * pmag; a.opy[j] = ny * pmag; a.opz[j] = nz * pmag;
                a.opid[j] = id;
                a.ostep[j] = step;
                a.ometa[j] = (uint8_t)((m == 0 ? SFQ_ELECTRON : SFQ_POSITRON) | ((m + 1) << 2) | (tag << 4));
            } else {
                ++c.v[C_DROP];
            }
            if (nspawn) {
                const unsigned long long s = bs + m;
                if (s < (unsigned long long)a.scap) {
                    a.spx[s] = nx * pmag; a.spy[s] = ny * pmag; a.spz[s] = nz * pmag;
                    a.stau[s] = -1.0;
                    a.sid[s] = CASC ? child_id(a.seed, id, tag, step, (uint32_t)(m + 1)) : id;
                    a.sflags[s] = (uint8_t)((pmag > (T)0 ? SFQ_ALIVE : 0) | SFQ_JUST_CREATED |
                                            ((m == 0 ? SFQ_ELECTRON : SFQ_POSITRON) << SFQ_SPECIES_SHIFT) |
                                            (CASC ? 0 : (m + 1) << SFQ_TAG_SHIFT));
                    if (a.sfp[0]) {
#pragma unroll
                        for (int d3 = 0; d3 < 3; ++d3) { a.sfp[d3][s] = (T)0; a.sdf[d3][s] = (T)0; }
                    }
                    if (a.sk0) a.sk0[s] = a.k0[ei];
                    if (a.samp) a.samp[s] = a.amp ? a.amp[ei] : a.amp0;
                } else {
                    ++c.v[C_SDROP];
                }
            }
        }
        o.fl = (uint8_t)(fl & ~SFQ_ALIVE);
        o.what = 4;
    } else if (nprod) {
        // photon emission: xi = s/(1+s) to the photon, the lepton keeps gamma/(1+s)
        const T s = xa;
        const T inv1s = (T)1 / ((T)1 + s);
        const T gph = eg * s * inv1s;
        const T pnew = lepton_pmag(eg * inv1s, c);
        const unsigned long long j = bp;
        if (j < (unsigned long long)a.cap) {
            a.opx[j] = nx * gph; a.opy[j] = ny * gph; a.opz[j] = nz * gph;
            a.opid[j] = id;
            a.ostep[j] = step;
            a.ometa[j] = (uint8_t)(SFQ_PHOTON | (tag << 4));
        } else {
            ++c.v[C_DROP];
        }
        if (CASC && nspawn) {
            // full cascade: the photon is also a particle, stepped from the next step on
            const unsigned long long sj = bs;
            if (sj < (unsigned long long)a.scap) {
                a.spx[sj] = nx * gph; a.spy[sj] = ny * gph; a.spz[sj] = nz * gph;
                a.stau[sj] = -1.0;
                a.sid[sj] = child_id(a.seed, id, tag, step, 0u);
                a.sflags[sj] = (uint8_t)((gph > (T)0 ? SFQ_ALIVE : 0) | SFQ_JUST_CREATED |
                                         (SFQ_PHOTON << SFQ_SPECIES_SHIFT));
                if (a.sfp[0]) {
#pragma unroll
                    for (int d3 = 0; d3 < 3; ++d3) { a.sfp[d3][sj] = (T)0; a.sdf[d3][sj] = (T)0; }
                }
                if (a.sk0) a.sk0[sj] = a.k0[ei];
                if (a.samp) a.samp[sj] = a.amp ? a.amp[ei] : a.amp0;
            } else {
                ++c.v[C_SDROP];
            }
        }
        o.px = nx * pnew; o.py = ny * pnew; o.pz = nz * pnew;
        o.what = 1;
        if (xb > (T)0) {                                        // fresh optical depth, word 0 (Sec. 2)
            o.tau = to_tau<T>(fresh_tau(xb));
            o.what |= 2;
        }
        // a lepton left without momentum is outside the ultrarelativistic regime of the rates
        // and has no direction for collinear emission: it leaves the step
        if (!(pnew > (T)0)) {
            o.fl = (uint8_t)(fl & ~SFQ_ALIVE);
            o.what |= 4;
        }
    }
}

// process_events_core at the launch's step with the parent's new state stored to the
// population in global memory.
template <typename T, bool TRUNC = false, bool CASC = false, bool SURR = false>
__device__ __forceinline__ void process_events(const StepArgs<T> &a, int64_t ei, T eg, T echi, T e_aux, T px,
                                               T py, T pz, uint8_t fl, bool valid, Cnt &c) {
    EvOut<T> o;
    process_events_core<T, TRUNC, CASC, SURR>(a, a.step, ei, eg, echi, e_aux, px, py, pz, fl, valid, c, o);
    if (o.what & 1) { a.px[ei] = o.px; a.py[ei] = o.py; a.pz[ei] = o.pz; }
    if (o.what & 2) a.tau[ei] = o.tau;
    if (o.what & 4) a.flags[ei] = o.fl;
}

// Per-lane computation of the rate and the optical-depth test for one particle held
// in registers; returns true on an event (tau is then left to the event path).  Every
// kernel shape calls this one routine, so results do not depend on the launch shape.
template <typename T, bool PW = false>
__device__ __forceinline__ bool step_particle(const StepArgs<T> &a, const T *s_nlc, const T *s_nbw, int64_t i,
                                              uint8_t fl, T px, T py, T pz, const T E[3], const T B[3],
                                              double tau_in, T &g, T &chi, Cnt &c) {
    const bool photon = ((fl >> SFQ_SPECIES_SHIFT) & 3) == SFQ_PHOTON;
    const T p2 = fma(px, px, fma(py, py, pz * pz));
    // gamma and 1/gamma from one reciprocal square root
    const T g2 = photon ? p2 : (T)1 + p2;
    const T inv_g = g2 > (T)0 ? rsqrt_nr(g2) : (T)0;
    g = g2 * inv_g;                                  // sqrt(g2) from the same reciprocal square root
    chi = PW ? chi_pw<T>(g, px, py, E[1], a.inv_rho) : chi_of<T>(g, px, py, pz, E, B, a.inv_rho);
    ++c.v[C_UPD];
    bool oor = false;
    T d;
    if (!(chi >= (T)0) || !(g > (T)0)) {
        ++c.v[C_NAN];
        d = (T)0;
    } else if (photon) {
        d = a.prefdt * wtilde_pair<T>(s_nbw, chi, oor, a.pair_chi_min) * inv_g;
    } else {
        d = a.prefdt * (chi * inv_g) * wtilde_rad<T>(s_nlc, chi, oor);
    }
    c.v[C_OOR] += oor;
    c.v[C_RDT] += d > (T)0.1;
    const auto id_of = [&]() { return a.id ? a.id[i] : a.id_base + (uint64_t)i; };
    double tau_v = tau_in;
    const bool ev = od_update(&tau_v, d, a.seed, id_of, a.step, (fl >> SFQ_TAG_SHIFT) & 3u);
    if (!ev) a.tau[i] = tau_v;
    return ev;
}

// As step_particle, with the optical depth passed in and out (stored by the caller).
template <typename T, bool PW = false>
__device__ __forceinline__ bool step_particle_v(const StepArgs<T> &a, const T *s_nlc, const T *s_nbw, int64_t i,
                                                uint8_t fl, T px, T py, T pz, const T E[3], const T B[3],
                                                double &tau, T &g, T &chi, Cnt &c, uint32_t step) {
    const bool photon = ((fl >> SFQ_SPECIES_SHIFT) & 3) == SFQ_PHOTON;
    const T p2 = fma(px, px, fma(py, py, pz * pz));
    const T g2 = photon ? p2 : (T)1 + p2;
    const T inv_g = g2 > (T)0 ? rsqrt_nr(g2) : (T)0;
    g = g2 * inv_g;                                  // sqrt(g2) from the same reciprocal square root
    chi = PW ? chi_pw<T>(g, px, py, E[1], a.inv_rho) : chi_of<T>(g, px, py, pz, E, B, a.inv_rho);
    ++c.v[C_UPD];
    bool oor = false;
    T d;
    if (!(chi >= (T)0) || !(g > (T)0)) {
        ++c.v[C_NAN];
        d = (T)0;
    } else if (photon) {
        d = a.prefdt * wtilde_pair<T>(s_nbw, chi, oor, a.pair_chi_min) * inv_g;
    } else {
        d = a.prefdt * (chi * inv_g) * wtilde_rad<T>(s_nlc, chi, oor);
    }
    c.v[C_OOR] += oor;
    c.v[C_RDT] += d > (T)0.1;
    const auto id_of = [&]() { return a.id ? a.id[i] : a.id_base + (uint64_t)i; };
    return od_update(&tau, d, a.seed, id_of, step, (fl >> SFQ_TAG_SHIFT) & 3u);
}

// Two alive leptons of one lane, binary32: the arithmetic of step_particle_v for each,
// written as one block with the rare optical-depth draw in front, so that nothing
// branches between the two dependency chains and they interleave.  The NaN guard of
// step_particle_v becomes a select (the rate is evaluated at chi = 0 and discarded).
template <bool PW>
__device__ __forceinline__ void step_lepton_pair(const StepArgs<float> &a, const float *s_nlc, int64_t i0,
                                                 const uint8_t fl[2], const float px[2], const float py[2],
                                                 const float pz[2], const float E[2][3], const float B[2][3],
                                                 double tau[2], float g[2], float chi[2], bool ev[2], Cnt &c) {
    uint64_t b[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const auto id_of = [&]() { return a.id ? a.id[i0 + k] : a.id_base + (uint64_t)(i0 + k); };
        b[k] = od_fill((uint64_t)__double_as_longlong(tau[k]), a.seed, id_of, a.step, (fl[k] >> SFQ_TAG_SHIFT) & 3u);
    }
    float d[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float p2 = fmaf(px[k], px[k], fmaf(py[k], py[k], pz[k] * pz[k]));
        const float g2 = 1.0f + p2;
        const float inv_g = g2 > 0.0f ? rsqrt_nr(g2) : 0.0f;
        g[k] = g2 * inv_g;
        chi[k] = PW ? chi_pw<float>(g[k], px[k], py[k], E[k][1], a.inv_rho)
                    : chi_of<float>(g[k], px[k], py[k], pz[k], E[k], B[k], a.inv_rho);
        const bool ok = chi[k] >= 0.0f && g[k] > 0.0f;
        bool oor = false;
        const float w = wtilde_rad<float>(s_nlc, ok ? chi[k] : 0.0f, oor);
        d[k] = ok ? a.prefdt * (chi[k] * inv_g) * w : 0.0f;
        c.v[C_UPD] += 1;
        c.v[C_NAN] += !ok;
        c.v[C_OOR] += ok && oor;
        c.v[C_RDT] += d[k] > 0.1f;
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) ev[k] = od_sub(&tau[k], b[k], d[k]);
}

// T: float (mixed) or double; FK: field source; PPT: particles per lane per chunk.
// Each warp streams chunks of 32*PPT particles and compacts event lanes into a
// warp-private ring in shared memory; a full batch of 32 events is sampled by the
// whole warp.  No block-wide barrier inside the loop.
// CASC: the full-cascade instance (every product is also spawned, with its own id).
// MINB: resident blocks per SM the register allocation aims for (the beyond-LCFA lepton and
// full-cascade instances take SFQ_LEPTON_MINB: their event paths hold more state).
template <typename T, int FK, int PPT, bool TRUNC = false, bool CASC = false, bool SURR = false,
          int MINB = SFQ_STEP_MINB>
__global__ void __launch_bounds__(STEP_BS, MINB) mc_step_kernel(const StepArgs<T> a) {
    using Q = L<T>;
    constexpr int WARPS = STEP_BS / 32;
    constexpr int QS = (32 * (PPT + 1) <= 64) ? 64 : ((32 * (PPT + 1) <= 128) ? 128 : 256);
    using RS = RateSmem<T>;
    __shared__ __align__(16) T s_nlc[RS::NLC_N];
    __shared__ __align__(16) T s_nbw[RS::NBW_N];
    __shared__ QEntryX<T> wq[WARPS][QS];

    stage_rate_table<T, Q::NLC_DEG, RS::NLC_STRIDE>(s_nlc, a.tab.nlc_rate, Q::RATE_NLC_N / (Q::NLC_DEG + 1),
                                                     threadIdx.x, STEP_BS);
    stage_rate_table<T, Q::NBW_DEG, RS::NBW_STRIDE>(s_nbw, a.tab.nbw_rate, Q::RATE_NBW_N / (Q::NBW_DEG + 1),
                                                     threadIdx.x, STEP_BS);
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    QEntryX<T> *q = wq[warp];
    unsigned head = 0, tail = 0;            // warp-uniform ring indices
    Cnt c;
    c.zero();
    constexpr int CH = 32 * PPT;
    const int64_t n_eff = effective_n(a);
    const int64_t nchunks = (n_eff + CH - 1) / CH;
    const int64_t gw = (int64_t)blockIdx.x * WARPS + warp, nw = (int64_t)gridDim.x * WARPS;
    for (int64_t ch = gw; ch < nchunks; ch += nw) {
        const int64_t base = ch * CH;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const int64_t i = base + k * 32 + lane;
            bool ev = false;
            T g = (T)0, chi = (T)0, aux = (T)-1;
            if (i < n_eff) {
                const uint8_t fl = a.flags[i];
                const bool photon_f = ((fl >> SFQ_SPECIES_SHIFT) & 3) == SFQ_PHOTON;
                if ((fl & SFQ_ALIVE) && !photon_f && a.lepton_model != SFQ_LEPTON_LCFA_OD) {
                    T E[3], B[3];
                    load_fields<T, FK>(a, i, E, B);
                    ev = blcfa_phase_a<T>(a, s_nlc, i, fl, a.px[i], a.py[i], a.pz[i], E, B, g, chi, aux, c);
                } else if (fl & SFQ_ALIVE) {
                    T E[3], B[3];
                    load_fields<T, FK>(a, i, E, B);
                    ev = step_particle<T, FK == FK_PW>(a, s_nlc, s_nbw, i, fl, a.px[i], a.py[i], a.pz[i], E, B,
                                                       a.tau[i], g, chi, c);
                }
            }
            const unsigned m = __ballot_sync(0xFFFFFFFFu, ev);
            if (ev) {
                const unsigned r = __popc(m & ((1u << lane) - 1u));
                QEntryX<T> e;
                e.i = i;
                e.g = g;
                e.chi = chi;
                e.aux = aux;
                q[(tail + r) & (QS - 1)] = e;
            }
            tail += __popc(m);
        }
        __syncwarp();
        while (tail - head >= 32u) {
            const QEntryX<T> e = q[(head + lane) & (QS - 1)];
            __syncwarp();
            head += 32;
            process_events<T, TRUNC, CASC, SURR>(a, e.i, e.g, e.chi, e.aux, a.px[e.i], a.py[e.i], a.pz[e.i], a.flags[e.i], true,
                                     c);
        }
    }
    // drain the partial batch
    __syncwarp();
    if (tail != head) {
        const unsigned nv = tail - head;
        const QEntryX<T> e = q[(head + lane) & (QS - 1)];
        const bool v = (unsigned)lane < nv;
        process_events<T, TRUNC, CASC, SURR>(a, e.i, e.g, e.chi, e.aux, v ? a.px[e.i] : (T)0, v ? a.py[e.i] : (T)0,
                          v ? a.pz[e.i] : (T)0, v ? a.flags[e.i] : (uint8_t)0, v, c);
    }
    flush_counters(c, a.counters);
}

}  // namespace sfq
