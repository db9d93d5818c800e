// sfq_step_tma.cuh -- the Monte Carlo step with the particle stream staged by TMA.
//
// One persistent CTA per SM: a producer warp copies each tile's structure-of-arrays
// slices (momenta, optical depth, flags, fields or phase index) from global to
// shared memory with 1D bulk copies (cp.async.bulk), NSTAGE tiles ahead, and 16
// consumer warps compute the step (Sec. 2 and 4 of Montefiori & Tamburini,
// arXiv:2301.07684) from shared memory.  A tile is cut into one slice per consumer warp;
// with fields in memory the warps claim the slices in order from a shared counter, so a
// warp busy with its events delays no stage's release.  Each consumer warp queues its event particles, with the
// state it read, in a ring of its own and samples them 32 at a time.  Stages are handed over with mbarriers
// (full: producer -> consumers, completed by the copies' transaction bytes;
// empty: consumers -> producer).  Every wait is bounded: on a timeout the kernel
// raises the timeout word of the counters and leaves its loops after its copies
// have landed.  The last, partial tile is read from global memory directly.
#pragma once
#include "sfq_step.cuh"

namespace sfq {

constexpr uint32_t TMA_WAIT_LIMIT = 1u << 24;   // try_wait polls before a wait is declared failed

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// Bounded wait for the phase of parity `parity` to complete: at most `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit = TMA_WAIT_LIMIT) {
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Layout of one stage for TILE particles.
template <typename T, int FK, int CW>
struct TmaStage {
    static constexpr int TILE = CW * (sizeof(T) == 4 ? 64 : 32);     // 2 (binary32) or 1 particle per lane
    static constexpr int NF = FK == FK_SOA ? 6 : 0;
    static constexpr size_t O_PX = 0, O_PY = O_PX + TILE * sizeof(T), O_PZ = O_PY + TILE * sizeof(T);
    static constexpr size_t O_TAU = O_PZ + TILE * sizeof(T);
    static constexpr size_t O_FL = O_TAU + TILE * 8;
    static constexpr size_t O_F = O_FL + TILE;                       // 6 field arrays (SoA)
    static constexpr size_t O_K0 = O_FL + TILE;                      // phase index (plane wave)
    static constexpr size_t O_AMP = O_K0 + TILE * 4;                 // amplitude (plane wave, optional)
    static constexpr size_t BYTES = FK == FK_SOA ? O_F + NF * TILE * sizeof(T) : O_AMP + TILE * sizeof(T);
};

// Dynamic shared memory of one CTA: NSTAGE stages, then the consumer warps' event queues
// (QS entries each: one tile's events plus a partial batch), then the mbarriers.  Three
// stages where they fit beside the queues and the static rate tables, else two.
template <typename T, int FK, int CW>
struct TmaCfg {
    using S = TmaStage<T, FK, CW>;
    static constexpr int PPL = S::TILE / CW / 32;                  // particles per lane per tile
    static constexpr int QS = 32 * (PPL + 1) <= 64 ? 64 : (32 * (PPL + 1) <= 128 ? 128 : 256);
    static constexpr size_t QBYTES = (size_t)CW * QS * sizeof(QEntry<T>);
    static constexpr size_t STATIC = (RateSmem<T>::NLC_N + RateSmem<T>::NBW_N) * sizeof(T);
    static constexpr size_t LIMIT = 227 * 1024;                    // shared memory per CTA
    static constexpr int NSTAGE = 3 * S::BYTES + QBYTES + STATIC + 1024 <= LIMIT ? 3 : 2;
    static constexpr size_t O_Q = (size_t)NSTAGE * S::BYTES;
    static constexpr size_t O_BAR = O_Q + QBYTES;
    static constexpr size_t SMEM = O_BAR + 2 * NSTAGE * sizeof(uint64_t) + 64;
    static_assert(S::BYTES % 16 == 0 && QBYTES % 16 == 0, "stage and queue offsets keep 16-byte alignment");
    static_assert(SMEM + STATIC <= LIMIT, "shared memory of the TMA-staged step");
};

template <typename T, int FK, int CW>
constexpr size_t tma_smem_bytes() {
    return TmaCfg<T, FK, CW>::SMEM;
}

// A wait that gave up is recorded in the counters.
__device__ __forceinline__ void raise_timeout(sfq_counters *c) {
    if (c) atomicAdd(&c->timeouts, 1ull);
}

// Check of the bounded waits: one thread waits, with the kernels' bounded wait, on an
// mbarrier that nothing completes (one arrival expected, none made), gives up after `polls`
// polls and records the timeout as the step kernel does.
template <int = 0>
__global__ void wait_check_kernel(uint32_t polls, sfq_counters *c) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (!mbar_wait(&bar, 0, polls)) raise_timeout(c);
    }
}

template <typename T, int FK, int CW, bool TRUNC = false, bool SURR = false>
__global__ void __launch_bounds__(32 * (CW + 1), 1) mc_step_tma_kernel(const StepArgs<T> a) {
    using Q = L<T>;
    using S = TmaStage<T, FK, CW>;
    using CFG = TmaCfg<T, FK, CW>;
    constexpr int TMA_NSTAGE = CFG::NSTAGE;
    constexpr int TMA_CONSUMER_WARPS = CW;
    constexpr int TMA_THREADS = 32 * (CW + 1);
    constexpr int TILE = S::TILE;
    constexpr int PER_WARP = TILE / TMA_CONSUMER_WARPS;    // particles per consumer warp per tile
    constexpr int PPL = CFG::PPL;                          // particles per lane per tile
    constexpr int QS = CFG::QS;                            // one tile + a partial batch
    constexpr bool PAIRED = sizeof(T) == 4 && PPL == 2;     // adjacent-pair vector layout
    extern __shared__ __align__(128) unsigned char smem[];
    QEntry<T> *wq = reinterpret_cast<QEntry<T> *>(smem + CFG::O_Q);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + CFG::O_BAR);
    uint64_t *empty = full + TMA_NSTAGE;
    int *abort_flag = reinterpret_cast<int *>(empty + TMA_NSTAGE);
    unsigned *slice_ctr = reinterpret_cast<unsigned *>(empty + TMA_NSTAGE + 1);
    using RS = RateSmem<T>;
    __shared__ __align__(16) T s_nlc[RS::NLC_N];
    __shared__ __align__(16) T s_nbw[RS::NBW_N];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    stage_rate_table<T, Q::NLC_DEG, RS::NLC_STRIDE>(s_nlc, a.tab.nlc_rate, Q::RATE_NLC_N / (Q::NLC_DEG + 1),
                                                     threadIdx.x, TMA_THREADS);
    stage_rate_table<T, Q::NBW_DEG, RS::NBW_STRIDE>(s_nbw, a.tab.nbw_rate, Q::RATE_NBW_N / (Q::NBW_DEG + 1),
                                                     threadIdx.x, TMA_THREADS);
    if (threadIdx.x == 0) {
        for (int s = 0; s < TMA_NSTAGE; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], TMA_CONSUMER_WARPS);
        }
        *abort_flag = 0;
        *slice_ctr = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const int64_t n_eff = effective_n(a);
    const int64_t ntiles = (n_eff + TILE - 1) / TILE;
    const bool has_amp = a.amp != nullptr;

    if (warp == TMA_CONSUMER_WARPS) {
        // ------------------------------------------------------------- producer
        if (lane == 0) {
            int issued_last[TMA_NSTAGE];
            for (int s = 0; s < TMA_NSTAGE; ++s) issued_last[s] = -1;
            for (int t = 0;; ++t) {
                const int64_t tile = blockIdx.x + (int64_t)t * gridDim.x;
                if (tile >= ntiles || *(volatile int *)abort_flag) break;
                const int s = t % TMA_NSTAGE;
                if (t >= TMA_NSTAGE && !mbar_wait(&empty[s], ((t / TMA_NSTAGE) - 1) & 1)) {
                    raise_timeout(a.counters);
                    *(volatile int *)abort_flag = 1;
                    break;
                }
                const int64_t start = tile * TILE;
                unsigned char *st = smem + (size_t)s * S::BYTES;
                if (start + TILE <= n_eff) {
                    const uint32_t bytes = (uint32_t)(FK == FK_SOA ? S::BYTES
                                                                   : (has_amp ? S::BYTES : S::O_AMP));
                    mbar_arrive_tx(&full[s], bytes);
                    bulk_g2s(st + S::O_PX, a.px + start, TILE * sizeof(T), &full[s]);
                    bulk_g2s(st + S::O_PY, a.py + start, TILE * sizeof(T), &full[s]);
                    bulk_g2s(st + S::O_PZ, a.pz + start, TILE * sizeof(T), &full[s]);
                    bulk_g2s(st + S::O_TAU, a.tau + start, TILE * 8, &full[s]);
                    bulk_g2s(st + S::O_FL, a.flags + start, TILE, &full[s]);
                    if (FK == FK_SOA) {
                        const T *fs[6] = {a.ex, a.ey, a.ez, a.bx, a.by, a.bz};
#pragma unroll
                        for (int f = 0; f < 6; ++f)
                            bulk_g2s(st + S::O_F + f * TILE * sizeof(T), fs[f] + start, TILE * sizeof(T), &full[s]);
                    } else {
                        bulk_g2s(st + S::O_K0, a.k0 + start, TILE * 4, &full[s]);
                        if (has_amp) bulk_g2s(st + S::O_AMP, a.amp + start, TILE * sizeof(T), &full[s]);
                    }
                } else {
                    mbar_arrive(&full[s]);          // partial tile: consumers read global memory
                }
                issued_last[s] = t;
            }
            // before leaving, every copy this warp issued has landed; a drain that times out is
            // counted (the step's results are then invalid) and waited for once more, so that the
            // block does not exit while its copies may still be writing its shared memory
            for (int s = 0; s < TMA_NSTAGE; ++s) {
                if (issued_last[s] < 0) continue;
                const uint32_t par = (issued_last[s] / TMA_NSTAGE) & 1;
                if (!mbar_wait(&full[s], par)) {
                    raise_timeout(a.counters);
                    mbar_wait(&full[s], par);
                }
            }
        }
        return;
    }

    // ------------------------------------------------------------------ consumers
    QEntry<T> *q = wq + (size_t)warp * QS;
    unsigned head = 0, tail = 0;
    Cnt c;
    c.zero();
    // With fields in memory (SoA) the step waits on HBM and on its events: a warp takes the
    // block's next slice (one warp's share, PER_WARP particles, of tile t) from a shared
    // counter, so a warp that is sampling its events leaves the next slices to the others
    // instead of holding up the release of their stage.  Slices are claimed in order and each
    // warp holds one claim, so no warp can wait on a stage two phases ahead.  With the plane
    // wave the step is bound by issue, and warp w keeps slice w of every tile (no claim).
    constexpr bool CLAIM = FK == FK_SOA;
    for (unsigned it = 0;; ++it) {
        unsigned g = it * TMA_CONSUMER_WARPS + (unsigned)warp;
        if constexpr (CLAIM) {
            if (lane == 0) g = atomicAdd(slice_ctr, 1u);
            g = __shfl_sync(0xFFFFFFFFu, g, 0);
        }
        const unsigned t = g / TMA_CONSUMER_WARPS;
        const int sl = (int)(g % TMA_CONSUMER_WARPS);
        const int64_t tile = blockIdx.x + (int64_t)t * gridDim.x;
        if (tile >= ntiles) break;
        const int s = (int)(t % TMA_NSTAGE);
        if (!mbar_wait(&full[s], (t / TMA_NSTAGE) & 1u)) {
            raise_timeout(a.counters);
            *(volatile int *)abort_flag = 1;
            break;
        }
        const int64_t start = tile * TILE;
        const bool staged = start + TILE <= n_eff;
        const unsigned char *st = smem + (size_t)s * S::BYTES;
        const T *spx = reinterpret_cast<const T *>(st + S::O_PX);
        const T *spy = reinterpret_cast<const T *>(st + S::O_PY);
        const T *spz = reinterpret_cast<const T *>(st + S::O_PZ);
        const double *stau = reinterpret_cast<const double *>(st + S::O_TAU);
        const uint8_t *sfl = st + S::O_FL;
        bool ev[PPL];
        T gk[PPL], ck[PPL], pk[PPL][3];
        uint8_t fk[PPL];
        if (staged && PAIRED) {
            // full tile, binary32: lane takes the adjacent particles li0, li0 + 1 (vector loads)
            const int li0 = sl * PER_WARP + 2 * lane;
            const float2 vx = *reinterpret_cast<const float2 *>(spx + li0);
            const float2 vy = *reinterpret_cast<const float2 *>(spy + li0);
            const float2 vz = *reinterpret_cast<const float2 *>(spz + li0);
            const double2 vt = *reinterpret_cast<const double2 *>(stau + li0);
            const uint16_t vf = *reinterpret_cast<const uint16_t *>(sfl + li0);
            float2 vE[3], vB[3];
            if (FK == FK_SOA) {
                const float *sf = reinterpret_cast<const float *>(st + S::O_F);
#pragma unroll
                for (int c3 = 0; c3 < 3; ++c3) {
                    vE[c3] = *reinterpret_cast<const float2 *>(sf + c3 * TILE + li0);
                    vB[c3] = *reinterpret_cast<const float2 *>(sf + (3 + c3) * TILE + li0);
                }
            }
            double tau_out[2] = {vt.x, vt.y};
            // the fields of particle li0 + k
            const auto fields = [&](int k, T E[3], T B[3]) {
                if (FK == FK_SOA) {
#pragma unroll
                    for (int c3 = 0; c3 < 3; ++c3) {
                        E[c3] = k == 0 ? vE[c3].x : vE[c3].y;
                        B[c3] = k == 0 ? vB[c3].x : vB[c3].y;
                    }
                } else {
                    uint32_t kk = reinterpret_cast<const uint32_t *>(st + S::O_K0)[li0 + k] + a.pw_offset;
                    kk -= (kk >= a.n_table) ? a.n_table : 0u;
                    kk = kk < a.n_table ? kk : a.n_table - 1u;
                    const T amp = has_amp ? reinterpret_cast<const T *>(st + S::O_AMP)[li0 + k] : a.amp0;
                    const T f = amp * __ldg(a.pw_table + kk);
                    E[0] = (T)0; E[1] = f; E[2] = (T)0;
                    B[0] = (T)0; B[1] = (T)0; B[2] = f;
                }
            };
            const uint8_t fl2[2] = {(uint8_t)(vf & 0xFF), (uint8_t)(vf >> 8)};
            const auto lepton = [](uint8_t fl) {
                return (fl & SFQ_ALIVE) && ((fl >> SFQ_SPECIES_SHIFT) & 3) != SFQ_PHOTON;
            };
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                pk[k][0] = k == 0 ? vx.x : vx.y;
                pk[k][1] = k == 0 ? vy.x : vy.y;
                pk[k][2] = k == 0 ? vz.x : vz.y;
                fk[k] = fl2[k];
            }
            bool done = false;
            if constexpr (PAIRED) {
                if (lepton(fl2[0]) && lepton(fl2[1])) {
                    // the common case: two alive leptons, stepped as one straight-line block
                    T E2[2][3], B2[2][3];
                    fields(0, E2[0], B2[0]);
                    fields(1, E2[1], B2[1]);
                    const T px2[2] = {vx.x, vx.y}, py2[2] = {vy.x, vy.y}, pz2[2] = {vz.x, vz.y};
                    step_lepton_pair<FK == FK_PW>(a, s_nlc, start + li0, fl2, px2, py2, pz2, E2, B2, tau_out, gk,
                                                  ck, ev, c);
                    done = true;
                }
            }
            if (!done) {
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    ev[k] = false;
                    gk[k] = (T)0;
                    ck[k] = (T)0;
                    if (fl2[k] & SFQ_ALIVE) {
                        T E[3], B[3];
                        fields(k, E, B);
                        ev[k] = step_particle_v<T, FK == FK_PW>(a, s_nlc, s_nbw, start + li0 + k, fl2[k], pk[k][0],
                                                                pk[k][1], pk[k][2], E, B, tau_out[k], gk[k], ck[k],
                                                                c, a.step);
                    }
                }
            }
            // both optical depths in one 16-byte store (an event particle's value is
            // rewritten later by this warp's event path)
            *reinterpret_cast<double2 *>(a.tau + start + li0) = make_double2(tau_out[0], tau_out[1]);
        } else if (staged) {
            // full tile: everything from shared memory, no bounds checks
#pragma unroll
            for (int k = 0; k < PPL; ++k) {
                const int li = sl * PER_WARP + k * 32 + lane;
                const uint8_t fl = sfl[li];
                ev[k] = false;
                gk[k] = (T)0;
                ck[k] = (T)0;
                pk[k][0] = spx[li];
                pk[k][1] = spy[li];
                pk[k][2] = spz[li];
                fk[k] = fl;
                if (fl & SFQ_ALIVE) {
                    T E[3], B[3];
                    if (FK == FK_SOA) {
                        const T *sf = reinterpret_cast<const T *>(st + S::O_F);
                        E[0] = sf[li]; E[1] = sf[TILE + li]; E[2] = sf[2 * TILE + li];
                        B[0] = sf[3 * TILE + li]; B[1] = sf[4 * TILE + li]; B[2] = sf[5 * TILE + li];
                    } else {
                        uint32_t kk = reinterpret_cast<const uint32_t *>(st + S::O_K0)[li] + a.pw_offset;
                        kk -= (kk >= a.n_table) ? a.n_table : 0u;
                        kk = kk < a.n_table ? kk : a.n_table - 1u;
                        const T amp = has_amp ? reinterpret_cast<const T *>(st + S::O_AMP)[li] : a.amp0;
                        const T f = amp * __ldg(a.pw_table + kk);
                        E[0] = (T)0; E[1] = f; E[2] = (T)0;
                        B[0] = (T)0; B[1] = (T)0; B[2] = f;
                    }
                    ev[k] = step_particle<T, FK == FK_PW>(a, s_nlc, s_nbw, start + li, fl, pk[k][0], pk[k][1], pk[k][2], E, B,
                                             stau[li], gk[k], ck[k], c);
                }
            }
        } else {
            // last, partial tile: global memory with bounds checks
#pragma unroll
            for (int k = 0; k < PPL; ++k) {
                const int li = sl * PER_WARP + k * 32 + lane;
                const int64_t i = start + li;
                ev[k] = false;
                gk[k] = (T)0;
                ck[k] = (T)0;
                pk[k][0] = pk[k][1] = pk[k][2] = (T)0;
                fk[k] = 0;
                if (i < n_eff) {
                    const uint8_t fl = a.flags[i];
                    fk[k] = fl;
                    if (fl & SFQ_ALIVE) {
                        T E[3], B[3];
                        load_fields<T, FK>(a, i, E, B);
                        pk[k][0] = a.px[i]; pk[k][1] = a.py[i]; pk[k][2] = a.pz[i];
                        ev[k] = step_particle<T, FK == FK_PW>(a, s_nlc, s_nbw, i, fl, pk[k][0], pk[k][1], pk[k][2], E, B, a.tau[i],
                                                 gk[k], ck[k], c);
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            const unsigned m = __ballot_sync(0xFFFFFFFFu, ev[k]);
            if (ev[k]) {
                const unsigned r = __popc(m & ((1u << lane) - 1u));
                QEntry<T> e;
                e.i = (staged && PAIRED) ? start + sl * PER_WARP + 2 * lane + k
                                         : start + sl * PER_WARP + k * 32 + lane;
                e.g = gk[k];
                e.chi = ck[k];
                e.px = pk[k][0];
                e.py = pk[k][1];
                e.pz = pk[k][2];
                e.fl = fk[k];
                q[(tail + r) & (QS - 1)] = e;
            }
            tail += __popc(m);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);        // this slice of the stage is done
        while (tail - head >= 32u) {
            const QEntry<T> e = q[(head + lane) & (QS - 1)];
            __syncwarp();
            head += 32;
            process_events<T, TRUNC, false, SURR>(a, e.i, e.g, e.chi, (T)-1, e.px, e.py, e.pz, (uint8_t)e.fl, true, c);
        }
    }
    __syncwarp();
    if (tail != head) {
        const unsigned nv = tail - head;
        const QEntry<T> e = q[(head + lane) & (QS - 1)];
        process_events<T, TRUNC, false, SURR>(a, e.i, e.g, e.chi, (T)-1, e.px, e.py, e.pz, (uint8_t)e.fl, (unsigned)lane < nv,
                                 c);
    }
    // counters of the consumer warps (the producer warp has returned)
    if (a.counters) {
#pragma unroll
        for (int k = 0; k < (SURR ? 13 : 12); ++k) {
            unsigned long long v = (unsigned long long)c.v[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
            if (lane == 0 && v) atomicAdd(reinterpret_cast<unsigned long long *>(a.counters) + (k < 12 ? k : 13), v);
        }
    }
}

}  // namespace sfq
