// sfq_fused.cuh -- many Monte Carlo steps in one launch for the analytic plane-wave field,
// each particle's state held in registers from the first step to the last.
//
// The per-step interface reads momenta, optical depth and fields from memory and writes
// them back at every step (Sec. 2 of Montefiori & Tamburini, arXiv:2301.07684, with the
// fields a PIC code provides).  When the field is the analytic wave E = (0, a C, 0),
// B = (0, 0, a C), C = cos table[(k0 + step k_step) mod K], nothing has to leave the SM
// between steps: this kernel loads a particle once, runs steps step0 ... step0+nsteps-1
// on it and stores it once.  The arithmetic of every update and of every event is the
// per-step kernels' own (step_particle_v with the plane-wave chi, process_events_core),
// so the records, final states and counters equal those of nsteps sfq_mc_step calls.
//
// Each lane holds PPL particles ("slots"), each with its own step counter.  An update
// that ends in an event puts the slot on the warp's event queue and the slot waits; the
// other slots keep stepping.  The queue is sampled 32 events at a time, the parents' new
// states are handed back through shared memory and the waiting slots resume.  A partial
// batch is sampled only when no slot of the warp can step.  So the sampler, whose cost is
// per batch, always runs on full batches except at the end of a chunk of particles.
#pragma once
#include "sfq_step.cuh"

namespace sfq {

constexpr int FUSED_BS = 256;                  // threads per block
constexpr int FUSED_TABLE_MAX = SFQ_FUSED_TABLE_MAX;   // largest cosine table (kept in shared memory)

template <typename T>
struct FEntry {                                // queued event
    int64_t i;
    T g, chi, px, py, pz;
    uint32_t step;
    uint32_t fl;
};

template <typename T, int PPL>
struct FusedCfg {
    static constexpr int WARPS = FUSED_BS / 32;
    static constexpr int QS = 32 * PPL;        // one pending event per slot at most
    static constexpr size_t O_RES = (size_t)WARPS * QS * sizeof(FEntry<T>);
    static constexpr size_t O_TAB = O_RES + (size_t)WARPS * QS * sizeof(EvOut<T>);
    static size_t smem(uint32_t n_table) { return O_TAB + (size_t)n_table * sizeof(T); }
    static_assert(O_RES % 16 == 0 && O_TAB % 16 == 0, "shared-memory offsets keep 16-byte alignment");
};

// kstep: k_step mod K; off0: (step0 k_step) mod K.
template <typename T, int PPL, bool TRUNC = false>
__global__ void __launch_bounds__(FUSED_BS, 2) mc_fused_kernel(const StepArgs<T> a, uint32_t step0, uint32_t nsteps,
                                                            uint32_t off0, uint32_t kstep) {
    using Q = L<T>;
    using CFG = FusedCfg<T, PPL>;
    constexpr int QS = CFG::QS;
    using RS = RateSmem<T>;
    __shared__ __align__(16) T s_nlc[RS::NLC_N];
    __shared__ __align__(16) T s_nbw[RS::NBW_N];
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    FEntry<T> *q = reinterpret_cast<FEntry<T> *>(smem) + (size_t)warp * QS;
    EvOut<T> *res = reinterpret_cast<EvOut<T> *>(smem + CFG::O_RES) + (size_t)warp * QS;
    T *s_tab = reinterpret_cast<T *>(smem + CFG::O_TAB);

    stage_rate_table<T, Q::NLC_DEG, RS::NLC_STRIDE>(s_nlc, a.tab.nlc_rate, Q::RATE_NLC_N / (Q::NLC_DEG + 1),
                                                     threadIdx.x, FUSED_BS);
    stage_rate_table<T, Q::NBW_DEG, RS::NBW_STRIDE>(s_nbw, a.tab.nbw_rate, Q::RATE_NBW_N / (Q::NBW_DEG + 1),
                                                     threadIdx.x, FUSED_BS);
    const uint32_t K = a.n_table;
    for (uint32_t k = threadIdx.x; k < K; k += FUSED_BS) s_tab[k] = a.pw_table[k];
    __syncthreads();

    Cnt c;
    c.zero();
    constexpr int CH = 32 * PPL;
    const int64_t n_eff = effective_n(a);
    const int64_t nchunks = (n_eff + CH - 1) / CH;
    const int64_t gw = (int64_t)blockIdx.x * CFG::WARPS + warp, nw = (int64_t)gridDim.x * CFG::WARPS;
    for (int64_t ch = gw; ch < nchunks; ch += nw) {
        const int64_t base = ch * CH;
        T px[PPL], py[PPL], pz[PPL], amp[PPL];
        double tau[PPL];
        uint32_t fl[PPL], st[PPL], off[PPL], k0[PPL], pos[PPL];
        bool pend[PPL], in[PPL];
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            const int64_t i = base + k * 32 + lane;
            in[k] = i < n_eff;
            px[k] = py[k] = pz[k] = amp[k] = (T)0;
            tau[k] = 0.0;
            fl[k] = 0u;
            k0[k] = 0u;
            if (in[k]) {
                px[k] = a.px[i]; py[k] = a.py[i]; pz[k] = a.pz[i];
                tau[k] = a.tau[i];
                fl[k] = a.flags[i];
                k0[k] = a.k0[i];
                amp[k] = a.amp ? a.amp[i] : a.amp0;
            }
            st[k] = 0u;
            off[k] = off0;
            pend[k] = false;
            pos[k] = 0u;
        }
        unsigned qt = 0, qh = 0;               // warp-uniform queue tail and head
        for (;;) {
            bool ran = false;
#pragma unroll
            for (int k = 0; k < PPL; ++k) {
                const int64_t i = base + k * 32 + lane;
                const bool run = in[k] && (fl[k] & SFQ_ALIVE) && !pend[k] && st[k] < nsteps;
                bool ev = false;
                T g = (T)0, chi = (T)0;
                if (run) {
                    ran = true;
                    uint32_t kk = k0[k] + off[k];               // as the per-step field source
                    kk -= (kk >= K) ? K : 0u;
                    kk = kk < K ? kk : K - 1u;
                    const T f = amp[k] * s_tab[kk];
                    const T E[3] = {(T)0, f, (T)0}, B[3] = {(T)0, (T)0, f};
                    ev = step_particle_v<T, true>(a, s_nlc, s_nbw, i, (uint8_t)fl[k], px[k], py[k], pz[k], E, B,
                                                  tau[k], g, chi, c, step0 + st[k]);
                    if (!ev) {
                        ++st[k];
                        off[k] += kstep;
                        off[k] -= (off[k] >= K) ? K : 0u;
                    }
                }
                const unsigned m = __ballot_sync(0xFFFFFFFFu, ev);
                if (ev) {
                    const unsigned r = qt + __popc(m & ((1u << lane) - 1u));
                    FEntry<T> e;
                    e.i = i;
                    e.g = g;
                    e.chi = chi;
                    e.px = px[k]; e.py = py[k]; e.pz = pz[k];
                    e.step = step0 + st[k];
                    e.fl = fl[k];
                    q[r & (QS - 1)] = e;
                    pend[k] = true;
                    pos[k] = r;
                }
                qt += __popc(m);
            }
            const bool any_ran = __any_sync(0xFFFFFFFFu, ran);
            if (!any_ran && qt == qh) break;              // every slot finished
            // sample full batches; a partial one only when no slot could step
            while (qt - qh >= 32u || (!any_ran && qt != qh)) {
                __syncwarp();
                const unsigned nb = qt - qh < 32u ? qt - qh : 32u;
                const bool v = (unsigned)lane < nb;
                FEntry<T> e{};
                if (v) e = q[(qh + lane) & (QS - 1)];
                EvOut<T> o;
                process_events_core<T, TRUNC>(a, e.step, e.i, e.g, e.chi, (T)-1, e.px, e.py, e.pz, (uint8_t)e.fl, v,
                                              c, o);
                if (v) res[(qh + lane) & (QS - 1)] = o;
                __syncwarp();
                // the waiting slots take their new state and finish their step
#pragma unroll
                for (int k = 0; k < PPL; ++k) {
                    if (pend[k] && pos[k] - qh < nb) {
                        const EvOut<T> r = res[pos[k] & (QS - 1)];
                        if (r.what & 1) { px[k] = r.px; py[k] = r.py; pz[k] = r.pz; }
                        if (r.what & 2) tau[k] = r.tau;
                        if (r.what & 4) fl[k] = r.fl;
                        pend[k] = false;
                        ++st[k];
                        off[k] += kstep;
                        off[k] -= (off[k] >= K) ? K : 0u;
                    }
                }
                qh += nb;
                if (!any_ran) break;                      // re-check which slots can step
            }
        }
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            const int64_t i = base + k * 32 + lane;
            if (in[k]) {
                a.px[i] = px[k]; a.py[i] = py[k]; a.pz[i] = pz[k];
                a.tau[i] = tau[k];
                a.flags[i] = (uint8_t)fl[k];
            }
        }
    }
    flush_counters(c, a.counters);
}

}  // namespace sfq
