/*
 * sfq.h -- C ABI of libsfq, a GB300 (sm_103a) implementation of the per-particle,
 * per-timestep strong-field QED Monte Carlo step of Montefiori & Tamburini,
 * "SFQEDtoolkit" (arXiv:2301.07684): nonlinear Compton photon emission (NLC) and
 * nonlinear Breit-Wheeler pair creation (NBW) in the locally-constant-field
 * approximation (LCFA), and photon emission beyond it (BLCFA, Sec. 5).
 *
 * Conventions for every entry point
 *  - Units are the paper's normalised units (Sec. 4.1, App. A): times in 1/omega_r,
 *    fields in E_r = m c omega_r/|e| (B in E_r/c), momenta in m c, energies in m c^2.
 *  - Floating-point buffers hold binary32 when the context was created with
 *    SFQ_FP32 and binary64 with SFQ_FP64 ("real" below).  The optical depth is
 *    binary64 in both.
 *  - Buffers are device pointers owned by the caller, 16-byte aligned; they are not
 *    retained after the call returns.  Sizes are element counts (int64_t).
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *    Work is enqueued asynchronously; argument errors are returned synchronously
 *    and nothing is enqueued.  Conditions found on the device (buffer overflow,
 *    chi outside the fitted range, NaN input) are counted in sfq_counters and never
 *    stop the kernel.
 *  - No entry point falls back to the CPU.  Every call returns an sfq_status;
 *    sfq_last_error() gives a message for the last failure of a context.
 */
#ifndef SFQ_H
#define SFQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SFQ_OK = 0,
    SFQ_ERR_ARG = 1,       /* invalid argument: NULL, misaligned, negative size, bad enum */
    SFQ_ERR_CUDA = 2,      /* a CUDA runtime call failed (message in sfq_last_error) */
    SFQ_ERR_CAPACITY = 3,  /* reported by sfq_counters_check: product records or children were dropped */
    SFQ_ERR_TABLE = 4,     /* sfq_init: a fitted table is missing, of inconsistent size, or not finite */
    SFQ_ERR_RANGE = 5,     /* reported by sfq_counters_check: inputs outside the fitted range, or NaN */
    SFQ_ERR_TIMEOUT = 6    /* reported by sfq_counters_check: a bounded device wait gave up */
} sfq_status;

enum { SFQ_FP32 = 0, SFQ_FP64 = 1 };

/* Library configuration, the counterpart of SFQED_INIT_ALL_ref_len / _ref_freq
 * (App. A, functions 1 and 2). */
typedef struct {
    double ref_len_m;      /* reference length lambda_r = c/omega_r in metres, or 0 */
    double ref_omega_si;   /* reference angular frequency omega_r in rad/s, or 0; exactly one > 0 */
    double dt;             /* timestep in units of 1/omega_r (> 0) */
    int32_t precision;     /* SFQ_FP32 (binary32 arithmetic, binary64 optical depth) or SFQ_FP64 */
    int32_t device;        /* CUDA device ordinal the context uses */
    uint64_t seed;         /* key of the Philox4x32-10 generator */
} sfq_config;

typedef struct sfq_ctx sfq_ctx;   /* opaque; owns the approximation tables on the device */

/* Create a context: validates the configuration, uploads the fitted tables of
 * this library to the device.  *out receives the context (NULL on failure).
 * Returns SFQ_ERR_ARG for an invalid configuration, SFQ_ERR_CUDA on a device error. */
sfq_status sfq_init(const sfq_config *cfg, sfq_ctx **out);

/* Free the context and its device tables (App. A, function 14).  NULL is ignored. */
void sfq_finalize(sfq_ctx *ctx);

/* Message describing the last error of this context ("" if none).  The string is
 * owned by the context. */
const char *sfq_last_error(const sfq_ctx *ctx);

/* Constants of the context: rho = lambda_r/lambda_C (the critical field in units of
 * E_r, and 1/tau_C in units of 1/omega_r) and pref = alpha/(sqrt(3) pi) * rho, the
 * common factor of Eq. pe_rate_3 and Eq. pp_tot_real. */
sfq_status sfq_constants(const sfq_ctx *ctx, double *rho, double *pref);

/* ------------------------------------------------------------------------- */
/* Rates (App. A functions 5 and 6)                                            */
/* ------------------------------------------------------------------------- */
/* rate[i] = W_rad(gamma[i], chi[i]) = pref (chi/gamma) W~_rad(chi), Eq. pe_rate_3 with
 * Eq. wtilde, in units of omega_r.  Inputs real[n]: lepton energy gamma (m c^2) and
 * quantum parameter chi >= 0; output real[n].  chi above 2^20 is evaluated at 2^20 and
 * counted; NaN gives 0.  `counters` may be NULL. */
struct sfq_counters;
sfq_status sfq_photon_rate(sfq_ctx *ctx, int64_t n, const void *gamma, const void *chi, void *rate,
                           struct sfq_counters *counters, void *stream);

/* rate[i] = W_pair(gamma[i], chi[i]) = pref W~_pair(chi)/gamma, Eq. pp_tot_real with
 * Eq. wtilde_pair; 0 for chi < 0.01, where the paper neglects the process (Sec. 4.2). */
sfq_status sfq_pair_rate(sfq_ctx *ctx, int64_t n, const void *gamma, const void *chi, void *rate,
                         struct sfq_counters *counters, void *stream);

/* ------------------------------------------------------------------------- */
/* Random numbers and energy sampling (App. A functions 9 and 11)              */
/* ------------------------------------------------------------------------- */
/* Four uniforms per particle from Philox4x32-10 with key = seed and counter
 * (id_lo, id_hi, step, tag): u[4i+k] = (floor(w_k / 2^9) + 1/2) 2^-23 (real).
 * Word 0 resets the optical depth (or is r of the local test), word 1 is the r of
 * the energy sampling, word 2 the r_2 of the BLCFA rejection, word 3 the first
 * optical depth of a particle created without one.  id: uint64[n] device. */
sfq_status sfq_uniforms(sfq_ctx *ctx, int64_t n, const uint64_t *id, uint32_t step, uint32_t tag,
                        void *u, void *stream);

/* Photon energy fraction by inverse-transform sampling, Eq. ITS_pe in the form of
 * Eq. again: w-bar solves I~_pe(w, chi) = r W~_rad(chi) (Eq. pe_eff_int_2), s = 3 chi w^3/2
 * (Eq. subs_altri), xi = eps_gamma/eps_e = s/(1+s).  Inputs real[n] chi (>= 0) and r in
 * (0,1); outputs real[n] xi and, if xi_c != NULL, xi_c = 1 - xi = 1/(1+s) with relative
 * precision.  chi above 2^12 and 1 - r below 2^-24 are clamped and counted. */
sfq_status sfq_sample_photon_xi(sfq_ctx *ctx, int64_t n, const void *chi, const void *r, void *xi,
                                void *xi_c, struct sfq_counters *counters, void *stream);

/* Electron energy share by inverse-transform sampling, Eq. again_pp: r' = 2r - 1,
 * v-bar solves I~_pp(v, chi) = |r'| W~_pair(chi) (Eq. tilde_I_pp), xi_e = (1 + sgn(r') v)/2
 * (Eq. return_to_nrg).  Outputs real[n] xi_e and, if xi_p != NULL, the positron share
 * 1 - xi_e, both with relative precision.  chi outside [2^-7, 2^12) is clamped and counted. */
sfq_status sfq_sample_pair_xi(sfq_ctx *ctx, int64_t n, const void *chi, const void *r, void *xi_e,
                              void *xi_p, struct sfq_counters *counters, void *stream);

/* ------------------------------------------------------------------------- */
/* The Monte Carlo step                                                         */
/* ------------------------------------------------------------------------- */
/* Per-particle flags (uint8). */
enum {
    SFQ_ALIVE = 1,          /* the particle takes part in the step */
    SFQ_JUST_CREATED = 2,   /* BLCFA: no force history yet (Sec. 5, App. A function 15) */
    SFQ_SPECIES_SHIFT = 2,  /* bits 2-3: SFQ_ELECTRON, SFQ_POSITRON or SFQ_PHOTON */
    SFQ_TAG_SHIFT = 4       /* bits 4-5: tag, the 4th word of the Philox counter */
};
enum { SFQ_ELECTRON = 0, SFQ_POSITRON = 1, SFQ_PHOTON = 2 };
/* Lepton emission models: LCFA with the optical-depth method; beyond-LCFA (Sec. 5) by the
 * local method with the Lorentz force E + beta x B at the particle; beyond-LCFA with the
 * force taken from the pusher (Eqs. fl): the step first advances p^(n-1/2) by one Boris push
 * (as sfq_push) to p^(n+1/2), which the particle keeps, and uses
 * F_L = (p^(n+1/2) - p^(n-1/2)) / dt at p_L = (p^(n+1/2) + p^(n-1/2)) / 2. */
enum { SFQ_LEPTON_LCFA_OD = 0, SFQ_LEPTON_BLCFA_LOCAL = 1, SFQ_LEPTON_BLCFA_PUSHED = 2 };

/* Structure-of-arrays particle population (all device pointers). */
typedef struct {
    int64_t n;                /* number of particles */
    void *px, *py, *pz;       /* real[n] momentum (in/out) */
    double *tau;              /* binary64[n] optical depth tau_d (Sec. 2); negative = draw at the next step */
    const uint64_t *id;       /* uint64[n] particle ids (Philox counter), or NULL: id = id_base + index */
    uint64_t id_base;
    uint8_t *flags;           /* uint8[n] (in/out) */
    void *fprev[3];           /* real[n] each: BLCFA F_perp^(n-1) (in/out), NULL if unused */
    void *dfprev[3];          /* real[n] each: BLCFA F_perp^(n-1) - F_perp^(n-2) (in/out) */
    int32_t lepton_model;     /* SFQ_LEPTON_LCFA_OD, SFQ_LEPTON_BLCFA_LOCAL or SFQ_LEPTON_BLCFA_PUSHED */
    int32_t reserved;
    const unsigned long long *n_dev;  /* optional device count: the step covers min(*n_dev, n)
                                         particles (a population grown on the device, e.g. the
                                         children of sfq_spawn); NULL = n */
} sfq_particles;

enum { SFQ_FIELDS_SOA = 0, SFQ_FIELDS_PLANE_WAVE = 1 };

/* Fields at the particles for this step.
 *  SFQ_FIELDS_SOA: ex..bz real[n] each (the fields a PIC code interpolates to the particles).
 *  SFQ_FIELDS_PLANE_WAVE: a linearly polarised wave along +x,
 *    E = (0, a C, 0), B = (0, 0, a C), C = table[(k0[i] + step * k_step) mod n_table],
 *    a = amp[i] (real[n]) or amp0 when amp == NULL; the product a*C is formed in the
 *    context's precision. */
typedef struct {
    int32_t kind;
    int32_t reserved;
    const void *ex, *ey, *ez, *bx, *by, *bz;
    const uint32_t *k0;
    const void *amp;
    double amp0;
    const void *table;
    uint32_t n_table;
    uint32_t k_step;
} sfq_fields;

/* Product records, appended by the step (device pointers, capacity elements each). */
typedef struct {
    int64_t capacity;
    void *px, *py, *pz;       /* real[capacity]: collinear momentum (Sec. 4, App. A function 17) */
    uint64_t *parent_id;      /* uint64[capacity] */
    uint32_t *step;           /* uint32[capacity]: step of creation */
    uint8_t *meta;            /* uint8[capacity]: species | member << 2 | parent tag << 4;
                                 member 0 = emitted photon, 1 = electron, 2 = positron */
    unsigned long long *count;/* device counter of requested records (caller zeroes it);
                                 records at index >= capacity are dropped and counted */
} sfq_products;

/* Optional stepped children: leptons created by pair creation are appended here
 * as particles (flags ALIVE | JUST_CREATED | species | member tag, id = parent id,
 * tau = -1, BLCFA state 0, k0/amp copied from the parent).  */
typedef struct {
    sfq_particles p;          /* p.n is the capacity */
    uint32_t *k0;             /* uint32[capacity] or NULL */
    void *amp;                /* real[capacity] or NULL */
    unsigned long long *count;/* device counter of requested children */
} sfq_spawn;

/* Device counters (binary layout shared with the host; zero before use). */
typedef struct sfq_counters {
    unsigned long long updates;          /* particle-updates performed */
    unsigned long long events;           /* events deemed to occur (Sec. 2 tests) */
    unsigned long long emitted;          /* photons emitted (after BLCFA acceptance) */
    unsigned long long pairs;            /* photons converted */
    unsigned long long dropped;          /* product records beyond capacity */
    unsigned long long spawn_dropped;    /* children beyond capacity */
    unsigned long long out_of_range;     /* chi beyond the fitted tables (clamped) */
    unsigned long long nan_input;        /* NaN chi or gamma (treated as zero rate) */
    unsigned long long gamma_below_one;  /* products with gamma < 1 (|p| set to 0) */
    unsigned long long large_rdt;        /* R dt > 0.1 (Sec. 2: R dt << 1 is assumed) */
    unsigned long long blcfa_no_emission;/* threshold >= 0.75 gamma (Sec. 5) */
    unsigned long long blcfa_rejected;   /* rejected by Eq. rej_cond */
    unsigned long long timeouts;         /* bounded device waits that gave up (0 in a correct run) */
    unsigned long long surrogate_fallbacks; /* surrogate draws taken by the plain sampler */
    unsigned long long reserved[2];
} sfq_counters;

/* Status of a run from a HOST copy of its counters (copy them back after the stream has
 * synchronised): SFQ_ERR_TIMEOUT if a bounded device wait gave up (the run's results are
 * then invalid), else SFQ_ERR_CAPACITY if product records or children were dropped, else
 * SFQ_ERR_RANGE if chi fell outside the fitted range (evaluated clamped) or an input was
 * NaN, else SFQ_OK.  SFQ_ERR_ARG for NULL.  Reads no device memory and needs no context. */
sfq_status sfq_counters_check(const sfq_counters *host_counters);

/* Check of the bounded device waits the kernels use (no counterpart in the paper): one CTA
 * waits, with the step kernel's bounded mbarrier wait, on a barrier that nothing completes,
 * gives up after `polls` polls, adds 1 to counters->timeouts and returns, so that a host
 * can see that a wait which gives up is reported and leaves the context usable.
 * polls in [1, 65536] (else SFQ_ERR_ARG); `counters` a device pointer, not NULL.
 * Asynchronous on `stream`. */
sfq_status sfq_check_bounded_wait(sfq_ctx *ctx, uint32_t polls, sfq_counters *counters, void *stream);

/* Check of the binary32 square roots every kernel uses for gamma = sqrt(1 + p^2), |p| and
 * 1/gamma: the hardware reciprocal-square-root estimate refined by one Newton step (about
 * 1 ulp).  For each of the n device values x[i] writes sqrt_out[i] (0 for x <= 0 or NaN)
 * and rsqrt_out[i] (defined for finite x > 0), so that a test can compare them with
 * correctly rounded results.  All pointers are device pointers of n floats (n >= 0; NULL only when
 * n == 0).  Asynchronous on `stream`. */
sfq_status sfq_check_sqrt(sfq_ctx *ctx, int64_t n, const float *x, float *sqrt_out, float *rsqrt_out, void *stream);

/* One Monte Carlo step for every alive particle of `p` (Sec. 2 and 4; Sec. 5 for
 * BLCFA leptons):
 *   chi (Eq. chi_exact) -> rate (Eq. pe_rate_3 / Eq. pp_tot_real) -> leptons with
 *   SFQ_LEPTON_LCFA_OD and photons: tau_d -= R dt (binary64), event iff tau_d < 0, then
 *   a fresh tau from word 0; BLCFA leptons: local test R dt > r (word 0) with the
 *   threshold and rejection of Sec. 5 -> energy sampling (word 1) -> recoil of the
 *   emitter or removal of the converted photon -> product records (and children).
 * `step` is the timestep number (Philox counter word 2 and the plane-wave phase).
 * `spawn` and `counters` may be NULL.  Counters are accumulated with atomics. */
sfq_status sfq_mc_step(sfq_ctx *ctx, const sfq_particles *p, const sfq_fields *f, uint32_t step,
                       const sfq_products *out, const sfq_spawn *spawn, sfq_counters *counters,
                       void *stream);

/* `nsteps` consecutive steps step0 ... step0+nsteps-1, recorded once into a CUDA graph and
 * replayed (the graph is cached in the context for the same arguments, so a repeated call
 * costs one graph launch).  Each step runs `children` first (if not NULL: a population
 * with its own field source, typically the sfq_spawn target of `p` with a device count)
 * and then `p`; it is equivalent to calling sfq_mc_step in that order for every step.
 * The call must not be made while `stream` is being captured. */
sfq_status sfq_mc_run(sfq_ctx *ctx, const sfq_particles *p, const sfq_fields *f, const sfq_particles *children,
                      const sfq_fields *children_fields, uint32_t step0, uint32_t nsteps, const sfq_products *out,
                      const sfq_spawn *spawn, sfq_counters *counters, void *stream);

/* Steps step0 ... step0+nsteps-1 of `p` in the analytic plane-wave field, fused into one
 * launch: each particle is loaded once, stepped nsteps times with its momentum, optical
 * depth, flags and phase held in registers, and stored once, so the run reads and writes
 * the population once instead of once per step.  Per update and per event it performs
 * exactly the arithmetic of sfq_mc_step (Sec. 2 and 4: chi, rate, binary64 optical depth,
 * Philox draws keyed by the particle's own step, energy sampling, recoil), so the product
 * records (in another order), the final state and the counters equal those of sfq_mc_step
 * called for step0, step0+1, ... in turn without children.
 * Requirements (else SFQ_ERR_ARG): f->kind == SFQ_FIELDS_PLANE_WAVE with
 * n_table <= SFQ_FUSED_TABLE_MAX; p->lepton_model == SFQ_LEPTON_LCFA_OD; step0 + nsteps
 * < 2^32.  Photons that convert are removed and leave their two product records; their
 * leptons are not stepped (no sfq_spawn).  Buffers and alignment as for sfq_mc_step;
 * `out` must hold the records of all nsteps steps (records past its capacity are counted
 * as dropped).  Asynchronous on `stream`. */
#define SFQ_FUSED_TABLE_MAX 8192
sfq_status sfq_mc_run_fused(sfq_ctx *ctx, const sfq_particles *p, const sfq_fields *f, uint32_t step0,
                            uint32_t nsteps, const sfq_products *out, sfq_counters *counters, void *stream);

/* Full cascade (every product is stepped again): `nsteps` steps step0 ... of a population
 * that grows by its own products.  Each step is the step of sfq_mc_step (Sec. 2 and 4, and
 * Sec. 5 for beyond-LCFA leptons) over the particles [0, *p->n_dev), and every product of
 * the step -- the photon of an emission, the two leptons of a conversion -- is also
 * appended to `p` as a particle: momentum of its record, tau = -1 (drawn at its first step),
 * flags ALIVE | JUST_CREATED | species with tag 0, BLCFA state 0, k0 and amp copied from the
 * parent, and its own id: bit 63 over the first two Philox words of the counter
 * (parent id lo, parent id hi, step, 0x100 | parent tag << 2 | member) under the seed
 * (member 0 photon, 1 electron, 2 positron).  A particle appended during a step is stepped
 * from the next step on; after each step *p->n_dev = min(appended total, p->n).  Product
 * records are written to `out` as by sfq_mc_step.
 *   p: p->n is the capacity; p->n_dev (device uint64, in/out) the live count; p->id
 *      (uint64[capacity], written for appended particles, kept below 2^63 for primaries so
 *      that descendants are told apart) must not be NULL.
 *   f: SFQ_FIELDS_PLANE_WAVE with k0 (and amp, if not NULL) of capacity elements; the
 *      cascade writes them for appended particles, so every descendant sees the wave at
 *      its primary's phase.
 *   next: device uint64 scratch (the append counter of a step).
 * Particles that would be appended beyond the capacity are counted in spawn_dropped and
 * lost; a caller that must lose none keeps 3 * count <= capacity per step (each particle
 * creates at most two) and makes room with sfq_cascade_compact.  Asynchronous on `stream`;
 * SFQ_ERR_ARG for invalid descriptors. */
sfq_status sfq_cascade_run(sfq_ctx *ctx, const sfq_particles *p, const sfq_fields *f, unsigned long long *next,
                           uint32_t step0, uint32_t nsteps, const sfq_products *out, sfq_counters *counters,
                           void *stream);

/* Stream compaction of a cascade population: the alive particles of src [0, *src->n_dev)
 * are moved, in their order, to dst [0, m), and *dst->n_dev = m.  Every per-particle array
 * moves: momentum, tau, id, flags, the BLCFA state (when src->lepton_model uses it) and the
 * plane-wave k0 and amp of fsrc -> fdst.  dst->n (its capacity) must be at least src->n, so
 * a larger dst also grows the population.  The buffers of src and dst must not overlap.
 * `scratch` (device, 16-byte aligned) holds sfq_cascade_compact_scratch_bytes(src->n) bytes.
 * Asynchronous on `stream`. */
size_t sfq_cascade_compact_scratch_bytes(int64_t capacity);
sfq_status sfq_cascade_compact(sfq_ctx *ctx, const sfq_particles *src, const sfq_fields *fsrc,
                               const sfq_particles *dst, const sfq_fields *fdst, void *scratch, size_t scratch_bytes,
                               void *stream);

/* One Boris push of the momenta (Boris 1970), the particle pusher a PIC code runs between
 * Monte Carlo steps; the paper's library leaves it to the host code.  For every alive
 * electron (charge -1) and positron (+1) of `p`, in the fields `f` at `step` (as
 * sfq_mc_step reads them): u- = u + q E dt/2, t = q B dt / (2 gamma(u-)),
 * s = 2 t / (1 + t.t), u+ = u- + (u- + u- x t) x s, u = u+ + q E dt/2, in the normalised
 * units of the step (u = p / m c, fields in E_r, dt in 1/omega_r).  Photons and dead
 * particles are left unchanged; positions are not tracked.  dt must be positive and finite,
 * buffers as for sfq_mc_step, else SFQ_ERR_ARG.  Asynchronous on `stream`. */
sfq_status sfq_push(sfq_ctx *ctx, const sfq_particles *p, const sfq_fields *f, uint32_t step, double dt,
                    void *stream);

/* Options of a context.  Both are read when work is enqueued; a CUDA graph recorded by
 * sfq_mc_run keeps the options it was recorded with, and a later call with other options
 * records a new graph.
 *
 * Pair-rate cutoff: the NBW rate (sfq_pair_rate and the photon step) is zero below
 * chi_min.  The default 0.01 is the lower end of the fitted domain (Sec. 4.2).  The paper's
 * "fast" rate returns zero below chi = 0.3, where W_pair <~ 9.1e-6 alpha rho / gamma
 * (Sec. 4.2, App. A functions 7 and 12): set 0.3 for it.  chi_min must lie in
 * [0.01, 2000], else SFQ_ERR_ARG. */
sfq_status sfq_set_pair_rate_cutoff(sfq_ctx *ctx, double chi_min);

/* Coefficient count of the energy samplers, the accuracy/speed knob of Sec. 4.5.  Each
 * piece of the two inverse-CDF tables holds n x n coefficients: n = 9 in binary32 and
 * n = 12 in binary64.  With k < n, every piece is rewritten once in the Chebyshev basis,
 * cut to its leading k x k coefficients, returned to monomials and uploaded.  The samplers
 * of sfq_sample_*_xi and of the Monte Carlo steps then evaluate k x k coefficients per
 * event.  Fewer loads and FMAs, a larger error.  Worst cases relative to the full table
 * (evaluated on a grid of every piece): binary32 w-bar (photon) 6.3e-7 at k = 8 and 3.6e-6
 * at k = 7, 1 - v-bar (pair) 1.7e-6 and 8.6e-6; binary64 w-bar 6.5e-12 at k = 11 and
 * 6.2e-11 at k = 10, 1 - v-bar 2.2e-11 and 2.0e-10.  The photon fraction xi inherits up to
 * three times the error of w-bar.  k must be n, n - 1 or n - 2,
 * else SFQ_ERR_ARG; k = n restores the full tables.  The call allocates device memory and
 * synchronises the device: make it outside stream capture, between runs.  The learned
 * surrogate's fallback keeps the full tables.  sfq_sampler_coefficients returns n and the
 * current k. */
sfq_status sfq_set_sampler_coefficients(sfq_ctx *ctx, int32_t k);
sfq_status sfq_sampler_coefficients(const sfq_ctx *ctx, int32_t *n, int32_t *k);

/* Evaluator of the fitted tables behind sfq_photon_rate, sfq_pair_rate, sfq_sample_photon_xi
 * and sfq_sample_pair_xi.  SFQ_EVAL_HORNER (default): every piece as a polynomial in the
 * monomial basis, evaluated by Horner's rule.  SFQ_EVAL_CLENSHAW: the same pieces converted
 * to the Chebyshev basis (on the host, in binary64, then rounded to the context's precision)
 * and evaluated by Clenshaw's recurrence, the layout of the paper's own piecewise Chebyshev
 * fits (Sec. 4), offered as a comparison; results agree with Horner's to rounding.  The
 * Monte Carlo step kernels always use Horner.  SFQ_EVAL_CLENSHAW needs the full sampler
 * tables (sfq_set_sampler_coefficients with k = n), else SFQ_ERR_ARG; the first switch to it
 * allocates and uploads the Chebyshev tables (synchronously). */
enum { SFQ_EVAL_HORNER = 0, SFQ_EVAL_CLENSHAW = 1 };
sfq_status sfq_set_evaluator(sfq_ctx *ctx, int32_t kind);

/* Host copy of a fitted table, without a device or a context: `which` is one of
 * SFQ_TABLE_NLC_RATE (W~_rad, Eq. wtilde), SFQ_TABLE_NBW_RATE (h of W~_pair, Eq. wtilde_pair),
 * SFQ_TABLE_NLC_INV (w-bar of Eq. again), SFQ_TABLE_NBW_INV (1 - v-bar of Eq. again_pp), in
 * `precision`'s element type; `basis` SFQ_EVAL_HORNER gives the monomial pieces,
 * SFQ_EVAL_CLENSHAW the same pieces in the Chebyshev basis.  Layout as on the device: rate
 * tables (deg + 1) coefficients per piece; inverse-CDF tables n x n per piece, each row of
 * n padded to 16 bytes.  *bytes (in: capacity of `out`; out: the table's size) must not be
 * NULL; `out` may be NULL to query the size, else SFQ_ERR_CAPACITY when it is too small. */
enum { SFQ_TABLE_NLC_RATE = 0, SFQ_TABLE_NBW_RATE = 1, SFQ_TABLE_NLC_INV = 2, SFQ_TABLE_NBW_INV = 3 };
sfq_status sfq_table_pieces(int32_t precision, int32_t which, int32_t basis, void *out, size_t *bytes);

/* Autotuner: times every launch shape of sfq_mc_step (kernel variant, particles per lane
 * or warps per block) on a copy of up to `sample_n` particles of `p` (the caller's state
 * is not modified; the copy lives in temporary device memory for the duration of the
 * call), keeps the fastest in the context (sfq_set_step_shape) and returns it.  Products
 * of the trial steps go to a temporary buffer.  Synchronises `stream`. */
sfq_status sfq_autotune_step(sfq_ctx *ctx, const sfq_particles *p, const sfq_fields *f, uint32_t step,
                             int64_t sample_n, int32_t *variant, int32_t *shape, double *ms_per_step, void *stream);

/* Sort the first n product records in place by (parent id, step, member, parent tag)
 * (a stable LSD radix sort).  `scratch` is caller-owned device memory of at least
 * sfq_sort_scratch_bytes(n) bytes, 256-byte aligned; nothing in it needs to start at zero.
 * Synchronises `stream` once (to learn which key bits occur, so that passes over
 * all-zero digits are skipped).  Returns SFQ_ERR_ARG if scratch is NULL, misaligned or
 * too small, or if n exceeds the capacity of `out` or 2^32 - 1. */
size_t sfq_sort_scratch_bytes(int64_t n);
sfq_status sfq_sort_products(sfq_ctx *ctx, const sfq_products *out, int64_t n, void *scratch, size_t scratch_bytes,
                             void *stream);

/* sfq_sort_products without caller scratch and without allocating (the paper has no
 * counterpart: this is a runtime service).  The scratch is a fixed array of
 * SFQ_SORT_NOALLOC_SCRATCH_BYTES in the library's own device memory, for callers that
 * cannot allocate at the point of the call: host codes that give all device memory to
 * their own pool at start-up and have no spare buffer, and step loops where a
 * cudaMalloc/cudaFree would synchronise the device.
 *   n: at most SFQ_SORT_NOALLOC_MAX_N records, else SFQ_ERR_ARG (use sfq_sort_products).
 *   Nothing in the scratch needs to start at zero.
 *   The array is shared by all calls on a device: calls that overlap in time on one
 *   device race, so issue them on one stream or order their streams.
 *   The first call with each context looks up the array's address on the context's device
 *   (cudaGetSymbolAddress) and keeps it in the context; make that first call before any
 *   stream capture begins.
 *   Synchronises `stream` once, as sfq_sort_products does. */
#define SFQ_SORT_NOALLOC_MAX_N (1 << 20)
#define SFQ_SORT_NOALLOC_SCRATCH_BYTES (44u << 20)
sfq_status sfq_sort_products_noalloc(sfq_ctx *ctx, const sfq_products *out, int64_t n, void *stream);

/* ---------------------------------------------------------------------------------
 * Learned surrogate of the photon-emission inverse CDF (Sec. 4.3, Eq. again).
 * A 2 -> 64 -> 64 -> 64 -> 1 SiLU network maps (ln chi, u) to the paper's inverse-CDF
 * variable:  x1 = (ln chi - C) / S with C, S centring ln chi in [ln 1e-3, ln 100] on
 * [-1, 1],  x2 = -ln(1 - u) / 8 - 1,  ln w-bar = network(x1, x2) + ln u,  and
 * xi = s / (1 + s), s = 3 chi w-bar^3 / 2 (Eq. subs_altri).  Parameters are one binary32
 * vector of sfq_mlp_num_params() = 8577 values, layer by layer, each layer its weights
 * (row-major [out][in]) then its biases.  Inference rounds weights and the inputs of
 * layers 2-4 to bfloat16 and accumulates in binary32; the two 64 x 64 layers run on the
 * tensor cores.  Binary32 contexts only.  Device buffers are caller-owned; the object
 * owns its parameters, optimiser state and calibration flags. */
typedef struct sfq_mlp sfq_mlp;
int32_t sfq_mlp_num_params(void);
/* Parameters drawn from U(-1/sqrt(fan_in), 1/sqrt(fan_in)) with Philox(seed). */
sfq_status sfq_mlp_create(sfq_ctx *ctx, uint64_t seed, sfq_mlp **out);
void sfq_mlp_destroy(sfq_mlp *m);
/* Copy the 8577 binary32 parameters to / from host memory (set resets the optimiser). */
sfq_status sfq_mlp_get_params(sfq_mlp *m, float *host);
sfq_status sfq_mlp_set_params(sfq_mlp *m, const float *host);
/* Loss = sum_i (ln w_pred,i - lnw_i)^2 / n over n samples (binary32 device arrays chi,
 * u in (0, 1), lnw = ln w-bar targets) and its gradient (device, 8577 floats); `loss`
 * (device float) may be NULL.  quantize != 0 rounds as inference does (the rounding is
 * passed straight through to the gradient).  Deterministic (fixed reduction order). */
sfq_status sfq_mlp_loss_grad(sfq_mlp *m, int64_t n, const float *chi, const float *u, const float *lnw,
                             int32_t quantize, float *grad, float *loss, void *stream);
/* `steps` Adam steps (beta 0.9, 0.999, eps 1e-8) on minibatches of `batch` samples (a
 * multiple of 64) drawn with replacement by Philox(seed, sample, step); learning rate
 * lr * (1 + cos(pi t / steps)) / 2.  loss_history (device, `steps` floats) may be NULL. */
sfq_status sfq_mlp_train(sfq_mlp *m, int64_t n, const float *chi, const float *u, const float *lnw, int64_t steps,
                         int32_t batch, float lr, int32_t quantize, uint64_t seed, float *loss_history,
                         void *stream);
/* ln w-bar of the network (CUDA-core kernel, the same rounding as inference; no fallback). */
sfq_status sfq_mlp_predict_lnw(sfq_mlp *m, int64_t n, const float *chi, const float *u, float *lnw, void *stream);
/* Training targets from the plain fitted sampler: lnw = ln w-bar with s = 3 chi w-bar^3 / 2
 * the value sfq_sample_photon_xi uses (for training without oracle data). */
sfq_status sfq_mlp_plain_targets(sfq_mlp *m, int64_t n, const float *chi, const float *u, float *lnw, void *stream);
/* Flags the cells of a 64 x 64 grid over (ln chi in [ln 1e-3, ln 100], u in (0, 1)) where
 * |u_network - u| = |ln w_network - ln w_plain| / (d ln w_plain / du), over 8 x 8 points
 * of the cell, exceeds tol_u (the plain fitted sampler of sfq_sample_photon_xi is the
 * judge).  Returns the number of flagged cells and the largest error of the others.
 * Synchronises `stream`. */
sfq_status sfq_mlp_calibrate(sfq_mlp *m, float tol_u, int32_t *n_flagged, float *max_err, void *stream);
/* As sfq_sample_photon_xi, through the network on the tensor cores.  With use_flags (after
 * sfq_mlp_calibrate) draws in flagged cells, and every chi outside [1e-3, 100], take the
 * plain sampler (counted in counters->surrogate_fallbacks). */
sfq_status sfq_mlp_sample_photon_xi(sfq_mlp *m, int64_t n, const void *chi, const void *r, void *xi, void *xi_c,
                                    int32_t use_flags, sfq_counters *counters, void *stream);

/* The same network for pair creation (f4): a second surrogate object stands for the
 * inverse CDF of Eq. again_pp.  Input u = |r'| = |2r - 1| and chi in [0.1, 100]:
 * x1 = (ln chi - C) / S with C, S centring ln chi in [ln 0.1, ln 100] on [-1, 1],
 * x2 = -ln(1 - u) / 8 - 1; the sampler variable is ln(-ln y) with y = 1 - v-bar, the
 * network output that variable minus ln u (-ln y ~ v-bar ~ u as u -> 0), so that
 * y = exp(-u e^output) <= 1; the electron share is xi_e = (1 + sgn(r') v-bar) / 2, the
 * positron's 1 - xi_e (Eq. return_to_nrg).  sfq_mlp_train, _loss_grad, _predict_lnw
 * (which returns ln(-ln y)), _plain_targets (ln(-ln y) of the fitted pair sampler, NaN
 * where 1 - y falls below the binary32 table's resolution, |r'| below about 1e-5) and
 * _calibrate work on either kind; training and the loss skip samples whose target is not
 * finite.
 * sfq_mlp_sample_pair_xi writes real[n] xi_e and, if xi_p != NULL, xi_p with relative
 * precision; draws outside the chi range or in flagged cells use the fitted pair
 * sampler.  Calling the sampler of the other kind returns SFQ_ERR_ARG.  The paper has no
 * surrogate. */
sfq_status sfq_mlp_create_pair(sfq_ctx *ctx, uint64_t seed, sfq_mlp **out);
sfq_status sfq_mlp_sample_pair_xi(sfq_mlp *m, int64_t n, const void *chi, const void *r, void *xi_e, void *xi_p,
                                  int32_t use_flags, struct sfq_counters *counters, void *stream);

/* The Monte Carlo step with the photon surrogate on its event path (the survey's
 * use_surrogate; the paper has no surrogate).  Caller-owned queue of photon-emission
 * events (device pointers, `capacity` entries each, 16-byte aligned): */
typedef struct {
    int64_t capacity;
    int64_t *index;            /* int64: the emitter's index in the stepped population */
    float *chi, *r;            /* binary32: chi at the event and the energy draw r_1 (word 1) */
    float *gamma;              /* binary32: the emitter's energy before the event */
    float *px, *py, *pz;       /* binary32: its momentum before the event */
    float *xi;                 /* binary32: the fraction the surrogate pass sampled (output) */
    unsigned long long *count; /* device counter of requested entries; each step zeroes it */
} sfq_event_queue;
/* Attach a trained photon surrogate (binary32 context, the object's own context) and a
 * queue, or detach with net == NULL.  While attached, every sfq_mc_step (and sfq_mc_run)
 * of the context runs photon emission by the optical-depth method (Sec. 2, 4.1) in three
 * launches on the step's stream: the step kernel decides the events as without the
 * surrogate (the decision does not depend on the sampler) and appends each emission to
 * the queue instead of sampling it; the tensor-core surrogate samples xi = s/(1 + s) for
 * the queued events (Eq. again through the network; with use_flags, flagged cells and chi
 * outside [1e-3, 100] take the plain sampler, counted in surrogate_fallbacks); a finishing
 * pass applies the recoil and appends the photon records (Sec. 3, collinear).  Events past
 * the queue's capacity are sampled by the plain sampler in the step kernel (also counted
 * in surrogate_fallbacks).  Pair creation, beyond-LCFA leptons, sfq_mc_run_fused and
 * sfq_cascade_run keep the plain samplers.  After a step the queue holds that step's
 * emissions (index, chi, r, gamma, momentum and the sampled xi), in no particular order.
 * use_flags requires sfq_mlp_calibrate first.  SFQ_ERR_ARG for a binary64 context, a pair
 * surrogate, a net of another context, or NULL/misaligned queue buffers. */
sfq_status sfq_set_surrogate(sfq_ctx *ctx, sfq_mlp *net, const sfq_event_queue *queue, int32_t use_flags);

/* The deferred event path with the plain fitted sampler (no counterpart in the paper: a
 * launch structure).  With a queue set (binary32 context), every sfq_mc_step and sfq_mc_run
 * of the context runs photon emission by the optical-depth method in two launches: the
 * step kernel streams the population, decides the events (Sec. 2) and appends each
 * emission to the queue; an event pass samples the queued emissions (Eq. again with the
 * fitted tables, as sfq_sample_photon_xi), recoils each emitter and appends the photon's
 * record (Sec. 3).  The arithmetic is the inline path's, so the records (in another order),
 * the state and the counters equal those of the step without a queue.  Emissions past
 * the capacity are finished inline by the step kernel (counted in surrogate_fallbacks).
 * The queue's xi column is not written.  A surrogate attached with sfq_set_surrogate takes
 * precedence.  On GB300 the inline path is the faster one for dense populations (the event
 * pass gathers each sample's coefficients without the stream to hide them behind).  queue == NULL restores the inline path.  SFQ_ERR_ARG for a binary64 context,
 * truncated samplers, or NULL/misaligned queue buffers. */
sfq_status sfq_set_event_queue(sfq_ctx *ctx, const sfq_event_queue *queue);

/* Launch shape of sfq_mc_step for this context, the knob the autotuner turns.
 *   variant: 0 = automatic; 1 = warp-streaming kernel (each warp loads its particles
 *            directly); 2 = TMA-staged kernel (bulk copies of each tile into shared
 *            memory, one persistent block per SM).
 *   ppt:     shape of the chosen kernel: particles per lane per chunk of the
 *            warp-streaming kernel (1, 2 or 4), or consumer warps per block of the
 *            TMA-staged kernel (8, 16 or 20); 0 = default.
 *   grid_blocks: grid size (0 = one wave of resident blocks on every SM).
 * Returns SFQ_ERR_ARG for other values.  Results do not depend on the shape. */
sfq_status sfq_set_step_shape(sfq_ctx *ctx, int32_t variant, int32_t ppt, int32_t grid_blocks);

/* Library version string. */
const char *sfq_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SFQ_H */
