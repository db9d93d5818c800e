/*
 * sfq_oracle.c -- reference ("oracle") implementation of the strong-field QED
 * Monte Carlo step of Montefiori & Tamburini, "SFQEDtoolkit" (arXiv:2301.07684).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library, its
 * Python binding, the table generator) may include, link, load or call this
 * file.  Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark use it.
 *
 * Everything is plain IEEE double precision on the CPU and follows the
 * defining formulas of the paper directly:
 *   - K_nu(x) and Ki_nu(x) = int_x^inf K_nu(y) dy from the integral
 *     representation K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt
 *     (DLMF 10.32.9) and its integral in x, by adaptive Gauss-Kronrod (7,15);
 *   - the rates  W~_rad (Eq. wtilde, Sec. 4.1) and W~_pair (Eq. wtilde_pair,
 *     Sec. 4.2) by quadrature, with the normalised prefactors of
 *     Eq. pe_rate_3 and Eq. pp_tot_real;
 *   - the cumulative functions I~_pe (Eq. pe_eff_int_2, Sec. 4.3) and
 *     I~_pp (Eq. tilde_I_pp, Sec. 4.4) by quadrature;
 *   - inverse-transform sampling (Eq. again, Eq. again_pp) by Brent's
 *     bracketing root finder;
 *   - chi (Eq. chi_exact), the optical-depth and local event tests (Sec. 2),
 *     the beyond-LCFA update, threshold and rejection (Sec. 5,
 *     Eqs. fl ... condit, gammaLCFA, rej_cond) and collinear products (Sec. 3).
 * No piecewise fits, no tables, no blocking and no reordering beyond what the
 * formulas state.  Readings of points the paper leaves open are marked
 * "READING" below.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------- */
/* Physical constants (CODATA 2018).                                          */
/* ------------------------------------------------------------------------- */
static const double ORC_ALPHA = 7.2973525693e-3;          /* fine-structure constant */
static const double ORC_LAMBDA_C = 3.8615926796e-13;      /* reduced Compton length hbar/(m c) [m] */
static const double ORC_C = 299792458.0;                   /* speed of light [m/s] */

/* rho = lambda_r / lambda_C: the critical field in units of E_r = m c omega_r/|e|
 * and the inverse of the Compton time in units of 1/omega_r (Sec. 4.1, App. A). */
double orc_rho_from_ref_len(double ref_len_m) { return ref_len_m / ORC_LAMBDA_C; }
double orc_rho_from_ref_freq(double omega_si) { return (ORC_C / omega_si) / ORC_LAMBDA_C; }
/* alpha/(sqrt(3) pi) * lambda_r/lambda_C: the common factor of Eq. pe_rate_3 and Eq. pp_tot_real. */
double orc_rate_prefactor(double rho) { return ORC_ALPHA / (sqrt(3.0) * ORC_PI) * rho; }

/* ------------------------------------------------------------------------- */
/* Adaptive Gauss-Kronrod (7,15) quadrature.                                  */
/* Nodes and weights of the 15-point Kronrod extension of the 7-point Gauss-  */
/* Legendre rule (Piessens et al., QUADPACK, 1983).                          */
/* ------------------------------------------------------------------------- */
static const double XGK[8] = {
    0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
    0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
    0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
    0.207784955007898467600689403773245, 0.000000000000000000000000000000000};
static const double WGK[8] = {
    0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
    0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
    0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
    0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
static const double WG[4] = {
    0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
    0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

typedef double (*orc_fn)(double x, const void *ctx);

/* One (7,15) panel on [a,b]: Kronrod estimate and |Kronrod - Gauss|. */
static void gk15(orc_fn f, const void *ctx, double a, double b, double *res, double *err) {
    const double c = 0.5 * (a + b), h = 0.5 * (b - a);
    const double fc = f(c, ctx);
    double rk = fc * WGK[7], rg = fc * WG[3];
    for (int j = 0; j < 7; ++j) {
        const double dx = h * XGK[j];
        const double s = f(c - dx, ctx) + f(c + dx, ctx);
        rk += WGK[j] * s;
        if (j & 1) rg += WG[j / 2] * s;
    }
    *res = rk * h;
    *err = fabs((rk - rg) * h);
}

/* Globally adaptive bisection (the strategy of QUADPACK's QAG): keep a list of
 * panels, split the one with the largest error estimate until the summed
 * estimate is below rel * |integral| or the panel budget is spent. */
enum { GK_MAXP = 4000, GK_NP0 = 8 };
typedef struct { double a, b, r, e; } gk_panel;

static double integrate(orc_fn f, const void *ctx, double a, double b, double rel) {
    if (!(b > a)) return 0.0;
    gk_panel *P = (gk_panel *)malloc(sizeof(gk_panel) * GK_MAXP);
    int np = 0;
    const double h = (b - a) / GK_NP0;
    for (int i = 0; i < GK_NP0; ++i) {
        gk_panel *q = &P[np++];
        q->a = a + i * h;
        q->b = (i == GK_NP0 - 1) ? b : a + (i + 1) * h;
        gk15(f, ctx, q->a, q->b, &q->r, &q->e);
    }
    double sum = 0.0;
    for (;;) {
        double R = 0.0, E = 0.0, emax = -1.0;
        int imax = -1;
        for (int i = 0; i < np; ++i) {
            R += P[i].r;
            E += P[i].e;
            if (P[i].e > emax) { emax = P[i].e; imax = i; }
        }
        sum = R;
        if (E != E || R != R) break;                 /* NaN integrand: no refinement helps */
        if (E <= rel * fabs(R) || E == 0.0 || np >= GK_MAXP - 1) break;
        gk_panel *q = &P[imax];
        const double m = 0.5 * (q->a + q->b);
        if (!(m > q->a && m < q->b)) { q->e = 0.0; continue; }   /* cannot split further */
        gk_panel right = {m, q->b, 0.0, 0.0};
        q->b = m;
        gk15(f, ctx, q->a, q->b, &q->r, &q->e);
        gk15(f, ctx, right.a, right.b, &right.r, &right.e);
        P[np++] = right;
    }
    free(P);
    return sum;
}

/* Public, for the quadrature self-test: int_a^b x^k dx. */
static double orc_mono(double x, const void *ctx) { return pow(x, *(const double *)ctx); }
double orc_test_gk15_monomial(double k, double a, double b) {
    double r, e;
    gk15(orc_mono, &k, a, b, &r, &e);
    return r;
}
double orc_test_gauss7_monomial(double k, double a, double b) {
    const double c = 0.5 * (a + b), h = 0.5 * (b - a);
    double s = WG[3] * pow(c, k);
    for (int j = 1; j < 7; j += 2) s += WG[j / 2] * (pow(c - h * XGK[j], k) + pow(c + h * XGK[j], k));
    return s * h;
}

/* ------------------------------------------------------------------------- */
/* Modified Bessel functions of the second kind by quadrature.               */
/* ------------------------------------------------------------------------- */
static const double REL_INNER = 1e-14;   /* special functions */
static const double REL_OUTER = 1e-13;   /* rates, spectra and cumulative functions */

typedef struct { double x, nu; } kctx;

/* exp(-x (cosh t - 1)) cosh(nu t); cosh t - 1 = 2 sinh^2(t/2) avoids cancellation. */
static double k_scaled_integrand(double t, const void *c) {
    const kctx *k = (const kctx *)c;
    const double sh = sinh(0.5 * t);
    return exp(-k->x * 2.0 * sh * sh) * cosh(k->nu * t);
}
/* exp(-x (cosh t - 1)) cosh(nu t) / cosh t */
static double ki_scaled_integrand(double t, const void *c) {
    const kctx *k = (const kctx *)c;
    const double sh = sinh(0.5 * t);
    return exp(-k->x * 2.0 * sh * sh) * cosh(k->nu * t) / cosh(t);
}

/* Upper cut T of the t-integral: beyond it the scaled integrand is below
 * exp(-800) times a factor that grows at most like exp(nu t). */
static double t_cut(double x) {
    if (x > 0.0) return acosh(1.0 + 800.0 / x);
    return 120.0; /* x = 0: only for Ki, integrand ~ exp((nu-1) t) */
}

/* exp(x) K_nu(x), x > 0 (DLMF 10.32.9). */
double orc_besselk_scaled(double nu, double x) {
    kctx c = {x, nu};
    return integrate(k_scaled_integrand, &c, 0.0, t_cut(x), REL_INNER);
}
/* K_nu(x), x > 0. */
double orc_besselk(double nu, double x) {
    if (x > 745.0) return 0.0;
    return exp(-x) * orc_besselk_scaled(nu, x);
}
/* exp(x) Ki_nu(x),  Ki_nu(x) = int_x^inf K_nu(y) dy = int_0^inf exp(-x cosh t) cosh(nu t)/cosh t dt
 * (the x-integral of DLMF 10.32.9; it vanishes at infinity and its x-derivative is -K_nu). */
double orc_besselk_int_scaled(double nu, double x) {
    kctx c = {x, nu};
    return integrate(ki_scaled_integrand, &c, 0.0, t_cut(x), REL_INNER);
}
double orc_besselk_int(double nu, double x) {
    if (x > 745.0) return 0.0;
    return exp(-x) * orc_besselk_int_scaled(nu, x);
}

/* ------------------------------------------------------------------------- */
/* Photon emission (nonlinear Compton), Sec. 4.1 and Sec. 4.3.                */
/* ------------------------------------------------------------------------- */

/* Integrand of Eq. wtilde after v = t^3 (removes the v^{-2/3} end-point singularity). */
static double wrad_integrand(double t, const void *c) {
    const double chi = *(const double *)c;
    const double v = t * t * t;
    const double x = v * chi;
    const double den = 2.0 + 3.0 * x;
    const double f = (45.0 * x * x + 42.0 * x + 20.0) / (den * den * den);
    return f * orc_besselk(2.0 / 3.0, v) * 3.0 * t * t;
}
/* W~_rad(chi), Eq. wtilde; upper limit v = 700 (footnote to Eq. wtilde). */
double orc_wtilde_rad(double chi) {
    return integrate(wrad_integrand, &chi, 0.0, cbrt(700.0), REL_OUTER);
}
/* W_rad(gamma, chi) = R_pe/omega_r, Eq. pe_rate_3. */
double orc_photon_rate(double gamma, double chi, double pref) {
    if (chi <= 0.0) return 0.0;
    return pref * (chi / gamma) * orc_wtilde_rad(chi);
}

/* Integrand of Eq. pe_eff_int_2 (s = 3 chi w^3 / 2). */
static double ipe_integrand(double w, const void *c) {
    const double chi = *(const double *)c;
    const double x = w * w * w;
    const double s = 1.5 * chi * x;
    const double ops = 1.0 + s;
    const double k23 = orc_besselk(2.0 / 3.0, x);
    const double ki13 = orc_besselk_int(1.0 / 3.0, x);
    return 9.0 * w * w / (2.0 * ops * ops * ops) * ((1.0 + ops * ops) * k23 - ops * ki13);
}
static double w_max(void) { return cbrt(700.0); }
/* I~_pe(w, chi), Eq. pe_eff_int_2. */
double orc_itilde_pe(double w, double chi) {
    if (w <= 0.0) return 0.0;
    return integrate(ipe_integrand, &chi, 0.0, fmin(w, w_max()), REL_OUTER);
}
/* int_w^inf of the same integrand (= W~_rad - I~_pe); evaluated directly so that
 * the far tail keeps its relative precision. */
double orc_itilde_pe_upper(double w, double chi) {
    if (w >= w_max()) return 0.0;
    return integrate(ipe_integrand, &chi, fmax(w, 0.0), w_max(), REL_OUTER);
}

/* ------------------------------------------------------------------------- */
/* Pair creation (nonlinear Breit-Wheeler), Sec. 4.2 and Sec. 4.4.            */
/* ------------------------------------------------------------------------- */

/* om = 1 - v^2 is passed separately so that the end v -> 1 keeps relative precision. */
static double wpair_integrand_vo(double v, double om, double chi) {
    const double eta = 8.0 / (3.0 * chi * om);
    if (eta > 745.0) return 0.0;
    return (9.0 - v * v) / (3.0 * om) * orc_besselk(2.0 / 3.0, eta);
}
static double wpair_integrand(double v, const void *c) {
    return wpair_integrand_vo(v, (1.0 - v) * (1.0 + v), *(const double *)c);
}
/* W~_pair(chi), Eq. wtilde_pair. */
double orc_wtilde_pair(double chi) {
    if (chi <= 0.0) return 0.0;
    return integrate(wpair_integrand, &chi, 0.0, 1.0, REL_OUTER);
}
/* W_pair(gamma, chi) = R_pp/omega_r, Eq. pp_tot_real; zero below chi = 0.01
 * where the paper neglects the process (Sec. 4.2, below Eq. low_chi). */
double orc_pair_rate(double gamma, double chi, double pref) {
    if (chi < 0.01) return 0.0;
    return pref * orc_wtilde_pair(chi) / gamma;
}

/* Integrand of Eq. tilde_I_pp, eta_v = 8/(3 chi (1 - v^2)). */
static double ipp_integrand_vo(double om, double v, double chi) {
    const double eta = 8.0 / (3.0 * chi * om);
    if (eta > 745.0) return 0.0;
    return 2.0 * (1.0 + v * v) / om * orc_besselk(2.0 / 3.0, eta) + orc_besselk_int(1.0 / 3.0, eta);
}
static double ipp_integrand_v(double v, const void *c) {
    return ipp_integrand_vo((1.0 - v) * (1.0 + v), v, *(const double *)c);
}
/* same integrand as a function of y = 1 - v: 1 - v^2 = y (2 - y) */
static double ipp_integrand_y(double y, const void *c) {
    return ipp_integrand_vo(y * (2.0 - y), 1.0 - y, *(const double *)c);
}
/* I~_pp(v, chi), Eq. tilde_I_pp. */
double orc_itilde_pp(double v, double chi) {
    if (v <= 0.0) return 0.0;
    return integrate(ipp_integrand_v, &chi, 0.0, fmin(v, 1.0), REL_OUTER);
}
/* int_{1-y}^{1} of the same integrand (= W~_pair - I~_pp(1-y)), integrated in y. */
double orc_itilde_pp_upper_y(double y, double chi) {
    if (y <= 0.0) return 0.0;
    return integrate(ipp_integrand_y, &chi, 0.0, fmin(y, 1.0), REL_OUTER);
}

/* ------------------------------------------------------------------------- */
/* Brent's bracketing root finder (Brent 1973: bisection safeguarding secant */
/* and inverse quadratic interpolation).                                      */
/* ------------------------------------------------------------------------- */
static double brent(orc_fn g, const void *ctx, double a, double b, double fa, double fb, double rtol) {
    double c = a, fc = fa, d = b - a, e = d;
    for (int it = 0; it < 400; ++it) {
        if ((fb > 0.0) == (fc > 0.0)) { c = a; fc = fa; d = e = b - a; }
        if (fabs(fc) < fabs(fb)) { a = b; b = c; c = a; fa = fb; fb = fc; fc = fa; }
        const double tol = 2.0 * DBL_EPSILON * fabs(b) + 0.5 * rtol * fabs(b) + 1e-300;
        const double m = 0.5 * (c - b);
        if (fabs(m) <= tol || fb == 0.0) return b;
        if (fabs(e) >= tol && fabs(fa) > fabs(fb)) {
            const double s = fb / fa;
            double p, q;
            if (a == c) {            /* secant */
                p = 2.0 * m * s;
                q = 1.0 - s;
            } else {                 /* inverse quadratic interpolation */
                const double qa = fa / fc, r = fb / fc;
                p = s * (2.0 * m * qa * (qa - r) - (b - a) * (r - 1.0));
                q = (qa - 1.0) * (r - 1.0) * (s - 1.0);
            }
            if (p > 0.0) q = -q; else p = -p;
            if (2.0 * p < fmin(3.0 * m * q - fabs(tol * q), fabs(e * q))) { e = d; d = p / q; }
            else { d = m; e = m; }
        } else {
            d = m; e = m;
        }
        a = b; fa = fb;
        b += (fabs(d) > tol) ? d : (m > 0.0 ? tol : -tol);
        fb = g(b, ctx);
    }
    return b;
}
static const double RTOL_ROOT = 1e-14;

typedef struct { double chi, target; } rctx;
static double g_pe_lower(double w, const void *c) {
    const rctx *r = (const rctx *)c; return orc_itilde_pe(w, r->chi) - r->target;
}
static double g_pe_upper(double w, const void *c) {
    const rctx *r = (const rctx *)c; return orc_itilde_pe_upper(w, r->chi) - r->target;
}

/* w-bar = G~_pe(r, chi): the root of Eq. again, I~_pe(w, chi) = r W~_rad(chi).
 * READING: for r >= 1/2 the equivalent complementary form
 * int_w^inf (...) = (1 - r) W~_rad(chi) is solved, which keeps the relative
 * precision of the root in the upper tail (r -> 1). */
double orc_photon_wbar(double r, double chi) {
    const double W = orc_wtilde_rad(chi);
    if (r < 0.5) {
        rctx c = {chi, r * W};
        return brent(g_pe_lower, &c, 0.0, w_max(), -r * W, (1.0 - r) * W, RTOL_ROOT);
    }
    rctx c = {chi, (1.0 - r) * W};
    return brent(g_pe_upper, &c, 0.0, w_max(), r * W, -(1.0 - r) * W, RTOL_ROOT);
}
/* s = u = eps_gamma/(eps_e - eps_gamma) = 3 chi w^3 / 2 (Eq. subs_altri); xi = s/(1+s). */
double orc_photon_s(double r, double chi) {
    const double w = orc_photon_wbar(r, chi);
    return 1.5 * chi * w * w * w;
}

static double g_pp_lower(double v, const void *c) {
    const rctx *r = (const rctx *)c; return orc_itilde_pp(v, r->chi) - r->target;
}
static double g_pp_upper(double y, const void *c) {
    const rctx *r = (const rctx *)c; return orc_itilde_pp_upper_y(y, r->chi) - r->target;
}
/* v-bar = G~_pp(a, chi), a = |r'|: the root of Eq. again_pp,
 * I~_pp(v, chi) = a W~_pair(chi).  Returns v-bar and y = 1 - v-bar.
 * READING: for a >= 1/2 the complementary form in y = 1 - v,
 * int_{1-y}^1 (...) dv = (1 - a) W~_pair, is solved so that 1 - v-bar (the
 * smaller lepton share) keeps its relative precision. */
void orc_pair_vbar(double a, double chi, double *vbar, double *ybar) {
    const double W = orc_wtilde_pair(chi);
    if (a < 0.5) {
        rctx c = {chi, a * W};
        const double v = brent(g_pp_lower, &c, 0.0, 1.0, -a * W, (1.0 - a) * W, RTOL_ROOT);
        *vbar = v; *ybar = 1.0 - v;
        return;
    }
    rctx c = {chi, (1.0 - a) * W};
    const double y = brent(g_pp_upper, &c, 0.0, 1.0, -(1.0 - a) * W, a * W, RTOL_ROOT);
    *ybar = y; *vbar = 1.0 - y;
}
/* Electron share xi_e = eps_e/eps_gamma = (1 + sgn(r') v)/2 (Eq. return_to_nrg),
 * r' = 2 r - 1; the positron gets 1 - xi_e.  Both shares are returned with
 * relative precision. */
void orc_pair_shares(double r, double chi, double *xi_e, double *xi_p) {
    const double rp = 2.0 * r - 1.0;
    double v, y;
    orc_pair_vbar(fabs(rp), chi, &v, &y);
    const double big = 1.0 - 0.5 * y, small = 0.5 * y;
    if (rp >= 0.0) { *xi_e = big; *xi_p = small; }
    else { *xi_e = small; *xi_p = big; }
}

/* ------------------------------------------------------------------------- */
/* Spectra, Eq. pe_dp and Eq. pp_dp, in units of omega_r per unit of         */
/* normalised energy.                                                         */
/* ------------------------------------------------------------------------- */
/* d^2W_pe/(dt d gamma_gamma) at photon energy gg from a lepton of energy ge. */
double orc_spectrum_pe(double gg, double ge, double chi, double pref) {
    if (gg <= 0.0 || gg >= ge || chi <= 0.0) return 0.0;
    const double u = gg / (ge - gg);
    const double x = 2.0 * u / (3.0 * chi);
    if (x > 745.0) return 0.0;
    const double opu = 1.0 + u;
    return pref / (ge * ge) / opu *
           ((1.0 + opu * opu) * orc_besselk(2.0 / 3.0, x) - opu * orc_besselk_int(1.0 / 3.0, x));
}
/* d^2W_pp/(dt d gamma_e) at electron energy ge from a photon of energy gg. */
double orc_spectrum_pp(double ge, double gg, double chi, double pref) {
    const double gp = gg - ge;
    if (ge <= 0.0 || gp <= 0.0 || chi <= 0.0) return 0.0;
    const double eta = 2.0 * gg * gg / (3.0 * ge * gp * chi);
    if (eta > 745.0) return 0.0;
    return pref / (gg * gg) *
           ((ge * ge + gp * gp) / (ge * gp) * orc_besselk(2.0 / 3.0, eta) + orc_besselk_int(1.0 / 3.0, eta));
}

/* ------------------------------------------------------------------------- */
/* chi, Eq. chi_exact, in normalised units (fields in units of E_r, momenta  */
/* in m c, energies in m c^2): chi = (gamma/rho) sqrt((E + beta x B)^2 -     */
/* (beta . E)^2), beta = p / gamma.                                           */
/* ------------------------------------------------------------------------- */
double orc_chi(double gamma, const double p[3], const double E[3], const double B[3], double rho) {
    const double b[3] = {p[0] / gamma, p[1] / gamma, p[2] / gamma};
    const double f[3] = {E[0] + b[1] * B[2] - b[2] * B[1],
                         E[1] + b[2] * B[0] - b[0] * B[2],
                         E[2] + b[0] * B[1] - b[1] * B[0]};
    const double be = b[0] * E[0] + b[1] * E[1] + b[2] * E[2];
    const double q = f[0] * f[0] + f[1] * f[1] + f[2] * f[2] - be * be;
    return (gamma / rho) * sqrt(q > 0.0 ? q : 0.0);
}
double orc_chi_components(double gamma, double px, double py, double pz, double ex, double ey,
                          double ez, double bx, double by, double bz, double rho) {
    const double p[3] = {px, py, pz}, E[3] = {ex, ey, ez}, B[3] = {bx, by, bz};
    return orc_chi(gamma, p, E, B, rho);
}

/* ------------------------------------------------------------------------- */
/* Beyond-LCFA photon emission, Sec. 5.                                       */
/* ------------------------------------------------------------------------- */
/* zeta ~ 2.22e-16, "assuming double precision" (footnote in Sec. 5). */
static const double ORC_ZETA = 2.220446049250313080847263336181640625e-16;

typedef struct {
    double F[3];       /* F_perp^{(n)} */
    double gamma, chi, delta;
    int gate;          /* the two conditions below Eq. condit */
} blcfa_eval;

/* The common part of one update of the per-particle state (Eqs. fl_perp ... condit): pL is
 * the momentum at the step, FL the Lorentz force on it.
 * READING (first step after creation): F^(n-2) = F^(n-1) = F^(n) as stated in Sec. 5, i.e.
 * the stored difference becomes zero; the call signals no emission at this step.  Returns
 * the gate (0 for a just-created particle). */
static int blcfa_core(const double pL[3], const double FL[3], double dt, double rho, double Fprev[3],
                      double dF[3], uint8_t *just_created, blcfa_eval *out) {
    const double tauC = 1.0 / rho;
    const double gamma = sqrt(1.0 + pL[0] * pL[0] + pL[1] * pL[1] + pL[2] * pL[2]);   /* Eq. gammaBLCFA */
    const double fp = (FL[0] * pL[0] + FL[1] * pL[1] + FL[2] * pL[2]) / (gamma * gamma);
    double F[3];
    for (int k = 0; k < 3; ++k) F[k] = FL[k] - fp * pL[k];               /* Eq. fl_perp */
    const double F2 = F[0] * F[0] + F[1] * F[1] + F[2] * F[2];
    out->gamma = gamma;
    out->chi = tauC * gamma * sqrt(F2);                                    /* Eq. chi_p */
    for (int k = 0; k < 3; ++k) out->F[k] = F[k];
    if (*just_created) {
        for (int k = 0; k < 3; ++k) { Fprev[k] = F[k]; dF[k] = 0.0; }
        *just_created = 0;
        out->delta = 0.0;
        out->gate = 0;
        return 0;
    }
    double Fd[3], Fdd[3], d1[3];
    for (int k = 0; k < 3; ++k) {
        d1[k] = F[k] - Fprev[k];
        Fd[k] = d1[k] / dt;
        Fdd[k] = (d1[k] - dF[k]) / (dt * dt);
    }
    const double Fd2 = Fd[0] * Fd[0] + Fd[1] * Fd[1] + Fd[2] * Fd[2];
    const double FFdd = F[0] * Fdd[0] + F[1] * Fdd[1] + F[2] * Fdd[2];
    const double delta = tauC * tauC * (Fd2 + fabs(FFdd));                /* Eq. condit */
    for (int k = 0; k < 3; ++k) { Fprev[k] = F[k]; dF[k] = d1[k]; }
    out->delta = delta;
    out->gate = (gamma * gamma * delta / (ORC_ZETA * ORC_ZETA) > out->chi * out->chi * F2) &&
                (out->chi > ORC_ZETA);
    return out->gate;
}

/* One update without a pusher.  READING: the Lorentz force is the normalised
 * F_L = E + beta x B at the particle and p_L = p. */
int orc_blcfa_update(const double p[3], const double E[3], const double B[3], double dt, double rho,
                     double Fprev[3], double dF[3], uint8_t *just_created, blcfa_eval *out) {
    const double gamma = sqrt(1.0 + p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    const double b[3] = {p[0] / gamma, p[1] / gamma, p[2] / gamma};
    const double FL[3] = {E[0] + b[1] * B[2] - b[2] * B[1],
                          E[1] + b[2] * B[0] - b[0] * B[2],
                          E[2] + b[0] * B[1] - b[1] * B[0]};
    return blcfa_core(p, FL, dt, rho, Fprev, dF, just_created, out);
}

/* One update with the force from the pusher (Eqs. fl): p is p^(n-1/2), pn = p_L^(n+1/2) its
 * push over dt; F_L = (pn - p) / dt and p_L = (pn + p) / 2. */
int orc_blcfa_update_pushed(const double p[3], const double pn[3], double dt, double rho, double Fprev[3],
                            double dF[3], uint8_t *just_created, blcfa_eval *out) {
    double FL[3], pL[3];
    for (int k = 0; k < 3; ++k) {
        FL[k] = (pn[k] - p[k]) / dt;
        pL[k] = 0.5 * (pn[k] + p[k]);
    }
    return blcfa_core(pL, FL, dt, rho, Fprev, dF, just_created, out);
}

/* gamma_{gamma,LCFA}, Eq. gammaLCFA, with tau/tau_C = 2 pi sqrt(F^2/delta). */
double orc_blcfa_threshold(const double F[3], double delta, double gamma, double chi) {
    const double F2 = F[0] * F[0] + F[1] * F[1] + F[2] * F[2];
    const double tau_ratio = 2.0 * ORC_PI * sqrt(F2 / delta);
    return 0.7 * gamma /
           (1.0 + 4.0 / (3.0 * ORC_PI * chi) * sinh(3.0 * asinh(chi / (8.0 * gamma) * tau_ratio)));
}

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from its       */
/* published definition.                                                      */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}
/* READING: uniform in (0,1) from one 32-bit word, u = (floor(w/2^9) + 1/2) 2^-23.
 * Both u and 1 - u are exact in binary32 and binary64; u never is 0 or 1 and
 * 2u - 1 never is 0. */
double orc_uniform(uint32_t w) { return ((double)(w >> 9) + 0.5) * 0x1p-23; }

/* Draws of one (particle, step): counter (id_lo, id_hi, step, tag), key = seed.
 * Word 0: optical-depth reset after an event, or r of the local test;
 * word 1: r_1 of the energy sampling; word 2: r_2 of the beyond-LCFA rejection;
 * word 3: first optical depth of a particle created without one. */
static void draws(uint64_t seed, uint64_t id, uint32_t step, uint32_t tag, double u[4]) {
    const uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), step, tag};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    for (int k = 0; k < 4; ++k) u[k] = orc_uniform(w[k]);
}
void orc_uniforms(uint64_t seed, uint64_t id, uint32_t step, uint32_t tag, double u[4]) {
    draws(seed, id, step, tag, u);
}

/* READING (the paper keys no random numbers by particle): the id of a particle created
 * in a full cascade, a function of its parent (id, tag), the creation step and its member
 * number (0 emitted photon, 1 electron, 2 positron).  The first two Philox words of the
 * counter (parent id lo, hi, step, 0x100 | parent tag << 2 | member) under the run's key,
 * with bit 63 set: the counter's last word lies outside the 0 ... 3 of the step draws, and
 * the set bit keeps descendants apart from primaries, whose ids are below 2^63. */
uint64_t orc_child_id(uint64_t seed, uint64_t parent, uint32_t parent_tag, uint32_t step, uint32_t member) {
    const uint32_t ctr[4] = {(uint32_t)parent, (uint32_t)(parent >> 32), step,
                             0x100u | ((parent_tag & 3u) << 2) | member};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    return (1ull << 63) | ((uint64_t)(w[1] & 0x7FFFFFFFu) << 32) | w[0];
}

/* ------------------------------------------------------------------------- */
/* Batched entry points (OpenMP over independent elements).                   */
/* ------------------------------------------------------------------------- */
void orc_batch_wtilde_rad(int64_t n, const double *chi, double *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i) out[i] = orc_wtilde_rad(chi[i]);
}
void orc_batch_wtilde_pair(int64_t n, const double *chi, double *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i) out[i] = orc_wtilde_pair(chi[i]);
}
void orc_batch_photon_rate(int64_t n, const double *gamma, const double *chi, double pref, double *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i) out[i] = orc_photon_rate(gamma[i], chi[i], pref);
}
void orc_batch_pair_rate(int64_t n, const double *gamma, const double *chi, double pref, double *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i) out[i] = orc_pair_rate(gamma[i], chi[i], pref);
}
void orc_batch_photon_s(int64_t n, const double *r, const double *chi, double *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i) out[i] = orc_photon_s(r[i], chi[i]);
}
void orc_batch_photon_wbar(int64_t n, const double *r, const double *chi, double *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i) out[i] = orc_photon_wbar(r[i], chi[i]);
}
void orc_batch_pair_vbar(int64_t n, const double *a, const double *chi, double *vbar, double *ybar) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i) orc_pair_vbar(a[i], chi[i], &vbar[i], &ybar[i]);
}
void orc_batch_pair_shares(int64_t n, const double *r, const double *chi, double *xi_e, double *xi_p) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i) orc_pair_shares(r[i], chi[i], &xi_e[i], &xi_p[i]);
}
void orc_batch_itilde_pe(int64_t n, const double *w, const double *chi, double *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i) out[i] = orc_itilde_pe(w[i], chi[i]);
}
void orc_batch_itilde_pe_upper(int64_t n, const double *w, const double *chi, double *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i) out[i] = orc_itilde_pe_upper(w[i], chi[i]);
}
void orc_batch_itilde_pp(int64_t n, const double *v, const double *chi, double *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i) out[i] = orc_itilde_pp(v[i], chi[i]);
}
void orc_batch_itilde_pp_upper_y(int64_t n, const double *y, const double *chi, double *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i) out[i] = orc_itilde_pp_upper_y(y[i], chi[i]);
}
/* ------------------------------------------------------------------------- */
/* Boris push of the momentum (the pusher a PIC code runs between Monte Carlo */
/* steps; Boris 1970, in the normalised units of the step: du/dt = q (E + u x */
/* B / gamma), u = p / m c, fields in E_r, time in 1/omega_r):               */
/*   u- = u + q E dt/2;  t = q B dt / (2 gamma(u-));  s = 2 t / (1 + t.t);    */
/*   u' = u- + u- x t;  u+ = u- + u' x s;  u_new = u+ + q E dt/2.             */
/* ------------------------------------------------------------------------- */
static void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
void orc_boris_push(double u[3], const double E[3], const double B[3], double q, double dt) {
    double um[3], t[3], s[3], c[3], up[3];
    for (int k = 0; k < 3; ++k) um[k] = u[k] + 0.5 * q * dt * E[k];
    const double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    for (int k = 0; k < 3; ++k) t[k] = 0.5 * q * dt * B[k] / gm;
    const double tt = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    for (int k = 0; k < 3; ++k) s[k] = 2.0 * t[k] / (1.0 + tt);
    cross3(um, t, c);
    double uprime[3];
    for (int k = 0; k < 3; ++k) uprime[k] = um[k] + c[k];
    cross3(uprime, s, c);
    for (int k = 0; k < 3; ++k) up[k] = um[k] + c[k];
    for (int k = 0; k < 3; ++k) u[k] = up[k] + 0.5 * q * dt * E[k];
}
/* n particles: u (n x 3, in/out), E, B (n x 3), q (n; 0 leaves u unchanged). */
void orc_batch_boris_push(int64_t n, double *u, const double *E, const double *B, const double *q, double dt) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        if (q[i] != 0.0) orc_boris_push(u + 3 * i, E + 3 * i, B + 3 * i, q[i], dt);
}

void orc_batch_philox(int64_t n, const uint64_t *id, uint32_t step, uint32_t tag, uint64_t seed,
                      uint32_t *out4) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t ctr[4] = {(uint32_t)id[i], (uint32_t)(id[i] >> 32), step, tag};
        orc_philox4x32_10(ctr, key, out4 + 4 * i);
    }
}
int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Monte Carlo step (Sec. 2, Sec. 3, Sec. 5) for independent lineages.        */
/* ------------------------------------------------------------------------- */
enum { SP_ELECTRON = 0, SP_POSITRON = 1, SP_PHOTON = 2 };
enum { FL_ALIVE = 1, FL_JUST_CREATED = 2 };
enum { MODE_LCFA_OD = 0, MODE_BLCFA_LOCAL = 1, MODE_BLCFA_PUSHED = 2 };

/* Run parameters shared by all lineages. */
typedef struct {
    double rho, pref, dt;
    uint64_t seed;
    uint32_t step0, nsteps;
    int32_t lepton_mode;        /* MODE_LCFA_OD, MODE_BLCFA_LOCAL or MODE_BLCFA_PUSHED */
    int32_t step_children;      /* 1: created leptons are stepped (beyond-LCFA chain) */
    double near_od;             /* |tau_d| <= near_od * tau0: optical-depth decision near threshold */
    double near_local;          /* |R dt - r| <= near_local * r: local decision near threshold */
    double near_blcfa;          /* relative window of the beyond-LCFA comparisons */
    int32_t cascade;            /* 1: full cascade, every product is a particle stepped from the next step on */
    int32_t reserved;
} orc_run_params;

/* One recorded product. */
typedef struct {
    double p[3];
    uint64_t parent_id;
    uint32_t step;
    uint32_t parent_tag;
    uint32_t species;
    uint32_t member;            /* 0: photon of an emission; 1: electron; 2: positron */
} orc_product;

/* Per-lineage output and counters. */
typedef struct {
    int64_t n_products;
    int64_t cap_products;
    orc_product *prod;          /* caller-owned, capacity cap_products */
    int64_t *counter;           /* shared product counter (atomic) */
} orc_prod_sink;

/* Events, near-threshold information and overflow, per primary.  The last three count the
 * beyond-LCFA branches of Sec. 5 taken in the lineage: local events whose gate held (the
 * threshold of Eq. gammaLCFA applied), events stopped by the 0.75 gamma_e rule, and samples
 * rejected by Eq. rej_cond. */
typedef struct {
    int32_t first_near_step;    /* first step with a near-threshold decision in the lineage, or -1 */
    int32_t n_events;
    int32_t n_gated, n_no_emission, n_rejected;
} orc_lineage_info;

typedef struct {
    double p[3];
    double tau, tau0;
    uint64_t id;
    uint32_t tag;
    uint8_t flags, species;
    double Fprev[3], dF[3];
    uint64_t parent;            /* descendants: parent id, creation step and member */
    uint32_t born, member;
} orc_state;

/* The particles a lineage has created, in order of creation (growable). */
typedef struct {
    orc_state *v;
    int n, cap;
} orc_kids;

static orc_state *kid_new(orc_kids *k) {
    if (k->n == k->cap) {
        k->cap = k->cap ? 2 * k->cap : 8;
        k->v = (orc_state *)realloc(k->v, (size_t)k->cap * sizeof(orc_state));
        if (!k->v) abort();
    }
    orc_state *c = &k->v[k->n++];
    memset(c, 0, sizeof(*c));
    return c;
}

/* A created particle: momentum pc, no optical depth yet, BLCFA state zero.  In a cascade it
 * takes its own id (orc_child_id) and tag 0; otherwise (stepped children of a converted
 * photon) the parent's id and the member as tag. */
static void kid_init(orc_state *c, const orc_state *parent, const double pc[3], uint32_t step, uint32_t member,
                     uint8_t species, const orc_run_params *P) {
    c->p[0] = pc[0]; c->p[1] = pc[1]; c->p[2] = pc[2];
    c->tau = -1.0; c->tau0 = 0.0;
    if (P->cascade) {
        c->id = orc_child_id(P->seed, parent->id, parent->tag, step, member);
        c->tag = 0u;
    } else {
        c->id = parent->id;
        c->tag = member;
    }
    /* a particle created without momentum does not take part in later steps */
    c->flags = (uint8_t)((pc[0] != 0.0 || pc[1] != 0.0 || pc[2] != 0.0 ? FL_ALIVE : 0) | FL_JUST_CREATED);
    c->species = species;
    c->parent = parent->id;
    c->born = step;
    c->member = member;
}

static void push_product(orc_prod_sink *sink, const double p[3], uint64_t parent_id, uint32_t step,
                         uint32_t parent_tag, uint32_t species, uint32_t member) {
    int64_t k;
#pragma omp atomic capture
    k = (*sink->counter)++;
    if (k < sink->cap_products) {
        orc_product *q = &sink->prod[k];
        q->p[0] = p[0]; q->p[1] = p[1]; q->p[2] = p[2];
        q->parent_id = parent_id; q->step = step; q->parent_tag = parent_tag;
        q->species = species; q->member = member;
    }
}

static void note_near(orc_lineage_info *info, uint32_t step) {
    if (info->first_near_step < 0) info->first_near_step = (int32_t)step;
}

/* Collinear momentum of magnitude |p| along the unit vector n (Sec. 3, App. A). */
static void collinear(const double n[3], double pmag, double out[3]) {
    out[0] = n[0] * pmag; out[1] = n[1] * pmag; out[2] = n[2] * pmag;
}
static double lepton_pmag(double g) { const double q = g * g - 1.0; return q > 0.0 ? sqrt(q) : 0.0; }

/* One step of a photon: nonlinear Breit-Wheeler by the optical-depth method. */
static void step_photon(orc_state *s, const double E[3], const double B[3], uint32_t n,
                        const orc_run_params *P, orc_prod_sink *sink, orc_lineage_info *info, orc_kids *kids) {
    double u[4];
    draws(P->seed, s->id, n, s->tag, u);
    if (s->tau < 0.0) { s->tau = -log(u[3]); s->tau0 = s->tau; }
    const double g = sqrt(s->p[0] * s->p[0] + s->p[1] * s->p[1] + s->p[2] * s->p[2]);
    const double chi = orc_chi(g, s->p, E, B, P->rho);
    const double R = orc_pair_rate(g, chi, P->pref);
    const double tn = s->tau - R * P->dt;                       /* Sec. 2: tau_d -= R dt */
    if (fabs(tn) <= P->near_od * s->tau0) note_near(info, n);
    if (!(tn < 0.0)) { s->tau = tn; return; }
    info->n_events++;
    double xe, xp;
    orc_pair_shares(u[1], chi, &xe, &xp);
    const double nh[3] = {s->p[0] / g, s->p[1] / g, s->p[2] / g};
    const double ge = xe * g, gp = xp * g;
    double pe[3], pp[3];
    collinear(nh, lepton_pmag(ge), pe);
    collinear(nh, lepton_pmag(gp), pp);
    push_product(sink, pe, s->id, n, s->tag, SP_ELECTRON, 1);
    push_product(sink, pp, s->id, n, s->tag, SP_POSITRON, 2);
    s->flags &= (uint8_t)~FL_ALIVE;                             /* the photon is converted */
    if (kids)
        for (int m = 0; m < 2; ++m)
            kid_init(kid_new(kids), s, m == 0 ? pe : pp, n, (uint32_t)(m + 1),
                     (uint8_t)(m == 0 ? SP_ELECTRON : SP_POSITRON), P);
}

/* Recoil of the emitting lepton and the emitted photon for s = u. */
static void emit_photon(orc_state *s, double gamma, double su, uint32_t n, orc_prod_sink *sink,
                        const orc_run_params *P, orc_kids *kids) {
    const double pm = sqrt(s->p[0] * s->p[0] + s->p[1] * s->p[1] + s->p[2] * s->p[2]);
    const double nh[3] = {s->p[0] / pm, s->p[1] / pm, s->p[2] / pm};
    const double gph = gamma * su / (1.0 + su);                 /* xi gamma_e */
    const double gnew = gamma / (1.0 + su);                     /* (1 - xi) gamma_e */
    double pph[3], pnew[3];
    collinear(nh, gph, pph);                                    /* photon: |p| = gamma */
    const double pm_new = lepton_pmag(gnew);
    collinear(nh, pm_new, pnew);
    push_product(sink, pph, s->id, n, s->tag, SP_PHOTON, 0);
    if (kids && P->cascade) kid_init(kid_new(kids), s, pph, n, 0u, SP_PHOTON, P);
    s->p[0] = pnew[0]; s->p[1] = pnew[1]; s->p[2] = pnew[2];
    /* READING: a lepton left without momentum is outside the ultrarelativistic regime the
     * rates assume (Sec. 4) and has no direction for collinear emission: it leaves the step */
    if (!(pm_new > 0.0)) s->flags &= (uint8_t)~FL_ALIVE;
}

/* One step of a lepton, LCFA emission by the optical-depth method. */
static void step_lepton_od(orc_state *s, const double E[3], const double B[3], uint32_t n,
                           const orc_run_params *P, orc_prod_sink *sink, orc_lineage_info *info, orc_kids *kids) {
    double u[4];
    draws(P->seed, s->id, n, s->tag, u);
    if (s->tau < 0.0) { s->tau = -log(u[3]); s->tau0 = s->tau; }
    const double g = sqrt(1.0 + s->p[0] * s->p[0] + s->p[1] * s->p[1] + s->p[2] * s->p[2]);
    const double chi = orc_chi(g, s->p, E, B, P->rho);
    const double R = orc_photon_rate(g, chi, P->pref);
    const double tn = s->tau - R * P->dt;
    if (fabs(tn) <= P->near_od * s->tau0) note_near(info, n);
    if (!(tn < 0.0)) { s->tau = tn; return; }
    info->n_events++;
    const double su = orc_photon_s(u[1], chi);
    emit_photon(s, g, su, n, sink, P, kids);
    s->tau = -log(u[0]);                                        /* fresh optical depth, Sec. 2 */
    s->tau0 = s->tau;
}

/* Unnormalised LCFA spectrum at photon energy gg (the prefactor of Eq. pe_dp is
 * common to both sides of Eq. rej_cond). */
static double rej_spectrum(double gg, double ge, double chi) {
    return orc_spectrum_pe(gg, ge, chi, 1.0);
}

/* One step of a lepton, beyond-LCFA emission by the local method (Sec. 5). */
static void step_lepton_blcfa(orc_state *s, const double E[3], const double B[3], uint32_t n,
                              const orc_run_params *P, orc_prod_sink *sink, orc_lineage_info *info,
                              orc_kids *kids) {
    blcfa_eval ev;
    const int was_new = (s->flags & FL_JUST_CREATED) != 0;
    uint8_t jc = (uint8_t)was_new;
    int gate;
    if (P->lepton_mode == MODE_BLCFA_PUSHED) {
        /* the pusher advances p^(n-1/2) to p^(n+1/2) first; the particle keeps it */
        double pn[3] = {s->p[0], s->p[1], s->p[2]};
        orc_boris_push(pn, E, B, s->species == SP_ELECTRON ? -1.0 : 1.0, P->dt);
        gate = orc_blcfa_update_pushed(s->p, pn, P->dt, P->rho, s->Fprev, s->dF, &jc, &ev);
        for (int k = 0; k < 3; ++k) s->p[k] = pn[k];
    } else {
        gate = orc_blcfa_update(s->p, E, B, P->dt, P->rho, s->Fprev, s->dF, &jc, &ev);
    }
    s->flags = (uint8_t)((s->flags & ~FL_JUST_CREATED) | (jc ? FL_JUST_CREATED : 0));
    if (was_new) return;                                        /* no emission after creation */
    double u[4];
    draws(P->seed, s->id, n, s->tag, u);
    const double R = orc_photon_rate(ev.gamma, ev.chi, P->pref);
    const double Rdt = R * P->dt;
    if (fabs(Rdt - u[0]) <= P->near_local * u[0]) note_near(info, n);
    if (!(Rdt > u[0])) return;                                  /* local test, Sec. 2 */
    info->n_events++;
    const double g = ev.gamma;
    const double su = orc_photon_s(u[1], ev.chi);
    const double gbar = g * su / (1.0 + su);
    if (gate) {
        info->n_gated++;
        const double gL = orc_blcfa_threshold(ev.F, ev.delta, g, ev.chi);
        if (fabs(gL - 0.75 * g) <= P->near_blcfa * 0.75 * g) note_near(info, n);
        if (!(gL < 0.75 * g)) { info->n_no_emission++; return; }   /* no emission, Sec. 5 */
        if (fabs(gbar - gL) <= P->near_blcfa * gL) note_near(info, n);
        if (!(gbar > gL)) {
            const double Sb = rej_spectrum(gbar, g, ev.chi), SL = rej_spectrum(gL, g, ev.chi);
            if (fabs(u[2] * Sb - SL) <= P->near_blcfa * SL) note_near(info, n);
            if (!(u[2] * Sb <= SL)) { info->n_rejected++; return; }  /* rejected, Eq. rej_cond */
        }
    }
    /* READING: without the gate the field is locally constant (or chi is
     * negligible) and the LCFA spectrum applies unchanged. */
    emit_photon(s, g, su, n, sink, P, kids);
}

/* One step of one particle.  `kids` (may be NULL) receives the particles it creates:
 * in a cascade every product, otherwise the leptons of a converted photon. */
static void step_particle(orc_state *s, const double *EB, uint32_t n, const orc_run_params *P,
                          orc_prod_sink *sink, orc_lineage_info *info, orc_kids *kids) {
    if (!(s->flags & FL_ALIVE)) return;
    const double *E = EB, *B = EB + 3;
    if (s->species == SP_PHOTON) step_photon(s, E, B, n, P, sink, info, kids);
    else if (P->lepton_mode != MODE_LCFA_OD) step_lepton_blcfa(s, E, B, n, P, sink, info, kids);
    else step_lepton_od(s, E, B, n, P, sink, info, kids);
}

/* Run `nsteps` steps (numbered step0 ...) for `n` independent primaries.
 *   p[3n], tau[n] (negative: drawn at the first step), id[n], tag[n],
 *   flags[n] (bit 0 alive, bit 1 just created), species[n],
 *   fprev[3n], dfprev[3n] (beyond-LCFA state; may be NULL when unused),
 *   fields[n * nsteps * 6]: (Ex,Ey,Ez,Bx,By,Bz) seen by primary i at step j,
 *     index (i*nsteps + j)*6; children created by a primary see its fields.
 * Updates the primaries' state in place, writes products (atomic counter),
 * and per-primary lineage info: first_near_step[n] and stats[4n] = (events, gated
 * beyond-LCFA events, events stopped by the 0.75 gamma_e rule, rejected samples).  Returns 0. */
int orc_mc_run(int64_t n, double *p, double *tau, const uint64_t *id, const uint32_t *tag,
               uint8_t *flags, const uint8_t *species, double *fprev, double *dfprev,
               const double *fields, const orc_run_params *P, orc_product *prod, int64_t cap_products,
               int64_t *n_products, int32_t *first_near_step, int32_t *stats) {
    *n_products = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i) {
        orc_state s;
        memset(&s, 0, sizeof(s));
        s.p[0] = p[3 * i]; s.p[1] = p[3 * i + 1]; s.p[2] = p[3 * i + 2];
        s.tau = tau[i]; s.tau0 = tau[i] > 0.0 ? tau[i] : 0.0;
        s.id = id[i]; s.tag = tag ? tag[i] : 0u;
        s.flags = flags[i]; s.species = species[i];
        if (fprev) for (int k = 0; k < 3; ++k) { s.Fprev[k] = fprev[3 * i + k]; s.dF[k] = dfprev[3 * i + k]; }
        orc_prod_sink sink = {0, cap_products, prod, n_products};
        orc_lineage_info info = {-1, 0, 0, 0, 0};
        orc_kids kids = {NULL, 0, 0};
        for (uint32_t j = 0; j < P->nsteps; ++j) {
            const uint32_t step = P->step0 + j;
            const double *EB = fields + ((size_t)i * P->nsteps + j) * 6;
            /* children created at earlier steps are stepped first (they were
             * created before this step began); then the primary */
            const int nk = kids.n;
            for (int c = 0; c < nk; ++c) step_particle(&kids.v[c], EB, step, P, &sink, &info, NULL);
            step_particle(&s, EB, step, P, &sink, &info, P->step_children ? &kids : NULL);
        }
        free(kids.v);
        p[3 * i] = s.p[0]; p[3 * i + 1] = s.p[1]; p[3 * i + 2] = s.p[2];
        tau[i] = s.tau; flags[i] = s.flags;
        if (fprev) for (int k = 0; k < 3; ++k) { fprev[3 * i + k] = s.Fprev[k]; dfprev[3 * i + k] = s.dF[k]; }
        first_near_step[i] = info.first_near_step;
        stats[4 * i] = info.n_events;
        stats[4 * i + 1] = info.n_gated;
        stats[4 * i + 2] = info.n_no_emission;
        stats[4 * i + 3] = info.n_rejected;
    }
    return 0;
}

/* One particle of a cascade as orc_mc_cascade returns it. */
typedef struct {
    double p[3];
    double tau;
    uint64_t id, parent_id;
    int64_t root;               /* index of the primary whose lineage it belongs to */
    uint32_t step;              /* step of creation */
    uint32_t member;            /* 0 emitted photon, 1 electron, 2 positron */
    uint8_t flags, species, pad[6];
} orc_cascade_particle;

/* Full cascade (the step of Sec. 2 with the collinear products of Sec. 3; READING: the
 * paper hands products back to the host code, here every product is stepped again):
 * as orc_mc_run, and every product (the photon of an emission, the two
 * leptons of a conversion) is also a particle of the lineage, with its own id
 * (orc_child_id), no optical depth yet and zero BLCFA state, stepped from the step after
 * its creation on, in the field of the lineage's primary, and creating particles in turn.
 * Within a step the particles created at earlier steps are stepped, then the primary; a
 * particle created during the step waits for the next one.  Primaries carry tag 0.  The
 * primaries' final state is written in place; every created particle (alive or not) goes
 * to `out` (atomic counter n_out; entries past cap_out are counted, not written). */
int orc_mc_cascade(int64_t n, double *p, double *tau, const uint64_t *id, uint8_t *flags, const uint8_t *species,
                   double *fprev, double *dfprev, const double *fields, const orc_run_params *P,
                   orc_product *prod, int64_t cap_products, int64_t *n_products,
                   orc_cascade_particle *out, int64_t cap_out, int64_t *n_out,
                   int32_t *first_near_step, int32_t *stats) {
    if (!P->cascade) return -1;
    *n_products = 0;
    *n_out = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; ++i) {
        orc_state s;
        memset(&s, 0, sizeof(s));
        s.p[0] = p[3 * i]; s.p[1] = p[3 * i + 1]; s.p[2] = p[3 * i + 2];
        s.tau = tau[i]; s.tau0 = tau[i] > 0.0 ? tau[i] : 0.0;
        s.id = id[i]; s.tag = 0u;
        s.flags = flags[i]; s.species = species[i];
        if (fprev) for (int k = 0; k < 3; ++k) { s.Fprev[k] = fprev[3 * i + k]; s.dF[k] = dfprev[3 * i + k]; }
        orc_prod_sink sink = {0, cap_products, prod, n_products};
        orc_lineage_info info = {-1, 0, 0, 0, 0};
        orc_kids kids = {NULL, 0, 0};
        for (uint32_t j = 0; j < P->nsteps; ++j) {
            const uint32_t step = P->step0 + j;
            const double *EB = fields + ((size_t)i * P->nsteps + j) * 6;
            const int nk = kids.n;
            for (int c = 0; c < nk; ++c) {
                orc_state t = kids.v[c];                        /* kids.v may move while t steps */
                step_particle(&t, EB, step, P, &sink, &info, &kids);
                kids.v[c] = t;
            }
            step_particle(&s, EB, step, P, &sink, &info, &kids);
        }
        p[3 * i] = s.p[0]; p[3 * i + 1] = s.p[1]; p[3 * i + 2] = s.p[2];
        tau[i] = s.tau; flags[i] = s.flags;
        if (fprev) for (int k = 0; k < 3; ++k) { fprev[3 * i + k] = s.Fprev[k]; dfprev[3 * i + k] = s.dF[k]; }
        first_near_step[i] = info.first_near_step;
        stats[4 * i] = info.n_events;
        stats[4 * i + 1] = info.n_gated;
        stats[4 * i + 2] = info.n_no_emission;
        stats[4 * i + 3] = info.n_rejected;
        for (int c = 0; c < kids.n; ++c) {
            int64_t k;
#pragma omp atomic capture
            k = (*n_out)++;
            if (k < cap_out) {
                const orc_state *t = &kids.v[c];
                orc_cascade_particle *o = &out[k];
                memset(o, 0, sizeof(*o));
                o->p[0] = t->p[0]; o->p[1] = t->p[1]; o->p[2] = t->p[2];
                o->tau = t->tau;
                o->id = t->id; o->parent_id = t->parent;
                o->root = i;
                o->step = t->born; o->member = t->member;
                o->flags = t->flags; o->species = t->species;
            }
        }
        free(kids.v);
    }
    return 0;
}

