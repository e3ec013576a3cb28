/*
 * qed_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU statement of the per-super-particle QED step of
 * Lobet, d'Humieres, Grech, Ruyer, Davoine, Gremillet, "Modeling of radiative
 * and quantum electrodynamics effects in PIC simulations of ultra-relativistic
 * laser-plasma interaction" (arXiv:1311.1107).  It exists to check the CUDA
 * library, shares no code with it, and is used only by the tests, the smoke
 * check and the benchmark's CPU-baseline leg.  Nothing in the product path may
 * call it.
 *
 * Everything is written in the order the paper states it:
 *   section 2  : chi_e / chi_gamma (Eq. 1), photon spectrum (Eq. 2), pair
 *                spectrum (Eq. 3);
 *   section 3  : Sokolov damping (Eq. 4), radiated power (Eq. 5), optical
 *                depth (Eq. 6), final optical depth tau^f = -log(xi), inverse
 *                CDF (Eq. 7), collinear recoil (Eq. 8), Monte-Carlo pair
 *                creation, the 2 m c^2 photon cut.
 * Readings of garbled or silent passages are marked READING and listed in the
 * design notes of the repository.
 *
 * Units: time in 1/omega, length in c/omega, momentum u = p/(m c), fields in
 * m c omega / e (E) and m omega / e (B), for a reference wavelength lambda.
 *
 * Parity: pinned by the tests in tests/test_oracle_*.py (scipy Bessel
 * functions, closed-form limits, Philox known-answer vectors, boost
 * invariance, Boris invariants, conservation at each emission).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* Physical constants (CODATA 2018) and normalised units                      */
/* ------------------------------------------------------------------------- */

typedef struct {
    double lambda_m;  /* reference wavelength [m]                               */
    double omega;     /* 2 pi c / lambda [1/s]                                  */
    double tau_c;     /* hbar / (m c^2) [s]  (section 2, after Eq. 2; READING:
                         the paper calls it a length, it is the Compton time)  */
    double a_S;       /* Schwinger field E_s = m^2 c^3/(e hbar) in m c omega/e */
    double C_rate;    /* alpha / (sqrt(3) pi tau_c omega): prefactor of Eq. 2,3
                         in units of omega                                      */
    double tau0w;     /* tau_0 omega, tau_0 = 2 e^2 / (12 pi eps0 m c^3), Eq. 4 */
    double alpha;
} or_units;

void or_units_init(double lambda_m, or_units *U)
{
    const double c = 299792458.0;
    const double hbar = 1.054571817e-34;
    const double me = 9.1093837015e-31;
    const double qe = 1.602176634e-19;
    const double eps0 = 8.8541878128e-12;
    const double alpha = 7.2973525693e-3;
    U->lambda_m = lambda_m;
    U->omega = 2.0 * OR_PI * c / lambda_m;
    U->tau_c = hbar / (me * c * c);
    /* E_s / (m c omega / e) = m c^2 / (hbar omega) = 1 / (tau_c omega) */
    U->a_S = 1.0 / (U->tau_c * U->omega);
    U->C_rate = alpha / (sqrt(3.0) * OR_PI * U->tau_c * U->omega);
    U->tau0w = 2.0 * qe * qe / (12.0 * OR_PI * eps0 * me * c * c * c) * U->omega;
    U->alpha = alpha;
}

/* ------------------------------------------------------------------------- */
/* Modified Bessel functions from their integral representation              */
/*   K_nu(x)             = int_0^inf exp(-x cosh t) cosh(nu t) dt            */
/*   int_x^inf K_1/3(s)ds = int_0^inf exp(-x cosh t) cosh(t/3)/cosh(t) dt    */
/* evaluated by the trapezoid rule in t (the integrands are analytic in the  */
/* strip |Im t| < pi/2, so the rule converges geometrically in 1/h).         */
/* ------------------------------------------------------------------------- */

/* Step: 1/16 for small x; for large x the integrand narrows like 1/sqrt(x)
 * and grows like exp(x y^2/2) off the real axis, so the step shrinks as
 * 0.6/sqrt(x) to keep the discretisation error below exp(-50). */
static double or_bessel_step(double x)
{
    double h = 0.6 / sqrt(x);
    return h < 0.0625 ? h : 0.0625;
}

/* cosh(t), sinh(t), cosh(2t/3), cosh(t/3)/cosh(t) at t = k/16 (cached) */
#define OR_BNODES 1024
static double or_bn_ch[OR_BNODES], or_bn_sh[OR_BNODES], or_bn_c23[OR_BNODES],
    or_bn_c13[OR_BNODES], or_bn_cnu[OR_BNODES];
static double or_bn_nu = -1.0;
static int or_bn_ready = 0;

static void or_bessel_nodes(void)
{
    if (or_bn_ready) return;
    for (int k = 0; k < OR_BNODES; k++) {
        double t = k * 0.0625;
        or_bn_ch[k] = cosh(t);
        or_bn_sh[k] = sinh(t);
        or_bn_c23[k] = cosh(2.0 * t / 3.0);
        or_bn_c13[k] = cosh(t / 3.0) / cosh(t);
    }
    or_bn_ready = 1;
}

/* One trapezoid pass giving K_nu(x) and int_x^inf K_1/3 together (they share
 * exp(-x cosh t)).  Results carry the factor exp(-x) scaled back in. */
static void or_bessel_both(double x, double nu, double *knu, double *ik13)
{
    if (!(x > 0.0)) {
        *knu = INFINITY;
        *ik13 = INFINITY;
        return;
    }
    if (x > 740.0) {
        *knu = 0.0;
        *ik13 = 0.0;
        return;
    }
    const double h = or_bessel_step(x);
    const int cached = (h == 0.0625);
    if (cached) or_bessel_nodes();
    if (cached && nu != or_bn_nu && nu != 2.0 / 3.0) {
        for (int k = 0; k < OR_BNODES; k++) or_bn_cnu[k] = cosh(nu * k * 0.0625);
        or_bn_nu = nu;
    }
    double s1 = 0.0, s2 = 0.0;
    for (int k = 0; k < 1000000; k++) {
        double t = k * h, ch, sh, gnu, g13;
        if (cached && k < OR_BNODES) {
            ch = or_bn_ch[k];
            sh = or_bn_sh[k];
            gnu = (nu == 2.0 / 3.0) ? or_bn_c23[k] : or_bn_cnu[k];
            g13 = or_bn_c13[k];
        } else {
            ch = cosh(t);
            sh = sinh(t);
            gnu = cosh(nu * t);
            g13 = cosh(t / 3.0) / ch;
        }
        double e = exp(-x * (ch - 1.0));
        double a = e * gnu, b = e * g13;
        if (k == 0) {
            a *= 0.5;
            b *= 0.5;
        }
        s1 += a;
        s2 += b;
        /* stop once past the maximum of the integrands and negligible */
        if (x * sh > (nu > 1.0 ? nu : 1.0) && a < 1e-18 * s1 && b < 1e-18 * s2) break;
    }
    double sc = exp(-x) * h;
    *knu = s1 * sc;
    *ik13 = s2 * sc;
}

double or_bessel_K(double nu, double x)
{
    double k, i;
    or_bessel_both(x, nu, &k, &i);
    return k;
}

double or_int_K13(double x)
{
    double k, i;
    or_bessel_both(x, 2.0 / 3.0, &k, &i);
    return i;
}

/* ------------------------------------------------------------------------- */
/* Spectra (section 2)                                                        */
/* ------------------------------------------------------------------------- */

/* Eq. 2 in the variable u = chi_gamma / chi_e = gamma_gamma / gamma_e:
 *   d2N/(dt du) = C_rate / gamma_e * F_gamma(u; chi_e),
 *   F_gamma = (2 + 3 chi_gamma y) K_2/3(2y) - int_2y^inf K_1/3,
 *   y = chi_gamma / (3 chi_e (chi_e - chi_gamma)),  2y = 2u/(3 chi (1-u)),
 *   3 chi_gamma y = u^2/(1-u).
 * READING: the bracket of Eq. 2 is printed with the opposite overall sign,
 * which makes the rate negative for every u; the positive form is used.
 * omu = 1 - u is passed separately to avoid cancellation near u = 1. */
double or_F_gamma(double u, double omu, double chi)
{
    if (!(u > 0.0) || !(omu > 0.0) || !(chi > 0.0)) return 0.0;
    double z = 2.0 * u / (3.0 * chi * omu), k23, ik13;
    or_bessel_both(z, 2.0 / 3.0, &k23, &ik13);
    return (2.0 + u * u / omu) * k23 - ik13;
}

/* Eq. 3 in the variable v = chi_- / chi_gamma (created electron):
 *   d2N/(dt dv) = C_rate / gamma_gamma * F_pair(v; chi_gamma),
 *   F_pair = int_2y^inf K_1/3 - (2 - 3 chi_gamma y) K_2/3(2y),
 * READING: y is the emission y with chi_e -> chi_-, (chi_e - chi_gamma) ->
 * chi_+ = chi_gamma - chi_-, i.e. y = 1/(3 chi v (1-v)), 3 chi_gamma y =
 * 1/(v(1-v)). */
double or_F_pair(double v, double omv, double chi)
{
    if (!(v > 0.0) || !(omv > 0.0) || !(chi > 0.0)) return 0.0;
    double vv = v * omv;
    double z = 2.0 / (3.0 * chi * vv), k23, ik13;
    or_bessel_both(z, 2.0 / 3.0, &k23, &ik13);
    return ik13 - (2.0 - 1.0 / vv) * k23;
}

/* ------------------------------------------------------------------------- */
/* Quadrature over (0,1): composite Gauss-Legendre in w with the map          */
/*   u(w) = w^3 / (w^3 + (1-w)^3)                                             */
/* which removes the u^(-2/3) end-point behaviour of Eq. 2 (and its mirror).  */
/* ------------------------------------------------------------------------- */

#define OR_GL_N 8
static double or_gl_x[OR_GL_N], or_gl_w[OR_GL_N];
static int or_gl_ready = 0;

/* Gauss-Legendre nodes on [-1,1]: roots of P_n by Newton iteration. */
static void or_gl_init(void)
{
    if (or_gl_ready) return;
    const int n = OR_GL_N;
    for (int i = 0; i < n; i++) {
        double x = cos(OR_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
        }
        or_gl_x[i] = x;
        or_gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    or_gl_ready = 1;
}

static void or_cubic_map(double w, double *u, double *omu, double *dudw)
{
    double a = w * w * w, b = (1.0 - w) * (1.0 - w) * (1.0 - w), d = a + b;
    *u = a / d;
    *omu = b / d;
    *dudw = 3.0 * w * w * (1.0 - w) * (1.0 - w) / (d * d);
}

/* which: 0 -> int F_gamma du, 1 -> int u F_gamma du, 2 -> int F_pair dv */
static double or_integrand(int which, double w, double chi)
{
    double u, omu, dudw;
    or_cubic_map(w, &u, &omu, &dudw);
    if (which == 0) return or_F_gamma(u, omu, chi) * dudw;
    if (which == 1) return u * or_F_gamma(u, omu, chi) * dudw;
    return or_F_pair(u, omu, chi) * dudw;
}

#define OR_PANELS 256

/* int over w in [wa, wb] with panels of width <= 1/OR_PANELS */
static double or_integrate_w(int which, double chi, double wa, double wb)
{
    or_gl_init();
    if (!(wb > wa)) return 0.0;
    int np = (int)ceil((wb - wa) * OR_PANELS);
    if (np < 1) np = 1;
    double hw = (wb - wa) / np, sum = 0.0;
    for (int p = 0; p < np; p++) {
        double a = wa + p * hw, mid = a + 0.5 * hw;
        for (int i = 0; i < OR_GL_N; i++)
            sum += or_gl_w[i] * or_integrand(which, mid + 0.5 * hw * or_gl_x[i], chi);
    }
    return sum * 0.5 * hw;
}

/* H and G together over w in [0, 1] (same quadrature as or_integrate_w) */
static void or_integrate_HG(double chi, double *H, double *G)
{
    or_gl_init();
    const int np = OR_PANELS;
    double hw = 1.0 / np, sh = 0.0, sg = 0.0;
    for (int p = 0; p < np; p++) {
        double mid = (p + 0.5) * hw;
        for (int i = 0; i < OR_GL_N; i++) {
            double u, omu, dudw;
            or_cubic_map(mid + 0.5 * hw * or_gl_x[i], &u, &omu, &dudw);
            double f = or_F_gamma(u, omu, chi) * dudw;
            sh += or_gl_w[i] * f;
            sg += or_gl_w[i] * u * f;
        }
    }
    *H = sh * 0.5 * hw;
    *G = sg * 0.5 * hw;
}

/* w such that u(w) = u, i.e. logit(w) = logit(u)/3 */
static double or_w_of_logit(double s) { return 1.0 / (1.0 + exp(-s / 3.0)); }

/* H(chi) = int_0^1 F_gamma du  (Eq. 6: dtau/dt = C_rate H / gamma) */
double or_H_exact(double chi) { return or_integrate_w(0, chi, 0.0, 1.0); }
/* G(chi) = int_0^1 u F_gamma du (Eq. 5: P_rad = m c^2 omega C_rate G) */
double or_G_exact(double chi) { return or_integrate_w(1, chi, 0.0, 1.0); }
/* T(chi) = int_0^1 F_pair dv (pair rate C_rate T / gamma_gamma) */
double or_T_exact(double chi) { return or_integrate_w(2, chi, 0.0, 1.0); }

/* Eq. 7: P_gamma(0 -> u) = int_0^u F_gamma / int_0^1 F_gamma, u given by its
 * logit s = log(u/(1-u)) */
double or_cdf_gamma_exact(double s, double chi)
{
    double tot = or_H_exact(chi);
    if (!(tot > 0.0)) return 0.0;
    return or_integrate_w(0, chi, 0.0, or_w_of_logit(s)) / tot;
}

/* pair CDF P_pm(0 -> v), v given by its logit */
double or_cdf_pair_exact(double s, double chi)
{
    double tot = or_T_exact(chi);
    if (!(tot > 0.0)) return 0.0;
    return or_integrate_w(2, chi, 0.0, or_w_of_logit(s)) / tot;
}

/* ------------------------------------------------------------------------- */
/* Tables (grid definition shared with the library as a specification only)  */
/*   rate grid : chi_j = 2^(-14 + j/32) (1 + (j mod 32)/32), j = 0..768      */
/*   CDF grid  : chi_j = 2^(-14 + j/4)  (1 + (j mod 4)/4),   j = 0..96       */
/*   emission u-grid: logit s_i = -30 + 50 i/255,  i = 0..255                 */
/*   pair v-grid    : logit s_i = -20 + 40 i/255,  i = 0..255                 */
/* Rate tables hold smooth scaled forms, interpolated linearly in chi:        */
/*   H(chi);  Gs = G(chi)/chi;  Ts = T(chi) exp(8/(3 chi)) for chi >= 2^-8     */
/* (the exponent is the small-chi law of the pair rate; below 2^-8 the pair    */
/* rate is below exp(-680) and is taken as zero).                             */
/* ------------------------------------------------------------------------- */

#define OR_NRATE 769
#define OR_RATE_PER_OCT 32
#define OR_NCDF 97
#define OR_CDF_PER_OCT 4
#define OR_NS 256
#define OR_CHI_EXP0 (-14)
#define OR_PAIR_CHI_MIN 0x1.0p-8
#define OR_SG_MIN (-30.0)
#define OR_SG_MAX (20.0)
#define OR_SP_MIN (-20.0)
#define OR_SP_MAX (20.0)

typedef struct {
    double chi[OR_NRATE], H[OR_NRATE], Gs[OR_NRATE], Ts[OR_NRATE];
    double chic[OR_NCDF];
    double sg[OR_NS], ug[OR_NS];      /* emission logit nodes and u values */
    double sp[OR_NS], vp[OR_NS];      /* pair logit nodes and v values     */
    double Cg[OR_NCDF * OR_NS];       /* emission CDF rows                 */
    double Cp[OR_NCDF * OR_NS];       /* pair CDF rows                     */
} or_tables;

size_t or_tables_size(void) { return sizeof(or_tables); }

static double or_grid_node(int j, int per_oct)
{
    return ldexp(1.0 + (double)(j % per_oct) / per_oct, OR_CHI_EXP0 + j / per_oct);
}

/* One CDF row: cumulative integral between consecutive logit nodes. */
static void or_cdf_row(int which, double chi, const double *s, double *C)
{
    double acc = 0.0, wprev = 0.0;
    for (int i = 0; i < OR_NS; i++) {
        double wi = or_w_of_logit(s[i]);
        acc += or_integrate_w(which, chi, wprev, wi);
        C[i] = acc;
        wprev = wi;
    }
    double tot = acc + or_integrate_w(which, chi, wprev, 1.0);
    if (tot > 0.0 && isfinite(tot)) {
        for (int i = 0; i < OR_NS; i++) C[i] /= tot;
    } else {
        /* READING: rows whose total rate underflows (pair rows at tiny chi)
         * carry the CDF of v itself; they are never reached by an event. */
        for (int i = 0; i < OR_NS; i++) C[i] = 1.0 / (1.0 + exp(-s[i]));
    }
}

void or_tables_build(or_tables *T)
{
    for (int j = 0; j < OR_NRATE; j++) {
        double chi = or_grid_node(j, OR_RATE_PER_OCT), G;
        T->chi[j] = chi;
        or_integrate_HG(chi, &T->H[j], &G);
        T->Gs[j] = G / chi;
        T->Ts[j] = chi >= OR_PAIR_CHI_MIN ? or_T_exact(chi) * exp(8.0 / (3.0 * chi)) : 0.0;
    }
    for (int i = 0; i < OR_NS; i++) {
        T->sg[i] = OR_SG_MIN + (OR_SG_MAX - OR_SG_MIN) * i / (OR_NS - 1);
        T->ug[i] = 1.0 / (1.0 + exp(-T->sg[i]));
        T->sp[i] = OR_SP_MIN + (OR_SP_MAX - OR_SP_MIN) * i / (OR_NS - 1);
        T->vp[i] = 1.0 / (1.0 + exp(-T->sp[i]));
    }
    for (int j = 0; j < OR_NCDF; j++) {
        double chi = or_grid_node(j, OR_CDF_PER_OCT);
        T->chic[j] = chi;
        or_cdf_row(0, chi, T->sg, &T->Cg[j * OR_NS]);
        or_cdf_row(2, chi, T->sp, &T->Cp[j * OR_NS]);
    }
}

/* Locate chi on a node array by bisection: largest j with nodes[j] <= chi,
 * and the linear weight f = (chi - nodes[j]) / (nodes[j+1] - nodes[j]).
 * Requires nodes[0] <= chi < nodes[n-1]. */
static int or_locate(const double *nodes, int n, double chi, double *f)
{
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (nodes[mid] <= chi) lo = mid;
        else hi = mid;
    }
    *f = (chi - nodes[lo]) / (nodes[lo + 1] - nodes[lo]);
    return lo;
}

static double or_lerp(double a, double b, double f)
{
    double d = b - a;
    double p = f * d;
    return a + p;
}

/* Rate lookups: which = 0 -> H, 1 -> G, 2 -> T.  Below the grid the
 * classical closed forms H = 5 pi chi / 2, G = 2 pi chi^2 / sqrt(3) are used
 * and T = 0; at or above the last node the last node value is used and
 * *clamped is set. */
double or_lookup_rate(const or_tables *T, int which, double chi, int *clamped)
{
    if (which == 2 && !(chi >= OR_PAIR_CHI_MIN)) return 0.0;
    if (!(chi >= T->chi[0])) {
        if (which == 0) return 2.5 * OR_PI * chi;
        return 2.0 * OR_PI * chi * chi / sqrt(3.0);
    }
    const double *V = which == 0 ? T->H : (which == 1 ? T->Gs : T->Ts);
    double v, c = chi;
    if (chi >= T->chi[OR_NRATE - 1]) {
        if (clamped) *clamped = 1;
        v = V[OR_NRATE - 1];
        c = T->chi[OR_NRATE - 1];
    } else {
        double f;
        int j = or_locate(T->chi, OR_NRATE, chi, &f);
        v = or_lerp(V[j], V[j + 1], f);
    }
    if (which == 1) return v * c;
    if (which == 2) return v * exp(-8.0 / (3.0 * c));
    return v;
}

/* Invert one CDF row at xi (Eq. 7).  Between nodes the CDF is linear in the
 * logit s.  Emission rows: below the first node P ~ u^(1/3) (small-u limit of
 * Eq. 2), so u = u_0 (xi / C_0)^3; pair rows: clamp to the first node.  Above
 * the last node: clamp to the last node. */
static double or_row_invert(const double *C, const double *s, const double *x,
                            double xi, int power_tail)
{
    if (xi <= C[0]) {
        if (power_tail && C[0] > 0.0) {
            double r = xi / C[0];
            return x[0] * r * r * r;
        }
        return x[0];
    }
    if (xi >= C[OR_NS - 1]) return x[OR_NS - 1];
    int lo = 0, hi = OR_NS - 1;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (C[mid] < xi) lo = mid;
        else hi = mid;
    }
    double ds = s[lo + 1] - s[lo];
    double t = (xi - C[lo]) / (C[lo + 1] - C[lo]);
    double sv = s[lo] + t * ds;
    return 1.0 / (1.0 + exp(-sv));
}

/* Sample the photon energy fraction u = chi_gamma/chi_e for a given chi_e
 * (Eq. 7): rows j, j+1 of the CDF grid bracketing chi are inverted and the
 * results interpolated linearly in chi.  Below the grid the spectrum shape
 * scales with chi (classical limit), so u = (chi/chi_0) R_0(xi). */
double or_sample_gamma(const or_tables *T, double chi, double xi, int *clamped)
{
    if (!(chi >= T->chic[0])) {
        double r0 = or_row_invert(&T->Cg[0], T->sg, T->ug, xi, 1);
        return (chi / T->chic[0]) * r0;
    }
    if (chi >= T->chic[OR_NCDF - 1]) {
        if (clamped) *clamped = 1;
        return or_row_invert(&T->Cg[(OR_NCDF - 1) * OR_NS], T->sg, T->ug, xi, 1);
    }
    double f;
    int j = or_locate(T->chic, OR_NCDF, chi, &f);
    double ra = or_row_invert(&T->Cg[j * OR_NS], T->sg, T->ug, xi, 1);
    double rb = or_row_invert(&T->Cg[(j + 1) * OR_NS], T->sg, T->ug, xi, 1);
    return or_lerp(ra, rb, f);
}

/* Sample v = chi_-/chi_gamma of the created electron (pair CDF). */
double or_sample_pair(const or_tables *T, double chi, double xi, int *clamped)
{
    if (!(chi >= T->chic[0])) return or_row_invert(&T->Cp[0], T->sp, T->vp, xi, 0);
    if (chi >= T->chic[OR_NCDF - 1]) {
        if (clamped) *clamped = 1;
        return or_row_invert(&T->Cp[(OR_NCDF - 1) * OR_NS], T->sp, T->vp, xi, 0);
    }
    double f;
    int j = or_locate(T->chic, OR_NCDF, chi, &f);
    double ra = or_row_invert(&T->Cp[j * OR_NS], T->sp, T->vp, xi, 0);
    double rb = or_row_invert(&T->Cp[(j + 1) * OR_NS], T->sp, T->vp, xi, 0);
    return or_lerp(ra, rb, f);
}

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from its        */
/* published definition; uniform maps for the random numbers of section 3.    */
/* ------------------------------------------------------------------------- */

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 53-bit uniform in ]0,1] from two 32-bit words (section 3 asks for
 * xi in ]0,1]; the same map serves xi' and xi''). */
double or_u53(uint32_t a, uint32_t b)
{
    uint64_t m = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
    return (double)(m + 1) * 0x1.0p-53;
}

enum { OR_SP_ELECTRON = 0, OR_SP_POSITRON = 1, OR_SP_PHOTON = 2 };
enum { OR_RNG_INIT = 0, OR_RNG_EMIT = 1, OR_RNG_PHOTON_TAU = 2, OR_RNG_PAIR = 3, OR_RNG_PAIR_POS = 4 };

/* Counter layout: (slot lo, slot hi, step, species<<24 | purpose<<16 | k),
 * key = (seed lo, seed hi). */
void or_draw(uint64_t seed, int species, int purpose, int64_t slot, int64_t step, int k,
             uint32_t out[4])
{
    uint32_t ctr[4], key[2];
    ctr[0] = (uint32_t)((uint64_t)slot & 0xFFFFFFFFu);
    ctr[1] = (uint32_t)((uint64_t)slot >> 32);
    ctr[2] = (uint32_t)((uint64_t)step & 0xFFFFFFFFu);
    ctr[3] = ((uint32_t)species << 24) | ((uint32_t)purpose << 16) | ((uint32_t)k & 0xFFFFu);
    key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
    key[1] = (uint32_t)(seed >> 32);
    or_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------- */
/* Fields                                                                     */
/* ------------------------------------------------------------------------- */

enum { OR_FIELD_NONE = 0, OR_FIELD_PLANE = 1, OR_FIELD_GAUSSIAN = 2, OR_FIELD_YEE2D = 3,
       OR_FIELD_UNIFORM_B = 4 };

typedef struct {
    int kind;
    double a0;          /* peak normalised amplitude                         */
    double w0;          /* Gaussian: waist (1/e field radius at focus)       */
    double tau_fwhm;    /* Gaussian: FWHM duration of the intensity          */
    double x_focus;     /* Gaussian: focal plane                             */
    double t_focus;     /* Gaussian: time the envelope peak crosses x_focus  */
    double b0;          /* uniform B_z                                       */
    const float *yee[6];/* Ex Ey Ez Bx By Bz, each ny rows of nx values      */
    int64_t nx, ny;
    double dx, dy, x0, y0;
} or_field;

/* Linear (cloud-in-cell) interpolation of one staggered Yee component.
 * Nodes outside the grid contribute zero field. */
static double or_yee_component(const or_field *F, int c, double x, double y)
{
    static const double ox[6] = {0.5, 0.0, 0.0, 0.0, 0.5, 0.5};
    static const double oy[6] = {0.0, 0.5, 0.0, 0.5, 0.0, 0.5};
    double gx = (x - F->x0) / F->dx - ox[c];
    double gy = (y - F->y0) / F->dy - oy[c];
    double fi = floor(gx), fj = floor(gy);
    double fx = gx - fi, fy = gy - fj;
    double sum = 0.0;
    for (int b = 0; b < 2; b++) {
        for (int a = 0; a < 2; a++) {
            double ii = fi + a, jj = fj + b;
            /* written so that NaN positions fail the test too */
            if (!(ii >= 0.0 && jj >= 0.0 && ii < (double)F->nx && jj < (double)F->ny)) continue;
            double wgt = (a ? fx : 1.0 - fx) * (b ? fy : 1.0 - fy);
            sum += wgt * (double)F->yee[c][(int64_t)jj * F->nx + (int64_t)ii];
        }
    }
    return sum;
}

void or_field_eval(const or_field *F, double x, double y, double z, double t, double E[3],
                   double B[3])
{
    E[0] = E[1] = E[2] = B[0] = B[1] = B[2] = 0.0;
    if (F->kind == OR_FIELD_PLANE) {
        /* linearly polarised plane wave along +x: E_y = B_z = a0 cos(t - x) */
        double f = F->a0 * cos(t - x);
        E[1] = f;
        B[2] = f;
    } else if (F->kind == OR_FIELD_GAUSSIAN) {
        /* lowest-order paraxial Gaussian pulse along +x, polarised along y,
         * transverse fields only (B_z = E_y) */
        double xi = x - F->x_focus;
        double eta = (t - F->t_focus) - xi;
        double zr = 0.5 * F->w0 * F->w0;
        double q = xi / zr;
        double wr2 = 1.0 + q * q;
        double r2 = y * y + z * z;
        double env = -r2 / (F->w0 * F->w0 * wr2) - 2.0 * log(2.0) * eta * eta /
                                                       (F->tau_fwhm * F->tau_fwhm);
        double amp = F->a0 / sqrt(wr2) * exp(env);
        double phase = -eta + r2 * xi / (2.0 * (xi * xi + zr * zr)) - atan(q);
        double f = amp * cos(phase);
        E[1] = f;
        B[2] = f;
    } else if (F->kind == OR_FIELD_YEE2D) {
        for (int c = 0; c < 3; c++) E[c] = or_yee_component(F, c, x, y);
        for (int c = 0; c < 3; c++) B[c] = or_yee_component(F, 3 + c, x, y);
    } else if (F->kind == OR_FIELD_UNIFORM_B) {
        B[2] = F->b0;
    }
}

/* ------------------------------------------------------------------------- */
/* Lorentz-invariant quantum parameters (Eq. 1)                               */
/* ------------------------------------------------------------------------- */

/* chi_e = (gamma/E_s) sqrt(E_par^2/gamma^2 + (E_perp + v x B)^2)
 *       = sqrt(|gamma E + u x B|^2 - (u.E)^2) / a_S  (normalised units) */
double or_chi_e(const double E[3], const double B[3], const double u[3], double gamma,
                double a_S)
{
    double ax = gamma * E[0] + (u[1] * B[2] - u[2] * B[1]);
    double ay = gamma * E[1] + (u[2] * B[0] - u[0] * B[2]);
    double az = gamma * E[2] + (u[0] * B[1] - u[1] * B[0]);
    double ue = u[0] * E[0] + u[1] * E[1] + u[2] * E[2];
    double s = ax * ax + ay * ay + az * az - ue * ue;
    return s > 0.0 ? sqrt(s) / a_S : 0.0;
}

/* chi_gamma = (gamma_gamma/E_s) |E_perp + c k^ x B| with k^ the photon
 * direction.  READING: the printed "c x B" stands for c k^ x B; equivalently
 * gamma_gamma sqrt(|E + k^ x B|^2 - (k^.E)^2) / a_S. */
double or_chi_gamma(const double E[3], const double B[3], const double u[3], double a_S)
{
    double g = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    if (!(g > 0.0)) return 0.0;
    double k[3] = {u[0] / g, u[1] / g, u[2] / g};
    double ax = E[0] + (k[1] * B[2] - k[2] * B[1]);
    double ay = E[1] + (k[2] * B[0] - k[0] * B[2]);
    double az = E[2] + (k[0] * B[1] - k[1] * B[0]);
    double ke = k[0] * E[0] + k[1] * E[1] + k[2] * E[2];
    double s = ax * ax + ay * ay + az * az - ke * ke;
    return s > 0.0 ? g * sqrt(s) / a_S : 0.0;
}

/* ------------------------------------------------------------------------- */
/* Boris push for the Lorentz force f_l of Eq. 4 (charge q = -1 e-, +1 e+)    */
/* ------------------------------------------------------------------------- */

void or_boris(double q, double dt, const double E[3], const double B[3], double u[3])
{
    double h = 0.5 * q * dt;
    double um[3] = {u[0] + h * E[0], u[1] + h * E[1], u[2] + h * E[2]};
    double g = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    double t[3] = {h * B[0] / g, h * B[1] / g, h * B[2] / g};
    double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    double s[3] = {2.0 * t[0] / (1.0 + t2), 2.0 * t[1] / (1.0 + t2), 2.0 * t[2] / (1.0 + t2)};
    double up[3] = {um[0] + (um[1] * t[2] - um[2] * t[1]),
                    um[1] + (um[2] * t[0] - um[0] * t[2]),
                    um[2] + (um[0] * t[1] - um[1] * t[0])};
    double upl[3] = {um[0] + (up[1] * s[2] - up[2] * s[1]),
                     um[1] + (up[2] * s[0] - up[0] * s[2]),
                     um[2] + (up[0] * s[1] - up[1] * s[0])};
    u[0] = upl[0] + h * E[0];
    u[1] = upl[1] + h * E[1];
    u[2] = upl[2] + h * E[2];
}

/* ------------------------------------------------------------------------- */
/* Species, parameters and the step                                           */
/* ------------------------------------------------------------------------- */

typedef struct {
    int64_t n;        /* live slots                                  */
    int64_t cap;      /* slot capacity                               */
    double *x, *y, *z;/* z may be NULL (2D)                          */
    double *ux, *uy, *uz, *tau, *w;
    double *chi;      /* optional: chi of the last step per slot     */
    double *margin;   /* optional: smallest |tau - dtau| / dtau seen */
    int32_t *nemit;   /* optional: emissions per slot (cumulative)   */
    int64_t *ids;     /* optional: the slot number each entry stands for
                         in the random streams (default: its index);
                         lets a test run a sample of a larger population */
    int64_t id_base;  /* without ids: slot i is particle id_base + i ...     */
    int64_t id_split; /* ... below id_split when id_split > 0, and particle
                         id_append + (i - id_split) from there on (the ids a
                         part of a split population gives what it appends) */
    int64_t id_append;
} or_species;

/* The particle id of slot i by the species' id rule (ids array aside). */
static int64_t or_slot_id(const or_species *S, int64_t i)
{
    if (S->id_split > 0 && i >= S->id_split) return S->id_append + (i - S->id_split);
    return S->id_base + i;
}

/* The particle id whose random streams slot i draws from. */
static int64_t or_id(const or_species *S, int64_t i) { return S->ids ? S->ids[i] : or_slot_id(S, i); }

typedef struct {
    double dt;
    int64_t step;
    uint64_t seed;
    double chi_th;           /* continuous (Sokolov) regime below this chi   */
    double photon_min_gamma; /* super-photons stored only above this energy  */
    int32_t pairs;           /* Monte-Carlo pair creation on/off             */
    int32_t max_emit;        /* emissions allowed per particle per step      */
    int32_t recoil;          /* 1 = apply Eq. 8 (0 only for spectrum tests)  */
    int32_t dims;            /* 2 or 3                                       */
    double noise;            /* test-only sensitivity probe: relative kick of
                                +-noise given to each lepton's momentum after
                                every step (0 = the method itself)           */
    uint64_t noise_key;      /* selects an independent pattern of kick signs  */
} or_params;

typedef struct {
    int64_t n_emit;          /* all emission events (stored or not)      */
    int64_t n_photon;        /* photons appended (stored)                */
    int64_t n_photon_drop;   /* photons over capacity                    */
    int64_t n_subthreshold;  /* photons below photon_min_gamma           */
    int64_t n_pair;          /* pair events                              */
    int64_t n_pair_drop;     /* pairs over capacity                      */
    int64_t n_saturated;     /* steps that reached max_emit              */
    int64_t n_clamped;       /* table lookups above the table range      */
    int64_t n_continuous;    /* particle-steps in the Sokolov regime     */
    double e_subthreshold;   /* sum w gamma_gamma below the photon cut   */
    double e_dropped;        /* sum w gamma of dropped particles         */
} or_stats;

static void or_record_margin(or_species *S, int64_t i, double tau, double dtau)
{
    if (!S->margin || !(dtau > 0.0)) return;
    double m = fabs(tau - dtau) / dtau;
    if (m < S->margin[i]) S->margin[i] = m;
}

/* Append a super-photon (section 3: created along the electron velocity,
 * with the emitter's weight and position).  ord = its ordinal this step. */
static void or_append_photon(or_species *P, int64_t base, int64_t *ord, const double x[3],
                             const double ku[3], double w, double tau, or_stats *st,
                             double egam)
{
    int64_t slot = base + (*ord)++;
    if (slot >= P->cap) {
        st->n_photon_drop++;
        st->e_dropped += w * egam;
        return;
    }
    P->x[slot] = x[0];
    P->y[slot] = x[1];
    if (P->z) P->z[slot] = x[2];
    P->ux[slot] = ku[0];
    P->uy[slot] = ku[1];
    P->uz[slot] = ku[2];
    P->tau[slot] = tau;
    P->w[slot] = w;
    if (P->chi) P->chi[slot] = 0.0;
    if (P->margin) P->margin[slot] = INFINITY;
    if (P->nemit) P->nemit[slot] = 0;
    if (P->ids) P->ids[slot] = or_slot_id(P, slot);
    st->n_photon++;
}

/* One step of one lepton (section 3, with the time discretisation READING:
 * fields at x^n, Boris to u^(n+1/2), Sokolov explicit on u^(n+1/2) below
 * chi_th, otherwise optical depth + Monte-Carlo emission, then x^(n+1)). */
static void or_lepton_step(const or_units *U, const or_tables *T, const or_field *F,
                           const or_params *P, int species, or_species *S, int64_t i,
                           or_species *Ph, int64_t ph_base, int64_t *ph_ord, or_stats *st)
{
    const double q = species == OR_SP_ELECTRON ? -1.0 : 1.0;
    const double dt = P->dt;
    const double t = (double)P->step * dt;
    double x[3] = {S->x[i], S->y[i], S->z ? S->z[i] : 0.0};
    double u[3] = {S->ux[i], S->uy[i], S->uz[i]};
    double tau = S->tau[i];
    double E[3], B[3];
    int clamped = 0;

    or_field_eval(F, x[0], x[1], x[2], t, E, B);
    or_boris(q, dt, E, B, u);
    double gam = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double chi = or_chi_e(E, B, u, gam, U->a_S);
    if (S->chi) S->chi[i] = chi;
    double dv[3] = {0.0, 0.0, 0.0};
    /* the regime choice is a decision too: record how close it was */
    if (S->margin && P->chi_th > 0.0) {
        double m = fabs(chi - P->chi_th) / P->chi_th;
        if (m < S->margin[i]) S->margin[i] = m;
    }

    if (chi < P->chi_th) {
        /* Eq. 4-5, continuous regime: f_l = q (E + v x B),
         * dv = tau0 (f_l - v (v.f_l)) / (1 + tau0 v.f_l)   (READING of the
         * printed numerator/denominator, see design notes),
         * du/dt = f_l + q dv x B - P_rad v, P_rad = C_rate G(chi). */
        st->n_continuous++;
        double v[3] = {u[0] / gam, u[1] / gam, u[2] / gam};
        double fl[3] = {q * (E[0] + (v[1] * B[2] - v[2] * B[1])),
                        q * (E[1] + (v[2] * B[0] - v[0] * B[2])),
                        q * (E[2] + (v[0] * B[1] - v[1] * B[0]))};
        double vf = v[0] * fl[0] + v[1] * fl[1] + v[2] * fl[2];
        double den = 1.0 + U->tau0w * vf;
        for (int c = 0; c < 3; c++) dv[c] = U->tau0w * (fl[c] - v[c] * vf) / den;
        double prad = U->C_rate * or_lookup_rate(T, 1, chi, &clamped);
        double dvxb[3] = {dv[1] * B[2] - dv[2] * B[1], dv[2] * B[0] - dv[0] * B[2],
                          dv[0] * B[1] - dv[1] * B[0]};
        for (int c = 0; c < 3; c++) u[c] = u[c] + dt * (q * dvxb[c] - prad * v[c]);
        gam = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    } else {
        /* Eq. 6 with the residual-time sub-loop (READING): after an event
         * the remaining fraction r of the step continues with the new state. */
        double r = 1.0;
        for (int k = 0;; k++) {
            double H = or_lookup_rate(T, 0, chi, &clamped);
            double wdt = U->C_rate * H / gam * dt;
            double dtau = wdt * r;
            or_record_margin(S, i, tau, dtau);
            if (!(dtau > 0.0) || tau > dtau) {
                tau = tau - dtau;
                break;
            }
            if (k == P->max_emit) {
                /* cap reached: the event is carried to the next step */
                tau = tau - dtau;
                st->n_saturated++;
                break;
            }
            r = r - tau / wdt;
            uint32_t rr[4];
            or_draw(P->seed, species, OR_RNG_EMIT, or_id(S, i), P->step, k, rr);
            double xi_p = or_u53(rr[0], rr[1]);   /* xi'  (Eq. 7) */
            double xi = or_u53(rr[2], rr[3]);     /* xi   (tau^f) */
            double ufrac = or_sample_gamma(T, chi, xi_p, &clamped);
            double pmag = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
            double gg = ufrac * gam;
            if (gg > pmag) gg = pmag; /* READING: photon cannot exceed |p| */
            /* a particle at rest (|p| = 0) emits nothing: gg = 0, no recoil */
            double khat[3] = {0.0, 0.0, 0.0};
            if (pmag > 0.0) {
                khat[0] = u[0] / pmag;
                khat[1] = u[1] / pmag;
                khat[2] = u[2] / pmag;
            }
            st->n_emit++;
            if (S->nemit) S->nemit[i]++;
            if (gg > P->photon_min_gamma) {
                uint32_t rp[4];
                or_draw(P->seed, species, OR_RNG_PHOTON_TAU, or_id(S, i), P->step, k, rp);
                double tau_g = -log(or_u53(rp[0], rp[1]));
                double ku[3] = {gg * khat[0], gg * khat[1], gg * khat[2]};
                if (Ph) {
                    or_append_photon(Ph, ph_base, ph_ord, x, ku, S->w[i], tau_g, st, gg);
                } else {
                    st->n_photon_drop++; /* no photon species: nowhere to store it */
                    st->e_dropped += S->w[i] * gg;
                }
            } else {
                st->n_subthreshold++;
                st->e_subthreshold += S->w[i] * gg;
            }
            if (P->recoil && pmag > 0.0) {
                /* Eq. 8: p_f = (|p| - eps_gamma/c) p/|p| */
                double scale = (pmag - gg) / pmag;
                u[0] *= scale;
                u[1] *= scale;
                u[2] *= scale;
            }
            tau = -log(xi);
            gam = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
            chi = or_chi_e(E, B, u, gam, U->a_S);
        }
    }
    if (clamped) st->n_clamped++;

    /* Eq. 4: dx/dt = v + dv */
    for (int c = 0; c < 3; c++) x[c] = x[c] + dt * (u[c] / gam + dv[c]);
    if (P->noise != 0.0) {
        /* test-only: deterministic +-noise kick (sign from the slot and step) */
        uint32_t rn[4];
        or_draw(P->seed ^ 0x5EEDull ^ (P->noise_key * 0x9E3779B97F4A7C15ull), species, 7,
                or_id(S, i), P->step, 0, rn);
        for (int c = 0; c < 3; c++) u[c] *= 1.0 + ((rn[c] & 1u) ? P->noise : -P->noise);
    }
    S->x[i] = x[0];
    S->y[i] = x[1];
    if (S->z) S->z[i] = x[2];
    S->ux[i] = u[0];
    S->uy[i] = u[1];
    S->uz[i] = u[2];
    S->tau[i] = tau;
}

static void or_append_lepton(or_species *S, int64_t slot, const double x[3], const double u[3],
                             double w, double tau)
{
    S->x[slot] = x[0];
    S->y[slot] = x[1];
    if (S->z) S->z[slot] = x[2];
    S->ux[slot] = u[0];
    S->uy[slot] = u[1];
    S->uz[slot] = u[2];
    S->tau[slot] = tau;
    S->w[slot] = w;
    if (S->chi) S->chi[slot] = 0.0;
    if (S->margin) S->margin[slot] = INFINITY;
    if (S->nemit) S->nemit[slot] = 0;
    if (S->ids) S->ids[slot] = or_slot_id(S, slot);
}

/* One step of one super-photon: ballistic motion at c along k, optical depth
 * against the pair rate above 2 m c^2 (section 2, P_pm; section 3, pair MC).
 * A photon with tau < 0 is dead (it decayed into a pair). */
static void or_photon_step(const or_units *U, const or_tables *T, const or_field *F,
                           const or_params *P, or_species *Ph, int64_t i, or_species *El,
                           or_species *Po, int64_t be, int64_t bp, int64_t *pair_ord,
                           or_stats *st)
{
    double tau = Ph->tau[i];
    if (tau < 0.0) return;
    const double dt = P->dt;
    const double t = (double)P->step * dt;
    double x[3] = {Ph->x[i], Ph->y[i], Ph->z ? Ph->z[i] : 0.0};
    double u[3] = {Ph->ux[i], Ph->uy[i], Ph->uz[i]};
    double g = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    int clamped = 0;
    if (P->pairs && g > 2.0) {
        double E[3], B[3];
        or_field_eval(F, x[0], x[1], x[2], t, E, B);
        double chi = or_chi_gamma(E, B, u, U->a_S);
        if (Ph->chi) Ph->chi[i] = chi;
        double Tr = or_lookup_rate(T, 2, chi, &clamped);
        double dtau = U->C_rate * Tr / g * dt;
        or_record_margin(Ph, i, tau, dtau);
        if (clamped) st->n_clamped++;
        if (dtau > 0.0 && !(tau > dtau)) {
            /* pair event: photon deleted, e- e+ created at its position */
            uint32_t r1[4], r2[4];
            or_draw(P->seed, OR_SP_PHOTON, OR_RNG_PAIR, or_id(Ph, i), P->step, 0, r1);
            or_draw(P->seed, OR_SP_PHOTON, OR_RNG_PAIR_POS, or_id(Ph, i), P->step, 0, r2);
            double v = or_sample_pair(T, chi, or_u53(r1[0], r1[1]), &clamped);
            double tau_m = -log(or_u53(r1[2], r1[3]));
            double tau_p = -log(or_u53(r2[0], r2[1]));
            /* READING: momentum shared along k, chi_+ = chi_gamma - chi_- */
            double um[3] = {v * u[0], v * u[1], v * u[2]};
            double omv = 1.0 - v;
            double up[3] = {omv * u[0], omv * u[1], omv * u[2]};
            st->n_pair++;
            if (Ph->nemit) Ph->nemit[i]++;
            int64_t ord = (*pair_ord)++;
            int64_t se = be + ord, sp = bp + ord;
            if (El && Po && se < El->cap && sp < Po->cap) {
                or_append_lepton(El, se, x, um, Ph->w[i], tau_m);
                or_append_lepton(Po, sp, x, up, Ph->w[i], tau_p);
            } else {
                st->n_pair_drop++;
                st->e_dropped += Ph->w[i] * g;
            }
            Ph->tau[i] = -1.0;
            return;
        }
        tau = tau - dtau;
    }
    if (g > 0.0)
        for (int c = 0; c < 3; c++) x[c] = x[c] + dt * (u[c] / g);
    Ph->x[i] = x[0];
    Ph->y[i] = x[1];
    if (Ph->z) Ph->z[i] = x[2];
    Ph->tau[i] = tau;
}

/* One PIC step of all species, in slot order: electrons, positrons (each may
 * append photons), then the photons that existed at the start of the step
 * (each may append a pair).  Particles created during a step first move in
 * the next step. */
int or_step(const or_units *U, const or_tables *T, const or_field *F, const or_params *P,
            or_species *El, or_species *Po, or_species *Ph, or_stats *st)
{
    int64_t n_e = El ? El->n : 0, n_p = Po ? Po->n : 0, n_g = Ph ? Ph->n : 0;
    int64_t ph_base = n_g, ph_ord = 0;
    for (int64_t i = 0; i < n_e; i++)
        or_lepton_step(U, T, F, P, OR_SP_ELECTRON, El, i, Ph, ph_base, &ph_ord, st);
    for (int64_t i = 0; i < n_p; i++)
        or_lepton_step(U, T, F, P, OR_SP_POSITRON, Po, i, Ph, ph_base, &ph_ord, st);
    if (Ph) {
        int64_t nn = ph_base + ph_ord;
        Ph->n = nn < Ph->cap ? nn : Ph->cap;
    }
    int64_t pair_ord = 0;
    for (int64_t i = 0; i < n_g; i++)
        or_photon_step(U, T, F, P, Ph, i, El, Po, n_e, n_p, &pair_ord, st);
    if (El && Po && pair_ord > 0) {
        int64_t room = El->cap - n_e;
        if (Po->cap - n_p < room) room = Po->cap - n_p;
        int64_t add = pair_ord < room ? pair_ord : room;
        if (add < 0) add = 0;
        El->n = n_e + add;
        Po->n = n_p + add;
    }
    return 0;
}

/* Initial optical depth of slots [first, last) of a species:
 * tau = -log(xi), xi from the INIT stream of each slot. */
void or_init_tau(uint64_t seed, int species, double *tau, int64_t first, int64_t last)
{
    for (int64_t i = first; i < last; i++) {
        uint32_t r[4];
        or_draw(seed, species, OR_RNG_INIT, i, 0, 0, r);
        tau[i] = -log(or_u53(r[0], r[1]));
    }
}

/* Run n_steps steps starting at P->step (P is not modified). */
int or_run(const or_units *U, const or_tables *T, const or_field *F, const or_params *P,
           int64_t n_steps, or_species *El, or_species *Po, or_species *Ph, or_stats *st)
{
    or_params Q = *P;
    for (int64_t s = 0; s < n_steps; s++) {
        Q.step = P->step + s;
        or_step(U, T, F, &Q, El, Po, Ph, st);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Super-photon compaction and coalescence (section 3, last paragraph)        */
/* ------------------------------------------------------------------------- */

/* The paper names a coalescence of super-photons that conserves energy and
 * momentum on average and gives no algorithm.  READING (design notes): the
 * live photons are grouped by (cell of a box grid, log2-energy bin,
 * direction bin on the faces of a cube); a group of at least min_group
 * photons is replaced by two photons of weight W/2 each, energy E/W each and
 * momenta P/W +- d, d perpendicular to P with |P/W|^2 + |d|^2 = (E/W)^2, so
 * that the group's weight W = sum w, energy E = sum w |u| and momentum
 * P = sum w u are conserved exactly (to rounding), and both stay massless.
 * d lies in the plane of P and the group's first photon (the lowest slot);
 * when that photon is parallel to P, in the plane of P and the coordinate
 * axis least aligned with it.  The merged pair sits at the weighted mean
 * position of the group and draws fresh optical depths -log(xi) (the
 * remaining optical depth of a photon is memoryless).  Decayed photons
 * (tau < 0) are removed; what remains keeps its slot order, a merged pair
 * taking the place of its group's first photon.  Slots are renumbered, so a
 * photon's later draws follow its new slot.  A group of more than max_group
 * photons is merged in runs of max_group (its members in slot order, the
 * last run the rest; a run of fewer than min_group is kept as it is), which
 * bounds the work of one merge. */

typedef struct {
    double x0, y0, z0, dx, dy, dz;
    int64_t nx, ny, nz;
    int32_t ebins_per_octave; /* power of two, 1 .. 64                      */
    int32_t dir_bins;         /* power of two, 1 .. 64, per face axis        */
    int32_t min_group;        /* >= 3                                        */
    int32_t dims;
    int32_t max_group;        /* >= min_group; 0: 256                        */
    int32_t pad;
    uint64_t seed;
    int64_t step;
} or_coalesce_params;

typedef struct {
    int64_t n_before, n_dead, n_after, groups_merged, photons_merged;
} or_coalesce_stats;

enum { OR_RNG_COALESCE = 5 };

#define OR_NOMERGE UINT64_MAX

static int or_log2i(int v)
{
    int k = 0;
    while ((1 << k) < v) k++;
    return k;
}

/* The group key of a live photon, or OR_NOMERGE (outside the box, zero or
 * non-finite momentum).  Every decision is an exact FP64 operation (a
 * subtraction, a division, a comparison) or a bit extraction. */
static uint64_t or_coalesce_key(const or_coalesce_params *C, double x, double y, double z,
                                double ux, double uy, double uz)
{
    /* cell: the offset times the reciprocal of the cell size */
    double gx = floor((x - C->x0) * (1.0 / C->dx));
    double gy = floor((y - C->y0) * (1.0 / C->dy));
    double gz = C->dims == 3 ? floor((z - C->z0) * (1.0 / C->dz)) : 0.0;
    if (!(gx >= 0.0 && gx < (double)C->nx && gy >= 0.0 && gy < (double)C->ny && gz >= 0.0 &&
          gz < (double)C->nz))
        return OR_NOMERGE;
    double e = sqrt(ux * ux + uy * uy + uz * uz);
    uint64_t eb;
    memcpy(&eb, &e, 8);
    uint64_t ex = (eb >> 52) & 0x7FF;
    if (ex == 0 || ex == 0x7FF) return OR_NOMERGE;
    /* energy bin: the exponent, then the leading mantissa bits */
    int lb = or_log2i(C->ebins_per_octave);
    uint64_t ebin = (ex << lb) | ((eb & ((1ull << 52) - 1)) >> (52 - lb));
    /* direction bin: the dominant axis with its sign (a cube face), then the
     * two other components over the dominant one, each in dir_bins bins */
    double u[3] = {ux, uy, uz};
    int f = 0;
    if (fabs(u[1]) > fabs(u[f])) f = 1;
    if (fabs(u[2]) > fabs(u[f])) f = 2;
    int face = 2 * f + (u[f] < 0.0 ? 1 : 0);
    double r = 1.0 / fabs(u[f]);
    double a = u[(f + 1) % 3] * r;
    double b = u[(f + 2) % 3] * r;
    int64_t D = C->dir_bins;
    int64_t ia = (int64_t)floor((a + 1.0) * (0.5 * (double)D));
    int64_t ib = (int64_t)floor((b + 1.0) * (0.5 * (double)D));
    if (ia > D - 1) ia = D - 1;
    if (ib > D - 1) ib = D - 1;
    uint64_t dbin = ((uint64_t)face * (uint64_t)D + (uint64_t)ia) * (uint64_t)D + (uint64_t)ib;
    uint64_t cell = ((uint64_t)gx * (uint64_t)C->ny + (uint64_t)gy) * (uint64_t)C->nz +
                    (uint64_t)gz;
    uint64_t n_e = 2048ull << lb, n_d = 6ull * (uint64_t)D * (uint64_t)D;
    return (cell * n_e + ebin) * n_d + dbin;
}

typedef struct {
    uint64_t key;
    int64_t slot;
} or_keyslot;

static int or_keyslot_cmp(const void *pa, const void *pb)
{
    const or_keyslot *a = (const or_keyslot *)pa, *b = (const or_keyslot *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->slot < b->slot ? -1 : (a->slot > b->slot ? 1 : 0);
}

/* The merged pair of one group (members m[0..n), in slot order). */
static void or_merge_group(const or_species *Ph, const int64_t *m, int64_t n,
                           const or_coalesce_params *C, int64_t anchor_id, double out[2][8])
{
    double W = 0.0, E = 0.0, P[3] = {0.0, 0.0, 0.0}, X[3] = {0.0, 0.0, 0.0};
    for (int64_t k = 0; k < n; k++) {
        int64_t i = m[k];
        double w = Ph->w[i];
        double ux = Ph->ux[i], uy = Ph->uy[i], uz = Ph->uz[i];
        double e = sqrt(ux * ux + uy * uy + uz * uz);
        W = W + w;
        E = E + w * e;
        P[0] = P[0] + w * ux;
        P[1] = P[1] + w * uy;
        P[2] = P[2] + w * uz;
        X[0] = X[0] + w * Ph->x[i];
        X[1] = X[1] + w * Ph->y[i];
        X[2] = X[2] + w * (Ph->z ? Ph->z[i] : 0.0);
    }
    double eps = E / W;
    double c[3] = {P[0] / W, P[1] / W, P[2] / W};
    double c2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    double d2 = eps * eps - c2;
    double dm = d2 > 0.0 ? sqrt(d2) : 0.0;
    /* unit vector of P, and the reference direction: the first photon */
    double cm = sqrt(c2);
    double ph[3] = {c[0] / cm, c[1] / cm, c[2] / cm};
    double r[3] = {Ph->ux[m[0]], Ph->uy[m[0]], Ph->uz[m[0]]};
    double rp = r[0] * ph[0] + r[1] * ph[1] + r[2] * ph[2];
    double v[3] = {r[0] - rp * ph[0], r[1] - rp * ph[1], r[2] - rp * ph[2]};
    double vm = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double rm = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (!(vm > 1e-12 * rm)) {
        /* the first photon is parallel to P: the axis least aligned with P */
        int a = 0;
        if (fabs(ph[1]) < fabs(ph[a])) a = 1;
        if (fabs(ph[2]) < fabs(ph[a])) a = 2;
        double ax[3] = {0.0, 0.0, 0.0};
        ax[a] = 1.0;
        double ap = ph[a];
        v[0] = ax[0] - ap * ph[0];
        v[1] = ax[1] - ap * ph[1];
        v[2] = ax[2] - ap * ph[2];
        vm = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    }
    double dv[3] = {dm * (v[0] / vm), dm * (v[1] / vm), dm * (v[2] / vm)};
    for (int s = 0; s < 2; s++) {
        double sg = s == 0 ? 1.0 : -1.0;
        uint32_t rr[4];
        or_draw(C->seed, OR_SP_PHOTON, OR_RNG_COALESCE, anchor_id, C->step, s, rr);
        out[s][0] = X[0] / W;
        out[s][1] = X[1] / W;
        out[s][2] = X[2] / W;
        out[s][3] = c[0] + sg * dv[0];
        out[s][4] = c[1] + sg * dv[1];
        out[s][5] = c[2] + sg * dv[2];
        out[s][6] = -log(or_u53(rr[0], rr[1]));
        out[s][7] = 0.5 * W;
    }
}

/* Compaction (min_group = 0: nothing merged) or coalescence of the live
 * photons of Ph, in place.  Returns 0, or -1 on bad parameters or memory. */
int or_coalesce(or_species *Ph, const or_coalesce_params *C, or_coalesce_stats *st)
{
    int64_t n = Ph->n;
    memset(st, 0, sizeof(*st));
    st->n_before = n;
    int merge = C && C->min_group > 0;
    if (merge && (C->min_group < 3 || (C->max_group != 0 && C->max_group < C->min_group) ||
                  C->ebins_per_octave < 1 || C->ebins_per_octave > 64 ||
                  C->dir_bins < 1 || C->dir_bins > 64 || !(C->dx > 0.0) || !(C->dy > 0.0) ||
                  (C->dims == 3 && !(C->dz > 0.0)) || C->nx < 1 || C->ny < 1 || C->nz < 1))
        return -1;
    /* role of each slot: 0 dead or merged away, 1 kept, 2 anchor of a pair */
    int8_t *role = (int8_t *)malloc((size_t)(n > 0 ? n : 1));
    int64_t *grp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    or_keyslot *ks = (or_keyslot *)malloc(sizeof(or_keyslot) * (size_t)(n > 0 ? n : 1));
    if (!role || !grp || !ks) {
        free(role);
        free(grp);
        free(ks);
        return -1;
    }
    int64_t nk = 0;
    for (int64_t i = 0; i < n; i++) {
        role[i] = Ph->tau[i] < 0.0 ? 0 : 1;
        grp[i] = -1;
        if (!role[i]) {
            st->n_dead++;
            continue;
        }
        if (!merge) continue;
        uint64_t key = or_coalesce_key(C, Ph->x[i], Ph->y[i], Ph->z ? Ph->z[i] : 0.0,
                                       Ph->ux[i], Ph->uy[i], Ph->uz[i]);
        if (key == OR_NOMERGE) continue;
        ks[nk].key = key;
        ks[nk].slot = i;
        nk++;
    }
    qsort(ks, (size_t)nk, sizeof(or_keyslot), or_keyslot_cmp);
    /* groups: runs of one key; merged ones are recorded at their anchor */
    double (*pairs)[2][8] = NULL;
    int64_t n_pairs = 0;
    int64_t *members = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nk > 0 ? nk : 1));
    const int64_t M = merge ? (C->max_group > 0 ? C->max_group : 256) : 1;
    for (int64_t g0 = 0; g0 < nk;) {
        int64_t g1 = g0;
        while (g1 < nk && ks[g1].key == ks[g0].key) g1++;
        for (int64_t a = g0; a < g1; a += M) {
            const int64_t b = a + M < g1 ? a + M : g1;
            if (b - a >= C->min_group) {
                for (int64_t k = a; k < b; k++) members[k - a] = ks[k].slot;
                double c2 = 0.0;
                {
                    double P[3] = {0.0, 0.0, 0.0};
                    for (int64_t k = a; k < b; k++) {
                        int64_t i = ks[k].slot;
                        P[0] = P[0] + Ph->w[i] * Ph->ux[i];
                        P[1] = P[1] + Ph->w[i] * Ph->uy[i];
                        P[2] = P[2] + Ph->w[i] * Ph->uz[i];
                    }
                    c2 = P[0] * P[0] + P[1] * P[1] + P[2] * P[2];
                }
                if (c2 > 0.0) {
                    pairs = realloc(pairs, sizeof(*pairs) * (size_t)(n_pairs + 1));
                    int64_t anchor = members[0];
                    or_merge_group(Ph, members, b - a, C, or_id(Ph, anchor), pairs[n_pairs]);
                    grp[anchor] = n_pairs;
                    for (int64_t k = a; k < b; k++) role[ks[k].slot] = 0;
                    role[anchor] = 2;
                    n_pairs++;
                    st->groups_merged++;
                    st->photons_merged += b - a;
                }
            }
        }
        g0 = g1;
    }
    /* the survivors in slot order, into fresh arrays, then back */
    int64_t out = 0;
    for (int64_t i = 0; i < n; i++) out += role[i];
    /* per survivor: x y z ux uy uz tau w, then chi, margin and nemit (kept
     * photons carry theirs along; a merged pair starts from 0, inf, 0) */
    enum { NB = 11 };
    double *buf = (double *)malloc(sizeof(double) * NB * (size_t)(out > 0 ? out : 1));
    int64_t j = 0;
    for (int64_t i = 0; i < n; i++) {
        if (role[i] == 1) {
            double *o = buf + NB * j++;
            o[0] = Ph->x[i];
            o[1] = Ph->y[i];
            o[2] = Ph->z ? Ph->z[i] : 0.0;
            o[3] = Ph->ux[i];
            o[4] = Ph->uy[i];
            o[5] = Ph->uz[i];
            o[6] = Ph->tau[i];
            o[7] = Ph->w[i];
            o[8] = Ph->chi ? Ph->chi[i] : 0.0;
            o[9] = Ph->margin ? Ph->margin[i] : INFINITY;
            o[10] = Ph->nemit ? (double)Ph->nemit[i] : 0.0;
        } else if (role[i] == 2) {
            for (int s = 0; s < 2; s++) {
                double *o = buf + NB * j++;
                memcpy(o, pairs[grp[i]][s], 8 * sizeof(double));
                o[8] = 0.0;
                o[9] = INFINITY;
                o[10] = 0.0;
            }
        }
    }
    for (int64_t k = 0; k < out; k++) {
        const double *o = buf + NB * k;
        Ph->x[k] = o[0];
        Ph->y[k] = o[1];
        if (Ph->z) Ph->z[k] = o[2];
        Ph->ux[k] = o[3];
        Ph->uy[k] = o[4];
        Ph->uz[k] = o[5];
        Ph->tau[k] = o[6];
        Ph->w[k] = o[7];
        if (Ph->chi) Ph->chi[k] = o[8];
        if (Ph->margin) Ph->margin[k] = o[9];
        if (Ph->nemit) Ph->nemit[k] = (int32_t)o[10];
        if (Ph->ids) Ph->ids[k] = or_slot_id(Ph, k);
    }
    Ph->n = out;
    st->n_after = out;
    free(buf);
    free(pairs);
    free(members);
    free(role);
    free(grp);
    free(ks);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Refill of a 2D Yee grid from the analytic pulse                            */
/* ------------------------------------------------------------------------- */

/* The fields of a 2D paraxial Gaussian pulse along +x, polarised along y
 * (the laser of the foil workload; not in the paper), at time t:
 *   xi = x - x_focus, eta = (t - t_focus) - xi, zr = w0^2/2, q = xi/zr,
 *   E_y = B_z = a0 (1 + q^2)^(-1/4) exp(-r^2/(w0^2 (1 + q^2)) - 2 ln2 eta^2/tau^2)
 *               cos(-eta + r^2 xi / (2 (xi^2 + zr^2)) - atan(q)/2),
 * r = y - y_axis (the Gouy phase of a 2D beam is half that of a 3D one).
 * READING: the per-step refill of the fixed snapshot (the workload's fields
 * follow the pulse as it crosses the foil); E and B both at t. */
typedef struct {
    double a0, w0, tau_fwhm, x_focus, t_focus, y_axis;
} or_pulse2d;

double or_pulse2d_eval(const or_pulse2d *p, double x, double y, double t)
{
    double xi = x - p->x_focus;
    double eta = (t - p->t_focus) - xi;
    double zr = 0.5 * p->w0 * p->w0;
    double q = xi / zr;
    double wr2 = 1.0 + q * q;
    double r2 = (y - p->y_axis) * (y - p->y_axis);
    double env = -r2 / (p->w0 * p->w0 * wr2) -
                 2.0 * log(2.0) * eta * eta / (p->tau_fwhm * p->tau_fwhm);
    double amp = p->a0 * pow(wr2, -0.25) * exp(env);
    double phase = -eta + r2 * xi / (2.0 * (xi * xi + zr * zr)) - 0.5 * atan(q);
    return amp * cos(phase);
}

/* E_y at (x0 + i dx, y0 + (j + 1/2) dy) and B_z at (x0 + (i + 1/2) dx,
 * y0 + (j + 1/2) dy), each rounded to float; ny rows of nx values.  The
 * other components are not touched. */
void or_fill_pulse2d(const or_pulse2d *p, float *ey, float *bz, int64_t nx, int64_t ny,
                     double dx, double dy, double x0, double y0, double t)
{
    for (int64_t j = 0; j < ny; j++) {
        double y = y0 + ((double)j + 0.5) * dy;
        for (int64_t i = 0; i < nx; i++) {
            ey[j * nx + i] = (float)or_pulse2d_eval(p, x0 + (double)i * dx, y, t);
            bz[j * nx + i] = (float)or_pulse2d_eval(p, x0 + ((double)i + 0.5) * dx, y, t);
        }
    }
}

/* ------------------------------------------------------------------------- */
/* PIC coupling around the step: 2D Yee Maxwell solver, current deposition,  */
/* particle sorting (section 3: the QED step runs inside a PIC code)          */
/* ------------------------------------------------------------------------- */

/* The six float components of a 2D Yee grid, ny rows of nx values, on the
 * staggering of or_yee_component: Ex (i+1/2, j), Ey (i, j+1/2), Ez (i, j),
 * Bx (i, j+1/2), By (i+1/2, j), Bz (i+1/2, j+1/2); values outside the grid
 * are 0.  Normalised units (c = 1): dB/dt = -curl E, dE/dt = curl B - J,
 * with J in units of e n_c c (the charge density of the reference density
 * moving at c).  READING: the paper uses CALDER's solver and describes none;
 * this is the standard leapfrog on Yee's lattice, d/dz = 0. */
static float or_at(const float *a, int64_t nx, int64_t ny, int64_t i, int64_t j)
{
    if (i < 0 || j < 0 || i >= nx || j >= ny) return 0.0f;
    return a[j * nx + i];
}

/* B -= dtb curl E (each new value rounded to float). */
void or_yee_advance_b(float *const F[6], int64_t nx, int64_t ny, double dx, double dy, double dtb)
{
    float *Bx = F[3], *By = F[4], *Bz = F[5];
    const float *Ex = F[0], *Ey = F[1], *Ez = F[2];
    size_t n = (size_t)(nx * ny);
    float *nbx = malloc(n * sizeof(float)), *nby = malloc(n * sizeof(float)),
          *nbz = malloc(n * sizeof(float));
    for (int64_t j = 0; j < ny; j++)
        for (int64_t i = 0; i < nx; i++) {
            int64_t k = j * nx + i;
            /* Bx (i, j+1/2): d Ez/dy between (i, j+1) and (i, j) */
            double dEz_dy = ((double)or_at(Ez, nx, ny, i, j + 1) - (double)Ez[k]) / dy;
            /* By (i+1/2, j): -(-dEz/dx) = +dEz/dx */
            double dEz_dx = ((double)or_at(Ez, nx, ny, i + 1, j) - (double)Ez[k]) / dx;
            /* Bz (i+1/2, j+1/2): dEy/dx - dEx/dy */
            double dEy_dx = ((double)or_at(Ey, nx, ny, i + 1, j) - (double)Ey[k]) / dx;
            double dEx_dy = ((double)or_at(Ex, nx, ny, i, j + 1) - (double)Ex[k]) / dy;
            nbx[k] = (float)((double)Bx[k] - dtb * dEz_dy);
            nby[k] = (float)((double)By[k] + dtb * dEz_dx);
            nbz[k] = (float)((double)Bz[k] - dtb * (dEy_dx - dEx_dy));
        }
    memcpy(Bx, nbx, n * sizeof(float));
    memcpy(By, nby, n * sizeof(float));
    memcpy(Bz, nbz, n * sizeof(float));
    free(nbx);
    free(nby);
    free(nbz);
}

/* E += dt (curl B - J); J on E's staggering (NULL: no current). */
void or_yee_advance_e(float *const F[6], const float *const J[3], int64_t nx, int64_t ny,
                      double dx, double dy, double dt)
{
    float *Ex = F[0], *Ey = F[1], *Ez = F[2];
    const float *Bx = F[3], *By = F[4], *Bz = F[5];
    size_t n = (size_t)(nx * ny);
    float *nex = malloc(n * sizeof(float)), *ney = malloc(n * sizeof(float)),
          *nez = malloc(n * sizeof(float));
    for (int64_t j = 0; j < ny; j++)
        for (int64_t i = 0; i < nx; i++) {
            int64_t k = j * nx + i;
            /* Ex (i+1/2, j): dBz/dy between (i+1/2, j+1/2) and (i+1/2, j-1/2) */
            double dBz_dy = ((double)Bz[k] - (double)or_at(Bz, nx, ny, i, j - 1)) / dy;
            /* Ey (i, j+1/2): -dBz/dx between (i+1/2, j+1/2) and (i-1/2, j+1/2) */
            double dBz_dx = ((double)Bz[k] - (double)or_at(Bz, nx, ny, i - 1, j)) / dx;
            /* Ez (i, j): dBy/dx - dBx/dy */
            double dBy_dx = ((double)By[k] - (double)or_at(By, nx, ny, i - 1, j)) / dx;
            double dBx_dy = ((double)Bx[k] - (double)or_at(Bx, nx, ny, i, j - 1)) / dy;
            double jx = J ? (double)J[0][k] : 0.0, jy = J ? (double)J[1][k] : 0.0,
                   jz = J ? (double)J[2][k] : 0.0;
            nex[k] = (float)((double)Ex[k] + dt * (dBz_dy - jx));
            ney[k] = (float)((double)Ey[k] + dt * (-dBz_dx - jy));
            nez[k] = (float)((double)Ez[k] + dt * (dBy_dx - dBx_dy - jz));
        }
    memcpy(Ex, nex, n * sizeof(float));
    memcpy(Ey, ney, n * sizeof(float));
    memcpy(Ez, nez, n * sizeof(float));
    free(nex);
    free(ney);
    free(nez);
}

/* Current of the live slots of a lepton species, added to J (FP64 arrays on
 * E's staggering, ny rows of nx): each particle deposits q w v / (dx dy)
 * with the linear (cloud-in-cell) weights of each component's staggering at
 * the mid-step position x - v dt/2 (x^(n+1) and v^(n+1/2) after a step).
 * READING: direct (not charge-conserving) deposition. */
void or_deposit_current(const or_species *S, double q, double dt, double *const J[3], int64_t nx,
                        int64_t ny, double dx, double dy, double x0, double y0)
{
    static const double ox[3] = {0.5, 0.0, 0.0}, oy[3] = {0.0, 0.5, 0.0};
    for (int64_t p = 0; p < S->n; p++) {
        double u[3] = {S->ux[p], S->uy[p], S->uz[p]};
        double g = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        double v[3] = {u[0] / g, u[1] / g, u[2] / g};
        double xm = S->x[p] - 0.5 * dt * v[0], ym = S->y[p] - 0.5 * dt * v[1];
        double a = q * S->w[p] / (dx * dy);
        for (int c = 0; c < 3; c++) {
            double gx = (xm - x0) / dx - ox[c], gy = (ym - y0) / dy - oy[c];
            double fi = floor(gx), fj = floor(gy);
            double fx = gx - fi, fy = gy - fj;
            for (int b = 0; b < 2; b++)
                for (int e = 0; e < 2; e++) {
                    double ii = fi + e, jj = fj + b;
                    if (!(ii >= 0.0 && jj >= 0.0 && ii < (double)nx && jj < (double)ny)) continue;
                    double wgt = (e ? fx : 1.0 - fx) * (b ? fy : 1.0 - fy);
                    J[c][(int64_t)jj * nx + (int64_t)ii] += a * v[c] * wgt;
                }
        }
    }
}

/* Stable sort of the live slots of a species by the cell of the grid that
 * holds them (row-major, floor((y - y0)/dy) nx + floor((x - x0)/dx));
 * particles outside the grid after all others, in slot order.  Every array
 * moves with its particle; slots are renumbered (later draws follow the new
 * slots).  Returns 0, or -1 without memory. */
int or_sort_by_cell(or_species *S, int64_t nx, int64_t ny, double dx, double dy, double x0,
                    double y0)
{
    int64_t n = S->n;
    or_keyslot *ks = malloc(sizeof(or_keyslot) * (size_t)(n > 0 ? n : 1));
    double *buf = malloc(sizeof(double) * 11 * (size_t)(n > 0 ? n : 1));
    if (!ks || !buf) {
        free(ks);
        free(buf);
        return -1;
    }
    for (int64_t i = 0; i < n; i++) {
        double gx = floor((S->x[i] - x0) / dx), gy = floor((S->y[i] - y0) / dy);
        uint64_t key = (uint64_t)nx * (uint64_t)ny;  /* outside: after every cell */
        if (gx >= 0.0 && gy >= 0.0 && gx < (double)nx && gy < (double)ny)
            key = (uint64_t)gy * (uint64_t)nx + (uint64_t)gx;
        ks[i].key = key;
        ks[i].slot = i;
    }
    qsort(ks, (size_t)n, sizeof(or_keyslot), or_keyslot_cmp);
    for (int64_t k = 0; k < n; k++) {
        int64_t i = ks[k].slot;
        double *o = buf + 11 * k;
        o[0] = S->x[i];
        o[1] = S->y[i];
        o[2] = S->z ? S->z[i] : 0.0;
        o[3] = S->ux[i];
        o[4] = S->uy[i];
        o[5] = S->uz[i];
        o[6] = S->tau[i];
        o[7] = S->w[i];
        o[8] = S->chi ? S->chi[i] : 0.0;
        o[9] = S->margin ? S->margin[i] : INFINITY;
        o[10] = S->nemit ? (double)S->nemit[i] : 0.0;
    }
    for (int64_t k = 0; k < n; k++) {
        const double *o = buf + 11 * k;
        S->x[k] = o[0];
        S->y[k] = o[1];
        if (S->z) S->z[k] = o[2];
        S->ux[k] = o[3];
        S->uy[k] = o[4];
        S->uz[k] = o[5];
        S->tau[k] = o[6];
        S->w[k] = o[7];
        if (S->chi) S->chi[k] = o[8];
        if (S->margin) S->margin[k] = o[9];
        if (S->nemit) S->nemit[k] = (int32_t)o[10];
        if (S->ids) S->ids[k] = or_slot_id(S, k);
    }
    free(ks);
    free(buf);
    return 0;
}
