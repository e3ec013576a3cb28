// Host construction of the rate and CDF tables of libqedpic (FP64).
//
// The tables tabulate the nonlinear-Compton photon spectrum (Eq. 2 of
// Lobet et al., with its bracket read with the positive sign) and the
// Breit-Wheeler pair spectrum (Eq. 3), in the variables
//   u = chi_gamma / chi_e :  F_gamma(u) = (2 + u^2/(1-u)) K_2/3(z) - Ki_1/3(z),
//                            z = 2u / (3 chi (1-u))
//   v = chi_- / chi_gamma :  F_pm(v)    = Ki_1/3(z) + (1/(v(1-v)) - 2) K_2/3(z),
//                            z = 2 / (3 chi v (1-v))
// with Ki_1/3(z) = int_z^inf K_1/3.  The Bessel functions come from their
// integral representation K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt
// (and Ki_1/3(x) = int_0^inf exp(-x cosh t) cosh(t/3)/cosh(t) dt) by the
// trapezoid rule; the spectra are integrated by tanh-sinh quadrature on the
// intervals with an end-point singularity and 12-point Gauss-Legendre on the
// intervals between CDF nodes.  Rows are built in parallel on host threads.
#include <math.h>

#include <algorithm>
#include <thread>
#include <vector>

#include "qp_internal.h"

namespace qp {

void units_for_wavelength(double lambda_m, Units *u)
{
    const double c = 299792458.0, hbar = 1.054571817e-34, me = 9.1093837015e-31;
    const double qe = 1.602176634e-19, eps0 = 8.8541878128e-12, alpha = 7.2973525693e-3;
    const double pi = 3.14159265358979323846;
    const double omega = 2.0 * pi * c / lambda_m;
    const double tau_c = hbar / (me * c * c);  // Compton time
    u->a_S = me * c * c / (hbar * omega);
    u->C_rate = alpha / (sqrt(3.0) * pi * tau_c * omega);
    u->tau0w = qe * qe / (6.0 * pi * eps0 * me * c * c * c) * omega;  // 2e^2/(12 pi eps0 m c^3)
}

namespace {

constexpr double kPi = 3.14159265358979323846;

// K_2/3(x) and Ki_1/3(x) from one trapezoid sweep of their integrands.
void bessel_k23_ki13(double x, double *k23, double *ki13)
{
    if (x > 745.0) {
        *k23 = 0.0;
        *ki13 = 0.0;
        return;
    }
    const double h = x > 64.0 ? 0.4 / sqrt(x) : 0.05;
    double a = 0.0, b = 0.0;
    for (long k = 0;; ++k) {
        const double t = h * (double)k;
        const double ch = cosh(t);
        const double e = exp(-x * (ch - 1.0));  // exp(-x) factored out
        const double fa = e * cosh(t * (2.0 / 3.0));
        const double fb = e * cosh(t * (1.0 / 3.0)) / ch;
        const double wk = k == 0 ? 0.5 : 1.0;
        a += wk * fa;
        b += wk * fb;
        if ((x * sinh(t) > 1.0 && fa < 1e-17 * a && fb < 1e-17 * b) || k > 200000) break;
    }
    const double s = h * exp(-x);
    *k23 = a * s;
    *ki13 = b * s;
}

// Emission spectrum with 1-u passed separately (no cancellation near u = 1).
double f_gamma(double u, double omu, double chi)
{
    if (u <= 0.0 || omu <= 0.0) return 0.0;
    double k23, ki13;
    bessel_k23_ki13(2.0 * u / (3.0 * chi * omu), &k23, &ki13);
    return (2.0 + u * u / omu) * k23 - ki13;
}

double f_pair(double v, double omv, double chi)
{
    if (v <= 0.0 || omv <= 0.0) return 0.0;
    const double vv = v * omv;
    double k23, ki13;
    bessel_k23_ki13(2.0 / (3.0 * chi * vv), &k23, &ki13);
    return ki13 + (1.0 / vv - 2.0) * k23;
}

// tanh-sinh rule on [0,1]: sigma(t) = 1/(1+exp(-pi sinh t)), its complement,
// and weight h (pi/2) cosh t / (2 cosh^2(pi/2 sinh t)).
struct TanhSinh {
    std::vector<double> s, sc, w;
    TanhSinh()
    {
        const double h = 1.0 / 32.0, tmax = 4.6;
        for (double t = -tmax; t <= tmax + 1e-12; t += h) {
            const double a = kPi * sinh(t);
            const double c = cosh(0.5 * a);
            s.push_back(1.0 / (1.0 + exp(-a)));
            sc.push_back(1.0 / (1.0 + exp(a)));
            w.push_back(h * 0.5 * kPi * cosh(t) / (2.0 * c * c));
        }
    }
};

// 12-point Gauss-Legendre on [-1, 1] (Newton iteration on P_12).
struct GaussLegendre12 {
    double x[12], w[12];
    GaussLegendre12()
    {
        const int n = 12;
        for (int i = 0; i < n; ++i) {
            double z = cos(kPi * (i + 0.75) / (n + 0.5)), dp = 0.0;
            for (int it = 0; it < 64; ++it) {
                double p1 = 1.0, p2 = 0.0;
                for (int k = 1; k <= n; ++k) {
                    const double p3 = p2;
                    p2 = p1;
                    p1 = ((2.0 * k - 1.0) * z * p2 - (k - 1.0) * p3) / k;
                }
                dp = n * (z * p1 - p2) / (z * z - 1.0);
                const double dz = p1 / dp;
                z -= dz;
                if (fabs(dz) < 1e-15) {
                    // one more evaluation of P'_n at the converged node
                    p1 = 1.0;
                    p2 = 0.0;
                    for (int k = 1; k <= n; ++k) {
                        const double p3 = p2;
                        p2 = p1;
                        p1 = ((2.0 * k - 1.0) * z * p2 - (k - 1.0) * p3) / k;
                    }
                    dp = n * (z * p1 - p2) / (z * z - 1.0);
                    break;
                }
            }
            x[i] = z;
            w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
        }
    }
};

const TanhSinh &ts()
{
    static const TanhSinh r;
    return r;
}
const GaussLegendre12 &gl()
{
    static const GaussLegendre12 r;
    return r;
}

using Spectrum = double (*)(double, double, double);

// int_a^b f over [a, b] (with 1-b given as omb to keep the complement exact)
// by tanh-sinh: handles end-point singularities and fast decay.
double integrate_ts(Spectrum f, double chi, double a, double b, double omb)
{
    const TanhSinh &r = ts();
    const double len = b - a;
    double sum = 0.0;
    for (size_t k = 0; k < r.s.size(); ++k) {
        const double u = a + len * r.s[k];
        const double omu = omb + len * r.sc[k];
        sum += r.w[k] * f(u, omu, chi);
    }
    return sum * len;
}

// int_a^b by 12-point Gauss-Legendre (smooth interior intervals).
double integrate_gl(Spectrum f, double chi, double a, double b, double omb)
{
    const GaussLegendre12 &g = gl();
    const double half = 0.5 * (b - a), mid = 0.5 * (a + b);
    const double ommid = omb + half;
    double sum = 0.0;
    for (int i = 0; i < 12; ++i) sum += g.w[i] * f(mid + half * g.x[i], ommid - half * g.x[i], chi);
    return sum * half;
}

double u_gamma_weighted(double u, double omu, double chi) { return u * f_gamma(u, omu, chi); }

double chi_node(int j, int per_oct)
{
    return ldexp(1.0 + (double)(j % per_oct) / per_oct, kChiExp0 + j / per_oct);
}

// One CDF row: cumulative integrals up to the logit nodes s_i = smin + span i/255.
void cdf_row(Spectrum f, double chi, double smin, double span, double *row)
{
    double acc = 0.0, prev = 0.0, prev_om = 1.0;
    for (int i = 0; i < kNNode; ++i) {
        const double s = smin + span * i / (kNNode - 1);
        const double x = 1.0 / (1.0 + exp(-s)), omx = 1.0 / (1.0 + exp(s));
        acc += i == 0 ? integrate_ts(f, chi, 0.0, x, omx) : integrate_gl(f, chi, prev, x, omx);
        row[i] = acc;
        prev = x;
        prev_om = omx;
    }
    const double total = acc + integrate_ts(f, chi, prev, 1.0, 0.0);
    (void)prev_om;
    if (total > 0.0 && isfinite(total)) {
        for (int i = 0; i < kNNode; ++i) row[i] /= total;
    } else {
        // a row whose rate underflows carries the CDF of the variable itself
        for (int i = 0; i < kNNode; ++i) {
            const double s = smin + span * i / (kNNode - 1);
            row[i] = 1.0 / (1.0 + exp(-s));
        }
    }
}

template <class F>
void parallel_rows(int n, F fn)
{
    unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    for (unsigned t = 0; t < nt; ++t)
        pool.emplace_back([=] {
            for (int j = (int)t; j < n; j += (int)nt) fn(j);
        });
    for (auto &th : pool) th.join();
}

}  // namespace

void build_tables_host(HostTables *T)
{
    (void)ts();
    (void)gl();
    parallel_rows(kNRate, [T](int j) {
        const double chi = chi_node(j, kRatePerOct);
        // split the photon spectrum where it concentrates (u ~ chi at small chi)
        const double c = std::min(0.5, 2.0 * chi);
        const double H = integrate_ts(f_gamma, chi, 0.0, c, 1.0 - c) +
                         integrate_ts(f_gamma, chi, c, 1.0, 0.0);
        const double G = integrate_ts(u_gamma_weighted, chi, 0.0, c, 1.0 - c) +
                         integrate_ts(u_gamma_weighted, chi, c, 1.0, 0.0);
        T->H[j] = H;
        T->Gs[j] = G / chi;
        if (chi >= kPairChiMin) {
            const double P = integrate_ts(f_pair, chi, 0.0, 0.5, 0.5) +
                             integrate_ts(f_pair, chi, 0.5, 1.0, 0.0);
            T->Ts[j] = P * exp(8.0 / (3.0 * chi));
        } else {
            T->Ts[j] = 0.0;
        }
    });
    parallel_rows(2 * kNCdf, [T](int r) {
        const int j = r % kNCdf;
        const double chi = chi_node(j, kCdfPerOct);
        if (r < kNCdf)
            cdf_row(f_gamma, chi, kSgMin, kSgSpan, &T->Cg[j * kNNode]);
        else
            cdf_row(f_pair, chi, kSpMin, kSpSpan, &T->Cp[j * kNNode]);
    });
}

}  // namespace qp
