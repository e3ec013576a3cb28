// Host check of the double-float toolkit of the mixed-precision path
// (paper_1311_1107_gb300/csrc/qp_df.h) against long-double arithmetic.
// Prints one line per check: "<name> <failures> <worst>" and exits 0.
#include <math.h>
#include <stdio.h>
#include <stdint.h>

#include <random>

#include "qp_df.h"

using qp::df2;
typedef long double LD;

static double ulp(double x) { return nextafter(fabs(x), INFINITY) - fabs(x); }

int main()
{
    std::mt19937_64 rng(12345);
    std::uniform_real_distribution<double> u01(0.0, 1.0);
    auto rnd_double = [&](double lo_exp, double hi_exp) {
        double m = pow(10.0, lo_exp + (hi_exp - lo_exp) * u01(rng));
        return (rng() & 1) ? -m : m;
    };
    const int N = 400000;

    // split: hi + lo == d within 2^-46 |d| for |d| >= 2^-74; below that the
    // remainder is dropped (relative error 2^-23)
    long fail = 0;
    double worst = 0;
    for (int i = 0; i < N; ++i) {
        double d = rnd_double(-22, 30);
        df2 s = qp::split_d(d);
        double r = fabs(((double)s.hi + (double)s.lo) - d) / fabs(d);
        worst = fmax(worst, r);
        if (r > ldexp(1.0, -46) || fabs(s.hi) > fabs(d)) ++fail;
    }
    df2 z = qp::split_d(0.0);
    if (z.hi != 0.0f || z.lo != 0.0f) ++fail;
    for (int i = 0; i < 1000; ++i) {
        double d = rnd_double(-37, -23);
        df2 s = qp::split_d(d);
        if (fabs(((double)s.hi + (double)s.lo) - d) > ldexp(1.0, -23) * fabs(d)) ++fail;
    }
    printf("split %ld %.3e\n", fail, worst);

    // hi_d(d) == (float)d (round to nearest) except at exact ties, where it
    // rounds away from zero; includes values whose rounding carries into the
    // exponent (just below a power of two)
    fail = 0;
    for (int i = 0; i < N; ++i) {
        double d = rnd_double(-22, 30);
        if (i % 8 == 0) d = nextafter(ldexp(1.0, (int)(rng() % 40) - 20), 0.0) * ((rng() & 1) ? 1 : -1);
        float h = qp::hi_d(d), r = (float)d;
        if (h != r) {
            // allowed only at an exact tie
            double lo = fmin(fabs((double)h), fabs((double)r)), hi = fmax(fabs((double)h), fabs((double)r));
            if (fabs(fabs(d) - 0.5 * (lo + hi)) != 0.0 || fabs((double)h) < fabs((double)r)) ++fail;
        }
    }
    if (qp::hi_d(0.0) != 0.0f) ++fail;
    printf("hi_d %ld 0\n", fail);

    // merge(split(d)) == d within 2^-46 (a pair holds ~48 bits)
    fail = 0;
    worst = 0;
    for (int i = 0; i < N; ++i) {
        double d = rnd_double(-22, 30);
        double m = qp::merge_df(qp::split_d(d));
        double r = fabs(m - d) / fabs(d);
        worst = fmax(worst, r);
        if (r > ldexp(1.0, -46)) ++fail;
    }
    printf("roundtrip %ld %.3e\n", fail, worst);

    // add_fd(d, f) == round(d + f) within one ulp, over the magnitudes of
    // the step's increments (from far below d's last place to d / 4)
    fail = 0;
    worst = 0;
    for (int i = 0; i < N; ++i) {
        double d = rnd_double(-10, 10);
        double rel = pow(10.0, -20.0 * u01(rng));
        float f = (float)(d * rel * ((rng() & 1) ? 0.25 : -0.25));
        if (i % 17 == 0) f = 0.0f;
        LD exact = (LD)d + (LD)f;
        double m = qp::add_fd(d, f);
        double r = fabs((double)((LD)m - exact)) / ulp((double)exact);
        worst = fmax(worst, r);
        if (r > 1.0) ++fail;
    }
    for (int i = 0; i < 4000; ++i) {
        // zero d: exact; comparable magnitudes (the double-float path):
        // within 2^-46 of the result
        double d = (i % 2) ? 0.0 : rnd_double(-3, 3);
        float f = (float)rnd_double(-3, 3);
        LD exact = (LD)d + (LD)f;
        double m = qp::add_fd(d, f);
        double err = fabs((double)((LD)m - exact));
        if (d == 0.0 ? err != 0.0 : err > ldexp(fabs((double)exact) + fabs(d), -46)) ++fail;
    }
    printf("add_fd %ld %.3e\n", fail, worst);

    // merge of normalised pairs == round(hi + lo) within one ulp
    fail = 0;
    worst = 0;
    for (int i = 0; i < N; ++i) {
        float hi = (float)rnd_double(-20, 20);
        float uh = nextafterf(fabsf(hi), INFINITY) - fabsf(hi);
        float lo = (float)((u01(rng) - 0.5) * uh * (i % 7 == 0 ? 1.0 : 0.37));
        if (i % 11 == 0) lo = 0.0f;
        if (i % 13 == 0) lo = (float)((u01(rng) - 0.5) * uh * 1e-9);
        LD exact = (LD)hi + (LD)lo;
        double m = qp::merge_df({hi, lo});
        double r = fabs((double)((LD)m - exact)) / ulp((double)exact);
        worst = fmax(worst, r);
        if (r > 1.0) ++fail;
    }
    printf("merge %ld %.3e\n", fail, worst);

    // f_to_d exact
    fail = 0;
    for (int i = 0; i < N; ++i) {
        float f = (float)rnd_double(-30, 30);
        if (qp::f_to_d(f) != (double)f) ++fail;
    }
    printf("f_to_d %ld 0\n", fail);

    // TwoSum / TwoProd are exact
    fail = 0;
    for (int i = 0; i < N; ++i) {
        float a = (float)rnd_double(-10, 10), b = (float)rnd_double(-10, 10);
        df2 s = qp::two_sum(a, b);
        if ((LD)s.hi + (LD)s.lo != (LD)a + (LD)b) ++fail;
        df2 p = qp::two_prod(a, b);
        if ((LD)p.hi + (LD)p.lo != (LD)a * (LD)b) ++fail;
    }
    printf("eft %ld 0\n", fail);

    // df arithmetic: relative error bound 2^-44
    fail = 0;
    worst = 0;
    for (int i = 0; i < N; ++i) {
        double x = rnd_double(-5, 5), y = rnd_double(-5, 5);
        df2 a = qp::split_d(x), b = qp::split_d(y);
        LD ax = (LD)a.hi + a.lo, by = (LD)b.hi + b.lo;
        struct { df2 v; LD e; } cases[4] = {
            {qp::df_mul(a, b), ax * by},
            {qp::df_sqr(a), ax * ax},
            {qp::df_sqrt(qp::df_sqr(a)), fabsl(ax)},
            {qp::df_mul_f(a, b.hi), ax * (LD)b.hi},
        };
        for (auto &c : cases) {
            double r = (double)(fabsl(((LD)c.v.hi + c.v.lo) - c.e) / fabsl(c.e));
            worst = fmax(worst, r);
            if (r > ldexp(1.0, -44)) ++fail;
        }
        // additions: error relative to the operands' magnitude
        df2 s = qp::df_add(a, b);
        LD es = ax + by;
        double r = (double)(fabsl(((LD)s.hi + s.lo) - es) / (fabsl(ax) + fabsl(by)));
        worst = fmax(worst, r);
        if (r > ldexp(1.0, -45)) ++fail;
    }
    printf("arith %ld %.3e\n", fail, worst);

    // chi_e with the double-float formula for particles nearly co-moving with
    // a plane wave (the cancellation of Eq. 1): relative error against the
    // exact value, bounded by 1e-13 gamma^2 (the ~2^-44 error of a chain of
    // double-float operations amplified by 2 gamma^2)
    fail = 0;
    worst = 0;
    for (int i = 0; i < 20000; ++i) {
        double p = pow(10.0, 1.0 + 3.0 * u01(rng));  // |u| in [10, 1e4]
        double ang = 1e-3 * u01(rng);
        double ux = p * cos(ang), uy = p * sin(ang), uz = 0.0;
        float E = 50.0f, B = 50.0f;  // E_y = B_z
        df2 dx = qp::split_d(ux), dy = qp::split_d(uy), dz = qp::split_d(uz);
        df2 g2 = qp::df_add_f(qp::df_add(qp::df_add(qp::df_sqr(dx), qp::df_sqr(dy)), qp::df_sqr(dz)),
                              1.0f);
        df2 g = qp::df_sqrt(g2);
        // a = g E + u x B with E = (0,E,0), B = (0,0,B)
        df2 ax = qp::df_mul_f(dy, B);                               // uy Bz
        df2 ay = qp::df_sub(qp::df_mul_f(g, E), qp::df_mul_f(dx, B)); // g E - ux Bz
        df2 ue = qp::df_mul_f(dy, E);
        df2 s = qp::df_sub(qp::df_add(qp::df_sqr(ax), qp::df_sqr(ay)), qp::df_sqr(ue));
        double chi = sqrt(fmax((double)s.hi + (double)s.lo, 0.0));
        LD G = sqrtl(1.0L + (LD)ux * ux + (LD)uy * uy);
        LD AX = (LD)uy * B, AY = G * E - (LD)ux * B, UE = (LD)uy * E;
        LD CH = sqrtl(AX * AX + AY * AY - UE * UE);
        double r = (double)(fabsl(chi - CH) / CH);
        worst = fmax(worst, r / (double)(G * G));
        if (r > 1e-13 * (double)(G * G)) ++fail;
    }
    printf("chi_cancellation %ld %.3e\n", fail, worst);  // worst r / gamma^2
    return 0;
}
