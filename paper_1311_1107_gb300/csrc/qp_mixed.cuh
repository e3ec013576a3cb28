// Mixed-precision particle updates (QP_MIXED): FP32 gather, tables and
// sampling; chi_e, the Sokolov denominator and the accumulated momentum,
// position and optical depth carried in double-float (qp_df.h) and written
// back to the FP64 arrays by integer instructions.  On the common path no
// instruction uses the FP64 pipe, which issues at ~1/65 of the FP32 rate on
// GB300.
#pragma once

#include "qp_device.cuh"
#include "qp_df.h"

namespace qp {

// The reduction of a double-float phase to [-pi, pi] (2 pi as a pair); the
// hardware cosine is accurate to 2^-21.4 absolute on that interval.
__device__ __forceinline__ float reduce_phase(df2 ph)
{
    const float n = rintf(ph.hi * 0.15915494309189535f);
    const df2 m = df_mul_f({6.28318548202514648f, -1.74845553e-7f}, n);
    const df2 r = df_sub(ph, m);
    return r.hi + r.lo;
}

// Fields at the FP64 position (xd, yd, zd) and time of the step; each field
// model converts the coordinates it needs to the precision it needs them in
// (double-float where a phase or a cell index must resolve the position,
// the nearest float elsewhere).
template <int FK>
__device__ __forceinline__ void eval_field_mixed(const FieldDev &f, const MixedConsts &m,
                                                 double xd, double yd, double zd,
                                                 Vec3<float> &E, Vec3<float> &B)
{
    E = {0.0f, 0.0f, 0.0f};
    B = {0.0f, 0.0f, 0.0f};
    if constexpr (FK == QP_FIELD_PLANE) {
        // E_y = B_z = a0 cos(t - x)
        const float v = m.a0 * __cosf(reduce_phase(df_sub({m.t_hi, m.t_lo}, split_d(xd))));
        E.y = v;
        B.z = v;
    } else if constexpr (FK == QP_FIELD_GAUSSIAN) {
        const df2 xi = df_sub(split_d(xd), {m.xf_hi, m.xf_lo});
        const df2 eta = df_sub({m.tr_hi, m.tr_lo}, xi);  // (t - t_f) - xi
        const float xf = xi.hi, yf = hi_d(yd), zf = hi_d(zd);
        const float q = xf * m.inv_zr;
        const float wr2 = 1.0f + q * q;
        const float r2 = yf * yf + zf * zf;
        const float ef = df_to_f(eta);
        const float env = -r2 * m.inv_w0sq / wr2 - m.k_env * ef * ef;
        const float amp = m.a0 * rsqrtf(wr2) * __expf(env);
        const float curv = r2 * xf / (2.0f * (xf * xf + m.zr * m.zr));
        const float v = amp * __cosf(reduce_phase(df_add_f(df_neg(eta), curv - atanf(q))));
        E.y = v;
        B.z = v;
    } else if constexpr (FK == QP_FIELD_UNIFORM_B) {
        B.z = m.b0;
    } else if constexpr (FK == QP_FIELD_YEE2D) {
        // cell coordinates in double-float, then FP32 weights
        const df2 gx = df_sub(df_mul(split_d(xd), {m.idx_hi, m.idx_lo}), {m.x0s_hi, m.x0s_lo});
        const df2 gy = df_sub(df_mul(split_d(yd), {m.idy_hi, m.idy_lo}), {m.y0s_hi, m.y0s_lo});
        int ix[2], iy[2];
        float wx[2], wy[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const df2 ax = h ? df_add_f(gx, -0.5f) : gx, ay = h ? df_add_f(gy, -0.5f) : gy;
            float fx = floorf(ax.hi), fy = floorf(ay.hi);
            float rx = (ax.hi - fx) + ax.lo, ry = (ay.hi - fy) + ay.lo;
            if (rx < 0.0f) { rx += 1.0f; fx -= 1.0f; }
            if (rx >= 1.0f) { rx -= 1.0f; fx += 1.0f; }
            if (ry < 0.0f) { ry += 1.0f; fy -= 1.0f; }
            if (ry >= 1.0f) { ry -= 1.0f; fy += 1.0f; }
            wx[h] = rx;
            wy[h] = ry;
            // clamp before the conversion (NaN and huge values included)
            ix[h] = (int)fmaxf(-2.0f, fminf(m.nxf + 1.0f, fx));
            iy[h] = (int)fmaxf(-2.0f, fminf(m.nyf + 1.0f, fy));
        }
        yee_gather<float>(f, ix, iy, wx, wy, E, B);
    }
}

// r / a_S with 1/a_S as the pair (hi, lo): a rounding error of one unit that
// varies from particle to particle instead of the constant's fixed bias
__device__ __forceinline__ float over_aS(float r, float hi, float lo) { return fmaf(r, hi, r * lo); }

__device__ __forceinline__ df2 df_add_s(df2 a, df2 b)
{
    // "sloppy" sum: exact high parts, low parts added once (enough for the
    // sums below, including gamma E + u x B, see qp_df.h)
    const df2 s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, add_rn(s.lo, add_rn(a.lo, b.lo)));
}

// gamma = sqrt(1 + |u|^2) in double-float
__device__ __forceinline__ df2 gamma_df(df2 ux, df2 uy, df2 uz)
{
    return df_sqrt(df_add_f(df_add_s(df_add_s(df_sqr(ux), df_sqr(uy)), df_sqr(uz)), 1.0f));
}

// chi_e = sqrt(|gamma E + u x B|^2 - (u.E)^2) / a_S (Eq. 1), the
// differences carried in double-float
__device__ __forceinline__ float chi_mixed(df2 g, df2 ux, df2 uy, df2 uz, const Vec3<float> &E,
                                           const Vec3<float> &B, float ia_hi, float ia_lo)
{
    const df2 ax = df_add_s(df_mul_f(g, E.x), df_add_s(df_mul_f(uy, B.z), df_mul_f(uz, -B.y)));
    const df2 ay = df_add_s(df_mul_f(g, E.y), df_add_s(df_mul_f(uz, B.x), df_mul_f(ux, -B.z)));
    const df2 az = df_add_s(df_mul_f(g, E.z), df_add_s(df_mul_f(ux, B.y), df_mul_f(uy, -B.x)));
    const df2 ue = df_add_s(df_add_s(df_mul_f(ux, E.x), df_mul_f(uy, E.y)), df_mul_f(uz, E.z));
    const df2 s = df_add_s(df_add_s(df_add_s(df_sqr(ax), df_sqr(ay)), df_sqr(az)), df_neg(df_sqr(ue)));
    const float v = s.hi + s.lo;
    return v > 0.0f ? over_aS(sqrtf(v), ia_hi, ia_lo) : 0.0f;
}

// chi_e in double-float from the exact split of u0 plus du: the rare case of
// strong cancellation, called out of line so the FP32 path stays short
static __device__ __noinline__ float chi_mixed_split(double u0x, double u0y, double u0z,
                                                     float dux, float duy, float duz,
                                                     Vec3<float> E, Vec3<float> B, float ia_hi,
                                                     float ia_lo)
{
    const df2 UX = df_add_f(split_d(u0x), dux), UY = df_add_f(split_d(u0y), duy),
              UZ = df_add_f(split_d(u0z), duz);
    return chi_mixed(gamma_df(UX, UY, UZ), UX, UY, UZ, E, B, ia_hi, ia_lo);
}

// chi_e of u = u0 + du (u0 the FP64 state, du an FP32 increment): in FP32
// when |gamma E + u x B| and |a|^2 - (u.E)^2 show no strong cancellation (FP32
// then gives chi to ~1e-6), else in double-float from the exact split of u0.
__device__ __forceinline__ float chi_mixed_auto(double u0x, double u0y, double u0z, float dux,
                                                float duy, float duz, float ux, float uy, float uz,
                                                float g, const Vec3<float> &E,
                                                const Vec3<float> &B, float ia_hi, float ia_lo)
{
    const float cx = uy * B.z - uz * B.y, cy = uz * B.x - ux * B.z, cz = ux * B.y - uy * B.x;
    const float ax = fmaf(g, E.x, cx), ay = fmaf(g, E.y, cy), az = fmaf(g, E.z, cz);
    const float a2 = ax * ax + ay * ay + az * az;
    const float ue = ux * E.x + uy * E.y + uz * E.z;
    const float s = a2 - ue * ue;
    const float scale = g * g * (E.x * E.x + E.y * E.y + E.z * E.z) + cx * cx + cy * cy + cz * cz;
    if (a2 > 1e-2f * scale && s > 1e-2f * a2) return over_aS(sqrtf(s), ia_hi, ia_lo);
    if (!(scale > 0.0f)) return 0.0f;
    return chi_mixed_split(u0x, u0y, u0z, dux, duy, duz, E, B, ia_hi, ia_lo);
}

// The 53-bit uniform ((a>>5) 2^26 + (b>>6) + 1) 2^-53 of the FP64 path,
// rounded to FP32 (relative error 2^-24 at every magnitude) with 32-bit
// integer conversions only.
__device__ __forceinline__ float u53f(unsigned a, unsigned b)
{
    return fmaf((float)(b >> 6) + 1.0f, 0x1.0p-26f, (float)(a >> 5)) * 0x1.0p-27f;
}

// The same uniform and its complement 1 - u53 as unevaluated float pairs
// hi + lo (hi exact: the top 24 of the 27 bits of a >> 5; lo rounded, so the
// pair is within 2^-48 of the exact value).
__device__ __forceinline__ df2 u53_pair(unsigned a, unsigned b)
{
    const unsigned A = a >> 5, B = b >> 6;
    return {(float)(A & ~7u) * 0x1.0p-27f, (float)(((A & 7u) << 26) + B + 1u) * 0x1.0p-53f};
}

__device__ __forceinline__ df2 u53_pair_complement(unsigned a, unsigned b)
{
    const unsigned A = (~a) >> 5, B = (~b) >> 6;
    return {(float)(A & ~7u) * 0x1.0p-27f, (float)(((A & 7u) << 26) + B) * 0x1.0p-53f};
}

// ------------------------------------------------------------------ Eq. 7 in FP32
struct FracPair {
    float x, omx;  // the sampled fraction and 1 - fraction, each to FP32 relative precision
};

// x = 1/(1 + e^-s) and 1 - x at s = s_j + ds t (0 <= t <= 1), from the
// tabulated e^-s_j: no large logit is ever rounded to FP32
__device__ __forceinline__ FracPair logit_node(const float *__restrict__ En, int j, float ds,
                                               float t)
{
    const float e = __ldg(En + j) * expf(-ds * t);
    const float x = 1.0f / (1.0f + e);
    return {x, e * x};
}

// (a.hi + a.lo) - (c.x + c.y), exact to a rounding of the result
__device__ __forceinline__ float pair_diff(df2 a, float2 c) { return (a.hi - c.x) + (a.lo - c.y); }

__device__ __forceinline__ float2 ldg2(const float2 *p) { return __ldg(p); }

// Invert one row at xi (eta = 1 - xi, from the same random bits): the lower
// half searches the row C for xi, the upper half searches its complement
// Q = 1 - C for eta.  Rows, xi and eta are float pairs, so the position
// between two nodes, (xi - C_j)/(C_j+1 - C_j), keeps FP32 relative precision
// even where neighbouring nodes differ by 1e-3 or less.
__device__ __forceinline__ FracPair row_invert_f(const float2 *__restrict__ C,
                                                 const float2 *__restrict__ Q,
                                                 const unsigned char *__restrict__ guide,
                                                 const float *__restrict__ En, df2 xi, df2 eta,
                                                 float ds, bool power_tail)
{
    if (xi.hi <= 0.5f) {
        const float2 c0 = ldg2(C);
        if (pair_diff(xi, c0) <= 0.0f) {
            const FracPair p0 = logit_node(En, 0, ds, 0.0f);
            if (power_tail && c0.x > 0.0f) {
                // below the first node u grows as xi^3 (the u^(1/3) law)
                const float r = (xi.hi + xi.lo) / (c0.x + c0.y);
                const float x = p0.x * r * r * r;
                return {x, 1.0f - x};
            }
            return p0;
        }
        // the last node below xi: guide entry, then a forward scan
        int lo = (int)__ldg(guide + guide_bucket(xi.hi));
#pragma unroll 1
        while (lo < kNNode - 2 && pair_diff(xi, ldg2(C + lo + 1)) > 0.0f) ++lo;
        const float2 c_lo = ldg2(C + lo), c_hi = ldg2(C + lo + 1);
        const float den = (c_hi.x - c_lo.x) + (c_hi.y - c_lo.y);
        const float t = den > 0.0f ? fminf(pair_diff(xi, c_lo) / den, 1.0f) : 0.0f;
        return logit_node(En, lo, ds, t);
    }
    if (pair_diff(eta, ldg2(Q + kNNode - 1)) <= 0.0f) return logit_node(En, kNNode - 1, ds, 0.0f);
    // Q decreases along the row: the last node with Q > eta (guide, then scan)
    int lo = (int)__ldg(guide + kNCdf * kGuideBuckets + guide_bucket(eta.hi));
#pragma unroll 1
    while (lo < kNNode - 2 && pair_diff(eta, ldg2(Q + lo + 1)) < 0.0f) ++lo;
    const float2 q_lo = ldg2(Q + lo), q_hi = ldg2(Q + lo + 1);
    const float den = (q_lo.x - q_hi.x) + (q_lo.y - q_hi.y);
    const float t = den > 0.0f ? fminf(-pair_diff(eta, q_lo) / den, 1.0f) : 0.0f;
    return logit_node(En, lo, ds, fmaxf(t, 0.0f));
}

// Inverse CDF of Eq. 7 (emission rows) or of the pair spectrum, linear
// between the two chi rows around chi (same rule as the FP64 path).  One
// copy of the row inversion serves both rows (a loop of one or two).
__device__ __forceinline__ FracPair sample_cdf_f(const float2 *__restrict__ rows,
                                                 const float2 *__restrict__ qrows,
                                                 const unsigned char *__restrict__ guide,
                                                 const float *__restrict__ En, float chi, df2 xi,
                                                 df2 eta, float ds, bool emission, bool &clamped)
{
    const bool below = !(chi >= (float)kChiLo);
    int j = 0, nrow = 1;
    float f = 0.0f;
    if (below) {
        j = 0;
    } else if (chi >= (float)kChiHi) {
        clamped = true;
        j = kNCdf - 1;
    } else {
        j = grid_index32<2>(chi, f);
        nrow = 2;
    }
    FracPair a{0.0f, 1.0f}, b{0.0f, 1.0f};
#pragma unroll 1
    for (int k = 0; k < nrow; ++k, ++j) {
        const FracPair r = row_invert_f(rows + j * kNNode, qrows + j * kNNode,
                                        guide + j * kGuideBuckets, En, xi, eta, ds, emission);
        if (k == 0)
            a = r;
        else
            b = r;
    }
    if (nrow == 2) return {a.x + f * (b.x - a.x), a.omx + f * (b.omx - a.omx)};
    if (below && emission) {
        const float x = (chi / (float)kChiLo) * a.x;
        return {x, 1.0f - x};
    }
    return a;
}

}  // namespace qp
