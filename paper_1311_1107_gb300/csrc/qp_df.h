// Double-float arithmetic and FP64 <-> double-float conversion by integer
// operations, for the mixed-precision path.
//
// On GB300 every FP64 instruction, and every f32 <-> f64 conversion, issues
// at about 1/65 of the FP32 rate.  The mixed path therefore keeps the FP64
// storage of momenta, positions and optical depths, but converts them to
// double-float pairs (hi + lo, two FP32 numbers, ~47 significant bits) with
// integer and FP32 instructions only, carries the precision-critical
// quantities (chi_e's cancellation, the accumulated momentum, position and
// optical depth) in double-float, and converts back with integer
// instructions.  Everything here also compiles for the host, where it is
// tested bit-for-bit against exact double arithmetic.
//
// The error-free transformations are the classical ones: TwoSum (Knuth),
// FastTwoSum (Dekker) and TwoProd with a fused multiply-add.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define QP_HD __host__ __device__ __forceinline__
// rare cases: called, never inlined, so that the common path's code stays
// short and carries no predicated-off FP64 instructions
#define QP_HD_COLD __host__ __device__ inline __noinline__
// frequent but repeated many times per particle: one called copy keeps the
// step kernel's instruction footprint small (it measured faster than
// inlining every call site)
#define QP_HD_SHARED __host__ __device__ inline __noinline__
#else
#define QP_HD inline
#define QP_HD_COLD inline
#define QP_HD_SHARED inline
#include <math.h>
#include <string.h>
#endif

namespace qp {

// ------------------------------------------------------------------ bit casts

QP_HD uint32_t f2u(float f)
{
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
#endif
}

QP_HD float u2f(uint32_t u)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, 4);
    return f;
#endif
}

QP_HD uint64_t d2u(double d)
{
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(d);
#else
    uint64_t u;
    memcpy(&u, &d, 8);
    return u;
#endif
}

QP_HD double u2d(uint64_t u)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double d;
    memcpy(&d, &u, 8);
    return d;
#endif
}

QP_HD float fma32(float a, float b, float c)
{
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return fmaf(a, b, c);
#endif
}

// Plain FP32 operations that the compiler must neither fuse nor reorder
// (the error-free transformations depend on each rounding).
QP_HD float add_rn(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    volatile float r = a + b;
    return r;
#endif
}

QP_HD float sub_rn(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    volatile float r = a - b;
    return r;
#endif
}

QP_HD float mul_rn(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    volatile float r = a * b;
    return r;
#endif
}

// ------------------------------------------------------------------ double-float

struct df2 {
    float hi, lo;
};

QP_HD df2 two_sum(float a, float b)
{
    const float s = add_rn(a, b);
    const float bb = sub_rn(s, a);
    const float e = add_rn(sub_rn(a, sub_rn(s, bb)), sub_rn(b, bb));
    return {s, e};
}

// requires |a| >= |b| (or a == 0)
QP_HD df2 fast_two_sum(float a, float b)
{
    const float s = add_rn(a, b);
    return {s, sub_rn(b, sub_rn(s, a))};
}

QP_HD df2 two_prod(float a, float b)
{
    const float p = mul_rn(a, b);
    return {p, fma32(a, b, -p)};
}

QP_HD df2 df_add(df2 a, df2 b)
{
    const df2 s = two_sum(a.hi, b.hi);
    const df2 t = two_sum(a.lo, b.lo);
    df2 r = fast_two_sum(s.hi, add_rn(s.lo, t.hi));
    return fast_two_sum(r.hi, add_rn(r.lo, t.lo));
}

QP_HD df2 df_add_f(df2 a, float b)
{
    const df2 s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, add_rn(s.lo, a.lo));
}

QP_HD df2 df_neg(df2 a) { return {-a.hi, -a.lo}; }

QP_HD df2 df_sub(df2 a, df2 b) { return df_add(a, df_neg(b)); }

QP_HD df2 df_mul_f(df2 a, float b)
{
    const df2 p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, fma32(a.lo, b, p.lo));
}

QP_HD df2 df_mul(df2 a, df2 b)
{
    const df2 p = two_prod(a.hi, b.hi);
    return fast_two_sum(p.hi, fma32(a.hi, b.lo, fma32(a.lo, b.hi, p.lo)));
}

QP_HD df2 df_sqr(df2 a)
{
    const df2 p = two_prod(a.hi, a.hi);
    return fast_two_sum(p.hi, fma32(a.hi + a.hi, a.lo, p.lo));
}

// sqrt of a >= 0: one Newton correction of the FP32 root
QP_HD df2 df_sqrt(df2 a)
{
    if (!(a.hi > 0.0f)) return {0.0f, 0.0f};
#ifdef __CUDA_ARCH__
    const float s = __fsqrt_rn(a.hi);
#else
    const float s = sqrtf(a.hi);
#endif
    const df2 s2 = two_prod(s, s);
    const float r = (((a.hi - s2.hi) - s2.lo) + a.lo) / (2.0f * s);
    return fast_two_sum(s, r);
}

QP_HD float df_to_f(df2 a) { return a.hi + a.lo; }

// ------------------------------------------------------------------ FP64 <-> double-float

// Split a double into hi (its first 24 significand bits, truncated) and lo
// (the remainder rounded to FP32), using integer and FP32 instructions only.
// |d| below 2^-126 gives (0, 0); |d| at or above 2^128 is not supported
// (the caller's values are far inside this range).  hi + lo == d to within
// 2^-47 |d|.
QP_HD df2 split_d(double d)
{
    const uint64_t b = d2u(d);
    const uint32_t dh = (uint32_t)(b >> 32), dl = (uint32_t)b;
    const uint32_t e = (dh >> 20) & 0x7FFu;
    if (e < 897u) return {0.0f, 0.0f};
    // sign | (e - 896) << 23 | top 23 mantissa bits
    const uint32_t top = (dh << 3) | (dl >> 29);
    const uint32_t hb = ((top - (384u << 23)) & 0x7FFFFFFFu) | (dh & 0x80000000u);
    // remainder: the low 29 mantissa bits, worth 2^(e - 1075) each
    const uint32_t r29 = dl & 0x1FFFFFFFu;
    float lo = 0.0f;
    if (r29 && e >= 949u) {
        // exact FP32 values of the two halves, then one rounding in the fma
        const float fa = u2f(0x4B000000u | (r29 >> 15)) - 8388608.0f;
        const float fb = u2f(0x4B000000u | (r29 & 0x7FFFu)) - 8388608.0f;
        const float m = fma32(fa, 32768.0f, fb);
        lo = m * u2f((e - 948u) << 23);
        if (dh & 0x80000000u) lo = -lo;
    }
    return {u2f(hb), lo};
}

// d rounded to the nearest float (ties away from zero) by integer
// instructions; |d| below 2^-126 gives 0.  Rounding to nearest matters where
// an FP32 update acts on this value in place of d: a truncated (always
// smaller) value would let, e.g., a rotation shrink |u| by a biased amount
// every step.  A carry out of the mantissa rounds up into the exponent.
QP_HD float hi_d(double d)
{
    const uint64_t b = d2u(d);
    const uint32_t dh = (uint32_t)(b >> 32), dl = (uint32_t)b;
    const uint32_t e = (dh >> 20) & 0x7FFu;
    if (e < 897u) return 0.0f;
    const uint32_t top = ((dh << 3) | (dl >> 29)) + ((dl >> 28) & 1u);
    return u2f(((top - (384u << 23)) & 0x7FFFFFFFu) | (dh & 0x80000000u));
}

// Exact conversion of a float to double by integer instructions (normal
// floats; zero and denormals give 0).
QP_HD double f_to_d(float f)
{
    const uint32_t b = f2u(f);
    const uint32_t e = (b >> 23) & 0xFFu;
    if (e == 0u) return 0.0;
    return u2d(((uint64_t)(b & 0x80000000u) << 32) | ((uint64_t)(e + 896u) << 52) |
               ((uint64_t)(b & 0x7FFFFFu) << 29));
}

// hi + lo rounded to double (within one unit in the last place) by integer
// instructions, for a normalised pair (|lo| <= ulp(hi), as every df2
// operation above returns).  Pairs outside that range, zero hi, and
// non-finite values take an FP64 path.
QP_HD_COLD double merge_df_fp64(float hi, float lo) { return (double)hi + (double)lo; }

QP_HD double merge_df(df2 a)
{
    const uint32_t hb = f2u(a.hi), lb = f2u(a.lo);
    const uint32_t eh = (hb >> 23) & 0xFFu, el = (lb >> 23) & 0xFFu;
    if (eh == 0u || eh == 0xFFu || el == 0xFFu) return merge_df_fp64(a.hi, a.lo);
    const uint64_t sign = (uint64_t)(hb & 0x80000000u) << 32;
    int64_t S = (int64_t)((1ull << 52) | ((uint64_t)(hb & 0x7FFFFFu) << 29));
    if (el != 0u) {
        // lo in units of 2^-52 of hi's binade: ml * 2^(el - eh + 29)
        const int k = (int)el - (int)eh + 29;
        if (k > 8) return merge_df_fp64(a.hi, a.lo);  // not normalised
        const uint64_t ml = (1ull << 23) | (lb & 0x7FFFFFu);
        uint64_t L;
        if (k >= 0)
            L = ml << k;
        else if (k > -40)
            L = (ml + (1ull << (-k - 1))) >> (-k);
        else
            L = 0;
        if ((hb ^ lb) & 0x80000000u)
            S -= (int64_t)L;
        else
            S += (int64_t)L;
    }
    uint64_t e = (uint64_t)eh + 896u;
    if (S >= (int64_t)(1ull << 53)) {
        S = (S + 1) >> 1;
        e += 1;
    } else if (S < (int64_t)(1ull << 52)) {
        S <<= 1;
        e -= 1;
    }
    return u2d(sign | (e << 52) | ((uint64_t)S & ((1ull << 52) - 1)));
}

// d + f rounded to double (within one unit in the last place) by integer
// instructions: the FP64 accumulation of an FP32 increment.  The stored
// double keeps all its bits; only the increment carries FP32 error.
// add_fd handles the common case inline (d and f normal, f from half a unit
// of d's last place up to 2^27 units, the sum in d's binade) and calls
// add_fd_slow for the rest.

// The cases add_fd does not handle in integers (zero or tiny d, increments
// comparable to or larger than d, large cancellations): through a
// double-float sum, exact to 2^-47 relative, still without FP64
// instructions; non-finite values go through FP64.
QP_HD_COLD double add_fd_wide(double d, float f)
{
    const uint32_t ed = (uint32_t)(d2u(d) >> 52) & 0x7FFu;
    const uint32_t ef = (f2u(f) >> 23) & 0xFFu;
    if (ed == 0x7FFu || ef == 0xFFu || (ed != 0u && ed < 897u) || ed > 1150u)
        return d + (double)f;
    return merge_df(df_add_f(split_d(d), f));
}

// The general integer sum (the result may leave d's binade: renormalised,
// rounded once); zero, non-finite and subnormal operands, increments not
// much smaller than d, and large cancellations take add_fd_wide.
QP_HD_COLD double add_fd_slow(double d, float f)
{
    const uint32_t fb = f2u(f);
    if ((fb & 0x7FFFFFFFu) == 0u) return d;
    const uint64_t db = d2u(d);
    const uint32_t ed = (uint32_t)(db >> 52) & 0x7FFu, ef = (fb >> 23) & 0xFFu;
    if (ed == 0u || ed == 0x7FFu || ef == 0u || ef == 0xFFu) return add_fd_wide(d, f);
    // f in units of d's last place: mf * 2^k, k = ef - ed + 925
    const int k = (int)ef - (int)ed + 925;
    if (k > 28) return add_fd_wide(d, f);
    if (k < -25) return d;  // below half a unit of d
    const uint64_t mf = (1ull << 23) | (fb & 0x7FFFFFu);
    const uint64_t L = k >= 0 ? (mf << k) : ((mf + (1ull << (-k - 1))) >> (-k));
    int64_t S = (int64_t)((1ull << 52) | (db & ((1ull << 52) - 1)));
    if ((uint32_t)(db >> 63) != (fb >> 31))
        S -= (int64_t)L;
    else
        S += (int64_t)L;
    uint64_t e = ed;
    if (S >= (int64_t)(1ull << 53)) {
        S = (S + 1) >> 1;
        e += 1;
    } else if (S < (int64_t)(1ull << 52)) {
        if (S < (int64_t)(1ull << 51) || e <= 1u) return add_fd_wide(d, f);
        S <<= 1;
        e -= 1;
    }
    return u2d((db & 0x8000000000000000ull) | (e << 52) | ((uint64_t)S & ((1ull << 52) - 1)));
}

QP_HD_SHARED double add_fd(double d, float f)
{
    const uint32_t fb = f2u(f);
    if ((fb << 1) == 0u) return d;  // f = +-0
    const uint64_t db = d2u(d);
    const uint32_t dh = (uint32_t)(db >> 32);
    const uint32_t ed = (dh >> 20) & 0x7FFu, ef = (fb >> 23) & 0xFFu;
    // f in units of d's last place: mf * 2^k, k = ef - ed + 925
    const int k = (int)ef - (int)ed + 925;
    if ((ed - 1u) < 0x7FEu && (ef - 1u) < 0xFEu && k <= 27) {
        if (k < -25) return d;  // below half a unit of d's last place
        const uint32_t mf = (1u << 23) | (fb & 0x7FFFFFu);
        // the increment rounded to d's last place (half-way cases away from zero)
        const uint64_t L =
            k >= 0 ? ((uint64_t)mf << k) : (uint64_t)((mf + (1u << (-k - 1))) >> (-k));
        // added to (or taken from) the magnitude bits directly: exact while
        // the exponent field stays the same, which the test below confirms
        const uint64_t r = ((dh ^ fb) >> 31) ? db - L : db + L;
        if (((((uint32_t)(r >> 32)) ^ dh) & 0x7FF00000u) == 0u) return u2d(r);
    }
    return add_fd_slow(d, f);
}

}  // namespace qp
