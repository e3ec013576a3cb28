// Device building blocks of libqedpic: kernel argument layout, Philox,
// field models, chi, table lookups and inverse-CDF sampling.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "qp_internal.h"

namespace qp {

enum Prec { kFP64 = 0, kMixed = 1 };
constexpr int kTile = QP_STEP_TILE;  // particles per step tile = threads per block
constexpr int kWarps = kTile / 32;
constexpr int kDiagTile = 256;  // slots per block tile of the diagnostics

// ------------------------------------------------------------------ layout

struct SpeciesDev {
    double *x, *y, *z, *ux, *uy, *uz, *tau, *w, *chi;
    int32_t *nemit;
    int64_t *n_live;
    int64_t cap;
    int64_t id_base;     // global number of slot 0: particle id = id_base + slot
    int64_t id_split;    // > 0: slots from here on are id_append + (slot - id_split)
    int64_t id_append;
    int32_t present;
    int32_t slot_stats;  // index of this species' counter block
};

// The particle id of a slot: the counter of its random streams.
__device__ __forceinline__ int64_t particle_id(int64_t id_base, int64_t id_split,
                                               int64_t id_append, int64_t slot)
{
    return (id_split > 0 && slot >= id_split) ? id_append + (slot - id_split) : id_base + slot;
}
__device__ __forceinline__ int64_t particle_id(const SpeciesDev &S, int64_t slot)
{
    return particle_id(S.id_base, S.id_split, S.id_append, slot);
}

// Per-species event counters (device; atomics aggregated per block).
struct DevStats {
    unsigned long long n_emit, n_photon, n_photon_drop, n_subthreshold, n_pair, n_pair_drop,
        n_saturated, n_clamped, n_continuous;
    double e_subthreshold, e_dropped;
};

struct FieldDev {
    int32_t kind;
    double a0, w0, tau_fwhm, x_focus, t_focus, b0;
    const float *yee[6];
    int64_t nx, ny;
    double dx, dy, x0, y0;
    double inv_dx, inv_dy, x0s, y0s;  // 1/dx, 1/dy, x0/dx, y0/dy (mixed gather)
};

struct TablesDev {
    const double *H, *Gs, *Ts, *Cg, *Cp;       // FP64
    const float *Hf, *Gsf, *Tsf;               // FP32 copies of the rate rows
    // CDF rows C and their complements Q = 1 - C as hi + lo float pairs
    const float2 *Cg2, *Cp2, *Qg2, *Qp2;
    const float *Eg, *Ep;                      // e^(-s_j) at the logit nodes
    // guide tables of the CDF rows (see guide_bucket): [half][row][bucket]
    const unsigned char *Gg, *Gp;
};

// Step constants of the mixed path as FP32 values or double-float pairs
// (split on the host), so the kernel needs no FP64 arithmetic for them.
struct MixedConsts {
    float t_hi, t_lo;           // t = n dt
    float tr_hi, tr_lo;         // t - t_focus (Gaussian pulse)
    float xf_hi, xf_lo;         // x_focus
    float idx_hi, idx_lo, idy_hi, idy_lo;  // 1/dx, 1/dy (Yee grid)
    float x0s_hi, x0s_lo, y0s_hi, y0s_lo;  // x0/dx, y0/dy
    float h[2];                 // 0.5 q dt for electrons, positrons
    float dt, C_rate, inv_aS, tau0w, chi_th, gmin;
    float inv_aS_lo;            // 1/a_S - inv_aS: chi is scaled by the pair, so
                                // that no rounding of the constant biases every chi
    float a0, b0, zr, inv_zr, inv_w0sq, k_env;  // field shape (k_env = 2 ln2 / tau_fwhm^2)
    float nxf, nyf;                            // Yee grid size
};

// Device-resident control block of a launch sequence: the tile ticket, the
// count of finished blocks and the launch epoch that tags look-back words.  Blocks count their end in
// kDoneGroups group counters (one 32-byte sector each) and the last of each
// group in `done`: no counter sees more than a few tens of atomics at once.
constexpr int kDoneGroups = 32;
struct StepCtl {
    unsigned ticket, done, epoch, pad;
    unsigned grp[kDoneGroups][8];
};

constexpr int kMaxProblems = 64;  // problems (independent runs) per launch
// doubles per thread of one append record (see the stash of qp_step.cuh),
// and the append-record buffers per block: a tile's appends are written
// kStashBufs - 1 tiles after its physics
constexpr int kStashFieldsHost = 7 + 2 * QP_MAX_EMISSIONS;
constexpr int kStashBufs = 3;

// One independent run stepped by a launch: its species, field, step
// constants, look-back scratch and control words.  A launch steps either a
// single problem passed by value (qp_step) or a device table of problems
// (a batch); the kernel copies the problem of each tile to shared memory.
struct Problem {
    SpeciesDev sp[3];                 // electron, positron, photon
    FieldDev f;
    MixedConsts mc;                   // t_*, tr_* set per launch on the device
    unsigned long long *lep_words;    // look-back words of the lepton chain
    unsigned long long *pho_words;    // look-back words of the photon chain
    long long *pending;               // [3] new live counts, applied by the last block
    long long *step_ctr;              // device-stepped: next step index
    long long *left_ctr;              // device-stepped: launches still to run (0 = idle)
    long long *work_ctr;              // device-stepped: live slots stepped so far
    double dt, t;                     // t = step dt, set per launch on the device
    uint64_t step, seed;
    double chi_th, gmin;
    int32_t pairs, max_emit;
    int32_t device_step;              // 1: step and activity from step_ctr/left_ctr
    int32_t pad;
};

struct StepArgs {
    TablesDev tab;
    StepCtl *ctl;
    DevStats *stats;                  // counters, indexed by species handle
    int *status;                      // sticky status word
    double a_S, C_rate, tau0w;
    unsigned int spin_limit;          // bound of every device-side wait
    int32_t n_problems;               // 0: the single problem below
    const Problem *problems;          // device table of n_problems entries
    double *stash;                    // append records: [block][2][fields][kTile]
    Problem single;
};

// ------------------------------------------------------------------ status

__device__ __forceinline__ void raise_status(int *status, int code)
{
    // first error wins; a warning never overwrites an error
    int old = *((volatile int *)status);
    if (old < 0) return;
    if (code < 0)
        atomicCAS(status, old, code);
    else if (old == 0)
        atomicCAS(status, 0, code);
}

// ------------------------------------------------------------------ TMA bulk copies

__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// Global -> shared bulk copy completing on `bar`; both addresses 16-byte
// aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of `bar`; false on time-out.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity,
                                                  unsigned limit)
{
    for (unsigned k = 0; k < limit; ++k)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// ------------------------------------------------------------------ Philox4x32-10

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
    // two rounds per iteration: a short loop body keeps the several inlined
    // draws of the step kernel small in the instruction cache
#pragma unroll 1
    for (int r = 0; r < 10; r += 2) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
            const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
            c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
    }
    return c;
}

enum RngPurpose { kRngInit = 0, kRngEmit = 1, kRngPhotonTau = 2, kRngPair = 3, kRngPairPos = 4 };

// counter (slot lo, slot hi, step, species<<24 | purpose<<16 | k), key = seed
__device__ __forceinline__ uint4 draw(uint64_t seed, int species, int purpose, int64_t slot,
                                      uint64_t step, int k)
{
    const uint4 c = make_uint4((unsigned)((uint64_t)slot & 0xFFFFFFFFu),
                               (unsigned)((uint64_t)slot >> 32), (unsigned)(step & 0xFFFFFFFFu),
                               ((unsigned)species << 24) | ((unsigned)purpose << 16) |
                                   ((unsigned)k & 0xFFFFu));
    return philox4x32_10(c, make_uint2((unsigned)(seed & 0xFFFFFFFFu), (unsigned)(seed >> 32)));
}

// uniform in ]0,1] with 53 random bits
__device__ __forceinline__ double u53(unsigned a, unsigned b)
{
    const unsigned long long m = ((unsigned long long)(a >> 5) << 26) | (unsigned long long)(b >> 6);
    return (double)(m + 1ull) * 0x1.0p-53;
}

// ------------------------------------------------------------------ fields

template <typename R>
struct Vec3 {
    R x, y, z;
};

// Linear interpolation of the Yee components on their four staggered
// stencils (node/half-node in x and y): stencil (hx, hy) serves
// (0,0) Ez, (1,0) Ex and By, (0,1) Ey and Bx, (1,1) Bz.  Each stencil is
// bounds-checked once; nodes outside the grid contribute zero field.  The
// sum over the four nodes runs in the order (i,j), (i+1,j), (i,j+1),
// (i+1,j+1).
template <typename R>
struct YeeStencil {
    int base;      // index of node (i, j)
    int ix, iy;
    bool inside;   // all four nodes inside the grid
    R wx, wy;
};

template <typename R>
__device__ __forceinline__ R yee_interp(const float *__restrict__ F, const YeeStencil<R> &st,
                                        int nx, int ny)
{
    const R w00 = (R(1) - st.wx) * (R(1) - st.wy), w10 = st.wx * (R(1) - st.wy);
    const R w01 = (R(1) - st.wx) * st.wy, w11 = st.wx * st.wy;
    if (st.inside) {
        const float *p = F + st.base;
        R acc = R(0);
        acc += w00 * (R)__ldg(p);
        acc += w10 * (R)__ldg(p + 1);
        acc += w01 * (R)__ldg(p + nx);
        acc += w11 * (R)__ldg(p + nx + 1);
        return acc;
    }
    R acc = R(0);
    const R w[4] = {w00, w10, w01, w11};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int ii = st.ix + (k & 1), jj = st.iy + (k >> 1);
        if (ii < 0 || jj < 0 || ii >= nx || jj >= ny) continue;
        acc += w[k] * (R)__ldg(F + jj * nx + ii);
    }
    return acc;
}

template <typename R>
__device__ __forceinline__ void yee_gather(const FieldDev &f, const int ix[2], const int iy[2],
                                           const R wx[2], const R wy[2], Vec3<R> &E, Vec3<R> &B)
{
    const int nx = (int)f.nx, ny = (int)f.ny;
    // one check for all four stencils (their nodes span min(ix)..max(ix)+1)
    const bool all_inside = min(ix[0], ix[1]) >= 0 && min(iy[0], iy[1]) >= 0 &&
                            max(ix[0], ix[1]) + 1 < nx && max(iy[0], iy[1]) + 1 < ny;
    YeeStencil<R> st[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int hx = k & 1, hy = k >> 1;
        st[k].ix = ix[hx];
        st[k].iy = iy[hy];
        st[k].wx = wx[hx];
        st[k].wy = wy[hy];
        st[k].inside = all_inside || (ix[hx] >= 0 && iy[hy] >= 0 && ix[hx] + 1 < nx &&
                                      iy[hy] + 1 < ny);
        st[k].base = iy[hy] * nx + ix[hx];
    }
    if (all_inside) {
        // the common case: the 24 loads of the six components are issued
        // together (one round trip to memory), then combined in the order
        // of yee_interp
        const int comp_st[6] = {1, 2, 0, 2, 1, 3};  // stencil of Ex Ey Ez Bx By Bz
        float v[6][4];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const float *p = f.yee[c] + st[comp_st[c]].base;
            v[c][0] = __ldg(p);
            v[c][1] = __ldg(p + 1);
            v[c][2] = __ldg(p + nx);
            v[c][3] = __ldg(p + nx + 1);
        }
        R out[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const YeeStencil<R> &q = st[comp_st[c]];
            const R w00 = (R(1) - q.wx) * (R(1) - q.wy), w10 = q.wx * (R(1) - q.wy);
            const R w01 = (R(1) - q.wx) * q.wy, w11 = q.wx * q.wy;
            R acc = R(0);
            acc += w00 * (R)v[c][0];
            acc += w10 * (R)v[c][1];
            acc += w01 * (R)v[c][2];
            acc += w11 * (R)v[c][3];
            out[c] = acc;
        }
        E = {out[0], out[1], out[2]};
        B = {out[3], out[4], out[5]};
        return;
    }
    E.x = yee_interp<R>(f.yee[0], st[1], nx, ny);
    E.y = yee_interp<R>(f.yee[1], st[2], nx, ny);
    E.z = yee_interp<R>(f.yee[2], st[0], nx, ny);
    B.x = yee_interp<R>(f.yee[3], st[2], nx, ny);
    B.y = yee_interp<R>(f.yee[4], st[1], nx, ny);
    B.z = yee_interp<R>(f.yee[5], st[3], nx, ny);
}

// Fields at (x, y, z, t); R = double (FP64 path) or float (mixed path, with
// phases reduced in FP64 before the FP32 trigonometry).
template <int FK, typename R>
__device__ __forceinline__ void eval_field(const FieldDev &f, double x, double y, double z,
                                           double t, Vec3<R> &E, Vec3<R> &B)
{
    E = {R(0), R(0), R(0)};
    B = {R(0), R(0), R(0)};
    if constexpr (FK == QP_FIELD_PLANE) {
        R v;
        if constexpr (sizeof(R) == 8) {
            v = f.a0 * cos(t - x);
        } else {
            const double ph = t - x;
            const double red = ph - 6.283185307179586 * rint(ph * 0.15915494309189535);
            v = (float)f.a0 * cosf((float)red);
        }
        E.y = v;
        B.z = v;
    } else if constexpr (FK == QP_FIELD_GAUSSIAN) {
        const double xi = x - f.x_focus;
        const double eta = (t - f.t_focus) - xi;
        const double zr = 0.5 * f.w0 * f.w0;
        const double q = xi / zr;
        const double wr2 = 1.0 + q * q;
        const double r2 = y * y + z * z;
        R v;
        if constexpr (sizeof(R) == 8) {
            const double env = -r2 / (f.w0 * f.w0 * wr2) -
                               2.0 * 0.6931471805599453 * eta * eta / (f.tau_fwhm * f.tau_fwhm);
            const double amp = f.a0 / sqrt(wr2) * exp(env);
            const double phase = -eta + r2 * xi / (2.0 * (xi * xi + zr * zr)) - atan(q);
            v = amp * cos(phase);
        } else {
            const float env = (float)(-r2 / (f.w0 * f.w0 * wr2)) -
                              1.3862943611198906f * (float)(eta * eta / (f.tau_fwhm * f.tau_fwhm));
            const float amp = (float)f.a0 * rsqrtf((float)wr2) * __expf(env);
            double phase = -eta + r2 * xi / (2.0 * (xi * xi + zr * zr));
            phase -= 6.283185307179586 * rint(phase * 0.15915494309189535);
            v = amp * cosf((float)phase - atanf((float)q));
        }
        E.y = v;
        B.z = v;
    } else if constexpr (FK == QP_FIELD_UNIFORM_B) {
        B.z = (R)f.b0;
    } else if constexpr (FK == QP_FIELD_YEE2D) {
        // linear interpolation of the six staggered components
        //   Ex(i+1/2,j) Ey(i,j+1/2) Ez(i,j) Bx(i,j+1/2) By(i+1/2,j) Bz(i+1/2,j+1/2);
        // nodes outside the grid contribute zero field.  The cell index and
        // weight of each axis are found once for the node and the half-node
        // grids (FP64 path: in FP64; mixed path: the cell coordinate is formed
        // with one FP64 FMA, the rest in FP32).
        int ix[2], iy[2];
        R wx[2], wy[2];
        const double gx = (x - f.x0) / f.dx, gy = (y - f.y0) / f.dy;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const double ax = h ? gx - 0.5 : gx, ay = h ? gy - 0.5 : gy;
            const double fx = floor(ax), fy = floor(ay);
            wx[h] = (R)(ax - fx);
            wy[h] = (R)(ay - fy);
            // clamp before the conversion (NaN and huge values included)
            ix[h] = (int)fmax(-2.0, fmin((double)f.nx + 1.0, fx));
            iy[h] = (int)fmax(-2.0, fmin((double)f.ny + 1.0, fy));
        }
        yee_gather<R>(f, ix, iy, wx, wy, E, B);
    }
}

// ------------------------------------------------------------------ chi (Eq. 1)

// chi_e = sqrt(|gamma E + u x B|^2 - (u.E)^2) / a_S, in FP64
__device__ __forceinline__ double chi_e64(double Ex, double Ey, double Ez, double Bx, double By,
                                          double Bz, double ux, double uy, double uz, double g,
                                          double a_S)
{
    const double ax = g * Ex + (uy * Bz - uz * By);
    const double ay = g * Ey + (uz * Bx - ux * Bz);
    const double az = g * Ez + (ux * By - uy * Bx);
    const double ue = ux * Ex + uy * Ey + uz * Ez;
    const double s = ax * ax + ay * ay + az * az - ue * ue;
    return s > 0.0 ? sqrt(s) / a_S : 0.0;
}

// ------------------------------------------------------------------ rate tables

// Index and exact interpolation weight of chi on a grid of 2^k nodes per
// octave starting at 2^-14, from the bits of chi (no logarithm): the node is
// 2^e (1 + m/2^k) with m the top k mantissa bits; the weight is the rest of
// the mantissa.  Requires 2^-14 <= chi < 2^10.
template <int KBITS>
__device__ __forceinline__ int grid_index64(double chi, double &f)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(chi);
    const int e = (int)((b >> 52) & 0x7FF) - 1023;
    const int m = (int)((b >> (52 - KBITS)) & ((1u << KBITS) - 1));
    f = (double)(b & ((1ull << (52 - KBITS)) - 1)) * (1.0 / (double)(1ull << (52 - KBITS)));
    return ((e - kChiExp0) << KBITS) + m;
}

template <int KBITS>
__device__ __forceinline__ int grid_index32(float chi, float &f)
{
    const unsigned b = __float_as_uint(chi);
    const int e = (int)((b >> 23) & 0xFF) - 127;
    const int m = (int)((b >> (23 - KBITS)) & ((1u << KBITS) - 1));
    f = (float)(b & ((1u << (23 - KBITS)) - 1)) * (1.0f / (float)(1u << (23 - KBITS)));
    return ((e - kChiExp0) << KBITS) + m;
}

constexpr double kChiLo = 0x1.0p-14, kChiHi = 0x1.0p10;
constexpr double kPi = 3.14159265358979323846;

// which: 0 H, 1 G (table holds G/chi), 2 T (table holds T exp(8/(3 chi)))
// V points at the (shared-memory) table of that quantity.
template <int WHICH>
__device__ __forceinline__ double rate64(const double *V, double chi, bool &clamped)
{
    if (WHICH == 2 && !(chi >= kPairChiMin)) return 0.0;
    if (!(chi >= kChiLo)) {
        if (WHICH == 0) return __dmul_rn(2.5 * kPi, chi);
        return __dmul_rn(__dmul_rn(2.0 * kPi, chi), chi) / 1.7320508075688772;
    }
    double v, c = chi;
    if (chi >= kChiHi) {
        clamped = true;
        v = V[kNRate - 1];
        c = kChiHi;
    } else {
        double f;
        const int j = grid_index64<5>(chi, f);
        const double a = V[j], d = __dsub_rn(V[j + 1], a);
        v = __dadd_rn(a, __dmul_rn(f, d));
    }
    if (WHICH == 1) return __dmul_rn(v, c);
    if (WHICH == 2) return __dmul_rn(v, exp(-8.0 / (3.0 * c)));
    return v;
}

template <int WHICH>
__device__ __forceinline__ float rate32(const float *V, float chi, bool &clamped)
{
    if (WHICH == 2 && !(chi >= (float)kPairChiMin)) return 0.0f;
    if (!(chi >= (float)kChiLo)) {
        if (WHICH == 0) return (float)(2.5 * kPi) * chi;
        return (float)(2.0 * kPi / 1.7320508075688772) * chi * chi;
    }
    float v, c = chi;
    if (chi >= (float)kChiHi) {
        clamped = true;
        v = V[kNRate - 1];
        c = (float)kChiHi;
    } else {
        float f;
        const int j = grid_index32<5>(chi, f);
        const float a = V[j];
        v = fmaf(f, V[j + 1] - a, a);
    }
    if (WHICH == 1) return v * c;
    if (WHICH == 2) return v * __expf(-8.0f / (3.0f * c));
    return v;
}

// ------------------------------------------------------------------ inverse CDF (Eq. 7)

// Guide tables: the search of a CDF row for xi starts from a node read from
// a small table instead of bisecting the row (8 dependent loads on the rare
// emission branch, which every later tile of the launch waits for through
// the look-back).  xi <= 1/2 is located in the row by xi itself, xi > 1/2 by
// eta = 1 - xi; the bucket of a value in (0, 1/2] is four per octave, from
// its exponent and two leading mantissa bits.  Lower-half entry: the last
// node with C < the bucket's lower edge; upper-half entry: the last node
// with 1 - C > the bucket's upper edge.  A forward scan then finds the same
// interval as a bisection would (the last node below xi).
constexpr int kGuideBuckets = 224;

__device__ __forceinline__ int guide_bucket(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7FF) - 1023;
    const int m = ((-1 - e) << 2) | (int)((b >> 50) & 3u);
    return min(max(m, 0), kGuideBuckets - 1);
}

__device__ __forceinline__ int guide_bucket(float x)
{
    const unsigned b = __float_as_uint(x);
    const int e = (int)((b >> 23) & 0xFF) - 127;
    const int m = ((-1 - e) << 2) | (int)((b >> 21) & 3u);
    return min(max(m, 0), kGuideBuckets - 1);
}

// Invert one CDF row C (kNNode logit nodes s_i = smin + span i / 255) at xi.
// Emission rows follow u^(1/3) below the first node; pair rows clamp.
template <typename R>
__device__ __forceinline__ R row_invert(const R *__restrict__ C,
                                        const unsigned char *__restrict__ guide, R xi,
                                        double smin, double span, bool power_tail)
{
    const R c0 = __ldg(C);
    if (xi <= c0) {
        const R x0 = R(1) / (R(1) + (R)exp(-smin));
        if (power_tail && c0 > R(0)) {
            const R r = xi / c0;
            return x0 * r * r * r;
        }
        return x0;
    }
    const R clast = __ldg(C + kNNode - 1);
    if (xi >= clast) return R(1) / (R(1) + (R)exp(-(smin + span)));
    // the last node below xi: guide entry, then a forward scan
    int lo = xi <= R(0.5) ? (int)__ldg(guide + guide_bucket(xi))
                          : (int)__ldg(guide + kNCdf * kGuideBuckets + guide_bucket(R(1) - xi));
#pragma unroll 1
    while (lo < kNNode - 2 && __ldg(C + lo + 1) < xi) ++lo;
    const R clo = __ldg(C + lo), chi_ = __ldg(C + lo + 1);
    const double s_lo = smin + span * lo / (kNNode - 1);
    const double s_hi = smin + span * (lo + 1) / (kNNode - 1);
    if constexpr (sizeof(R) == 8) {
        const double t = (xi - clo) / (chi_ - clo);
        const double sv = s_lo + t * (s_hi - s_lo);
        return 1.0 / (1.0 + exp(-sv));
    } else {
        const float t = (xi - clo) / (chi_ - clo);
        const float sv = (float)s_lo + t * (float)(s_hi - s_lo);
        return 1.0f / (1.0f + __expf(-sv));
    }
}

// Photon fraction u = chi_gamma / chi_e for chi_e (rows j, j+1 interpolated
// linearly in chi; below the grid the classical scaling u ~ chi).
template <typename R>
__device__ __forceinline__ R sample_cdf(const R *__restrict__ rows,
                                        const unsigned char *__restrict__ guide, R chi, R xi,
                                        double smin, double span, bool emission, bool &clamped)
{
    if (!(chi >= (R)kChiLo)) {
        const R r0 = row_invert<R>(rows, guide, xi, smin, span, emission);
        return emission ? (chi / (R)kChiLo) * r0 : r0;
    }
    if (chi >= (R)kChiHi) {
        clamped = true;
        return row_invert<R>(rows + (kNCdf - 1) * kNNode, guide + (kNCdf - 1) * kGuideBuckets,
                             xi, smin, span, emission);
    }
    R f;
    int j;
    if constexpr (sizeof(R) == 8)
        j = grid_index64<2>(chi, f);
    else
        j = grid_index32<2>(chi, f);
    const R ra = row_invert<R>(rows + j * kNNode, guide + j * kGuideBuckets, xi, smin, span,
                               emission);
    const R rb = row_invert<R>(rows + (j + 1) * kNNode, guide + (j + 1) * kGuideBuckets, xi,
                               smin, span, emission);
    return ra + f * (rb - ra);
}

// ------------------------------------------------------------------ FP32 inverse CDF with complement

// Mixed path: the same inversion in FP32, returning x and 1 - x, both
// accurate (1 - x from the logit, not by subtraction), so that the recoil
// (|p| - u gamma) and the pair split (1 - v) keep their precision when the
// photon or the electron takes nearly everything.
}  // namespace qp
