// Kernels of libqedpic (sm_103a).
//
// One QED particle step is ONE launch of the persistent kernel k_step.  Its
// blocks take 256-particle tiles from one atomic ticket over a single tile
// space: first the electron tiles, then the positron tiles (together: the
// lepton chain), then the photon tiles (the photon chain).
//   lepton tile : gather, Boris, chi_e, Sokolov or optical depth + emission,
//                 position update; new photons appended in slot order;
//   photon tile : chi_gamma, pair optical depth, decay into an e-/e+ pair
//                 appended in slot order, ballistic motion.
// Lepton tiles only append photons at slots >= the photon count of the step
// start and photon tiles only append leptons at slots >= the lepton counts,
// so the two chains never touch the same slots and both run in the same
// launch.  The live counts are read-only during the launch; the last block to
// finish applies the new counts, resets the ticket and advances the launch
// epoch (device memory), which tags the look-back words: no memset and no
// host-side state between steps, so a step can be replayed in a CUDA graph.
#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "qp_device.cuh"
#include "qp_kernels.h"
#include "qp_mixed.cuh"

namespace qp {

namespace {

// Look-back word: epoch (24 bits) | flag (2 bits) | value (38 bits).
constexpr int kEpochShift = 40, kFlagShift = 38;
constexpr unsigned long long kValMask = (1ull << kFlagShift) - 1;
constexpr unsigned kEpochMask = 0xFFFFFFu;
constexpr unsigned kFlagAgg = 1u, kFlagPre = 2u;

__device__ __forceinline__ unsigned long long make_word(unsigned epoch, unsigned flag,
                                                        long long value)
{
    return ((unsigned long long)(epoch & kEpochMask) << kEpochShift) |
           ((unsigned long long)flag << kFlagShift) | ((unsigned long long)value & kValMask);
}

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long *p)
{
    return *((const volatile unsigned long long *)p);
}

// Exclusive prefix of this tile in its chain, computed by one full warp
// (decoupled look-back with a 32-tile window): lane l inspects tile
// base - l; a word counts only if it carries this launch's epoch.  The
// window is consumed up to the nearest tile that published its inclusive
// prefix, summing the aggregates in between.  Waits are bounded by
// spin_limit; on time-out the status is raised and the prefix is what was
// summed so far (the output is then wrong, the status says so, and the
// kernel still terminates).  Returns the prefix in every lane.
__device__ long long chain_prefix(unsigned long long *words, unsigned tile, long long aggregate,
                                  unsigned epoch, unsigned spin_limit, int *status)
{
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) atomicExch(words, make_word(epoch, kFlagPre, aggregate));
        return 0;
    }
    if (lane == 0) atomicExch(words + tile, make_word(epoch, kFlagAgg, aggregate));
    long long excl = 0;
    long long base = (long long)tile - 1;
    unsigned spins = 0;
    for (;;) {
        const long long idx = base - lane;
        // before tile 0 the chain is complete: read as "prefix 0"
        const unsigned long long w =
            idx >= 0 ? ld_volatile(words + idx) : make_word(epoch, kFlagPre, 0);
        const bool current = (unsigned)(w >> kEpochShift) == (epoch & kEpochMask);
        const unsigned flag = current ? (unsigned)(w >> kFlagShift) & 3u : 0u;
        const unsigned pre = __ballot_sync(0xFFFFFFFFu, flag == kFlagPre);
        const unsigned empty = __ballot_sync(0xFFFFFFFFu, flag == 0u);
        const int first = pre ? __ffs(pre) - 1 : 32;  // nearest inclusive prefix
        const unsigned need = first == 32 ? 0xFFFFFFFFu : (2u << first) - 1u;
        if (empty & need) {
            if (++spins > spin_limit) {
                if (lane == 0) raise_status(status, QP_ERR_TIMEOUT);
                break;
            }
            __nanosleep(32);
            continue;
        }
        long long v = lane <= first ? (long long)(w & kValMask) : 0;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, d);
        excl += v;
        if (first < 32) break;
        base -= 32;
    }
    if (lane == 0) atomicExch(words + tile, make_word(epoch, kFlagPre, excl + aggregate));
    return excl;
}

// Block-wide exclusive scan of one small count per thread; returns the
// thread's exclusive offset and writes the block total to *total.
__device__ __forceinline__ int block_scan(int v, int *s_warp, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = lane < kWarps ? s_warp[lane] : 0;
#pragma unroll
        for (int d = 1; d < kWarps; d <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, w, d);
            if (lane >= d) w += y;
        }
        if (lane < kWarps) s_warp[lane] = w;
    }
    __syncthreads();
    *total = s_warp[kWarps - 1];
    return inc - v + (warp ? s_warp[warp - 1] : 0);
}

// Counters kept in shared memory per block and species, flushed with one
// atomic per counter when the block leaves.
struct BlockStats {
    unsigned long long c[3][9];
    double e[3][2];
};
enum { cEmit, cPhoton, cPhotonDrop, cSub, cPair, cPairDrop, cSat, cClamp, cCont };

__device__ __forceinline__ void warp_count(unsigned long long *ctr, bool pred)
{
    const unsigned m = __ballot_sync(0xFFFFFFFFu, pred);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(ctr, (unsigned long long)__popc(m));
}

__device__ __forceinline__ void clear_stats(BlockStats &bs)
{
    const int t = threadIdx.x;
    if (t < 27) (&bs.c[0][0])[t] = 0ull;
    if (t < 6) (&bs.e[0][0])[t] = 0.0;
}

__device__ void flush_stats(const BlockStats &bs, const StepArgs &a)
{
    __syncthreads();
    const int t = threadIdx.x;
    if (t < 27) {
        const int s = t / 9, k = t % 9;
        if (bs.c[s][k] && a.sp[s].present)
            atomicAdd(&a.stats[a.sp[s].slot_stats].n_emit + k, bs.c[s][k]);
    } else if (t >= 32 && t < 38) {
        const int s = (t - 32) / 2, k = (t - 32) % 2;
        if (bs.e[s][k] != 0.0 && a.sp[s].present)
            atomicAdd(&a.stats[a.sp[s].slot_stats].e_subthreshold + k, bs.e[s][k]);
    }
}

// Shared-memory layout of k_step (dynamic part).
template <typename R>
struct Smem {
    R H[kNRatePad];                          // rate tables (TMA-staged)
    R G[kNRatePad];
    R T[kNRatePad];
    double gg[QP_MAX_EMISSIONS][kTile];      // stashed photon energies
    double tg[QP_MAX_EMISSIONS][kTile];      // and their optical depths
};

__device__ __forceinline__ void wait_tables(unsigned long long *bar, const StepArgs &a)
{
    if (!mbar_wait_bounded(bar, 0, a.spin_limit)) {
        raise_status(a.status, QP_ERR_TIMEOUT);
        (void)mbar_wait_bounded(bar, 0, a.spin_limit);  // never leave with a copy in flight
    }
}

// -------------------------------------------------------------------- lepton tile

template <int PREC, int FK, typename R>
__device__ void lepton_tile(const StepArgs &a, Smem<R> &sm, unsigned long long *bar,
                            bool &loaded, unsigned chain_tile, int sp, int64_t first, int64_t n,
                            int64_t ph_base, unsigned epoch, int *s_warp, long long *s_excl,
                            BlockStats &bs)
{
    const int tid = threadIdx.x;
    if (!loaded && tid == 0) {
        // stage the rate tables with one TMA bulk copy each; the copy
        // overlaps the particle loads, gather and push below
        const unsigned bytes = kNRatePad * sizeof(R);
        mbar_init(bar, 1);
        mbar_expect_tx(bar, 2 * bytes);
        if constexpr (PREC == kFP64) {
            bulk_g2s(sm.H, a.tab.H, bytes, bar);
            bulk_g2s(sm.G, a.tab.Gs, bytes, bar);
        } else {
            bulk_g2s(sm.H, a.tab.Hf, bytes, bar);
            bulk_g2s(sm.G, a.tab.Gsf, bytes, bar);
        }
    }
    if (!loaded) __syncthreads();
    const SpeciesDev &S = a.sp[sp];
    const SpeciesDev &Ph = a.sp[2];
    const bool photons = Ph.present != 0;
    const int64_t i = first + tid;
    const bool active = i < n;

    int nph = 0;
    double x0 = 0, y0 = 0, z0 = 0, kx = 0, ky = 0, kz = 0, wgt = 0;
    bool cont = false, sat = false, clamped = false;
    int n_emit = 0, n_sub = 0;
    double e_sub = 0.0;

    if constexpr (PREC == kFP64) {
    if (active) {
        const double q = sp == 0 ? -1.0 : 1.0;
        const double dt = a.dt;
        x0 = S.x[i];
        y0 = S.y[i];
        z0 = S.z ? S.z[i] : 0.0;
        double ux = S.ux[i], uy = S.uy[i], uz = S.uz[i];
        double tau = S.tau[i];
        Vec3<R> E, B;
        eval_field<FK, R>(a.f, x0, y0, z0, a.t, E, B);

        // ---- Boris push of the Lorentz force (f_l of Eq. 4)
        if constexpr (PREC == kFP64) {
            const double h = 0.5 * q * dt;
            const double mx = ux + h * E.x, my = uy + h * E.y, mz = uz + h * E.z;
            const double g = sqrt(1.0 + mx * mx + my * my + mz * mz);
            const double tx = h * B.x / g, ty = h * B.y / g, tz = h * B.z / g;
            const double t2 = tx * tx + ty * ty + tz * tz;
            const double sx = 2.0 * tx / (1.0 + t2), sy = 2.0 * ty / (1.0 + t2),
                         sz = 2.0 * tz / (1.0 + t2);
            const double px = mx + (my * tz - mz * ty), py = my + (mz * tx - mx * tz),
                         pz = mz + (mx * ty - my * tx);
            ux = mx + (py * sz - pz * sy) + h * E.x;
            uy = my + (pz * sx - px * sz) + h * E.y;
            uz = mz + (px * sy - py * sx) + h * E.z;
        } else {
            // FP32 rotation, FP64 accumulation of the momentum
            const float h = (float)(0.5 * q * dt);
            const float hx = h * E.x, hy = h * E.y, hz = h * E.z;
            const double mx = ux + hx, my = uy + hy, mz = uz + hz;
            const float fx = (float)mx, fy = (float)my, fz = (float)mz;
            const float ig = rsqrtf(1.0f + fx * fx + fy * fy + fz * fz);
            const float tx = h * B.x * ig, ty = h * B.y * ig, tz = h * B.z * ig;
            const float k2 = 2.0f / (1.0f + tx * tx + ty * ty + tz * tz);
            const float sx = k2 * tx, sy = k2 * ty, sz = k2 * tz;
            const float px = fx + (fy * tz - fz * ty), py = fy + (fz * tx - fx * tz),
                        pz = fz + (fx * ty - fy * tx);
            ux = mx + (double)((py * sz - pz * sy) + hx);
            uy = my + (double)((pz * sx - px * sz) + hy);
            uz = mz + (double)((px * sy - py * sx) + hz);
        }
        double gam = sqrt(1.0 + ux * ux + uy * uy + uz * uz);
        const double Ex = E.x, Ey = E.y, Ez = E.z, Bx = B.x, By = B.y, Bz = B.z;
        if (!loaded) wait_tables(bar, a);  // tables are needed from here on
        double chi = chi_e64(Ex, Ey, Ez, Bx, By, Bz, ux, uy, uz, gam, a.a_S);
        if (S.chi) S.chi[i] = chi;
        double dvx = 0.0, dvy = 0.0, dvz = 0.0;

        if (chi < a.chi_th) {
            // ---- Sokolov continuous regime (Eq. 4, P_rad of Eq. 5)
            cont = true;
            if constexpr (PREC == kFP64) {
                const double vx = ux / gam, vy = uy / gam, vz = uz / gam;
                const double fx = q * (Ex + (vy * Bz - vz * By));
                const double fy = q * (Ey + (vz * Bx - vx * Bz));
                const double fz = q * (Ez + (vx * By - vy * Bx));
                const double vf = vx * fx + vy * fy + vz * fz;
                const double den = 1.0 + a.tau0w * vf;
                dvx = a.tau0w * (fx - vx * vf) / den;
                dvy = a.tau0w * (fy - vy * vf) / den;
                dvz = a.tau0w * (fz - vz * vf) / den;
                const double prad = a.C_rate * rate64<1>(sm.G, chi, clamped);
                ux = ux + dt * (q * (dvy * Bz - dvz * By) - prad * vx);
                uy = uy + dt * (q * (dvz * Bx - dvx * Bz) - prad * vy);
                uz = uz + dt * (q * (dvx * By - dvy * Bx) - prad * vz);
            } else {
                const float ig = (float)(1.0 / gam), qf = (float)q;
                const float vx = (float)ux * ig, vy = (float)uy * ig, vz = (float)uz * ig;
                const float fx = qf * (E.x + (vy * B.z - vz * B.y));
                const float fy = qf * (E.y + (vz * B.x - vx * B.z));
                const float fz = qf * (E.z + (vx * B.y - vy * B.x));
                const float vf = vx * fx + vy * fy + vz * fz;
                const double den = 1.0 + a.tau0w * (double)vf;  // FP64 denominator
                const float c = (float)(a.tau0w / den);
                const float dx_ = c * (fx - vx * vf), dy_ = c * (fy - vy * vf),
                            dz_ = c * (fz - vz * vf);
                dvx = dx_;
                dvy = dy_;
                dvz = dz_;
                const float prad = (float)a.C_rate * rate32<1>(sm.G, (float)chi, clamped);
                const float dtf = (float)dt;
                ux += (double)(dtf * (qf * (dy_ * B.z - dz_ * B.y) - prad * vx));
                uy += (double)(dtf * (qf * (dz_ * B.x - dx_ * B.z) - prad * vy));
                uz += (double)(dtf * (qf * (dx_ * B.y - dy_ * B.x) - prad * vz));
            }
            gam = sqrt(1.0 + ux * ux + uy * uy + uz * uz);
        } else {
            // ---- optical depth (Eq. 6) with the residual-time sub-loop
            double r = 1.0;
            for (int k = 0;; ++k) {
                double wdt, dtau;
                if constexpr (PREC == kFP64) {
                    const double H = rate64<0>(sm.H, chi, clamped);
                    wdt = a.C_rate * H / gam * dt;
                    dtau = wdt * r;
                } else {
                    const float H = rate32<0>(sm.H, (float)chi, clamped);
                    const float wf = (float)a.C_rate * H / (float)gam * (float)dt;
                    wdt = wf;
                    dtau = (double)(wf * (float)r);
                }
                if (!(dtau > 0.0) || tau > dtau) {
                    tau = tau - dtau;
                    break;
                }
                if (k == a.max_emit) {
                    tau = tau - dtau;
                    sat = true;
                    break;
                }
                r = r - tau / wdt;
                // ---- emission: Eq. 7 sampling, Eq. 8 recoil
                const uint4 rr = draw(a.seed, sp, kRngEmit, i, a.step, k);
                const double xi_p = u53(rr.x, rr.y), xi = u53(rr.z, rr.w);
                double ufrac;
                ufrac = sample_cdf<double>(a.tab.Cg, chi, xi_p, kSgMin, kSgSpan, true, clamped);
                const double pmag = sqrt(ux * ux + uy * uy + uz * uz);
                double gg = ufrac * gam;
                if (gg > pmag) gg = pmag;
                if (n_emit == 0 && pmag > 0.0) {
                    kx = ux / pmag;
                    ky = uy / pmag;
                    kz = uz / pmag;
                }
                ++n_emit;
                if (gg > a.gmin) {
                    const uint4 rp = draw(a.seed, sp, kRngPhotonTau, i, a.step, k);
                    sm.gg[nph][tid] = gg;
                    sm.tg[nph][tid] = -log(u53(rp.x, rp.y));
                    ++nph;
                } else {
                    ++n_sub;
                    e_sub += gg;
                }
                if (pmag > 0.0) {
                    const double scale = (pmag - gg) / pmag;
                    ux *= scale;
                    uy *= scale;
                    uz *= scale;
                }
                tau = -log(xi);
                gam = sqrt(1.0 + ux * ux + uy * uy + uz * uz);
                chi = chi_e64(Ex, Ey, Ez, Bx, By, Bz, ux, uy, uz, gam, a.a_S);
            }
        }

        // ---- position (Eq. 4: dx/dt = v + delta v)
        if constexpr (PREC == kFP64) {
            S.x[i] = x0 + dt * (ux / gam + dvx);
            S.y[i] = y0 + dt * (uy / gam + dvy);
            if (S.z) S.z[i] = z0 + dt * (uz / gam + dvz);
        } else {
            const float ig = (float)(1.0 / gam), dtf = (float)dt;
            S.x[i] = x0 + (double)(dtf * ((float)ux * ig + (float)dvx));
            S.y[i] = y0 + (double)(dtf * ((float)uy * ig + (float)dvy));
            if (S.z) S.z[i] = z0 + (double)(dtf * ((float)uz * ig + (float)dvz));
        }
        S.ux[i] = ux;
        S.uy[i] = uy;
        S.uz[i] = uz;
        S.tau[i] = tau;
        if (nph || n_sub) wgt = S.w[i];
    }
    } else {
    if (active) {
        // ---- mixed precision: FP32 physics; the FP64 state is read once,
        // increments are formed in FP32 and added back by integer
        // instructions; chi_e falls back to double-float where FP32 cancels
        const MixedConsts &m = a.mc;
        const double xd = S.x[i], yd = S.y[i], zd = S.z ? S.z[i] : 0.0;
        x0 = xd;
        y0 = yd;
        z0 = zd;
        const double uxd = S.ux[i], uyd = S.uy[i], uzd = S.uz[i];
        const double taud = S.tau[i];
        Vec3<float> E, B;
        eval_field_mixed<FK>(a.f, m, split_d(xd), split_d(yd), split_d(zd), E, B);

        // Boris on the leading FP32 parts; the increment is kept in FP32
        const float u0x = hi_d(uxd), u0y = hi_d(uyd), u0z = hi_d(uzd);
        const float h = m.h[sp];
        const float hx = h * E.x, hy = h * E.y, hz = h * E.z;
        const float mx = u0x + hx, my = u0y + hy, mz = u0z + hz;
        const float ig = rsqrtf(1.0f + mx * mx + my * my + mz * mz);
        const float tx = h * B.x * ig, ty = h * B.y * ig, tz = h * B.z * ig;
        const float k2 = 2.0f / (1.0f + tx * tx + ty * ty + tz * tz);
        const float sx = k2 * tx, sy = k2 * ty, sz = k2 * tz;
        const float px = mx + (my * tz - mz * ty), py = my + (mz * tx - mx * tz),
                    pz = mz + (mx * ty - my * tx);
        float dux = (py * sz - pz * sy) + 2.0f * hx, duy = (pz * sx - px * sz) + 2.0f * hy,
              duz = (px * sy - py * sx) + 2.0f * hz;
        float ux = u0x + dux, uy = u0y + duy, uz = u0z + duz;
        float gam = sqrtf(1.0f + ux * ux + uy * uy + uz * uz);
        if (!loaded) wait_tables(bar, a);  // tables are needed from here on
        float chi = chi_mixed_auto(uxd, uyd, uzd, dux, duy, duz, ux, uy, uz, gam, E, B, m.inv_aS,
                                   m.inv_aS_lo);
        if (S.chi) S.chi[i] = f_to_d(chi);
        float dvx = 0.0f, dvy = 0.0f, dvz = 0.0f;
        float dtau_once = 0.0f;
        bool events = false;
        df2 TAU = {0.0f, 0.0f};

        if (chi < m.chi_th) {
            // ---- Sokolov (Eq. 4, 5); denominator 1 + tau0 v.f_l in double-float
            cont = true;
            const float q = sp == 0 ? -1.0f : 1.0f;
            const float gi = 1.0f / gam;
            const float vx = ux * gi, vy = uy * gi, vz = uz * gi;
            const float fx = q * (E.x + (vy * B.z - vz * B.y));
            const float fy = q * (E.y + (vz * B.x - vx * B.z));
            const float fz = q * (E.z + (vx * B.y - vy * B.x));
            const float vf = vx * fx + vy * fy + vz * fz;
            const df2 den = two_sum(1.0f, m.tau0w * vf);
            const float c = m.tau0w / den.hi * (1.0f - den.lo / den.hi);
            dvx = c * (fx - vx * vf);
            dvy = c * (fy - vy * vf);
            dvz = c * (fz - vz * vf);
            const float prad = m.C_rate * rate32<1>(sm.G, chi, clamped);
            const float sx_ = m.dt * (q * (dvy * B.z - dvz * B.y) - prad * vx);
            const float sy_ = m.dt * (q * (dvz * B.x - dvx * B.z) - prad * vy);
            const float sz_ = m.dt * (q * (dvx * B.y - dvy * B.x) - prad * vz);
            dux += sx_;
            duy += sy_;
            duz += sz_;
            ux += sx_;
            uy += sy_;
            uz += sz_;
            gam = sqrtf(1.0f + ux * ux + uy * uy + uz * uz);
        } else {
            // ---- optical depth (Eq. 6) with the residual-time sub-loop
            TAU = split_d(taud);
            float r = 1.0f;
            for (int k = 0;; ++k) {
                const float H = rate32<0>(sm.H, chi, clamped);
                const float wdt = m.C_rate * H / gam * m.dt;
                const float dtau = wdt * r;
                // tau > dtau decided on the double-float optical depth
                if (!(dtau > 0.0f) || TAU.hi > dtau || (TAU.hi == dtau && TAU.lo > 0.0f)) {
                    TAU = df_add_f(TAU, -dtau);
                    dtau_once = dtau;
                    break;
                }
                if (k == a.max_emit) {
                    TAU = df_add_f(TAU, -dtau);
                    dtau_once = dtau;
                    sat = true;
                    break;
                }
                events = true;
                r = r - df_to_f(TAU) / wdt;
                // ---- emission: Eq. 7 sampling, Eq. 8 recoil
                const uint4 rr = draw(a.seed, sp, kRngEmit, i, a.step, k);
                const float xi = u53f(rr.z, rr.w);
                const FracPair uf = sample_cdf_f(
                    a.tab.Cg2, a.tab.Qg2, a.tab.Eg, chi, u53_pair(rr.x, rr.y),
                    u53_pair_complement(rr.x, rr.y), (float)(kSgSpan / (kNNode - 1)), true,
                    clamped);
                const float pmag = sqrtf(ux * ux + uy * uy + uz * uz);
                float gg = uf.x * gam;
                // what the electron keeps, |p| - u gamma = (1-u) gamma - 1/(gamma + |p|),
                // formed without cancellation
                float keep = uf.omx * gam - 1.0f / (gam + pmag);
                if (gg > pmag || keep < 0.0f) {
                    gg = pmag;
                    keep = 0.0f;
                }
                if (n_emit == 0 && pmag > 0.0f) {
                    const float ip = 1.0f / pmag;
                    kx = f_to_d(ux * ip);
                    ky = f_to_d(uy * ip);
                    kz = f_to_d(uz * ip);
                }
                ++n_emit;
                if (gg > m.gmin) {
                    const uint4 rp = draw(a.seed, sp, kRngPhotonTau, i, a.step, k);
                    sm.gg[nph][tid] = f_to_d(gg);
                    sm.tg[nph][tid] = f_to_d(-logf(u53f(rp.x, rp.y)));
                    ++nph;
                } else {
                    ++n_sub;
                    e_sub += f_to_d(gg);
                }
                if (pmag > 0.0f) {
                    const float s1 = keep / pmag;
                    const float s1m = s1 - 1.0f;  // exact (Sterbenz) for s1 in [1/2, 1]
                    dux = fmaf(ux, s1m, dux);
                    duy = fmaf(uy, s1m, duy);
                    duz = fmaf(uz, s1m, duz);
                    ux *= s1;
                    uy *= s1;
                    uz *= s1;
                }
                TAU = {-logf(xi), 0.0f};
                gam = sqrtf(1.0f + ux * ux + uy * uy + uz * uz);
                chi = chi_mixed_auto(uxd, uyd, uzd, dux, duy, duz, ux, uy, uz, gam, E, B,
                                     m.inv_aS, m.inv_aS_lo);
            }
        }

        // ---- position and write-back: FP64 accumulation of FP32 increments
        const float gi = 1.0f / gam;
        S.x[i] = add_fd(xd, m.dt * (ux * gi + dvx));
        S.y[i] = add_fd(yd, m.dt * (uy * gi + dvy));
        if (S.z) S.z[i] = add_fd(zd, m.dt * (uz * gi + dvz));
        S.ux[i] = add_fd(uxd, dux);
        S.uy[i] = add_fd(uyd, duy);
        S.uz[i] = add_fd(uzd, duz);
        if (events)
            S.tau[i] = merge_df(TAU);
        else if (dtau_once != 0.0f)
            S.tau[i] = add_fd(taud, -dtau_once);
        if (nph || n_sub) wgt = S.w[i];
    }
    }
    if (active && n_emit && S.nemit) S.nemit[i] += n_emit;
    if (!loaded) {
        // threads without a particle also wait, so the block never leaves
        // (or reuses the tables) with the copy in flight
        if (!active) wait_tables(bar, a);
        loaded = true;
    }

    // ---- counters (warp-aggregated into shared memory)
    warp_count(&bs.c[sp][cCont], cont);
    warp_count(&bs.c[sp][cSat], sat);
    warp_count(&bs.c[sp][cClamp], clamped);
    if (__any_sync(0xFFFFFFFFu, n_emit > 0)) {
        if (n_emit) atomicAdd(&bs.c[sp][cEmit], (unsigned long long)n_emit);
        if (n_sub) {
            atomicAdd(&bs.c[sp][cSub], (unsigned long long)n_sub);
            atomicAdd(&bs.e[sp][0], wgt * e_sub);
        }
    }

    // ---- ordered append of the new photons
    int tile_total;
    const int local = block_scan(nph, s_warp, &tile_total);
    if (tid < 32) {
        const long long e =
            chain_prefix(a.lep_words, chain_tile, tile_total, epoch, a.spin_limit, a.status);
        if (tid == 0) *s_excl = e;
    }
    __syncthreads();
    const long long excl = *s_excl;
    if (nph) {
        const int64_t base = ph_base + excl + local;
        int stored = 0, dropped = 0;
        double e_drop = 0.0;
        for (int j = 0; j < nph; ++j) {
            const int64_t slot = base + j;
            const double gg = sm.gg[j][tid];
            if (photons && slot < Ph.cap) {
                Ph.x[slot] = x0;
                Ph.y[slot] = y0;
                if (Ph.z) Ph.z[slot] = z0;
                Ph.ux[slot] = gg * kx;
                Ph.uy[slot] = gg * ky;
                Ph.uz[slot] = gg * kz;
                Ph.tau[slot] = sm.tg[j][tid];
                Ph.w[slot] = wgt;
                if (Ph.chi) Ph.chi[slot] = 0.0;
                if (Ph.nemit) Ph.nemit[slot] = 0;
                ++stored;
            } else {
                ++dropped;
                e_drop += wgt * gg;
            }
        }
        if (stored) atomicAdd(&bs.c[sp][cPhoton], (unsigned long long)stored);
        if (dropped) {
            atomicAdd(&bs.c[sp][cPhotonDrop], (unsigned long long)dropped);
            atomicAdd(&bs.e[sp][1], e_drop);
        }
    }
    // s_excl and s_warp[kWarps - 1] (the tile total) stay valid for the caller
    // until its next barrier
}

// -------------------------------------------------------------------- photon tile

template <int PREC, int FK, typename R>
__device__ void photon_tile(const StepArgs &a, Smem<R> &sm, unsigned long long *bar,
                            bool &loaded, unsigned chain_tile, int64_t n, int64_t be, int64_t bp,
                            int64_t room, unsigned epoch, int *s_warp, long long *s_excl,
                            BlockStats &bs, int *tile_total_out)
{
    const int tid = threadIdx.x;
    const SpeciesDev &Ph = a.sp[2], &El = a.sp[0], &Po = a.sp[1];
    const bool pairs = a.pairs != 0;
    const bool leptons = El.present && Po.present;
    if (pairs && !loaded) {
        if (tid == 0) {
            const unsigned bytes = kNRatePad * sizeof(R);
            mbar_init(bar, 1);
            mbar_expect_tx(bar, bytes);
            if constexpr (PREC == kFP64)
                bulk_g2s(sm.T, a.tab.Ts, bytes, bar);
            else
                bulk_g2s(sm.T, a.tab.Tsf, bytes, bar);
        }
        __syncthreads();
        wait_tables(bar, a);
        loaded = true;
    }
    const int64_t i = (int64_t)chain_tile * kTile + tid;
    int npair = 0;
    double px = 0, py = 0, pz = 0, gux = 0, guy = 0, guz = 0, wg = 0, v = 0, omv = 0, tm = 0, tp = 0;
    bool clamped = false;

    if constexpr (PREC == kFP64) {
    if (i < n) {
        double tau = Ph.tau[i];
        if (tau >= 0.0) {
            px = Ph.x[i];
            py = Ph.y[i];
            pz = Ph.z ? Ph.z[i] : 0.0;
            gux = Ph.ux[i];
            guy = Ph.uy[i];
            guz = Ph.uz[i];
            const double g = sqrt(gux * gux + guy * guy + guz * guz);
            const double dt = a.dt;
            bool decayed = false;
            if (pairs && g > 2.0) {
                Vec3<R> E, B;
                eval_field<FK, R>(a.f, px, py, pz, a.t, E, B);
                double chi, dtau;
                if constexpr (PREC == kFP64) {
                    const double kx = gux / g, ky = guy / g, kz = guz / g;
                    const double ax = E.x + (ky * B.z - kz * B.y);
                    const double ay = E.y + (kz * B.x - kx * B.z);
                    const double az = E.z + (kx * B.y - ky * B.x);
                    const double ke = kx * E.x + ky * E.y + kz * E.z;
                    const double s = ax * ax + ay * ay + az * az - ke * ke;
                    chi = s > 0.0 ? g * sqrt(s) / a.a_S : 0.0;
                    const double Tr = rate64<2>(sm.T, chi, clamped);
                    dtau = a.C_rate * Tr / g * dt;
                } else {
                    const float ig = (float)(1.0 / g);
                    const float kx = (float)gux * ig, ky = (float)guy * ig, kz = (float)guz * ig;
                    const float ax = E.x + (ky * B.z - kz * B.y);
                    const float ay = E.y + (kz * B.x - kx * B.z);
                    const float az = E.z + (kx * B.y - ky * B.x);
                    const float ke = kx * E.x + ky * E.y + kz * E.z;
                    const float s = ax * ax + ay * ay + az * az - ke * ke;
                    const float cf = s > 0.0f ? (float)g * sqrtf(s) * (float)(1.0 / a.a_S) : 0.0f;
                    chi = cf;
                    const float Tr = rate32<2>(sm.T, cf, clamped);
                    dtau = (double)((float)a.C_rate * Tr / (float)g * (float)dt);
                }
                if (Ph.chi) Ph.chi[i] = chi;
                if (dtau > 0.0 && !(tau > dtau)) {
                    // ---- pair creation at the photon position
                    const uint4 r1 = draw(a.seed, QP_PHOTON, kRngPair, i, a.step, 0);
                    const uint4 r2 = draw(a.seed, QP_PHOTON, kRngPairPos, i, a.step, 0);
                    v = sample_cdf<double>(a.tab.Cp, chi, u53(r1.x, r1.y), kSpMin, kSpSpan, false,
                                           clamped);
                    omv = 1.0 - v;
                    tm = -log(u53(r1.z, r1.w));
                    tp = -log(u53(r2.x, r2.y));
                    wg = Ph.w[i];
                    npair = 1;
                    decayed = true;
                    Ph.tau[i] = -1.0;
                } else {
                    Ph.tau[i] = tau - dtau;
                }
            }
            if (!decayed && g > 0.0) {
                if constexpr (PREC == kFP64) {
                    Ph.x[i] = px + dt * (gux / g);
                    Ph.y[i] = py + dt * (guy / g);
                    if (Ph.z) Ph.z[i] = pz + dt * (guz / g);
                } else {
                    const float c = (float)(dt / g);
                    Ph.x[i] = px + (double)(c * (float)gux);
                    Ph.y[i] = py + (double)(c * (float)guy);
                    if (Ph.z) Ph.z[i] = pz + (double)(c * (float)guz);
                }
            }
        }
    }
    } else {
    if (i < n) {
        const double taud = Ph.tau[i];
        if (taud >= 0.0) {
            // ---- mixed precision: FP32 physics, FP64 accumulation by
            // integer instructions
            const MixedConsts &m = a.mc;
            px = Ph.x[i];
            py = Ph.y[i];
            pz = Ph.z ? Ph.z[i] : 0.0;
            gux = Ph.ux[i];
            guy = Ph.uy[i];
            guz = Ph.uz[i];
            const float fx = hi_d(gux), fy = hi_d(guy), fz = hi_d(guz);
            const float g = sqrtf(fx * fx + fy * fy + fz * fz);
            bool decayed = false;
            if (pairs && g > 2.0f) {
                Vec3<float> E, B;
                eval_field_mixed<FK>(a.f, m, split_d(px), split_d(py), split_d(pz), E, B);
                const float ig = 1.0f / g;
                const float kx = fx * ig, ky = fy * ig, kz = fz * ig;
                const float ax = E.x + (ky * B.z - kz * B.y);
                const float ay = E.y + (kz * B.x - kx * B.z);
                const float az = E.z + (kx * B.y - ky * B.x);
                const float ke = kx * E.x + ky * E.y + kz * E.z;
                const float s2 = ax * ax + ay * ay + az * az - ke * ke;
                const float chi = s2 > 0.0f ? over_aS(g * sqrtf(s2), m.inv_aS, m.inv_aS_lo) : 0.0f;
                const float Tr = rate32<2>(sm.T, chi, clamped);
                const float dtau = m.C_rate * Tr / g * m.dt;
                if (Ph.chi) Ph.chi[i] = f_to_d(chi);
                const df2 TAU = split_d(taud);
                if (dtau > 0.0f && !(TAU.hi > dtau || (TAU.hi == dtau && TAU.lo > 0.0f))) {
                    // ---- pair creation at the photon position
                    const uint4 r1 = draw(a.seed, QP_PHOTON, kRngPair, i, a.step, 0);
                    const uint4 r2 = draw(a.seed, QP_PHOTON, kRngPairPos, i, a.step, 0);
                    const FracPair vf = sample_cdf_f(
                        a.tab.Cp2, a.tab.Qp2, a.tab.Ep, chi, u53_pair(r1.x, r1.y),
                        u53_pair_complement(r1.x, r1.y), (float)(kSpSpan / (kNNode - 1)), false,
                        clamped);
                    v = f_to_d(vf.x);
                    omv = f_to_d(vf.omx);
                    tm = f_to_d(-logf(u53f(r1.z, r1.w)));
                    tp = f_to_d(-logf(u53f(r2.x, r2.y)));
                    wg = Ph.w[i];
                    npair = 1;
                    decayed = true;
                    Ph.tau[i] = -1.0;
                } else if (dtau != 0.0f) {
                    Ph.tau[i] = add_fd(taud, -dtau);
                }
            }
            if (!decayed && g > 0.0f) {
                const float c = m.dt / g;
                Ph.x[i] = add_fd(px, c * fx);
                Ph.y[i] = add_fd(py, c * fy);
                if (Ph.z) Ph.z[i] = add_fd(pz, c * fz);
            }
        }
    }
    }
    if (npair && Ph.nemit) Ph.nemit[i] += 1;
    warp_count(&bs.c[2][cClamp], clamped);
    warp_count(&bs.c[2][cPair], npair != 0);
    *tile_total_out = 0;
    if (!pairs) return;

    int tile_total;
    const int local = block_scan(npair, s_warp, &tile_total);
    if (tid < 32) {
        const long long e =
            chain_prefix(a.pho_words, chain_tile, tile_total, epoch, a.spin_limit, a.status);
        if (tid == 0) *s_excl = e;
    }
    __syncthreads();
    const long long excl = *s_excl;
    *tile_total_out = tile_total;
    if (npair) {
        const int64_t ord = excl + local;
        if (leptons && ord < room) {
            const int64_t se = be + ord, spo = bp + ord;
            const double om = omv;
            El.x[se] = px;
            El.y[se] = py;
            if (El.z) El.z[se] = pz;
            El.ux[se] = v * gux;
            El.uy[se] = v * guy;
            El.uz[se] = v * guz;
            El.tau[se] = tm;
            El.w[se] = wg;
            if (El.chi) El.chi[se] = 0.0;
            if (El.nemit) El.nemit[se] = 0;
            Po.x[spo] = px;
            Po.y[spo] = py;
            if (Po.z) Po.z[spo] = pz;
            Po.ux[spo] = om * gux;
            Po.uy[spo] = om * guy;
            Po.uz[spo] = om * guz;
            Po.tau[spo] = tp;
            Po.w[spo] = wg;
            if (Po.chi) Po.chi[spo] = 0.0;
            if (Po.nemit) Po.nemit[spo] = 0;
        } else {
            atomicAdd(&bs.c[2][cPairDrop], 1ull);
            atomicAdd(&bs.e[2][1], wg * sqrt(gux * gux + guy * guy + guz * guz));
        }
    }
}

}  // namespace

// -------------------------------------------------------------------- the step

// FP64: 4 blocks of 128 per SM (128 registers, no spills); mixed: 8 blocks
// (64 registers; the few spills cost less than the extra resident warps gain)
template <int PREC, int FK>
__global__ void __launch_bounds__(kTile, PREC == kFP64 ? 4 : 8)
    k_step(const __grid_constant__ StepArgs a)
{
    using R = typename std::conditional<PREC == kFP64, double, float>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<R> &sm = *reinterpret_cast<Smem<R> *>(smem_raw);
    __shared__ __align__(8) unsigned long long s_bar[2];   // TMA: lepton, photon tables
    __shared__ int s_warp[kWarps];
    __shared__ unsigned s_ticket;
    __shared__ long long s_excl;
    __shared__ BlockStats bs;

    const int tid = threadIdx.x;
    clear_stats(bs);
    const unsigned epoch = *((volatile unsigned *)&a.ctl->epoch);
    // live counts: read-only during the launch; clamped so that a bad caller
    // counter never indexes outside the buffers
    int64_t n[3];
    bool bad = false;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        n[s] = a.sp[s].present ? *a.sp[s].n_live : 0;
        if (n[s] < 0 || n[s] > a.sp[s].cap) {
            bad = true;
            n[s] = n[s] < 0 ? 0 : a.sp[s].cap;
        }
    }
    if (bad && blockIdx.x == 0 && tid == 0) raise_status(a.status, QP_ERR_INVALID_ARG);
    const int64_t tiles_e = (n[0] + kTile - 1) / kTile;
    const int64_t tiles_l = tiles_e + (n[1] + kTile - 1) / kTile;
    const int64_t tiles_g = (n[2] + kTile - 1) / kTile;
    const int64_t n_tiles = tiles_l + tiles_g;
    const int64_t be = n[0], bp = n[1];
    int64_t room = 0;
    if (a.sp[0].present && a.sp[1].present) {
        room = a.sp[0].cap - be;
        if (a.sp[1].cap - bp < room) room = a.sp[1].cap - bp;
        if (room < 0) room = 0;
    }
    bool lep_loaded = false, ph_loaded = false;

    if ((int64_t)blockIdx.x < n_tiles) {
        for (;;) {
            if (tid == 0) s_ticket = atomicAdd(&a.ctl->ticket, 1u);
            __syncthreads();
            const unsigned t = s_ticket;
            if ((int64_t)t >= n_tiles) break;
            if ((int64_t)t < tiles_l) {
                const int sp = (int64_t)t < tiles_e ? 0 : 1;
                const int64_t first = ((int64_t)t - (sp ? tiles_e : 0)) * kTile;
                lepton_tile<PREC, FK, R>(a, sm, &s_bar[0], lep_loaded, t, sp, first, n[sp], n[2],
                                         epoch, s_warp, &s_excl, bs);
                if ((int64_t)t == tiles_l - 1 && tid == 0) {
                    // last lepton tile: the new photon count, applied at the end
                    const int64_t tot = n[2] + s_excl + s_warp[kWarps - 1];
                    if (a.sp[2].present) {
                        a.ctl->pending[2] = tot < a.sp[2].cap ? tot : a.sp[2].cap;
                        if (tot > a.sp[2].cap) raise_status(a.status, QP_WARN_BUFFER_FULL);
                    } else if (tot > n[2]) {
                        raise_status(a.status, QP_WARN_BUFFER_FULL);
                    }
                }
            } else {
                const unsigned pt = (unsigned)((int64_t)t - tiles_l);
                int tile_total = 0;
                photon_tile<PREC, FK, R>(a, sm, &s_bar[1], ph_loaded, pt, n[2], be, bp, room, epoch,
                                         s_warp, &s_excl, bs, &tile_total);
                if ((int64_t)t == n_tiles - 1 && tid == 0 && a.pairs) {
                    // last photon tile: the new lepton counts, applied at the end
                    const int64_t tot = s_excl + tile_total;
                    const int64_t add = tot < room ? tot : room;
                    a.ctl->pending[0] = be + add;
                    a.ctl->pending[1] = bp + add;
                    if (tot > add) raise_status(a.status, QP_WARN_BUFFER_FULL);
                }
            }
            __syncthreads();
        }
    }
    flush_stats(bs, a);
    if (tid == 0 && (bs.c[0][cClamp] | bs.c[1][cClamp] | bs.c[2][cClamp]))
        raise_status(a.status, QP_WARN_TABLE_CLAMPED);

    // ---- the last block to finish publishes the step
    if (tid == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&a.ctl->done, 1u);
        if (prev == gridDim.x - 1) {
            __threadfence();
            volatile long long *pend = a.ctl->pending;
            if (tiles_l > 0 && a.sp[2].present) *a.sp[2].n_live = pend[2];
            if (tiles_g > 0 && a.pairs && a.sp[0].present && a.sp[1].present) {
                *a.sp[0].n_live = pend[0];
                *a.sp[1].n_live = pend[1];
            }
            *((volatile unsigned *)&a.ctl->ticket) = 0u;
            *((volatile unsigned *)&a.ctl->done) = 0u;
            *((volatile unsigned *)&a.ctl->epoch) = epoch + 1u;
            __threadfence();
        }
    }
}

// -------------------------------------------------------------------- wait self-test

// Tile 1 of a chain whose tile 0 never publishes: the bounded wait must
// give up, raise QP_ERR_TIMEOUT and return.
__global__ void k_wait_selftest(unsigned long long *words, unsigned spin_limit, int *status)
{
    if (threadIdx.x < 32 && blockIdx.x == 0) {
        if (threadIdx.x == 0) words[0] = 0ull;
        __syncwarp();
        (void)chain_prefix(words, 1u, 0, 7u, spin_limit, status);
    }
}

cudaError_t launch_wait_selftest(unsigned long long *words, unsigned spin_limit, int *status,
                                 cudaStream_t st)
{
    k_wait_selftest<<<1, 32, 0, st>>>(words, spin_limit, status);
    return cudaGetLastError();
}

// -------------------------------------------------------------------- initial optical depth

__global__ void k_init_tau(double *tau, int64_t first, int64_t count, uint64_t seed, int species)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += stride) {
        const int64_t i = first + k;
        const uint4 r = draw(seed, species, kRngInit, i, 0, 0);
        tau[i] = -log(u53(r.x, r.y));
    }
}

// -------------------------------------------------------------------- diagnostics

// Fixed-order reduction: block b takes tiles b, b + G, ... and every thread
// sums its own elements in order; the block tree and the final pass over
// blocks have a fixed shape, so the result is independent of timing.
constexpr int kDiagScalars = 8;  // n_alive, weight, energy, px, py, pz, w chi, (spare)

__global__ void __launch_bounds__(kDiagTile) k_diag_partial(SpeciesDev S, int is_photon,
                                                       double *partials)
{
    __shared__ double s_red[kDiagScalars][kDiagTile];
    __shared__ int s_bin[kDiagTile];
    __shared__ double s_w[kDiagTile];
    const int tid = threadIdx.x;
    int64_t n = *S.n_live;
    n = n < 0 ? 0 : (n > S.cap ? S.cap : n);
    double acc[kDiagScalars] = {0, 0, 0, 0, 0, 0, 0, 0};
    double hist = 0.0;  // thread tid < QP_HIST_BINS owns bin tid
    const double bin_scale = QP_HIST_BINS / (QP_HIST_LOG10_MAX - QP_HIST_LOG10_MIN);
    for (int64_t base = (int64_t)blockIdx.x * kDiagTile; base < n; base += (int64_t)gridDim.x * kDiagTile) {
        const int64_t i = base + tid;
        int bin = -1;
        double wv = 0.0;
        if (i < n) {
            const double tau = S.tau[i];
            if (!is_photon || tau >= 0.0) {
                const double ux = S.ux[i], uy = S.uy[i], uz = S.uz[i], w = S.w[i];
                const double p2 = ux * ux + uy * uy + uz * uz;
                const double g = is_photon ? sqrt(p2) : sqrt(1.0 + p2);
                acc[0] += 1.0;
                acc[1] += w;
                acc[2] += w * g;
                acc[3] += w * ux;
                acc[4] += w * uy;
                acc[5] += w * uz;
                if (S.chi) acc[6] += w * S.chi[i];
                double b = (log10(g) - QP_HIST_LOG10_MIN) * bin_scale;
                b = b < 0.0 ? 0.0 : (b > QP_HIST_BINS - 1 ? QP_HIST_BINS - 1 : b);
                bin = g > 0.0 ? (int)b : 0;
                wv = w;
            }
        }
        s_bin[tid] = bin;
        s_w[tid] = wv;
        __syncthreads();
        if (tid < QP_HIST_BINS)
            for (int k = 0; k < kDiagTile; ++k)
                if (s_bin[k] == tid) hist += s_w[k];
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < kDiagScalars; ++k) s_red[k][tid] = acc[k];
    __syncthreads();
    for (int h = kDiagTile / 2; h > 0; h >>= 1) {
        if (tid < h)
#pragma unroll
            for (int k = 0; k < kDiagScalars; ++k) s_red[k][tid] += s_red[k][tid + h];
        __syncthreads();
    }
    double *out = partials + (size_t)blockIdx.x * (kDiagScalars + QP_HIST_BINS);
    if (tid < kDiagScalars) out[tid] = s_red[tid][0];
    if (tid < QP_HIST_BINS) out[kDiagScalars + tid] = hist;
}

__global__ void k_diag_final(const double *partials, int nblocks, double *out)
{
    const int k = threadIdx.x;
    if (k >= kDiagScalars + QP_HIST_BINS) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partials[(size_t)b * (kDiagScalars + QP_HIST_BINS) + k];
    out[k] = s;
}

// -------------------------------------------------------------------- launchers

template <int PREC>
static const void *step_kernel(int fk)
{
    switch (fk) {
    case QP_FIELD_NONE: return (const void *)k_step<PREC, QP_FIELD_NONE>;
    case QP_FIELD_PLANE: return (const void *)k_step<PREC, QP_FIELD_PLANE>;
    case QP_FIELD_GAUSSIAN: return (const void *)k_step<PREC, QP_FIELD_GAUSSIAN>;
    case QP_FIELD_YEE2D: return (const void *)k_step<PREC, QP_FIELD_YEE2D>;
    case QP_FIELD_UNIFORM_B: return (const void *)k_step<PREC, QP_FIELD_UNIFORM_B>;
    default: return nullptr;
    }
}

static const void *step_fn(int precision, int fk)
{
    return precision == QP_MIXED ? step_kernel<kMixed>(fk) : step_kernel<kFP64>(fk);
}

size_t step_smem_bytes(int precision)
{
    return precision == QP_MIXED ? sizeof(Smem<float>) : sizeof(Smem<double>);
}

int step_blocks_per_sm(int precision, int field_kind)
{
    const void *fn = step_fn(precision, field_kind);
    if (!fn) return 1;
    const size_t smem = step_smem_bytes(precision);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 1;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kTile, smem) != cudaSuccess)
        return 1;
    return nb < 1 ? 1 : nb;
}

cudaError_t launch_step(const StepArgs &a, int precision, int grid, cudaStream_t st)
{
    const void *fn = step_fn(precision, a.f.kind);
    if (!fn) return cudaErrorInvalidValue;
    const size_t smem = step_smem_bytes(precision);
    void *args[] = {(void *)&a};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kTile), args, smem, st);
}

cudaError_t launch_init_tau(double *tau, int64_t first, int64_t count, uint64_t seed, int species,
                            cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    int64_t blocks = (count + kDiagTile - 1) / kDiagTile;
    if (blocks > 4096) blocks = 4096;
    k_init_tau<<<(int)blocks, kDiagTile, 0, st>>>(tau, first, count, seed, species);
    return cudaGetLastError();
}

cudaError_t launch_diag(const SpeciesDev &S, int is_photon, double *partials, int nblocks,
                        double *out, cudaStream_t st)
{
    k_diag_partial<<<nblocks, kDiagTile, 0, st>>>(S, is_photon, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_diag_final<<<1, 128, 0, st>>>(partials, nblocks, out);
    return cudaGetLastError();
}

}  // namespace qp
