// The step kernel of libqedpic (sm_103a), instantiated per precision in
// qp_step_fp64.cu and qp_step_mixed.cu.
//
// One QED particle step is ONE launch of the persistent kernel k_step.  Its
// blocks take 128-particle tiles from one atomic ticket over a single tile
// space: per problem, first the electron tiles, then the positron tiles
// (together: the lepton chain), then the photon tiles (the photon chain).
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
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include <stddef.h>

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

// *p += v at GPU scope with acquire-release semantics; returns the old value
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned *p, unsigned v)
{
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;"
                 : "=r"(old)
                 : "l"(p), "r"(v)
                 : "memory");
    return old;
}

// Decoupled look-back over a chain of tiles.  A tile first publishes its
// aggregate (the number of particles it appends); the exclusive prefix is
// then computed by one full warp with a 32-tile window: lane l inspects tile
// base - l; a word counts only if it carries this launch's epoch.  The
// window is consumed up to the nearest tile that published its inclusive
// prefix, summing the aggregates in between.  Waits are bounded by
// spin_limit; on time-out the status is raised and the prefix is what was
// summed so far (the output is then wrong, the status says so, and the
// kernel still terminates).  Returns the prefix in every lane.

// Publish a tile's aggregate (tile 0: its inclusive prefix); one thread.
__device__ __forceinline__ void publish_aggregate(unsigned long long *words, unsigned tile,
                                                  long long aggregate, unsigned epoch)
{
    atomicExch(words + tile, make_word(epoch, tile == 0 ? kFlagPre : kFlagAgg, aggregate));
}

// The exclusive prefix of a tile whose aggregate is published: one full
// warp; publishes the tile's inclusive prefix.
__device__ long long resolve_prefix(unsigned long long *words, unsigned tile, long long aggregate,
                                    unsigned epoch, unsigned spin_limit, int *status)
{
    const int lane = threadIdx.x & 31;
    if (tile == 0) return 0;
    long long excl = 0;
    long long base = (long long)tile - 1;
    unsigned spins = 0, nap = 32;
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
            // back off (32 ns doubling to 256 ns): a waiting warp takes few
            // issue slots from the warps still computing their tiles, and
            // wakes soon after the tile it waits on publishes (a 1 us cap:
            // foil 30.5 us per step, 256 ns: 30.1)
            __nanosleep(nap);
            if (nap < 256) nap <<= 1;
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

__device__ long long chain_prefix(unsigned long long *words, unsigned tile, long long aggregate,
                                  unsigned epoch, unsigned spin_limit, int *status)
{
    if ((threadIdx.x & 31) == 0) publish_aggregate(words, tile, aggregate, epoch);
    __syncwarp();
    return resolve_prefix(words, tile, aggregate, epoch, spin_limit, status);
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
// atomic per counter when the block leaves.  The counts are 32-bit (shared
// memory adds them natively; a block never counts 2^32 events in a launch),
// summed over a warp before one lane adds them.
struct BlockStats {
    unsigned c[3][9];
    double e[3][2];
};
enum { cEmit, cPhoton, cPhotonDrop, cSub, cPair, cPairDrop, cSat, cClamp, cCont };

__device__ __forceinline__ void warp_count(unsigned *ctr, bool pred)
{
    const unsigned m = __ballot_sync(0xFFFFFFFFu, pred);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(ctr, (unsigned)__popc(m));
}

// Sum of v over the (converged) warp, added by one lane.
__device__ __forceinline__ void warp_add(unsigned *ctr, unsigned v)
{
    const unsigned s = __reduce_add_sync(0xFFFFFFFFu, v);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(ctr, s);
}

__device__ __forceinline__ void warp_add(double *ctr, double v)
{
    if (!__any_sync(0xFFFFFFFFu, v != 0.0)) return;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, d);
    if ((threadIdx.x & 31) == 0) atomicAdd(ctr, v);
}

__device__ __forceinline__ void clear_stats(BlockStats &bs)
{
    const int t = threadIdx.x;
    if (t < 27) (&bs.c[0][0])[t] = 0u;
    if (t < 6) (&bs.e[0][0])[t] = 0.0;
}

__device__ void flush_stats(const BlockStats &bs, const StepArgs &a, const Problem &P)
{
    __syncthreads();
    const int t = threadIdx.x;
    if (t < 27) {
        const int s = t / 9, k = t % 9;
        if (bs.c[s][k] && P.sp[s].present)
            atomicAdd(&a.stats[P.sp[s].slot_stats].n_emit + k, (unsigned long long)bs.c[s][k]);
    } else if (t >= 32 && t < 38) {
        const int s = (t - 32) / 2, k = (t - 32) % 2;
        if (bs.e[s][k] != 0.0 && P.sp[s].present)
            atomicAdd(&a.stats[P.sp[s].slot_stats].e_subthreshold + k, bs.e[s][k]);
    }
    if (t == 0 && (bs.c[0][cClamp] | bs.c[1][cClamp] | bs.c[2][cClamp]))
        raise_status(a.status, QP_WARN_TABLE_CLAMPED);
}

// Append records of a tile, written during its physics to a per-block ring
// of kStashBufs buffers in device memory ([field][thread] per buffer) and
// read when the tile's slots are known, kStashBufs - 1 tiles later.
// Lepton tiles: emitter x, y, z, direction kx, ky, kz, weight, then the
// energies and the optical depths of up to QP_MAX_EMISSIONS photons.  Photon
// tiles: x, y, z, photon momentum, weight, v, 1 - v, electron and positron
// optical depths.
constexpr int kStashGg = 7, kStashTg = kStashGg + QP_MAX_EMISSIONS;
constexpr int kStashFields = kStashTg + QP_MAX_EMISSIONS;
static_assert(kStashFields == kStashFieldsHost, "stash layout");
// Append map of a stashed tile: entry j (the tile's j-th new particle) holds
// its parent thread (low byte) and the parent's emission index (high byte).
constexpr int kMapEntries = kTile * QP_MAX_EMISSIONS;
static_assert(kTile <= 256 && QP_MAX_EMISSIONS <= 256, "append map entries are two bytes");

// Shared-memory layout of k_step (dynamic part).
template <typename R>
struct Smem {
    R H[kNRatePad];                          // rate tables (TMA-staged)
    R G[kNRatePad];
    R T[kNRatePad];
};

__device__ __forceinline__ void wait_tables(unsigned long long *bar, const StepArgs &a)
{
    if (!mbar_wait_bounded(bar, 0, a.spin_limit)) {
        // the step's results are flagged invalid from here on; a second
        // bounded wait gives the copy more time to land before the block
        // reads the tables or leaves.  If it runs out too, the tile reads
        // tables that may be incomplete (the raised status says so) and the
        // kernel still terminates.
        raise_status(a.status, QP_ERR_TIMEOUT);
        (void)mbar_wait_bounded(bar, 0, a.spin_limit);
    }
}

// -------------------------------------------------------------------- lepton tile

// Issue the copy of the rate tables H and G into shared memory (one TMA
// bulk copy each, completing on `bar`); one thread, before a barrier that
// makes the barrier's initialisation visible to the block.
template <int PREC, typename R>
__device__ __forceinline__ void stage_rate_tables(const StepArgs &a, Smem<R> &sm,
                                                  unsigned long long *bar)
{
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

// State of one lepton at the start of a step (the FP64 storage of both
// paths; component c of the new state goes to the sink's put<c> as soon as
// it is formed, c = x y z ux uy uz tau, tau only when it changed).
struct LeptonState {
    double x, y, z, ux, uy, uz, tau;
};

// What one lepton's step produced besides its new state.
struct LeptonOut {
    int n_emit, nph, n_sub;
    double e_sub;   // sum of gamma_gamma of the photons below the cut
    bool cont, sat, clamped;
};

// One step of one lepton (a1..a8 of the hot path): fields at (x, t), Boris
// push, chi_e, then Sokolov damping below chi_th or the optical depth with
// its emission sub-loop (Eq. 6-8), then the position (Eq. 4).  The sink
// receives the new state (put<c>, see LeptonState) and what an append needs: tables() before the
// rate tables H and G are first read, chi(c) with chi_e after the push,
// direction(k) with the momentum direction before the first recoil,
// photon(j, gamma, tau) for the j-th stored photon, origin(x) with the
// position at the start of the step when photons were stored.  S, i: the
// particle's species and slot (its id keys the random streams).
template <int PREC, int FK, typename R, class Sink>
__device__ __forceinline__ void lepton_particle(const StepArgs &a, const Problem &P, const R *H,
                                                const R *G, int sp, const SpeciesDev &S,
                                                int64_t i, const LeptonState &s, LeptonOut &o,
                                                Sink &sink)
{
    o.n_emit = o.nph = o.n_sub = 0;
    o.e_sub = 0.0;
    o.cont = o.sat = o.clamped = false;
    bool clamped = false;
    int nph = 0, n_emit = 0, n_sub = 0;
    if constexpr (PREC == kFP64) {
        const double q = sp == 0 ? -1.0 : 1.0;
        const double dt = P.dt;
        const double x0 = s.x, y0 = s.y, z0 = s.z;
        double ux = s.ux, uy = s.uy, uz = s.uz;
        double tau = s.tau;
        Vec3<R> E, B;
        eval_field<FK, R>(P.f, x0, y0, z0, P.t, E, B);

        // ---- Boris push of the Lorentz force (f_l of Eq. 4)
        {
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
        }
        double gam = sqrt(1.0 + ux * ux + uy * uy + uz * uz);
        const double Ex = E.x, Ey = E.y, Ez = E.z, Bx = B.x, By = B.y, Bz = B.z;
        sink.tables();  // tables are needed from here on
        double chi = chi_e64(Ex, Ey, Ez, Bx, By, Bz, ux, uy, uz, gam, a.a_S);
        sink.chi(chi);
        double dvx = 0.0, dvy = 0.0, dvz = 0.0;

        if (chi < P.chi_th) {
            // ---- Sokolov continuous regime (Eq. 4, P_rad of Eq. 5)
            o.cont = true;
            const double vx = ux / gam, vy = uy / gam, vz = uz / gam;
            const double fx = q * (Ex + (vy * Bz - vz * By));
            const double fy = q * (Ey + (vz * Bx - vx * Bz));
            const double fz = q * (Ez + (vx * By - vy * Bx));
            const double vf = vx * fx + vy * fy + vz * fz;
            const double den = 1.0 + a.tau0w * vf;
            dvx = a.tau0w * (fx - vx * vf) / den;
            dvy = a.tau0w * (fy - vy * vf) / den;
            dvz = a.tau0w * (fz - vz * vf) / den;
            const double prad = a.C_rate * rate64<1>(G, chi, clamped);
            ux = ux + dt * (q * (dvy * Bz - dvz * By) - prad * vx);
            uy = uy + dt * (q * (dvz * Bx - dvx * Bz) - prad * vy);
            uz = uz + dt * (q * (dvx * By - dvy * Bx) - prad * vz);
            gam = sqrt(1.0 + ux * ux + uy * uy + uz * uz);
        } else {
            // ---- optical depth (Eq. 6) with the residual-time sub-loop
            double r = 1.0;
            for (int k = 0;; ++k) {
                const double Hv = rate64<0>(H, chi, clamped);
                const double wdt = a.C_rate * Hv / gam * dt;
                const double dtau = wdt * r;
                if (!(dtau > 0.0) || tau > dtau) {
                    tau = tau - dtau;
                    break;
                }
                if (k == P.max_emit) {
                    tau = tau - dtau;
                    o.sat = true;
                    break;
                }
                r = r - tau / wdt;
                // ---- emission: Eq. 7 sampling, Eq. 8 recoil
                const uint4 rr = draw(P.seed, sp, kRngEmit, particle_id(S, i), P.step, k);
                const double xi_p = u53(rr.x, rr.y), xi = u53(rr.z, rr.w);
                const double ufrac = sample_cdf<double>(a.tab.Cg, a.tab.Gg, chi, xi_p, kSgMin,
                                                        kSgSpan, true, clamped);
                const double pmag = sqrt(ux * ux + uy * uy + uz * uz);
                double gg = ufrac * gam;
                if (gg > pmag) gg = pmag;
                if (n_emit == 0 && pmag > 0.0) sink.direction(ux / pmag, uy / pmag, uz / pmag);
                ++n_emit;
                if (gg > P.gmin) {
                    const uint4 rp = draw(P.seed, sp, kRngPhotonTau, particle_id(S, i), P.step, k);
                    sink.photon(nph, gg, -log(u53(rp.x, rp.y)));
                    ++nph;
                } else {
                    ++n_sub;
                    o.e_sub += gg;
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
        if (nph) sink.origin(x0, y0, z0);
        sink.template put<0>(x0 + dt * (ux / gam + dvx));
        sink.template put<1>(y0 + dt * (uy / gam + dvy));
        sink.template put<2>(z0 + dt * (uz / gam + dvz));
        sink.template put<3>(ux);
        sink.template put<4>(uy);
        sink.template put<5>(uz);
        sink.template put<6>(tau);
    } else {
        // ---- mixed precision: FP32 physics; the FP64 state is read once,
        // increments are formed in FP32 and added back by integer
        // instructions; chi_e falls back to double-float where FP32 cancels
        const MixedConsts &m = P.mc;
        const double xd = s.x, yd = s.y, zd = s.z;
        const double uxd = s.ux, uyd = s.uy, uzd = s.uz;
        const double taud = s.tau;
        Vec3<float> E, B;
        eval_field_mixed<FK>(P.f, m, xd, yd, zd, E, B);

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
        sink.tables();  // tables are needed from here on
        float chi = chi_mixed_auto(uxd, uyd, uzd, dux, duy, duz, ux, uy, uz, gam, E, B, m.inv_aS,
                                   m.inv_aS_lo);
        sink.chi(f_to_d(chi));
        float dvx = 0.0f, dvy = 0.0f, dvz = 0.0f;
        float dtau_once = 0.0f, esub_f = 0.0f;
        bool events = false;
        df2 TAU = {0.0f, 0.0f};

        if (chi < m.chi_th) {
            // ---- Sokolov (Eq. 4, 5); denominator 1 + tau0 v.f_l in double-float
            o.cont = true;
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
            const float prad = m.C_rate * rate32<1>(G, chi, clamped);
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
                const float Hv = rate32<0>(H, chi, clamped);
                const float wdt = m.C_rate * Hv / gam * m.dt;
                const float dtau = wdt * r;
                // tau > dtau decided on the double-float optical depth
                if (!(dtau > 0.0f) || TAU.hi > dtau || (TAU.hi == dtau && TAU.lo > 0.0f)) {
                    TAU = df_add_f(TAU, -dtau);
                    dtau_once = dtau;
                    break;
                }
                if (k == P.max_emit) {
                    TAU = df_add_f(TAU, -dtau);
                    dtau_once = dtau;
                    o.sat = true;
                    break;
                }
                events = true;
                r = r - df_to_f(TAU) / wdt;
                // ---- emission: Eq. 7 sampling, Eq. 8 recoil
                const uint4 rr = draw(P.seed, sp, kRngEmit, particle_id(S, i), P.step, k);
                const float xi = u53f(rr.z, rr.w);
                const FracPair uf = sample_cdf_f(
                    a.tab.Cg2, a.tab.Qg2, a.tab.Gg, a.tab.Eg, chi, u53_pair(rr.x, rr.y),
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
                if (n_emit == 0) {
                    // the photons' direction goes to the append record now
                    // (fewer values live through the loop)
                    const float ip = pmag > 0.0f ? 1.0f / pmag : 0.0f;
                    sink.direction(f_to_d(ux * ip), f_to_d(uy * ip), f_to_d(uz * ip));
                }
                ++n_emit;
                if (gg > m.gmin) {
                    const uint4 rp = draw(P.seed, sp, kRngPhotonTau, particle_id(S, i), P.step, k);
                    sink.photon(nph, f_to_d(gg), f_to_d(-logf(u53f(rp.x, rp.y))));
                    ++nph;
                } else {
                    ++n_sub;
                    esub_f += gg;
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

        // ---- position and state: FP64 accumulation of FP32 increments
        if (nph) sink.origin(xd, yd, zd);
        const float gi = 1.0f / gam;
        sink.template put<0>(add_fd(xd, m.dt * (ux * gi + dvx)));
        sink.template put<1>(add_fd(yd, m.dt * (uy * gi + dvy)));
        sink.template put<2>(add_fd(zd, m.dt * (uz * gi + dvz)));
        sink.template put<3>(add_fd(uxd, dux));
        sink.template put<4>(add_fd(uyd, duy));
        sink.template put<5>(add_fd(uzd, duz));
        if (events)
            sink.template put<6>(merge_df(TAU));
        else if (dtau_once != 0.0f)
            sink.template put<6>(add_fd(taud, -dtau_once));
        if (n_sub) o.e_sub = f_to_d(esub_f);
    }
    o.n_emit = n_emit;
    o.nph = nph;
    o.n_sub = n_sub;
    o.clamped = clamped;
}

// The append sink of a step tile: the block's tables are waited for once,
// and the records go to the tile's stash ([field][thread]).
template <int PREC>
struct StashSink {
    const StepArgs &a;
    unsigned long long *bar;
    bool loaded;
    double *st;
    int tid;
    double *chi_slot;  // the particle's chi, or NULL
    const SpeciesDev &S;
    int64_t i;
    // each component is stored as soon as it is formed (a value kept across
    // the called write-back helpers would have to be saved and restored)
    template <int C>
    __device__ __forceinline__ void put(double v)
    {
        if constexpr (C == 0) S.x[i] = v;
        if constexpr (C == 1) S.y[i] = v;
        if constexpr (C == 2) {
            if (S.z) S.z[i] = v;
        }
        if constexpr (C == 3) S.ux[i] = v;
        if constexpr (C == 4) S.uy[i] = v;
        if constexpr (C == 5) S.uz[i] = v;
        if constexpr (C == 6) S.tau[i] = v;
    }
    __device__ __forceinline__ void tables()
    {
        if (!loaded) wait_tables(bar, a);
    }
    __device__ __forceinline__ void chi(double c)
    {
        if (chi_slot) *chi_slot = c;
    }
    __device__ __forceinline__ void direction(double kx, double ky, double kz)
    {
        st[3 * kTile + tid] = kx;
        st[4 * kTile + tid] = ky;
        st[5 * kTile + tid] = kz;
    }
    __device__ __forceinline__ void photon(int j, double gg, double tau)
    {
        st[(kStashGg + j) * kTile + tid] = gg;
        st[(kStashTg + j) * kTile + tid] = tau;
    }
    __device__ __forceinline__ void origin(double x, double y, double z)
    {
        st[0 * kTile + tid] = x;
        st[1 * kTile + tid] = y;
        st[2 * kTile + tid] = z;
    }
};

template <int PREC, int FK, typename R, class Hook>
__device__ int lepton_tile(const StepArgs &a, const Problem &P, Smem<R> &sm,
                           unsigned long long *bar, bool &loaded, unsigned chain_tile, int sp,
                           int64_t first, int64_t n, unsigned epoch, int *s_warp, BlockStats &bs,
                           double *st, unsigned short *s_map, Hook &&before_scan)
{
    const int tid = threadIdx.x;
    // the rate tables' copy was issued in the kernel's prologue
    // (stage_rate_tables); `loaded`: every thread has seen it land
    const SpeciesDev &S = P.sp[sp];
    const int64_t i = first + tid;
    const bool active = i < n;

    LeptonOut o{};
    double wgt = 0;
    if (active) {
        LeptonState s{S.x[i], S.y[i], S.z ? S.z[i] : 0.0, S.ux[i], S.uy[i], S.uz[i], S.tau[i]};
        StashSink<PREC> sink{a, bar, loaded, st, tid, S.chi ? S.chi + i : nullptr, S, i};
        lepton_particle<PREC, FK, R>(a, P, sm.H, sm.G, sp, S, i, s, o, sink);
        if (o.nph || o.n_sub) wgt = S.w[i];
        if (o.nph) st[6 * kTile + tid] = wgt;
        if (o.n_emit && S.nemit) S.nemit[i] += o.n_emit;
    }
    if (!loaded) {
        // every thread waits once (at once if its particle already did, or
        // if the copy has landed): later tiles read the tables without a
        // wait, and the block never leaves with the copy in flight
        wait_tables(bar, a);
        loaded = true;
    }

    // ---- counters (warp-aggregated into shared memory)
    warp_count(&bs.c[sp][cCont], o.cont);
    warp_count(&bs.c[sp][cSat], o.sat);
    warp_count(&bs.c[sp][cClamp], o.clamped);
    if (__any_sync(0xFFFFFFFFu, o.n_emit > 0)) {
        warp_add(&bs.c[sp][cEmit], (unsigned)o.n_emit);
        warp_add(&bs.c[sp][cSub], (unsigned)o.n_sub);
        warp_add(&bs.e[sp][0], o.n_sub ? wgt * o.e_sub : 0.0);
    }

    // ---- this tile's appends: the aggregate is published now, the records
    // stashed and mapped; their slots are written later (write_photons)
    int tile_total;
    const int nph = o.nph;
    before_scan();
    const int local = block_scan(nph, s_warp, &tile_total);
    if (tid == 0) publish_aggregate(P.lep_words, chain_tile, tile_total, epoch);
    for (int k = 0; k < nph; ++k) s_map[local + k] = (unsigned short)(tid | (k << 8));
    return tile_total;
}

// Photons of a stashed lepton tile: the tile's photon j (in emitter order)
// goes to slot base + j, one thread per photon (coalesced stores); those
// beyond the capacity are counted as dropped with their energy.
__device__ void write_photons(const Problem &P, const double *st, const unsigned short *s_map,
                              int total, long long base, int sp, BlockStats &bs, int t0,
                              int stride)
{
    const SpeciesDev &Ph = P.sp[2];
    const bool photons = Ph.present != 0;
    int stored = 0, dropped = 0;
    double e_drop = 0.0;
    for (int j = t0; j < total; j += stride) {
        const unsigned m = s_map[j];
        const int e = (int)(m & 0xFFu), k = (int)(m >> 8);
        const int64_t slot = base + j;
        const double gg = st[(kStashGg + k) * kTile + e];
        const double wgt = st[6 * kTile + e];
        if (photons && slot < Ph.cap) {
            Ph.x[slot] = st[0 * kTile + e];
            Ph.y[slot] = st[1 * kTile + e];
            if (Ph.z) Ph.z[slot] = st[2 * kTile + e];
            Ph.ux[slot] = gg * st[3 * kTile + e];
            Ph.uy[slot] = gg * st[4 * kTile + e];
            Ph.uz[slot] = gg * st[5 * kTile + e];
            Ph.tau[slot] = st[(kStashTg + k) * kTile + e];
            Ph.w[slot] = wgt;
            if (Ph.chi) Ph.chi[slot] = 0.0;
            if (Ph.nemit) Ph.nemit[slot] = 0;
            ++stored;
        } else {
            ++dropped;
            e_drop += wgt * gg;
        }
    }
    warp_add(&bs.c[sp][cPhoton], (unsigned)stored);
    if (__any_sync(0xFFFFFFFFu, dropped != 0)) {
        warp_add(&bs.c[sp][cPhotonDrop], (unsigned)dropped);
        warp_add(&bs.e[sp][1], e_drop);
    }
}

// Ballistic motion of a photon over one step, x += c k^ dt: one copy of the
// arithmetic for every place a photon moves (the step's photon tiles and
// the fused steps), with every rounding explicit (a product left to the
// compiler could be fused into the add in one place and hoisted out of a
// loop in the other), so both give the same bits.
__device__ __forceinline__ double photon_speed64(double ux, double uy, double uz)
{
    return __dsqrt_rn(__fma_rn(uz, uz, __fma_rn(uy, uy, __dmul_rn(ux, ux))));
}
__device__ __forceinline__ double photon_move64(double x, double u, double g, double dt)
{
    return __fma_rn(dt, __ddiv_rn(u, g), x);
}
__device__ __forceinline__ float photon_speed32(float fx, float fy, float fz)
{
    return sqrtf(fx * fx + fy * fy + fz * fz);
}
__device__ __forceinline__ double photon_move32(double x, float f, float c)
{
    return add_fd(x, c * f);
}

// -------------------------------------------------------------------- photon tile

template <int PREC, int FK, typename R, class Hook>
__device__ int photon_tile(const StepArgs &a, const Problem &P, Smem<R> &sm,
                           unsigned long long *bar, bool &loaded, unsigned chain_tile, int64_t n,
                           unsigned epoch, int *s_warp, BlockStats &bs, double *st,
                           unsigned short *s_map, Hook &&before_scan)
{
    const int tid = threadIdx.x;
    const SpeciesDev &Ph = P.sp[2];
    const bool pairs = P.pairs != 0;
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
            const double g = photon_speed64(gux, guy, guz);
            const double dt = P.dt;
            bool decayed = false;
            if (pairs && g > 2.0) {
                Vec3<R> E, B;
                eval_field<FK, R>(P.f, px, py, pz, P.t, E, B);
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
                    const uint4 r1 = draw(P.seed, QP_PHOTON, kRngPair, particle_id(Ph, i), P.step, 0);
                    const uint4 r2 = draw(P.seed, QP_PHOTON, kRngPairPos, particle_id(Ph, i), P.step, 0);
                    v = sample_cdf<double>(a.tab.Cp, a.tab.Gp, chi, u53(r1.x, r1.y), kSpMin,
                                           kSpSpan, false, clamped);
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
                    Ph.x[i] = photon_move64(px, gux, g, dt);
                    Ph.y[i] = photon_move64(py, guy, g, dt);
                    if (Ph.z) Ph.z[i] = photon_move64(pz, guz, g, dt);
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
            const MixedConsts &m = P.mc;
            px = Ph.x[i];
            py = Ph.y[i];
            pz = Ph.z ? Ph.z[i] : 0.0;
            gux = Ph.ux[i];
            guy = Ph.uy[i];
            guz = Ph.uz[i];
            const float fx = hi_d(gux), fy = hi_d(guy), fz = hi_d(guz);
            const float g = photon_speed32(fx, fy, fz);
            bool decayed = false;
            if (pairs && g > 2.0f) {
                Vec3<float> E, B;
                eval_field_mixed<FK>(P.f, m, px, py, pz, E, B);
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
                    const uint4 r1 = draw(P.seed, QP_PHOTON, kRngPair, particle_id(Ph, i), P.step, 0);
                    const uint4 r2 = draw(P.seed, QP_PHOTON, kRngPairPos, particle_id(Ph, i), P.step, 0);
                    const FracPair vf = sample_cdf_f(
                        a.tab.Cp2, a.tab.Qp2, a.tab.Gp, a.tab.Ep, chi, u53_pair(r1.x, r1.y),
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
                Ph.x[i] = photon_move32(px, fx, c);
                Ph.y[i] = photon_move32(py, fy, c);
                if (Ph.z) Ph.z[i] = photon_move32(pz, fz, c);
            }
        }
    }
    }
    if (npair && Ph.nemit) Ph.nemit[i] += 1;
    warp_count(&bs.c[2][cClamp], clamped);
    warp_count(&bs.c[2][cPair], npair != 0);
    before_scan();
    if (!pairs) return 0;

    // ---- this tile's pairs: aggregate published now, records stashed
    int tile_total;
    const int local = block_scan(npair, s_warp, &tile_total);
    if (tid == 0) publish_aggregate(P.pho_words, chain_tile, tile_total, epoch);
    if (npair) {
        st[0 * kTile + tid] = px;
        st[1 * kTile + tid] = py;
        st[2 * kTile + tid] = pz;
        st[3 * kTile + tid] = gux;
        st[4 * kTile + tid] = guy;
        st[5 * kTile + tid] = guz;
        st[6 * kTile + tid] = wg;
        st[7 * kTile + tid] = v;
        st[8 * kTile + tid] = omv;
        st[9 * kTile + tid] = tm;
        st[10 * kTile + tid] = tp;
        s_map[local] = (unsigned short)tid;
    }
    return tile_total;
}

// The e-/e+ pairs of a stashed photon tile, one thread per pair: pair number
// excl + j goes to slots be + that and bp + that while it is below `room`;
// beyond it the pair is dropped and its energy counted.
__device__ void write_pairs(const Problem &P, const double *st, const unsigned short *s_map,
                            int total, long long excl, long long be, long long bp, long long room,
                            BlockStats &bs, int t0, int stride)
{
    const SpeciesDev &El = P.sp[0], &Po = P.sp[1];
    const bool leptons = El.present && Po.present;
    for (int j = t0; j < total; j += stride) {
        const int e = (int)(s_map[j] & 0xFFu);
        const double px = st[0 * kTile + e], py = st[1 * kTile + e], pz = st[2 * kTile + e];
        const double gux = st[3 * kTile + e], guy = st[4 * kTile + e], guz = st[5 * kTile + e];
        const double wg = st[6 * kTile + e];
        const int64_t ord = excl + j;
        if (leptons && ord < room) {
            const double v = st[7 * kTile + e], om = st[8 * kTile + e];
            const int64_t se = be + ord, spo = bp + ord;
            El.x[se] = px;
            El.y[se] = py;
            if (El.z) El.z[se] = pz;
            El.ux[se] = v * gux;
            El.uy[se] = v * guy;
            El.uz[se] = v * guz;
            El.tau[se] = st[9 * kTile + e];
            El.w[se] = wg;
            if (El.chi) El.chi[se] = 0.0;
            if (El.nemit) El.nemit[se] = 0;
            Po.x[spo] = px;
            Po.y[spo] = py;
            if (Po.z) Po.z[spo] = pz;
            Po.ux[spo] = om * gux;
            Po.uy[spo] = om * guy;
            Po.uz[spo] = om * guz;
            Po.tau[spo] = st[10 * kTile + e];
            Po.w[spo] = wg;
            if (Po.chi) Po.chi[spo] = 0.0;
            if (Po.nemit) Po.nemit[spo] = 0;
        } else {
            atomicAdd(&bs.c[2][cPairDrop], 1u);
            atomicAdd(&bs.e[2][1], wg * sqrt(gux * gux + guy * guy + guz * guz));
        }
    }
}

// -------------------------------------------------------------------- the step

// Tile counts of one problem for this launch.  Live counts and step counters
// change only at the end of a launch (last block), so every block sees the
// same values.  Counts outside [0, capacity] are clamped (and reported).
struct ProbCounts {
    long long n[3];
    long long tiles_e, tiles_l, tiles_g;
    bool active, bad;
};

__device__ __forceinline__ ProbCounts problem_counts(const Problem &P)
{
    ProbCounts c{};
    // every counter is loaded before any is tested, so the (uncached) reads
    // overlap instead of following each other
    long long v[3], left = 1;
#pragma unroll
    for (int s = 0; s < 3; ++s) v[s] = P.sp[s].present ? __ldcg(P.sp[s].n_live) : 0;
    if (P.device_step) left = __ldcg(P.left_ctr);
    c.active = left > 0;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        long long x = c.active ? v[s] : 0;
        if (x < 0 || x > P.sp[s].cap) {
            c.bad = true;
            x = x < 0 ? 0 : P.sp[s].cap;
        }
        c.n[s] = x;
    }
    c.tiles_e = (c.n[0] + kTile - 1) / kTile;
    c.tiles_l = c.tiles_e + (c.n[1] + kTile - 1) / kTile;
    c.tiles_g = (c.n[2] + kTile - 1) / kTile;
    return c;
}

// FP32 / double-float time constants of the mixed path at time t (the same
// IEEE operations as a host-side split, so both give identical values).
__device__ __forceinline__ void set_time(Problem &P, long long step)
{
    P.step = (uint64_t)step;
    P.t = (double)step * P.dt;
    const double tr = P.t - P.f.t_focus;
    P.mc.t_hi = __double2float_rn(P.t);
    P.mc.t_lo = __double2float_rn(P.t - (double)P.mc.t_hi);
    P.mc.tr_hi = __double2float_rn(tr);
    P.mc.tr_lo = __double2float_rn(tr - (double)P.mc.tr_hi);
}

// Block-wide inclusive scan of v[0..n) in place (n <= 2 kTile).
__device__ void scan_offsets(long long *v, int n, long long *s_tmp)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long a = 2 * tid < n ? v[2 * tid] : 0, b = 2 * tid + 1 < n ? v[2 * tid + 1] : 0;
    long long inc = a + b;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const long long y = __shfl_up_sync(0xFFFFFFFFu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) s_tmp[warp] = inc;
    __syncthreads();
    long long before = 0;
    for (int w = 0; w < warp; ++w) before += s_tmp[w];
    const long long excl = before + inc - (a + b);
    __syncthreads();
    if (2 * tid < n) v[2 * tid] = excl + a;
    if (2 * tid + 1 < n) v[2 * tid + 1] = excl + a + b;
    __syncthreads();
}

// A tile whose appends are stashed and not yet written (a ring of
// kStashBufs per block; the record of tile number q of the block sits at
// q % kStashBufs, beside its stash buffer and append map).
struct Pending {
    int chain, last, sp, total;
    unsigned tile;
    long long base, be, bp, room;
};

// The writes of a stashed tile whose exclusive prefix excl is known:
// threads t0, t0 + stride, ... write its photons or pairs; `leader` (one
// thread) sets the new live count when it is the last tile of its chain.
__device__ __forceinline__ void flush_write(const StepArgs &a, const Problem &P, const Pending &pd,
                                           long long excl, BlockStats &bs, const double *st,
                                           const unsigned short *s_map, int t0, int stride,
                                           bool leader)
{
    if (pd.chain == 0) {
        if (pd.last && leader) {
            const long long tot = pd.base + excl + pd.total;
            if (P.sp[2].present) {
                P.pending[2] = tot < P.sp[2].cap ? tot : P.sp[2].cap;
                if (tot > P.sp[2].cap) raise_status(a.status, QP_WARN_BUFFER_FULL);
            } else if (tot > pd.base) {
                raise_status(a.status, QP_WARN_BUFFER_FULL);
            }
        }
        if (pd.total) write_photons(P, st, s_map, pd.total, pd.base + excl, pd.sp, bs, t0, stride);
    } else {
        if (pd.last && leader) {
            const long long tot = excl + pd.total;
            const long long add = tot < pd.room ? tot : pd.room;
            P.pending[0] = pd.be + add;
            P.pending[1] = pd.bp + add;
            if (tot > add) raise_status(a.status, QP_WARN_BUFFER_FULL);
        }
        if (pd.total)
            write_pairs(P, st, s_map, pd.total, excl, pd.be, pd.bp, pd.room, bs, t0, stride);
    }
}

// Resolve a stashed tile's prefix (its predecessors are, by now, almost
// always published) and write its photons or pairs; the last tile of a
// chain also sets the new live count applied at the end of the launch.
// All threads of the block (when the block leaves a problem or the launch);
// the record was written before a barrier.
__device__ __forceinline__ void flush_pending(const StepArgs &a, const Problem &P, const Pending &pd,
                                           unsigned epoch, long long *s_excl, BlockStats &bs,
                                           const double *st, const unsigned short *s_map)
{
    if (threadIdx.x < 32) {
        const long long e = resolve_prefix(pd.chain ? P.pho_words : P.lep_words, pd.tile,
                                           pd.total, epoch, a.spin_limit, a.status);
        if (threadIdx.x == 0) *s_excl = e;
    }
    __syncthreads();
    flush_write(a, P, pd, *s_excl, bs, st, s_map, threadIdx.x, kTile, threadIdx.x == 0);
    // the record, map, stash buffer and s_excl are free for reuse after this
    __syncthreads();
}

// The same by one warp, without a block barrier: the warp that finishes a
// tile's physics first flushes the block's oldest stashed tile while the
// others are still computing (the buffers are reused only after the tile
// loop's closing barrier).
__device__ void flush_pending_warp(const StepArgs &a, const Problem &P, const Pending &pd,
                                   unsigned epoch, BlockStats &bs, const double *st,
                                   const unsigned short *s_map)
{
    const int lane = threadIdx.x & 31;
    const long long excl = resolve_prefix(pd.chain ? P.pho_words : P.lep_words, pd.tile,
                                          pd.total, epoch, a.spin_limit, a.status);
    flush_write(a, P, pd, excl, bs, st, s_map, lane, 32, lane == 0);
}

// One launch = one step of every active problem.  Persistent blocks take
// 128-particle tiles by ticket (block b's first tile is b in a cooperative
// launch, every other ticket comes from an atomic counter; the next ticket
// is fetched while the current tile runs when more tiles than blocks
// remain); tickets enumerate, problem after problem, its electron tiles,
// positron tiles and photon tiles, so within each problem's chains start
// order is tile order and the decoupled look-back only ever waits on tiles
// that are running.  A tile's appends are written
// kStashBufs - 1 tiles later: its aggregate is published right after its
// physics, its records go to a stash, and its prefix is resolved after the
// block's next two tiles, when the earlier tiles have almost always
// published, so blocks do not wait on one another tile after tile (the
// smallest unpublished tile always progresses: every wait is for smaller
// tiles, and a block holds its next ticket only while it runs physics or
// flushes tiles older than that ticket).  BATCH = false: the single problem of the
// launch parameters (read in place, from the constant bank); BATCH = true: a
// device table of problems, each copied to shared memory for its tiles, with
// time and step counters advanced on the device.
// Resident blocks of 128 per SM.  FP64: 4 (128 registers, no spills).
// Mixed: 7 (72 registers): the Yee gather keeps its 24 loads in flight
// (the 2D foil: 30.4 us per step at 7, 32.7 at 8), and since the first warp
// past a tile's physics flushes the oldest stashed tile (its code in the
// tile loop) the analytic-field steps spill less at 72 than at 64 (the
// 2e6-electron collision: 0.371 ms per step at 7, 0.386 at 8; before that
// change, 366 us at 7 and 356 at 8).
template <int PREC, int FK>
constexpr int step_min_blocks()
{
    return PREC == kFP64 ? 4 : 7;
}

template <int PREC, int FK, bool BATCH>
__global__ void __launch_bounds__(kTile, step_min_blocks<PREC, FK>())
    k_step(const __grid_constant__ StepArgs a)
{
    using R = typename std::conditional<PREC == kFP64, double, float>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<R> &sm = *reinterpret_cast<Smem<R> *>(smem_raw);
    __shared__ __align__(8) unsigned long long s_bar[2];   // TMA: lepton, photon tables
    __shared__ int s_warp[kWarps];
    __shared__ unsigned s_ticket[2];
    __shared__ long long s_excl;
    __shared__ unsigned s_claim;  // warps past their tile's physics, all tiles so far
    __shared__ long long s_tmp[kWarps];
    __shared__ BlockStats bs;
    __shared__ __align__(16) Problem s_prob;        // batch: the problem of the current tile
    __shared__ long long s_off[kMaxProblems + 1];   // tickets of problems 0..b
    __shared__ int s_tl[kMaxProblems], s_tg[kMaxProblems];
    __shared__ ProbCounts s_pc;
    __shared__ int s_last;
    __shared__ Pending s_pq[kStashBufs];
    __shared__ unsigned short s_map[kStashBufs][kMapEntries];

    const int tid = threadIdx.x;
    // Tickets.  A tile must belong to a running block (its successors' look-
    // backs wait on it).  A single problem on the mixed path is launched
    // cooperatively (launch_step): every block is resident for the whole
    // launch, so block b takes tile b at entry and later tickets come from
    // the counter, offset by the grid; no block queues on the contended
    // counter before its first tile.  The FP64 path and batches take every
    // ticket from the counter, so a tile belongs to a block only once that
    // block runs (a batch's launches are captured in graphs next to other
    // streams' kernels; the FP64 path's one-launch-a-step runs of small
    // problems, 4096 e- on 608 blocks, took 75 -> 108 us a step when
    // launched cooperatively); the first atomic overlaps the reads of the
    // live counts below.  A block whose ticket is past the last tile leaves
    // without work.
    constexpr bool kFixedFirst = !BATCH && PREC != kFP64;
    const unsigned tbase = kFixedFirst ? gridDim.x : 0u;
    if (tid == 0) s_ticket[0] = kFixedFirst ? blockIdx.x : atomicAdd(&a.ctl->ticket, 1u);
    const int np = BATCH ? a.n_problems : 1;
    const Problem *table = BATCH ? a.problems : &a.single;
    const unsigned epoch = __ldcg(&a.ctl->epoch);
    clear_stats(bs);
    if (tid == 0) s_claim = 0u;  // visible after the barrier below
    // the lepton tiles' rate tables, staged from the start by a thread of
    // another warp than the ticket's and the counts' (their copy overlaps
    // the live counts' reads and the first tile's loads, gather and push)
    if (tid == 32) stage_rate_tables<PREC>(a, sm, &s_bar[0]);
    double *const stash_block = a.stash + (size_t)blockIdx.x * kStashBufs * kStashFields * kTile;
    // tiles of this block with stashed appends: numbers q_lo..q-1 are not
    // yet written (uniform over the block)
    unsigned q = 0, q_lo = 0;

    // tiles of every problem, and the ticket offset of each (threads 64 on:
    // not the ticket's or the tables' warp)
    bool bad = false;
    for (int b = (tid + kTile - 64) % kTile; b < np; b += kTile) {
        const ProbCounts c = problem_counts(table[b]);
        s_off[b] = c.tiles_l + c.tiles_g;
        s_tl[b] = (int)c.tiles_l;
        s_tg[b] = (int)c.tiles_g;
        bad |= c.bad;
        if (!BATCH) s_pc = c;
    }
    if (bad && blockIdx.x == 0) raise_status(a.status, QP_ERR_INVALID_ARG);
    __syncthreads();
    if (BATCH) scan_offsets(s_off, np, s_tmp);  // s_off[b] = tickets of problems 0..b
    const long long n_tickets = s_off[np - 1];

    bool lep_loaded = false, ph_loaded = false;
    int cur = BATCH ? -1 : 0;
    for (int buf = 0;; buf ^= 1) {
        const long long t = s_ticket[buf];
        const bool more = t < n_tickets;
        // fetch the next ticket while this tile runs, when another tile is
        // likely left for this block (else the atomic only adds contention)
        const bool early = t + (long long)gridDim.x < n_tickets;
        if (early && tid == 0) s_ticket[buf ^ 1] = tbase + atomicAdd(&a.ctl->ticket, 1u);
        int b = 0;
        if (BATCH && more) {
            // the problem of ticket t: the first b with s_off[b] > t
            int lo = 0, hi = np - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (s_off[mid] > t)
                    hi = mid;
                else
                    lo = mid + 1;
            }
            b = lo;
        }
        const bool leave = !more || (BATCH && b != cur);  // the current problem's last tile is done
        // ---- stashed appends: all of them when the block leaves its problem
        // (during a problem the first warp past a tile's physics flushes the
        // oldest one: see before_scan below; this loop then finds no full ring)
        {
            const Problem &F = BATCH ? s_prob : a.single;
            while (q_lo != q && (leave || q - q_lo == (unsigned)kStashBufs)) {
                const int ob = (int)(q_lo % kStashBufs);
                flush_pending(a, F, s_pq[ob], epoch, &s_excl, bs,
                              stash_block + (size_t)ob * kStashFields * kTile, s_map[ob]);
                ++q_lo;
            }
            if (leave && cur >= 0) {
                flush_stats(bs, a, F);
                __syncthreads();
                clear_stats(bs);
            }
        }
        if (!more) break;
        if (BATCH && b != cur) {
            // copy the problem descriptor to shared memory
            const int *src = reinterpret_cast<const int *>(table + b);
            int *dst = reinterpret_cast<int *>(&s_prob);
            for (int k = tid; k < (int)(sizeof(Problem) / sizeof(int)); k += kTile)
                dst[k] = src[k];
            __syncthreads();
            if (tid == 0) {
                s_pc = problem_counts(s_prob);
                set_time(s_prob, *((volatile long long *)s_prob.step_ctr));
            }
            __syncthreads();
            cur = b;
        }
        const Problem &P = BATCH ? s_prob : a.single;
        const ProbCounts pc = s_pc;                         // in registers for the tile
        const long long lt = t - (b > 0 ? s_off[b - 1] : 0);  // tile within the problem
        // this tile's stash buffer, append map and record: the oldest
        // pending tile is at most kStashBufs - 1 numbers back
        const int sb = (int)(q % kStashBufs);
        double *st = stash_block + (size_t)sb * kStashFields * kTile;
        bool stashed = true;
        // Right before a tile's own scan, every warp claims once (so each
        // tile adds kWarps to s_claim): the first warp past its physics
        // (claim a multiple of kWarps) flushes the oldest stashed tile, two
        // tiles back, when two are pending, while the others still compute.
        // Its buffers are reused only after the closing barrier of this tile.
        // Not on the 2D grid: its single-wave steps have one tile a block
        // (nothing to overlap) and the flush code would spill there.
        constexpr bool kEarlyFlush = FK != QP_FIELD_YEE2D;
        const bool flush_early = kEarlyFlush && q - q_lo == (unsigned)(kStashBufs - 1);
        const int ob = (int)(q_lo % kStashBufs);
        auto before_scan = [&]() {
            if constexpr (!kEarlyFlush) return;
            unsigned c = 0u;
            if ((tid & 31) == 0) c = atomicAdd(&s_claim, 1u);
            c = __shfl_sync(0xFFFFFFFFu, c, 0);
            if (flush_early && c % (unsigned)kWarps == 0u)
                flush_pending_warp(a, P, s_pq[ob], epoch, bs,
                                   stash_block + (size_t)ob * kStashFields * kTile, s_map[ob]);
        };
        if (lt < pc.tiles_l) {
            const int sp = lt < pc.tiles_e ? 0 : 1;
            const int64_t first = (lt - (sp ? pc.tiles_e : 0)) * kTile;
            const int total =
                lepton_tile<PREC, FK, R>(a, P, sm, &s_bar[0], lep_loaded, (unsigned)lt, sp,
                                         first, pc.n[sp], epoch, s_warp, bs, st, s_map[sb],
                                         before_scan);
            if (tid == 0) {
                Pending &r = s_pq[sb];
                r.chain = 0;
                r.last = lt == pc.tiles_l - 1;
                r.sp = sp;
                r.total = total;
                r.tile = (unsigned)lt;
                r.base = pc.n[2];
            }
        } else {
            const unsigned pt = (unsigned)(lt - pc.tiles_l);
            const long long be = pc.n[0], bp = pc.n[1];
            long long room = 0;
            if (P.sp[0].present && P.sp[1].present) {
                room = P.sp[0].cap - be;
                if (P.sp[1].cap - bp < room) room = P.sp[1].cap - bp;
                if (room < 0) room = 0;
            }
            const int total =
                photon_tile<PREC, FK, R>(a, P, sm, &s_bar[1], ph_loaded, pt, pc.n[2], epoch,
                                         s_warp, bs, st, s_map[sb], before_scan);
            stashed = P.pairs != 0;  // without pairs a photon tile appends nothing
            if (tid == 0 && stashed) {
                Pending &r = s_pq[sb];
                r.chain = 1;
                r.last = (long long)pt == pc.tiles_g - 1;
                r.sp = 2;
                r.total = total;
                r.tile = pt;
                r.be = be;
                r.bp = bp;
                r.room = room;
            }
        }
        if (!early && tid == 0) s_ticket[buf ^ 1] = tbase + atomicAdd(&a.ctl->ticket, 1u);
        __syncthreads();  // the record and the next ticket are visible
        if (flush_early) ++q_lo;
        if (stashed) ++q;
    }

    // a block that ran no lepton tile lets the tables' copy land before it
    // leaves
    if (!lep_loaded) wait_tables(&s_bar[0], a);

    // ---- the last block to finish publishes the step of every problem:
    // the last block of each group counts in `done`, the last of those is it
    // The counts are acquire-release atomics: a count releases the block's
    // writes (every thread's: the barrier that closed its last flush orders
    // them before thread 0's count) and the group's last count acquires the
    // group's, so the last block sees every block's pending counts.
    if (tid == 0) {
        const unsigned g = blockIdx.x % kDoneGroups;
        const unsigned in_group = (gridDim.x - 1 - g) / kDoneGroups + 1;
        const unsigned groups = gridDim.x < kDoneGroups ? gridDim.x : kDoneGroups;
        s_last = 0;
        if (atom_add_acq_rel(&a.ctl->grp[g][0], 1u) == in_group - 1) {
            a.ctl->grp[g][0] = 0u;  // every block of the group has counted
            s_last = atom_add_acq_rel(&a.ctl->done, 1u) == groups - 1;
        }
    }
    __syncthreads();
    if (s_last) {
        // thread 0 acquired with its count; the other threads' reads (a
        // batch's problems) follow this fence
        if (BATCH) __threadfence();
        for (int b = tid; b < np; b += kTile) {
            const Problem &Q = table[b];
            if (Q.device_step && *((volatile long long *)Q.left_ctr) <= 0) continue;
            if (Q.device_step) {
                // slots this launch stepped (before the new counts are applied)
                const ProbCounts c = problem_counts(Q);
                *Q.work_ctr += c.n[0] + c.n[1] + c.n[2];
            }
            // the three counts read together, then written
            volatile long long *pend = Q.pending;
            const long long p0 = pend[0], p1 = pend[1], p2 = pend[2];
            if (s_tl[b] > 0 && Q.sp[2].present) *Q.sp[2].n_live = p2;
            if (s_tg[b] > 0 && Q.pairs && Q.sp[0].present && Q.sp[1].present) {
                *Q.sp[0].n_live = p0;
                *Q.sp[1].n_live = p1;
            }
            if (Q.device_step) {
                *Q.step_ctr += 1;
                *Q.left_ctr -= 1;
            }
        }
        __syncthreads();
        // the next launch reads these after this one has ended: no fence
        if (tid == 0) {
            *((volatile unsigned *)&a.ctl->ticket) = 0u;
            *((volatile unsigned *)&a.ctl->done) = 0u;
            *((volatile unsigned *)&a.ctl->epoch) = epoch + 1u;
        }
    }
}

// -------------------------------------------------------------------- fused steps
//
// K steps of every lepton in one launch, the particle held in registers
// from the first step to the last (analytic or fixed fields, pairs off: the
// leptons then never change in number and the photons only move).  The
// physics is lepton_particle, the photon motion photon_move*: the same
// arithmetic as K launches of k_step, so the results are the same bits.
// New photons take provisional indices in arrival order (one atomic a warp
// and step) and are staged there with their order key: step, then emitter
// (tile, lane), then emission index, the slot order of K separate steps.
// The key sort (launch_fused_order) and k_fused_photons put them at those
// slots.  Tiles are one warp.

constexpr int kEmitBits = 3;
static_assert(QP_MAX_EMISSIONS <= (1 << kEmitBits), "emission index bits");

struct FusedArgs {
    StepArgs a;              // a.single: the problem at the window's first step
    int32_t K;               // steps in the window
    int32_t ob;              // bits of the emitter ordinal (tile * 32 + lane) in the key
    long long tiles_e, tiles; // lepton tiles (electron tiles first)
    FusedScratch fs;
    long long *win;          // [3] photons at the window start, stored and staged in it
};

// The append sink of a fused lepton: the state stays in registers, the
// emitted photons are kept for the warp's provisional indices.
struct FusedSink {
    LeptonState &cur;
    double chi_last, kx, ky, kz, ox, oy, oz;
    double gg[QP_MAX_EMISSIONS], tg[QP_MAX_EMISSIONS];
    template <int C>
    __device__ __forceinline__ void put(double v)
    {
        (&cur.x)[C] = v;
    }
    __device__ __forceinline__ void tables() {}
    __device__ __forceinline__ void chi(double c) { chi_last = c; }
    __device__ __forceinline__ void direction(double x, double y, double z)
    {
        kx = x;
        ky = y;
        kz = z;
    }
    __device__ __forceinline__ void photon(int j, double g, double t)
    {
        gg[j] = g;
        tg[j] = t;
    }
    __device__ __forceinline__ void origin(double x, double y, double z)
    {
        ox = x;
        oy = y;
        oz = z;
    }
};

static_assert(offsetof(LeptonState, tau) == 6 * sizeof(double), "LeptonState layout");

// One warp a block, at most 64 registers a thread (32 resident warps an SM).
template <int PREC, int FK>
__global__ void __launch_bounds__(32, 32) k_fused(const __grid_constant__ FusedArgs f)
{
    using R = typename std::conditional<PREC == kFP64, double, float>::type;
    __shared__ __align__(16) Problem sP;
    const int lane = threadIdx.x;
    const StepArgs &a = f.a;
    const R *H, *G;
    if constexpr (PREC == kFP64) {
        H = a.tab.H;
        G = a.tab.Gs;
    } else {
        H = a.tab.Hf;
        G = a.tab.Gsf;
    }
    // photons at the window start; new photons are staged up to the capacity
    // (the key order decides which of them the free slots keep), the rest
    // dropped here
    long long stage_cap = 0;
    {
        const SpeciesDev &Ph = a.single.sp[2];
        long long base = 0;
        if (Ph.present) {
            base = *((volatile long long *)Ph.n_live);
            if (base < 0 || base > Ph.cap) {
                if (lane == 0 && blockIdx.x == 0) raise_status(a.status, QP_ERR_INVALID_ARG);
                base = base < 0 ? 0 : Ph.cap;
            }
            stage_cap = Ph.cap;
        }
        if (blockIdx.x == 0 && lane == 0) f.win[0] = base;
    }
    for (long long tile = blockIdx.x; tile < f.tiles; tile += gridDim.x) {
        {
            const int *src = reinterpret_cast<const int *>(&a.single);
            int *dst = reinterpret_cast<int *>(&sP);
            for (int k = lane; k < (int)(sizeof(Problem) / sizeof(int)); k += 32) dst[k] = src[k];
        }
        __syncwarp();
        const int sp = tile < f.tiles_e ? 0 : 1;
        const SpeciesDev &S = sP.sp[sp];
        const int64_t i = (tile - (sp ? f.tiles_e : 0)) * 32 + lane;
        long long n = *((volatile long long *)S.n_live);
        if (n < 0 || n > S.cap) {
            if (lane == 0) raise_status(a.status, QP_ERR_INVALID_ARG);
            n = n < 0 ? 0 : S.cap;
        }
        const bool active = i < n;
        LeptonState cur{};
        double w = 0.0;
        if (active) {
            cur = {S.x[i], S.y[i], S.z ? S.z[i] : 0.0, S.ux[i], S.uy[i], S.uz[i], S.tau[i]};
            w = S.w[i];
        }
        const unsigned long long ordinal = (unsigned long long)(tile * 32 + lane) << kEmitBits;
        const uint64_t s0 = sP.step;
        unsigned c_emit = 0, c_sub = 0, c_cont = 0, c_sat = 0, c_clamp = 0, c_ph = 0, c_drop = 0;
        double e_sub = 0.0, e_drop = 0.0, chi_last = 0.0;
        for (int k = 0; k < f.K; ++k) {
            if (k > 0) {
                __syncwarp();
                if (lane == 0) set_time(sP, (long long)(s0 + k));
                __syncwarp();
            }
            LeptonOut o{};
            FusedSink sink{cur};
            if (active) {
                const LeptonState in = cur;
                lepton_particle<PREC, FK, R>(a, sP, H, G, sp, S, i, in, o, sink);
                chi_last = sink.chi_last;
            }
            // provisional indices: the warp's total from one atomic, the
            // lanes in order after it
            int inc = o.nph;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xFFFFFFFFu, inc, d);
                if (lane >= d) inc += y;
            }
            const int tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
            if (tot) {
                unsigned long long first = 0ull;
                if (lane == 31)
                    first = atomicAdd((unsigned long long *)f.fs.alloc, (unsigned long long)tot);
                first = __shfl_sync(0xFFFFFFFFu, first, 31) + (unsigned long long)(inc - o.nph);
                const unsigned long long kkey =
                    ((unsigned long long)k << (f.ob + kEmitBits)) | ordinal;
                for (int j = 0; j < o.nph; ++j) {
                    const long long pa = (long long)first + j;
                    const double g = sink.gg[j];
                    if (pa < stage_cap) {
                        f.fs.stage[0][pa] = sink.ox;
                        f.fs.stage[1][pa] = sink.oy;
                        f.fs.stage[2][pa] = sink.oz;
                        f.fs.stage[3][pa] = g * sink.kx;
                        f.fs.stage[4][pa] = g * sink.ky;
                        f.fs.stage[5][pa] = g * sink.kz;
                        f.fs.stage[6][pa] = sink.tg[j];
                        f.fs.stage[7][pa] = w;
                        f.fs.rkeys[pa] = kkey | (unsigned long long)j;
                        f.fs.moves_new[pa] = (unsigned short)(f.K - 1 - k);
                        ++c_ph;
                    } else {
                        ++c_drop;
                        e_drop += w * g;
                    }
                }
            }
            c_emit += (unsigned)o.n_emit;
            c_sub += (unsigned)o.n_sub;
            if (o.n_sub) e_sub += w * o.e_sub;
            c_cont += o.cont;
            c_sat += o.sat;
            c_clamp += o.clamped;
        }
        if (active) {
            S.x[i] = cur.x;
            S.y[i] = cur.y;
            if (S.z) S.z[i] = cur.z;
            S.ux[i] = cur.ux;
            S.uy[i] = cur.uy;
            S.uz[i] = cur.uz;
            S.tau[i] = cur.tau;
            if (S.chi) S.chi[i] = chi_last;
            if (c_emit && S.nemit) S.nemit[i] += (int)c_emit;
        }
        const unsigned t_emit = __reduce_add_sync(0xFFFFFFFFu, c_emit);
        const unsigned t_sub = __reduce_add_sync(0xFFFFFFFFu, c_sub);
        const unsigned t_cont = __reduce_add_sync(0xFFFFFFFFu, c_cont);
        const unsigned t_sat = __reduce_add_sync(0xFFFFFFFFu, c_sat);
        const unsigned t_clamp = __reduce_add_sync(0xFFFFFFFFu, c_clamp);
        const unsigned t_ph = __reduce_add_sync(0xFFFFFFFFu, c_ph);
        const unsigned t_drop = __reduce_add_sync(0xFFFFFFFFu, c_drop);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            e_sub += __shfl_xor_sync(0xFFFFFFFFu, e_sub, d);
            e_drop += __shfl_xor_sync(0xFFFFFFFFu, e_drop, d);
        }
        if (lane == 0) {
            DevStats &st = a.stats[S.slot_stats];
            if (t_emit) atomicAdd(&st.n_emit, (unsigned long long)t_emit);
            if (t_sub) atomicAdd(&st.n_subthreshold, (unsigned long long)t_sub);
            if (t_cont) atomicAdd(&st.n_continuous, (unsigned long long)t_cont);
            if (t_sat) atomicAdd(&st.n_saturated, (unsigned long long)t_sat);
            if (t_clamp) {
                atomicAdd(&st.n_clamped, (unsigned long long)t_clamp);
                raise_status(a.status, QP_WARN_TABLE_CLAMPED);
            }
            if (t_ph) atomicAdd(&st.n_photon, (unsigned long long)t_ph);
            if (t_drop) atomicAdd(&st.n_photon_drop, (unsigned long long)t_drop);
            if (e_sub != 0.0) atomicAdd(&st.e_subthreshold, e_sub);
            if (e_drop != 0.0) atomicAdd(&st.e_dropped, e_drop);
        }
        __syncwarp();
    }
}

// The photons of the window moved ballistically: those that existed at its
// start over its K steps in place (decayed ones, tau < 0, stay), the new
// ones gathered from the staging in key order into the slots after them and
// moved over the steps left after the step that emitted them.  One thread
// a slot; the new live count.  Launched for any photon capacity > 0.
template <int PREC>
__global__ void __launch_bounds__(256) k_fused_photons(const __grid_constant__ FusedArgs f)
{
    const Problem &P = f.a.single;
    const SpeciesDev &Ph = P.sp[2];
    const long long base = f.win[0], n = base + f.win[1];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        int moves;
        double x, y, z, ux, uy, uz, tau;
        long long pa = -1;
        if (i < base) {
            moves = f.K;
            tau = Ph.tau[i];
            if (!(tau >= 0.0)) continue;
            x = Ph.x[i];
            y = Ph.y[i];
            z = Ph.z ? Ph.z[i] : 0.0;
            ux = Ph.ux[i];
            uy = Ph.uy[i];
            uz = Ph.uz[i];
        } else {
            pa = f.fs.order[i - base];
            moves = f.fs.moves_new[pa];
            x = f.fs.stage[0][pa];
            y = f.fs.stage[1][pa];
            z = f.fs.stage[2][pa];
            ux = f.fs.stage[3][pa];
            uy = f.fs.stage[4][pa];
            uz = f.fs.stage[5][pa];
            tau = f.fs.stage[6][pa];
        }
        if (moves > 0 && tau >= 0.0) {
            if constexpr (PREC == kFP64) {
                const double g = photon_speed64(ux, uy, uz);
                if (g > 0.0)
                    for (int m = 0; m < moves; ++m) {
                        x = photon_move64(x, ux, g, P.dt);
                        y = photon_move64(y, uy, g, P.dt);
                        z = photon_move64(z, uz, g, P.dt);
                    }
            } else {
                const float fx = hi_d(ux), fy = hi_d(uy), fz = hi_d(uz);
                const float g = photon_speed32(fx, fy, fz);
                if (g > 0.0f) {
                    const float c = P.mc.dt / g;
                    for (int m = 0; m < moves; ++m) {
                        x = photon_move32(x, fx, c);
                        y = photon_move32(y, fy, c);
                        z = photon_move32(z, fz, c);
                    }
                }
            }
        }
        Ph.x[i] = x;
        Ph.y[i] = y;
        if (Ph.z) Ph.z[i] = z;
        if (pa >= 0) {
            Ph.ux[i] = ux;
            Ph.uy[i] = uy;
            Ph.uz[i] = uz;
            Ph.tau[i] = tau;
            Ph.w[i] = f.fs.stage[7][pa];
            if (Ph.chi) Ph.chi[i] = 0.0;
            if (Ph.nemit) Ph.nemit[i] = 0;
        }
    }
    // staged photons past the free slots: dropped, in key order, on the
    // counters of the species that emitted them
    const long long staged = f.win[2];
    for (long long r = f.win[1] + (long long)blockIdx.x * blockDim.x + threadIdx.x; r < staged;
         r += stride) {
        const long long pa = f.fs.order[r];
        const unsigned long long tile =
            (f.fs.sorted_keys[r] >> kEmitBits & ((1ull << f.ob) - 1ull)) >> 5;
        const int sp = tile < (unsigned long long)f.tiles_e ? 0 : 1;
        const double ux = f.fs.stage[3][pa], uy = f.fs.stage[4][pa], uz = f.fs.stage[5][pa];
        DevStats &st = f.a.stats[P.sp[sp].slot_stats];
        atomicAdd(&st.n_photon, (unsigned long long)-1ll);
        atomicAdd(&st.n_photon_drop, 1ull);
        atomicAdd(&st.e_dropped, f.fs.stage[7][pa] * sqrt(ux * ux + uy * uy + uz * uz));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && Ph.present) *Ph.n_live = n;
}

template <int PREC>
const void *fused_kernel_of(int fk)
{
    switch (fk) {
    case QP_FIELD_NONE: return (const void *)k_fused<PREC, QP_FIELD_NONE>;
    case QP_FIELD_PLANE: return (const void *)k_fused<PREC, QP_FIELD_PLANE>;
    case QP_FIELD_GAUSSIAN: return (const void *)k_fused<PREC, QP_FIELD_GAUSSIAN>;
    case QP_FIELD_YEE2D: return (const void *)k_fused<PREC, QP_FIELD_YEE2D>;
    case QP_FIELD_UNIFORM_B: return (const void *)k_fused<PREC, QP_FIELD_UNIFORM_B>;
    default: return nullptr;
    }
}

template <int PREC, bool BATCH>
const void *step_kernel_of(int fk)
{
    switch (fk) {
    case QP_FIELD_NONE: return (const void *)k_step<PREC, QP_FIELD_NONE, BATCH>;
    case QP_FIELD_PLANE: return (const void *)k_step<PREC, QP_FIELD_PLANE, BATCH>;
    case QP_FIELD_GAUSSIAN: return (const void *)k_step<PREC, QP_FIELD_GAUSSIAN, BATCH>;
    case QP_FIELD_YEE2D: return (const void *)k_step<PREC, QP_FIELD_YEE2D, BATCH>;
    case QP_FIELD_UNIFORM_B: return (const void *)k_step<PREC, QP_FIELD_UNIFORM_B, BATCH>;
    default: return nullptr;
    }
}

}  // namespace
}  // namespace qp
