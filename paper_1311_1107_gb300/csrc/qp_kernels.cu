// Kernels of libqedpic (sm_103a).
//
// One QED particle step is three launches on the caller's stream:
//   k_step_begin  snapshot the live counts, reset the two append chains;
//   k_lepton      electrons then positrons (one tile space, one chain):
//                 gather, Boris, chi_e, Sokolov or optical depth + emission,
//                 position update, ordered append of the new photons;
//   k_photon      photons alive at the start of the step: chi_gamma, pair
//                 optical depth, decay into an ordered e-/e+ append, motion.
// The kernels are persistent: a block takes tiles of 256 particles from an
// atomic ticket, so tile order is start order and the decoupled look-back
// that orders the appends only ever waits on tiles already being processed.
#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "qp_device.cuh"
#include "qp_kernels.h"

namespace qp {

namespace {

constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagPre = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long *p)
{
    return *((const volatile unsigned long long *)p);
}

// Exclusive prefix of this tile in its chain, computed by one full warp
// (decoupled look-back with a 32-tile window): lane l inspects tile
// base - l; the window is consumed up to the nearest tile that published its
// inclusive prefix, summing the aggregates in between.  Waits are bounded by
// spin_limit; on time-out the status is raised and the prefix is taken as
// what was summed so far (the output is then wrong, the status says so, and
// the kernel still terminates).  Returns the prefix in every lane.
__device__ long long chain_prefix(const ChainDev &ch, unsigned tile, long long aggregate,
                                  unsigned spin_limit, int *status)
{
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) atomicExch(ch.status, kFlagPre | (unsigned long long)aggregate);
        return 0;
    }
    if (lane == 0) atomicExch(ch.status + tile, kFlagAgg | (unsigned long long)aggregate);
    long long excl = 0;
    long long base = (long long)tile - 1;
    unsigned spins = 0;
    for (;;) {
        const long long idx = base - lane;
        // before tile 0 the chain is complete: read as "prefix 0"
        const unsigned long long w = idx >= 0 ? ld_volatile(ch.status + idx) : kFlagPre;
        const unsigned long long flag = w & ~kValMask;
        const unsigned pre = __ballot_sync(0xFFFFFFFFu, flag == kFlagPre);
        const unsigned empty = __ballot_sync(0xFFFFFFFFu, flag == 0ull);
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
    if (lane == 0) atomicExch(ch.status + tile, kFlagPre | (unsigned long long)(excl + aggregate));
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

// Counters kept in shared memory per block, per species (0, 1 or 2), and
// flushed with one atomic per counter at the end of the kernel.
struct BlockStats {
    unsigned long long c[2][9];
    double e[2][2];
};
enum { cEmit, cPhoton, cPhotonDrop, cSub, cPair, cPairDrop, cSat, cClamp, cCont };

__device__ __forceinline__ void warp_count(unsigned long long *ctr, bool pred)
{
    const unsigned m = __ballot_sync(0xFFFFFFFFu, pred);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(ctr, (unsigned long long)__popc(m));
}

__device__ void flush_stats(const BlockStats &bs, DevStats *const *dst, int nsp)
{
    __syncthreads();
    const int t = threadIdx.x;
    if (t < nsp * 9) {
        const int s = t / 9, k = t % 9;
        if (bs.c[s][k]) atomicAdd(&dst[s]->n_emit + k, bs.c[s][k]);
    } else if (t >= 64 && t < 64 + nsp * 2) {
        const int s = (t - 64) / 2, k = (t - 64) % 2;
        if (bs.e[s][k] != 0.0) atomicAdd(&dst[s]->e_subthreshold + k, bs.e[s][k]);
    }
}

__device__ __forceinline__ void clear_stats(BlockStats &bs)
{
    const int t = threadIdx.x;
    if (t < 18) (&bs.c[0][0])[t] = 0ull;
    if (t < 4) (&bs.e[0][0])[t] = 0.0;
}

}  // namespace

// -------------------------------------------------------------------- step begin

__global__ void k_step_begin(const __grid_constant__ StepArgs a)
{
    // live counts come from caller memory: clamp them to [0, capacity] so a
    // bad counter can never index outside the buffers, and report it
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
    const int64_t lep_tiles = (n[0] + kTile - 1) / kTile + (n[1] + kTile - 1) / kTile;
    const int64_t ph_tiles = (n[2] + kTile - 1) / kTile;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < lep_tiles; i += stride)
        a.lep.status[i] = 0ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ph_tiles; i += stride)
        a.pho.status[i] = 0ull;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (bad) raise_status(a.status, QP_ERR_INVALID_ARG);
        for (int s = 0; s < 3; ++s) a.n_start[s] = n[s];
        *a.lep.ticket = 0u;
        *a.pho.ticket = 0u;
    }
}

// -------------------------------------------------------------------- leptons

template <int PREC, int FK>
__global__ void __launch_bounds__(kTile) k_lepton(const __grid_constant__ StepArgs a)
{
    using R = typename std::conditional<PREC == kFP64, double, float>::type;
    __shared__ __align__(16) R s_H[kNRatePad];
    __shared__ __align__(16) R s_G[kNRatePad];
    __shared__ __align__(8) unsigned long long s_bar;   // TMA completion of the tables
    __shared__ double s_gg[QP_MAX_EMISSIONS][kTile];   // stashed photon energies
    __shared__ double s_tg[QP_MAX_EMISSIONS][kTile];   // and their optical depths
    __shared__ int s_warp[kWarps];
    __shared__ unsigned s_ticket;
    __shared__ long long s_excl;
    __shared__ BlockStats bs;

    const int tid = threadIdx.x;
    clear_stats(bs);
    const int64_t n_e = a.n_start[0], n_p = a.n_start[1];
    const int64_t tiles_e = (n_e + kTile - 1) / kTile;
    const int64_t n_tiles = tiles_e + (n_p + kTile - 1) / kTile;
    const SpeciesDev &Ph = a.sp[2];
    const bool photons = Ph.present != 0;
    const int64_t ph_base = a.n_start[2];
    bool loaded = false;
    // blocks beyond the tile count leave before touching the ticket
    if ((int64_t)blockIdx.x >= n_tiles) return;

    for (;;) {
        if (tid == 0) s_ticket = atomicAdd(a.lep.ticket, 1u);
        __syncthreads();
        const unsigned tile = s_ticket;
        if ((int64_t)tile >= n_tiles) break;
        if (!loaded) {
            // stage the rate tables with one TMA bulk copy each; the copy
            // overlaps the particle loads, gather and push below
            if (tid == 0) {
                const unsigned bytes = kNRatePad * sizeof(R);
                mbar_init(&s_bar, 1);
                mbar_expect_tx(&s_bar, 2 * bytes);
                if constexpr (PREC == kFP64) {
                    bulk_g2s(s_H, a.tab.H, bytes, &s_bar);
                    bulk_g2s(s_G, a.tab.Gs, bytes, &s_bar);
                } else {
                    bulk_g2s(s_H, a.tab.Hf, bytes, &s_bar);
                    bulk_g2s(s_G, a.tab.Gsf, bytes, &s_bar);
                }
            }
            __syncthreads();
        }
        const int sp = (int64_t)tile < tiles_e ? 0 : 1;
        const SpeciesDev &S = a.sp[sp];
        const int64_t first = ((int64_t)tile - (sp ? tiles_e : 0)) * kTile;
        const int64_t n = sp ? n_p : n_e;
        const int64_t i = first + tid;
        const bool active = i < n;

        int nph = 0;
        double x0 = 0, y0 = 0, z0 = 0, kx = 0, ky = 0, kz = 0, wgt = 0;
        bool cont = false, sat = false, clamped = false;
        int n_emit = 0, n_sub = 0;
        double e_sub = 0.0;

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
            if (!loaded) {
                // tables are needed from here on
                if (!mbar_wait_bounded(&s_bar, 0, a.spin_limit)) {
                    raise_status(a.status, QP_ERR_TIMEOUT);
                    (void)mbar_wait_bounded(&s_bar, 0, a.spin_limit);
                }
            }
            const double inv_aS = 1.0 / a.a_S;
            double chi = chi_e64(Ex, Ey, Ez, Bx, By, Bz, ux, uy, uz, gam, inv_aS);
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
                    const double prad = a.C_rate * rate64<1>(s_G, chi, clamped);
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
                    const float prad = (float)a.C_rate * rate32<1>(s_G, (float)chi, clamped);
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
                        const double H = rate64<0>(s_H, chi, clamped);
                        wdt = a.C_rate * H / gam * dt;
                        dtau = wdt * r;
                    } else {
                        const float H = rate32<0>(s_H, (float)chi, clamped);
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
                    if constexpr (PREC == kFP64)
                        ufrac = sample_cdf<double>(a.tab.Cg, chi, xi_p, kSgMin, kSgSpan, true,
                                                   clamped);
                    else
                        ufrac = sample_cdf<float>(a.tab.Cgf, (float)chi, (float)xi_p, kSgMin,
                                                  kSgSpan, true, clamped);
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
                        s_gg[nph][tid] = gg;
                        s_tg[nph][tid] = -log(u53(rp.x, rp.y));
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
                    chi = chi_e64(Ex, Ey, Ez, Bx, By, Bz, ux, uy, uz, gam, inv_aS);
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

        if (!loaded) {
            // threads without a particle also wait, so the block never leaves
            // (or reuses the tables) with the copy in flight
            if (!active && !mbar_wait_bounded(&s_bar, 0, a.spin_limit)) {
                raise_status(a.status, QP_ERR_TIMEOUT);
                (void)mbar_wait_bounded(&s_bar, 0, a.spin_limit);
            }
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
            const long long e = chain_prefix(a.lep, tile, tile_total, a.spin_limit, a.status);
            if (tid == 0) s_excl = e;
        }
        __syncthreads();
        if (nph) {
            const int64_t base = ph_base + s_excl + local;
            int stored = 0, dropped = 0;
            double e_drop = 0.0;
            for (int j = 0; j < nph; ++j) {
                const int64_t slot = base + j;
                const double gg = s_gg[j][tid];
                if (photons && slot < Ph.cap) {
                    Ph.x[slot] = x0;
                    Ph.y[slot] = y0;
                    if (Ph.z) Ph.z[slot] = z0;
                    Ph.ux[slot] = gg * kx;
                    Ph.uy[slot] = gg * ky;
                    Ph.uz[slot] = gg * kz;
                    Ph.tau[slot] = s_tg[j][tid];
                    Ph.w[slot] = wgt;
                    if (Ph.chi) Ph.chi[slot] = 0.0;
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
        if ((int64_t)tile == n_tiles - 1 && tid == 0 && photons) {
            const int64_t tot = ph_base + s_excl + tile_total;
            *Ph.n_live = tot < Ph.cap ? tot : Ph.cap;
            if (tot > Ph.cap) raise_status(a.status, QP_WARN_BUFFER_FULL);
        }
        if ((int64_t)tile == n_tiles - 1 && tid == 0 && !photons && s_excl + tile_total > 0)
            raise_status(a.status, QP_WARN_BUFFER_FULL);
        __syncthreads();
    }
    // an absent species has all-zero counters, so its slot is never written
    DevStats *dst[2] = {a.stats + (a.sp[0].present ? a.sp[0].slot_stats : 0),
                        a.stats + (a.sp[1].present ? a.sp[1].slot_stats : 0)};
    flush_stats(bs, dst, 2);
    if (tid == 0 && (bs.c[0][cClamp] | bs.c[1][cClamp])) raise_status(a.status, QP_WARN_TABLE_CLAMPED);
}

// -------------------------------------------------------------------- photons

template <int PREC, int FK>
__global__ void __launch_bounds__(kTile) k_photon(const __grid_constant__ StepArgs a)
{
    using R = typename std::conditional<PREC == kFP64, double, float>::type;
    __shared__ __align__(16) R s_T[kNRatePad];
    __shared__ __align__(8) unsigned long long s_bar;
    __shared__ int s_warp[kWarps];
    __shared__ unsigned s_ticket;
    __shared__ long long s_excl;
    __shared__ BlockStats bs;

    const int tid = threadIdx.x;
    clear_stats(bs);
    const SpeciesDev &Ph = a.sp[2], &El = a.sp[0], &Po = a.sp[1];
    const int64_t n = a.n_start[2];
    const int64_t n_tiles = (n + kTile - 1) / kTile;
    const int64_t be = a.n_start[0], bp = a.n_start[1];
    const bool leptons = El.present && Po.present;
    int64_t room = 0;
    if (leptons) {
        room = El.cap - be;
        if (Po.cap - bp < room) room = Po.cap - bp;
        if (room < 0) room = 0;
    }
    const bool pairs = a.pairs != 0;
    bool loaded = false;
    if ((int64_t)blockIdx.x >= n_tiles) return;

    for (;;) {
        if (tid == 0) s_ticket = atomicAdd(a.pho.ticket, 1u);
        __syncthreads();
        const unsigned tile = s_ticket;
        if ((int64_t)tile >= n_tiles) break;
        if (pairs && !loaded) {
            if (tid == 0) {
                const unsigned bytes = kNRatePad * sizeof(R);
                mbar_init(&s_bar, 1);
                mbar_expect_tx(&s_bar, bytes);
                if constexpr (PREC == kFP64)
                    bulk_g2s(s_T, a.tab.Ts, bytes, &s_bar);
                else
                    bulk_g2s(s_T, a.tab.Tsf, bytes, &s_bar);
            }
            __syncthreads();
            if (!mbar_wait_bounded(&s_bar, 0, a.spin_limit)) {
                raise_status(a.status, QP_ERR_TIMEOUT);
                (void)mbar_wait_bounded(&s_bar, 0, a.spin_limit);
            }
            loaded = true;
        }
        const int64_t i = (int64_t)tile * kTile + tid;
        int npair = 0;
        double px = 0, py = 0, pz = 0, gux = 0, guy = 0, guz = 0, wg = 0, v = 0, tm = 0, tp = 0;
        bool clamped = false;

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
                        const double Tr = rate64<2>(s_T, chi, clamped);
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
                        const float Tr = rate32<2>(s_T, cf, clamped);
                        dtau = (double)((float)a.C_rate * Tr / (float)g * (float)dt);
                    }
                    if (Ph.chi) Ph.chi[i] = chi;
                    if (dtau > 0.0 && !(tau > dtau)) {
                        // ---- pair creation at the photon position
                        const uint4 r1 = draw(a.seed, QP_PHOTON, kRngPair, i, a.step, 0);
                        const uint4 r2 = draw(a.seed, QP_PHOTON, kRngPairPos, i, a.step, 0);
                        if constexpr (PREC == kFP64)
                            v = sample_cdf<double>(a.tab.Cp, chi, u53(r1.x, r1.y), kSpMin, kSpSpan,
                                                   false, clamped);
                        else
                            v = sample_cdf<float>(a.tab.Cpf, (float)chi, (float)u53(r1.x, r1.y),
                                                  kSpMin, kSpSpan, false, clamped);
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
        warp_count(&bs.c[0][cClamp], clamped);
        warp_count(&bs.c[0][cPair], npair != 0);

        if (pairs) {
            int tile_total;
            const int local = block_scan(npair, s_warp, &tile_total);
            if (tid < 32) {
                const long long e = chain_prefix(a.pho, tile, tile_total, a.spin_limit, a.status);
                if (tid == 0) s_excl = e;
            }
            __syncthreads();
            if (npair) {
                const int64_t ord = s_excl + local;
                if (leptons && ord < room) {
                    const int64_t se = be + ord, spo = bp + ord;
                    const double om = 1.0 - v;
                    El.x[se] = px;
                    El.y[se] = py;
                    if (El.z) El.z[se] = pz;
                    El.ux[se] = v * gux;
                    El.uy[se] = v * guy;
                    El.uz[se] = v * guz;
                    El.tau[se] = tm;
                    El.w[se] = wg;
                    if (El.chi) El.chi[se] = 0.0;
                    Po.x[spo] = px;
                    Po.y[spo] = py;
                    if (Po.z) Po.z[spo] = pz;
                    Po.ux[spo] = om * gux;
                    Po.uy[spo] = om * guy;
                    Po.uz[spo] = om * guz;
                    Po.tau[spo] = tp;
                    Po.w[spo] = wg;
                    if (Po.chi) Po.chi[spo] = 0.0;
                } else {
                    atomicAdd(&bs.c[0][cPairDrop], 1ull);
                    atomicAdd(&bs.e[0][1], wg * sqrt(gux * gux + guy * guy + guz * guz));
                }
            }
            if ((int64_t)tile == n_tiles - 1 && tid == 0) {
                const int64_t tot = s_excl + tile_total;
                const int64_t add = tot < room ? tot : room;
                if (leptons) {
                    *El.n_live = be + add;
                    *Po.n_live = bp + add;
                }
                if (tot > add) raise_status(a.status, QP_WARN_BUFFER_FULL);
            }
        }
        __syncthreads();
    }
    DevStats *dst[1] = {a.stats + Ph.slot_stats};
    flush_stats(bs, dst, 1);
    if (tid == 0 && bs.c[0][cClamp]) raise_status(a.status, QP_WARN_TABLE_CLAMPED);
}

// -------------------------------------------------------------------- wait self-test

// Tile 1 of a chain whose tile 0 never publishes: the bounded wait must
// give up, raise QP_ERR_TIMEOUT and return.
__global__ void k_wait_selftest(ChainDev ch, unsigned spin_limit, int *status)
{
    if (threadIdx.x < 32 && blockIdx.x == 0) {
        if (threadIdx.x == 0) ch.status[0] = 0ull;
        __syncwarp();
        (void)chain_prefix(ch, 1u, 0, spin_limit, status);
    }
}

cudaError_t launch_wait_selftest(const ChainDev &ch, unsigned spin_limit, int *status,
                                 cudaStream_t st)
{
    k_wait_selftest<<<1, 32, 0, st>>>(ch, spin_limit, status);
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
constexpr int kDiagScalars = 8;  // n_alive, weight, energy, px, py, pz, wchi, wchi_norm

__global__ void __launch_bounds__(kTile) k_diag_partial(SpeciesDev S, int is_photon,
                                                       double *partials)
{
    __shared__ double s_red[kDiagScalars][kTile];
    __shared__ int s_bin[kTile];
    __shared__ double s_w[kTile];
    const int tid = threadIdx.x;
    int64_t n = *S.n_live;
    n = n < 0 ? 0 : (n > S.cap ? S.cap : n);
    double acc[kDiagScalars] = {0, 0, 0, 0, 0, 0, 0, 0};
    double hist = 0.0;  // thread tid < QP_HIST_BINS owns bin tid
    const double bin_scale = QP_HIST_BINS / (QP_HIST_LOG10_MAX - QP_HIST_LOG10_MIN);
    for (int64_t base = (int64_t)blockIdx.x * kTile; base < n; base += (int64_t)gridDim.x * kTile) {
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
            for (int k = 0; k < kTile; ++k)
                if (s_bin[k] == tid) hist += s_w[k];
        __syncthreads();
    }
    acc[7] = 0.0;
#pragma unroll
    for (int k = 0; k < kDiagScalars; ++k) s_red[k][tid] = acc[k];
    __syncthreads();
    for (int h = kTile / 2; h > 0; h >>= 1) {
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

template <int PREC, int FK>
static cudaError_t launch_one(const StepArgs &a, bool photon, int grid, cudaStream_t st)
{
    if (photon)
        k_photon<PREC, FK><<<grid, kTile, 0, st>>>(a);
    else
        k_lepton<PREC, FK><<<grid, kTile, 0, st>>>(a);
    return cudaGetLastError();
}

template <int PREC>
static cudaError_t dispatch_field(const StepArgs &a, bool photon, int grid, cudaStream_t st)
{
    switch (a.f.kind) {
    case QP_FIELD_NONE: return launch_one<PREC, QP_FIELD_NONE>(a, photon, grid, st);
    case QP_FIELD_PLANE: return launch_one<PREC, QP_FIELD_PLANE>(a, photon, grid, st);
    case QP_FIELD_GAUSSIAN: return launch_one<PREC, QP_FIELD_GAUSSIAN>(a, photon, grid, st);
    case QP_FIELD_YEE2D: return launch_one<PREC, QP_FIELD_YEE2D>(a, photon, grid, st);
    case QP_FIELD_UNIFORM_B: return launch_one<PREC, QP_FIELD_UNIFORM_B>(a, photon, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step_begin(const StepArgs &a, int grid, cudaStream_t st)
{
    k_step_begin<<<grid, kTile, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_species_kernel(const StepArgs &a, int precision, bool photon, int grid,
                                  cudaStream_t st)
{
    if (precision == QP_MIXED) return dispatch_field<kMixed>(a, photon, grid, st);
    return dispatch_field<kFP64>(a, photon, grid, st);
}

cudaError_t launch_init_tau(double *tau, int64_t first, int64_t count, uint64_t seed, int species,
                            cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    int64_t blocks = (count + kTile - 1) / kTile;
    if (blocks > 4096) blocks = 4096;
    k_init_tau<<<(int)blocks, kTile, 0, st>>>(tau, first, count, seed, species);
    return cudaGetLastError();
}

cudaError_t launch_diag(const SpeciesDev &S, int is_photon, double *partials, int nblocks,
                        double *out, cudaStream_t st)
{
    k_diag_partial<<<nblocks, kTile, 0, st>>>(S, is_photon, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_diag_final<<<1, 128, 0, st>>>(partials, nblocks, out);
    return cudaGetLastError();
}

// Occupancy of the persistent kernels (blocks per SM), for grid sizing.
template <int PREC>
static const void *step_kernel(bool photon, int fk)
{
    switch (fk) {
    case QP_FIELD_NONE:
        return photon ? (const void *)k_photon<PREC, QP_FIELD_NONE> : (const void *)k_lepton<PREC, QP_FIELD_NONE>;
    case QP_FIELD_PLANE:
        return photon ? (const void *)k_photon<PREC, QP_FIELD_PLANE> : (const void *)k_lepton<PREC, QP_FIELD_PLANE>;
    case QP_FIELD_GAUSSIAN:
        return photon ? (const void *)k_photon<PREC, QP_FIELD_GAUSSIAN> : (const void *)k_lepton<PREC, QP_FIELD_GAUSSIAN>;
    case QP_FIELD_YEE2D:
        return photon ? (const void *)k_photon<PREC, QP_FIELD_YEE2D> : (const void *)k_lepton<PREC, QP_FIELD_YEE2D>;
    case QP_FIELD_UNIFORM_B:
        return photon ? (const void *)k_photon<PREC, QP_FIELD_UNIFORM_B> : (const void *)k_lepton<PREC, QP_FIELD_UNIFORM_B>;
    default:
        return nullptr;
    }
}

int step_blocks_per_sm(int precision, bool photon, int field_kind)
{
    const void *fn = precision == QP_MIXED ? step_kernel<kMixed>(photon, field_kind)
                                           : step_kernel<kFP64>(photon, field_kind);
    int nb = 0;
    if (!fn || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kTile, 0) != cudaSuccess)
        return 1;
    return nb < 1 ? 1 : nb;
}

}  // namespace qp
