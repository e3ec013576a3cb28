// Compaction and coalescence of super-photons (qp_compact_photons,
// qp_coalesce_photons), and the stable sort of a species by cell
// (qp_sort_species) on the same radix sort.
//
// The paper (section 3, last paragraph) names a coalescence of super-photons
// that conserves energy and momentum on average, without an algorithm.
// Here: the live photons are grouped by (cell of a box grid, log2-energy
// bin, direction bin on the faces of a cube); a group of at least
// min_group photons becomes two photons of half its weight each, at its
// mean energy E/W, with momenta P/W +- d (d perpendicular to P, |P/W|^2 +
// |d|^2 = (E/W)^2) in the plane of P and the group's first photon, at its
// weighted mean position, with fresh optical depths.  Weight, energy and
// momentum of every group are conserved to rounding; both photons stay
// massless.  Decayed photons (tau < 0) are removed; what remains keeps its
// slot order, a merged pair in place of its group's first photon.
//
// Pipeline (one stream, every kernel over the live count read on the
// device, grids of G blocks each owning one contiguous chunk of slots):
//   k_co_prepare   roles (1 alive, 0 decayed) and group keys;
//   radix passes   stable LSD sort of (key, slot), 8 bits a pass:
//                  k_co_hist, k_co_scan_hist, k_co_scatter;
//   k_co_groups    groups (runs of one key) cut into runs of at most
//                  max_group members in slot order; runs of >= min_group
//                  listed;
//   k_co_runs      one thread a run: its momentum checked, roles set (2 at
//                  the first member, 0 at the others);
//   role scan      k_co_chunk_sums, k_co_scan_chunks, k_co_offsets: the
//                  output slot of every survivor in slot order;
//   k_co_kept      survivors copied to the staging arrays;
//   k_co_pairs     merged pairs computed and written to the staging arrays;
//   k_co_copy_back staging -> species, new live count.
// Group sums run in slot order in one thread per run, with the oracle's
// operations in the oracle's order; this unit is compiled without FMA
// contraction, so keys, sums and merged momenta are the oracle's bit for
// bit (the fresh optical depths -log(xi) differ by the last bit at most).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "qp_kernels.h"

namespace qp {
namespace {

constexpr int kCoThreads = 256;
constexpr int kRadix = 256;
constexpr int kCoWarps = kCoThreads / 32;
constexpr int kRngCoalesce = 5;

struct CoParams {
    double x0, y0, z0, dx, dy, dz;
    double idx, idy, idz;  // 1/dx, 1/dy, 1/dz
    long long nx, ny, nz;
    int lb;            // log2 of energy bins per octave
    int D;             // direction bins per face axis
    int min_group;
    int max_group;     // longest run of one group merged into one pair
    int dims;
    unsigned long long seed;
    long long step;
    unsigned long long nomerge;  // the key of photons that are not merged
    int merge;
};

__device__ __forceinline__ long long live_count(const SpeciesDev &S, int *status)
{
    long long n = *((volatile long long *)S.n_live);
    if (n < 0 || n > S.cap) {
        if (threadIdx.x == 0 && blockIdx.x == 0) raise_status(status, QP_ERR_INVALID_ARG);
        n = n < 0 ? 0 : S.cap;
    }
    return n;
}

// The chunk of block b: contiguous, a multiple of kCoThreads long.
__device__ __forceinline__ void chunk_of(long long n, long long *beg, long long *end)
{
    long long per = (n + gridDim.x - 1) / gridDim.x;
    per = (per + kCoThreads - 1) / kCoThreads * kCoThreads;
    *beg = (long long)blockIdx.x * per;
    *end = *beg + per < n ? *beg + per : n;
    if (*beg > n) *beg = n;
}

// e: the photon's energy |u| (sqrt(ux ux + uy uy + uz uz), formed by the caller)
__device__ unsigned long long group_key(const CoParams &C, double x, double y, double z, double ux,
                                        double uy, double uz, double e)
{
    // cell: the offset times the reciprocal of the cell size (formed on the host)
    const double gx = floor((x - C.x0) * C.idx);
    const double gy = floor((y - C.y0) * C.idy);
    const double gz = C.dims == 3 ? floor((z - C.z0) * C.idz) : 0.0;
    if (!(gx >= 0.0 && gx < (double)C.nx && gy >= 0.0 && gy < (double)C.ny && gz >= 0.0 &&
          gz < (double)C.nz))
        return C.nomerge;
    const unsigned long long eb = (unsigned long long)__double_as_longlong(e);
    const unsigned long long ex = (eb >> 52) & 0x7FFull;
    if (ex == 0ull || ex == 0x7FFull) return C.nomerge;
    const unsigned long long ebin = (ex << C.lb) | ((eb & ((1ull << 52) - 1ull)) >> (52 - C.lb));
    const double u[3] = {ux, uy, uz};
    int f = 0;
    if (fabs(u[1]) > fabs(u[f])) f = 1;
    if (fabs(u[2]) > fabs(u[f])) f = 2;
    const int face = 2 * f + (u[f] < 0.0 ? 1 : 0);
    const double r = 1.0 / fabs(u[f]);
    const double a = u[(f + 1) % 3] * r;
    const double b = u[(f + 2) % 3] * r;
    const long long D = C.D;
    long long ia = (long long)floor((a + 1.0) * (0.5 * (double)D));
    long long ib = (long long)floor((b + 1.0) * (0.5 * (double)D));
    if (ia > D - 1) ia = D - 1;
    if (ib > D - 1) ib = D - 1;
    const unsigned long long dbin =
        ((unsigned long long)face * (unsigned long long)D + (unsigned long long)ia) *
            (unsigned long long)D +
        (unsigned long long)ib;
    const unsigned long long cell =
        ((unsigned long long)gx * (unsigned long long)C.ny + (unsigned long long)gy) *
            (unsigned long long)C.nz +
        (unsigned long long)gz;
    const unsigned long long n_e = 2048ull << C.lb, n_d = 6ull * (unsigned long long)(D * D);
    return (cell * n_e + ebin) * n_d + dbin;
}

// ---------------------------------------------------------------- prepare

__global__ void __launch_bounds__(kCoThreads) k_co_prepare(SpeciesDev S, CoParams C,
                                                           unsigned long long *keys,
                                                           unsigned *vals, unsigned char *role,
                                                           double *en, long long *counts,
                                                           int *status)
{
    const long long n = live_count(S, status);
    if (blockIdx.x == 0 && threadIdx.x == 0) counts[0] = n;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const bool alive = S.tau[i] >= 0.0;
        role[i] = alive ? 1 : 0;
        if (C.merge) {
            unsigned long long key = C.nomerge;
            if (alive) {
                const double ux = S.ux[i], uy = S.uy[i], uz = S.uz[i];
                const double e = sqrt(ux * ux + uy * uy + uz * uz);
                en[i] = e;  // the merge sums these energies
                key = group_key(C, S.x[i], S.y[i], S.z ? S.z[i] : 0.0, ux, uy, uz, e);
            }
            keys[i] = key;
            vals[i] = (unsigned)i;
        }
    }
}

// ---------------------------------------------------------------- radix sort

__global__ void __launch_bounds__(kCoThreads) k_co_hist(const unsigned long long *keys, int shift,
                                                        unsigned *hist, const long long *counts)
{
    __shared__ unsigned h[kRadix];
    h[threadIdx.x] = 0u;
    __syncthreads();
    long long beg, end;
    chunk_of(counts[0], &beg, &end);
    for (long long i = beg + threadIdx.x; i < end; i += kCoThreads)
        atomicAdd(&h[(unsigned)(keys[i] >> shift) & 255u], 1u);
    __syncthreads();
    hist[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of m entries in place, one block of 1024 threads, in tiles
// of 8192 entries: a tile is loaded with coalesced reads into shared memory
// (one pad word per 32, so that a thread's 8 contiguous entries fall in
// distinct banks across the warp), each thread scans its 8 entries, the
// thread sums are scanned across the block, and the tile is written back
// coalesced with the running total of the earlier tiles added.  total: the
// sum of all entries, or nullptr.
constexpr int kScanThreads = 1024, kScanPer = 8, kScanTile = kScanThreads * kScanPer;

__global__ void __launch_bounds__(kScanThreads) k_co_scan(unsigned *v, int m, long long *total)
{
    __shared__ unsigned s[kScanTile + kScanTile / 32];
    __shared__ unsigned s_warp[32];
    __shared__ unsigned s_tile;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    unsigned carry = 0u;
    for (int base = 0; base < m; base += kScanTile) {
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) {
            const int i = k * kScanThreads + t;
            s[i + (i >> 5)] = base + i < m ? v[base + i] : 0u;
        }
        __syncthreads();
        unsigned loc[kScanPer], sum = 0u;
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) {
            const int i = t * kScanPer + k;
            loc[k] = s[i + (i >> 5)];
            sum += loc[k];
        }
        unsigned inc = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned y = __shfl_up_sync(0xFFFFFFFFu, inc, d);
            if (lane >= d) inc += y;
        }
        if (lane == 31) s_warp[w] = inc;
        __syncthreads();
        if (w == 0) {
            const unsigned x = s_warp[lane];
            unsigned xi = x;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned y = __shfl_up_sync(0xFFFFFFFFu, xi, d);
                if (lane >= d) xi += y;
            }
            s_warp[lane] = xi - x;
            if (lane == 31) s_tile = xi;
        }
        __syncthreads();
        unsigned run = carry + s_warp[w] + (inc - sum);
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) {
            const int i = t * kScanPer + k;
            s[i + (i >> 5)] = run;
            run += loc[k];
        }
        carry += s_tile;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) {
            const int i = k * kScanThreads + t;
            if (base + i < m) v[base + i] = s[i + (i >> 5)];
        }
        __syncthreads();  // s, s_warp and s_tile are reused by the next tile
    }
    if (total && t == 0) *total = (long long)carry;
}

// Stable scatter: the block walks its chunk tile by tile; within a tile an
// element's rank among equal digits is its rank in its warp (match_any)
// plus the counts of the earlier warps.
__global__ void __launch_bounds__(kCoThreads) k_co_scatter(const unsigned long long *kin,
                                                           const unsigned *vin,
                                                           unsigned long long *kout,
                                                           unsigned *vout, int shift,
                                                           const unsigned *hist,
                                                           const long long *counts)
{
    __shared__ unsigned base[kRadix];
    __shared__ unsigned wc[kCoWarps][kRadix];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    base[t] = hist[(size_t)t * gridDim.x + blockIdx.x];
    long long beg, end;
    chunk_of(counts[0], &beg, &end);
    const unsigned lt = (1u << lane) - 1u;
    for (long long t0 = beg; t0 < end; t0 += kCoThreads) {
        for (int w = 0; w < kCoWarps; ++w) wc[w][t] = 0u;
        __syncthreads();
        const long long i = t0 + t;
        const bool ok = i < end;
        unsigned long long k = 0ull;
        unsigned v = 0u;
        if (ok) {
            k = kin[i];
            v = vin[i];
        }
        const unsigned d = ok ? (unsigned)(k >> shift) & 255u : 256u + (unsigned)lane;
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
        const unsigned rank = (unsigned)__popc(peers & lt);
        if (ok && rank == 0u) wc[warp][d] = (unsigned)__popc(peers);
        __syncthreads();
        // per digit: exclusive prefix over the warps, and the tile's total
        unsigned run = 0u;
        for (int w = 0; w < kCoWarps; ++w) {
            const unsigned c = wc[w][t];
            wc[w][t] = run;
            run += c;
        }
        __syncthreads();
        if (ok) {
            const unsigned pos = base[d] + wc[warp][d] + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
        base[t] += run;
        __syncthreads();
    }
}

// ---------------------------------------------------------------- groups

struct GroupSums {
    double W, E, P[3], X[3];
};

// The sums of a run [a, b) of the sorted order, member by member in slot
// order; en: the members' energies |u| from k_co_prepare.
__device__ GroupSums group_sums(const SpeciesDev &S, const double *en, const unsigned *vals,
                                long long a, long long b)
{
    GroupSums g{0.0, 0.0, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
    for (long long k = a; k < b; ++k) {
        const unsigned i = vals[k];
        const double w = S.w[i];
        const double ux = S.ux[i], uy = S.uy[i], uz = S.uz[i];
        const double e = en[i];
        g.W = g.W + w;
        g.E = g.E + w * e;
        g.P[0] = g.P[0] + w * ux;
        g.P[1] = g.P[1] + w * uy;
        g.P[2] = g.P[2] + w * uz;
        g.X[0] = g.X[0] + w * S.x[i];
        g.X[1] = g.X[1] + w * S.y[i];
        g.X[2] = g.X[2] + w * (S.z ? S.z[i] : 0.0);
    }
    return g;
}

// A merged group (run [j, end) of the sorted keys) starts at j; its end.
__device__ __forceinline__ bool group_start(const unsigned long long *keys, long long j,
                                            long long n, unsigned long long nomerge,
                                            long long *end)
{
    const unsigned long long k = keys[j];
    if (k == nomerge || (j > 0 && keys[j - 1] == k)) return false;
    // the first index past j with another key (the keys are sorted): steps
    // doubling from j until one lands past the group, then bisection
    long long lo = j, step = 1;  // keys[lo] == k
    long long hi = n;            // keys[hi] != k, or hi == n
    while (lo + step < n && keys[lo + step] == k) {
        lo += step;
        step <<= 1;
    }
    if (lo + step < n) hi = lo + step;
    while (hi - lo > 1) {
        const long long mid = lo + (hi - lo) / 2;
        if (keys[mid] == k)
            lo = mid;
        else
            hi = mid;
    }
    *end = hi;
    return true;
}

// Runs of the sorted keys: every group (one key) is cut into runs of at
// most max_group members in slot order; the runs of at least min_group go to
// the run list (one thread a group: it only walks the group's keys).
__global__ void __launch_bounds__(kCoThreads) k_co_groups(CoParams C,
                                                          const unsigned long long *keys,
                                                          long long *counts, uint2 *runs)
{
    const long long n = counts[0];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        long long end;
        if (!group_start(keys, j, n, C.nomerge, &end)) continue;
        for (long long a = j; a < end; a += C.max_group) {
            const long long b = a + C.max_group < end ? a + C.max_group : end;
            if (b - a < C.min_group) continue;
            const unsigned long long r = atomicAdd((unsigned long long *)&counts[2], 1ull);
            runs[r] = make_uint2((unsigned)a, (unsigned)b);
        }
    }
}

// One thread a run: its sums, kept for k_co_pairs; a run whose momentum
// vanishes is kept as it is, the others become pairs (role 2 at the first
// member, 0 at the others).
__global__ void __launch_bounds__(kCoThreads) k_co_runs(SpeciesDev S, const double *en,
                                                        const unsigned *vals, const uint2 *runs,
                                                        unsigned char *role, GroupSums *rsum,
                                                        const long long *counts,
                                                        long long *stats)
{
    const long long nr = counts[2];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += stride) {
        const uint2 run = runs[r];
        const GroupSums g = group_sums(S, en, vals, run.x, run.y);
        rsum[r] = g;
        const double *P = g.P;
        if (!(P[0] * P[0] + P[1] * P[1] + P[2] * P[2] > 0.0)) continue;
        for (unsigned k = run.x; k < run.y; ++k) role[vals[k]] = 0;
        role[vals[run.x]] = 2;  // the sorted run is in slot order: its first
        atomicAdd((unsigned long long *)&stats[0], 1ull);
        atomicAdd((unsigned long long *)&stats[1], (unsigned long long)(run.y - run.x));
    }
}

// ---------------------------------------------------------------- role scan

__global__ void __launch_bounds__(kCoThreads) k_co_chunk_sums(const unsigned char *role,
                                                              unsigned *sums,
                                                              const long long *counts)
{
    __shared__ unsigned s[kCoWarps];
    long long beg, end;
    chunk_of(counts[0], &beg, &end);
    unsigned v = 0u;
    for (long long i = beg + threadIdx.x; i < end; i += kCoThreads) v += role[i];
    v = __reduce_add_sync(0xFFFFFFFFu, v);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0u;
        for (int w = 0; w < kCoWarps; ++w) t += s[w];
        sums[blockIdx.x] = t;
    }
}

// Output slot of every survivor: the chunk's offset plus the exclusive scan
// of the roles within the chunk, tile after tile.
__global__ void __launch_bounds__(kCoThreads) k_co_offsets(const unsigned char *role,
                                                           const unsigned *chunk_off,
                                                           unsigned *off, const long long *counts)
{
    __shared__ unsigned s_w[kCoWarps];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    long long beg, end;
    chunk_of(counts[0], &beg, &end);
    unsigned run = chunk_off[blockIdx.x];
    for (long long t0 = beg; t0 < end; t0 += kCoThreads) {
        const long long i = t0 + t;
        const unsigned v = i < end ? role[i] : 0u;
        unsigned inc = v;
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned y = __shfl_up_sync(0xFFFFFFFFu, inc, d);
            if (lane >= d) inc += y;
        }
        if (lane == 31) s_w[warp] = inc;
        __syncthreads();
        unsigned before = 0u, tot = 0u;
        for (int w = 0; w < kCoWarps; ++w) {
            if (w < warp) before += s_w[w];
            tot += s_w[w];
        }
        if (i < end) off[i] = run + before + inc - v;
        run += tot;
        __syncthreads();
    }
}

// ---------------------------------------------------------------- outputs

struct Stage {
    double *f[9];  // x y z ux uy uz tau w chi
    int *nemit;
};

__global__ void __launch_bounds__(kCoThreads) k_co_kept(SpeciesDev S, const unsigned char *role,
                                                        const unsigned *off, Stage st,
                                                        const long long *counts)
{
    const long long n = counts[0];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        if (role[i] != 1) continue;
        const unsigned o = off[i];
        st.f[0][o] = S.x[i];
        st.f[1][o] = S.y[i];
        st.f[2][o] = S.z ? S.z[i] : 0.0;
        st.f[3][o] = S.ux[i];
        st.f[4][o] = S.uy[i];
        st.f[5][o] = S.uz[i];
        st.f[6][o] = S.tau[i];
        st.f[7][o] = S.w[i];
        st.f[8][o] = S.chi ? S.chi[i] : 0.0;
        st.nemit[o] = S.nemit ? S.nemit[i] : 0;
    }
}

__global__ void __launch_bounds__(kCoThreads) k_co_pairs(SpeciesDev S, CoParams C,
                                                         const unsigned *vals, const uint2 *runs,
                                                         const unsigned char *role,
                                                         const GroupSums *rsum,
                                                         const unsigned *off, Stage st,
                                                         const long long *counts)
{
    const long long nr = counts[2];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nr; q += stride) {
        const uint2 run = runs[q];
        const unsigned anchor = vals[run.x];
        if (role[anchor] != 2) continue;
        const GroupSums g = rsum[q];
        const double W = g.W;
        const double eps = g.E / W;
        const double c[3] = {g.P[0] / W, g.P[1] / W, g.P[2] / W};
        const double c2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
        const double d2 = eps * eps - c2;
        const double dm = d2 > 0.0 ? sqrt(d2) : 0.0;
        const double cm = sqrt(c2);
        const double ph[3] = {c[0] / cm, c[1] / cm, c[2] / cm};
        const double r[3] = {S.ux[anchor], S.uy[anchor], S.uz[anchor]};
        const double rp = r[0] * ph[0] + r[1] * ph[1] + r[2] * ph[2];
        double v[3] = {r[0] - rp * ph[0], r[1] - rp * ph[1], r[2] - rp * ph[2]};
        double vm = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        const double rm = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        if (!(vm > 1e-12 * rm)) {
            // the first photon is parallel to P: the axis least aligned with P
            int a = 0;
            if (fabs(ph[1]) < fabs(ph[a])) a = 1;
            if (fabs(ph[2]) < fabs(ph[a])) a = 2;
            const double ap = ph[a];
            v[0] = (a == 0 ? 1.0 : 0.0) - ap * ph[0];
            v[1] = (a == 1 ? 1.0 : 0.0) - ap * ph[1];
            v[2] = (a == 2 ? 1.0 : 0.0) - ap * ph[2];
            vm = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        }
        const double dv[3] = {dm * (v[0] / vm), dm * (v[1] / vm), dm * (v[2] / vm)};
        const unsigned o = off[anchor];
        const long long id = particle_id(S, anchor);
        for (int s = 0; s < 2; ++s) {
            const double sg = s == 0 ? 1.0 : -1.0;
            const uint4 rr = draw(C.seed, QP_PHOTON, kRngCoalesce, id, (uint64_t)C.step, s);
            st.f[0][o + s] = g.X[0] / W;
            st.f[1][o + s] = g.X[1] / W;
            st.f[2][o + s] = g.X[2] / W;
            st.f[3][o + s] = c[0] + sg * dv[0];
            st.f[4][o + s] = c[1] + sg * dv[1];
            st.f[5][o + s] = c[2] + sg * dv[2];
            st.f[6][o + s] = -log(u53(rr.x, rr.y));
            st.f[7][o + s] = 0.5 * W;
            st.f[8][o + s] = 0.0;
            st.nemit[o + s] = 0;
        }
    }
}

__global__ void __launch_bounds__(kCoThreads) k_co_copy_back(SpeciesDev S, Stage st,
                                                             const long long *counts,
                                                             long long *stats)
{
    const long long n_after = counts[1];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n_after;
         k += stride) {
        S.x[k] = st.f[0][k];
        S.y[k] = st.f[1][k];
        if (S.z) S.z[k] = st.f[2][k];
        S.ux[k] = st.f[3][k];
        S.uy[k] = st.f[4][k];
        S.uz[k] = st.f[5][k];
        S.tau[k] = st.f[6][k];
        S.w[k] = st.f[7][k];
        if (S.chi) S.chi[k] = st.f[8][k];
        if (S.nemit) S.nemit[k] = st.nemit[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        stats[2] = counts[0];
        stats[3] = n_after;
        *S.n_live = n_after;
    }
}

// ---------------------------------------------------------------- sort by cell

// Cell keys of the live slots (row-major; outside the grid: nx ny, after
// every cell) and the identity order.
__global__ void __launch_bounds__(kCoThreads) k_sort_prepare(SpeciesDev S, YeeGrid g,
                                                             unsigned long long *keys,
                                                             unsigned *vals, long long *counts,
                                                             int *status)
{
    const long long n = live_count(S, status);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        counts[0] = n;
        counts[1] = n;
    }
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double gx = floor((S.x[i] - g.x0) / g.dx), gy = floor((S.y[i] - g.y0) / g.dy);
        unsigned long long key = (unsigned long long)g.nx * (unsigned long long)g.ny;
        if (gx >= 0.0 && gy >= 0.0 && gx < (double)g.nx && gy < (double)g.ny)
            key = (unsigned long long)gy * (unsigned long long)g.nx + (unsigned long long)gx;
        keys[i] = key;
        vals[i] = (unsigned)i;
    }
}

// Every array of the sorted slot k from its source slot, into the staging arrays.
__global__ void __launch_bounds__(kCoThreads) k_sort_gather(SpeciesDev S, const unsigned *vals,
                                                            Stage st, const long long *counts)
{
    const long long n = counts[0];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const unsigned i = vals[k];
        st.f[0][k] = S.x[i];
        st.f[1][k] = S.y[i];
        st.f[2][k] = S.z ? S.z[i] : 0.0;
        st.f[3][k] = S.ux[i];
        st.f[4][k] = S.uy[i];
        st.f[5][k] = S.uz[i];
        st.f[6][k] = S.tau[i];
        st.f[7][k] = S.w[i];
        st.f[8][k] = S.chi ? S.chi[i] : 0.0;
        st.nemit[k] = S.nemit ? S.nemit[i] : 0;
    }
}

}  // namespace

size_t coalesce_scratch_bytes(int64_t cap, int grid)
{
    const size_t c = (size_t)(cap > 0 ? cap : 1);
    return 2 * c * 8 + 2 * c * 4 + c + c * 4 + c * 9 * 8 + c * 4 +
           ((size_t)kRadix * grid + grid + 64) * 4 + 16 * 8 + (c / 3 + 1) * 8 +
           (c / 3 + 1) * sizeof(GroupSums) + 32 * 256;
}

namespace {

// The scratch of qp_coalesce_photons, qp_sort_species and the fused steps'
// photon order, carved in one layout (every piece 256-byte aligned).
struct CoScratch {
    unsigned long long *keys[2];
    unsigned *vals[2];
    unsigned char *role;
    unsigned *off;
    Stage stg;
    unsigned *hist, *chunk;
    long long *counts;
    uint2 *runs;
    GroupSums *rsum;  // the sums of each run (k_co_runs, for k_co_pairs)
};

CoScratch carve(void *scratch, int64_t cap, int grid)
{
    const size_t c = (size_t)(cap > 0 ? cap : 1);
    unsigned char *p = (unsigned char *)scratch;
    auto take = [&](size_t bytes) {
        unsigned char *q = p;
        p += (bytes + 255) / 256 * 256;
        return q;
    };
    CoScratch s;
    s.keys[0] = (unsigned long long *)take(c * 8);
    s.keys[1] = (unsigned long long *)take(c * 8);
    s.vals[0] = (unsigned *)take(c * 4);
    s.vals[1] = (unsigned *)take(c * 4);
    s.role = take(c);
    s.off = (unsigned *)take(c * 4);
    for (int f = 0; f < 9; ++f) s.stg.f[f] = (double *)take(c * 8);
    s.stg.nemit = (int *)take(c * 4);
    s.hist = (unsigned *)take((size_t)kRadix * grid * 4);
    s.chunk = (unsigned *)take((size_t)grid * 4 + 64);
    s.counts = (long long *)take(16 * 8);
    s.runs = (uint2 *)take((c / 3 + 1) * sizeof(uint2));
    s.rsum = (GroupSums *)take((c / 3 + 1) * sizeof(GroupSums));
    return s;
}

}  // namespace

cudaError_t launch_coalesce(const SpeciesDev &S, const qp_coalesce_params *P, void *scratch,
                            int grid, long long *stats, int *status, cudaStream_t st)
{
    const CoScratch cs = carve(scratch, S.cap, grid);
    unsigned long long *const *keys = cs.keys;
    unsigned *const *vals = cs.vals;
    unsigned char *role = cs.role;
    unsigned *off = cs.off;
    const Stage stg = cs.stg;
    unsigned *hist = cs.hist;
    unsigned *chunk = cs.chunk;
    long long *counts = cs.counts;
    uint2 *runs = cs.runs;
    // the photons' energies (k_co_prepare to k_co_runs) in the chi staging
    // array, which k_co_kept and k_co_pairs write only after k_co_runs
    double *en = stg.f[8];

    CoParams C{};
    int passes = 0;
    if (P) {
        C.x0 = P->x0;
        C.y0 = P->y0;
        C.z0 = P->z0;
        C.dx = P->dx;
        C.dy = P->dy;
        C.dz = P->dz;
        C.idx = 1.0 / P->dx;
        C.idy = 1.0 / P->dy;
        C.idz = P->dz > 0.0 ? 1.0 / P->dz : 0.0;  // used with dims 3 only
        C.nx = P->nx;
        C.ny = P->ny;
        C.nz = P->nz;
        int lb = 0;
        while ((1 << lb) < P->energy_bins_per_octave) ++lb;
        C.lb = lb;
        C.D = P->direction_bins;
        C.min_group = P->min_group;
        C.max_group = P->max_group > 0 ? P->max_group : 256;
        C.dims = S.z ? 3 : 2;
        C.seed = P->seed;
        C.step = P->step;
        C.merge = 1;
        const unsigned long long n_e = 2048ull << lb;
        const unsigned long long n_d = 6ull * (unsigned long long)C.D * (unsigned long long)C.D;
        C.nomerge = (unsigned long long)P->nx * (unsigned long long)P->ny *
                    (unsigned long long)P->nz * n_e * n_d;
        int bits = 0;
        while (bits < 64 && (C.nomerge >> bits) != 0ull) ++bits;
        passes = (bits + 7) / 8;
    }
    cudaError_t e = cudaMemsetAsync(counts, 0, 16 * 8, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(stats, 0, 4 * 8, st);
    if (e != cudaSuccess) return e;
    k_co_prepare<<<grid, kCoThreads, 0, st>>>(S, C, keys[0], vals[0], role, en, counts, status);
    int cur = 0;
    for (int ps = 0; ps < passes; ++ps) {
        k_co_hist<<<grid, kCoThreads, 0, st>>>(keys[cur], 8 * ps, hist, counts);
        k_co_scan<<<1, 1024, 0, st>>>(hist, kRadix * grid, nullptr);
        k_co_scatter<<<grid, kCoThreads, 0, st>>>(keys[cur], vals[cur], keys[cur ^ 1],
                                                   vals[cur ^ 1], 8 * ps, hist, counts);
        cur ^= 1;
    }
    if (passes) {
        k_co_groups<<<grid, kCoThreads, 0, st>>>(C, keys[cur], counts, runs);
        k_co_runs<<<grid, kCoThreads, 0, st>>>(S, en, vals[cur], runs, role, cs.rsum, counts,
                                                stats);
    }
    k_co_chunk_sums<<<grid, kCoThreads, 0, st>>>(role, chunk, counts);
    k_co_scan<<<1, 1024, 0, st>>>(chunk, grid, counts + 1);
    k_co_offsets<<<grid, kCoThreads, 0, st>>>(role, chunk, off, counts);
    k_co_kept<<<grid, kCoThreads, 0, st>>>(S, role, off, stg, counts);
    if (passes) {
        k_co_pairs<<<grid, kCoThreads, 0, st>>>(S, C, vals[cur], runs, role, cs.rsum, off, stg,
                                                 counts);
    }
    k_co_copy_back<<<grid, kCoThreads, 0, st>>>(S, stg, counts, stats);
    return cudaGetLastError();
}

cudaError_t launch_sort_cells(const SpeciesDev &S, const YeeGrid &g, void *scratch, int grid,
                              long long *stats, int *status, cudaStream_t st)
{
    const CoScratch cs = carve(scratch, S.cap, grid);
    unsigned long long *const *keys = cs.keys;
    unsigned *const *vals = cs.vals;
    const Stage stg = cs.stg;
    unsigned *hist = cs.hist;
    long long *counts = cs.counts;
    const unsigned long long top = (unsigned long long)g.nx * (unsigned long long)g.ny;
    int bits = 0;
    while (bits < 64 && (top >> bits) != 0ull) ++bits;
    const int passes = (bits + 7) / 8;
    cudaError_t e = cudaMemsetAsync(stats, 0, 4 * 8, st);
    if (e != cudaSuccess) return e;
    k_sort_prepare<<<grid, kCoThreads, 0, st>>>(S, g, keys[0], vals[0], counts, status);
    int cur = 0;
    for (int ps = 0; ps < passes; ++ps) {
        k_co_hist<<<grid, kCoThreads, 0, st>>>(keys[cur], 8 * ps, hist, counts);
        k_co_scan<<<1, 1024, 0, st>>>(hist, kRadix * grid, nullptr);
        k_co_scatter<<<grid, kCoThreads, 0, st>>>(keys[cur], vals[cur], keys[cur ^ 1],
                                                   vals[cur ^ 1], 8 * ps, hist, counts);
        cur ^= 1;
    }
    k_sort_gather<<<grid, kCoThreads, 0, st>>>(S, vals[cur], stg, counts);
    k_co_copy_back<<<grid, kCoThreads, 0, st>>>(S, stg, counts, stats);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- fused photon order

namespace {

// counts[3]: photons the fused window allocated; counts[0] and win[2]:
// those it staged (the capacity bounds them), sorted next; win[1]: those it
// stores (the free slots bound them); identity order to sort.
__global__ void __launch_bounds__(kCoThreads) k_fo_prepare(SpeciesDev Ph, long long *counts,
                                                           long long *win, unsigned *vals,
                                                           int *status)
{
    const long long base = win[0];
    const long long cap = Ph.present ? Ph.cap : 0;
    const long long alloc = counts[3];
    const long long staged = alloc < cap ? alloc : cap;
    const long long stored = staged < cap - base ? staged : cap - base;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        counts[0] = staged;
        win[1] = stored;
        win[2] = staged;
        if (alloc > stored) raise_status(status, QP_WARN_BUFFER_FULL);
    }
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x; a < staged; a += stride)
        vals[a] = (unsigned)a;
}

}  // namespace

FusedScratch fused_scratch(void *scratch, int64_t photon_cap, int grid, int key_bits)
{
    const CoScratch cs = carve(scratch, photon_cap, grid);
    FusedScratch f;
    for (int c = 0; c < 8; ++c) f.stage[c] = cs.stg.f[c];
    f.rkeys = cs.keys[0];
    f.moves_new = (unsigned short *)cs.off;
    f.alloc = cs.counts + 3;
    f.order = cs.vals[((key_bits + 7) / 8) & 1];
    f.sorted_keys = cs.keys[((key_bits + 7) / 8) & 1];
    return f;
}

cudaError_t launch_fused_order(const SpeciesDev &Ph, void *scratch, int grid, int key_bits,
                               long long *win, int *status, cudaStream_t st)
{
    const CoScratch cs = carve(scratch, Ph.present ? Ph.cap : 0, grid);
    k_fo_prepare<<<grid, kCoThreads, 0, st>>>(Ph, cs.counts, win, cs.vals[0], status);
    int cur = 0;
    for (int ps = 0; ps < (key_bits + 7) / 8; ++ps) {
        k_co_hist<<<grid, kCoThreads, 0, st>>>(cs.keys[cur], 8 * ps, cs.hist, cs.counts);
        k_co_scan<<<1, 1024, 0, st>>>(cs.hist, kRadix * grid, nullptr);
        k_co_scatter<<<grid, kCoThreads, 0, st>>>(cs.keys[cur], cs.vals[cur], cs.keys[cur ^ 1],
                                                   cs.vals[cur ^ 1], 8 * ps, cs.hist,
                                                   cs.counts);
        cur ^= 1;
    }
    return cudaGetLastError();
}

}  // namespace qp
