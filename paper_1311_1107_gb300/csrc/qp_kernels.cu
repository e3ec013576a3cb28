// Auxiliary kernels of libqedpic (sm_103a): initial optical depths,
// diagnostics, the bounded-wait self-test, and the launchers of all kernels
// (the step kernel itself is in qp_step.cuh).
#include <cuda_runtime.h>
#include <math.h>

#include "qp_kernels.h"
#include "qp_step.cuh"

namespace qp {

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

__global__ void k_init_tau(double *tau, int64_t first, int64_t count, int64_t id_base,
                           int64_t id_split, int64_t id_append, uint64_t seed, int species)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += stride) {
        const int64_t i = first + k;
        const uint4 r =
            draw(seed, species, kRngInit, particle_id(id_base, id_split, id_append, i), 0, 0);
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

static const void *step_fn(int precision, int fk, bool batch)
{
    return precision == QP_MIXED ? step_kernel_mixed(fk, batch) : step_kernel_fp64(fk, batch);
}

size_t step_smem_bytes(int precision)
{
    return precision == QP_MIXED ? step_smem_mixed() : step_smem_fp64();
}

int step_blocks_per_sm(int precision, int field_kind, bool batch)
{
    const void *fn = step_fn(precision, field_kind, batch);
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

cudaError_t launch_step(const StepArgs &a, int precision, int field_kind, bool batch, int grid,
                        cudaStream_t st)
{
    const void *fn = step_fn(precision, field_kind, batch);
    if (!fn) return cudaErrorInvalidValue;
    const size_t smem = step_smem_bytes(precision);
    void *args[] = {(void *)&a};
    // the single-problem mixed-path kernel takes fixed first tiles, which
    // need every block resident at once: a cooperative launch guarantees it
    // (or fails to launch)
    if (!batch && precision == QP_MIXED)
        return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kTile), args, smem, st);
    return cudaLaunchKernel(fn, dim3(grid), dim3(kTile), args, smem, st);
}

static int bits_of(unsigned long long v)
{
    int b = 0;
    while (v) {
        ++b;
        v >>= 1;
    }
    return b;
}

int fused_key_bits(int K, long long tiles, int *ordinal_bits)
{
    const int ob = bits_of((unsigned long long)(tiles > 0 ? tiles : 1) * 32ull - 1ull);
    if (ordinal_bits) *ordinal_bits = ob;
    return bits_of((unsigned long long)(K > 1 ? K - 1 : 0)) + ob + kEmitBits;
}

cudaError_t launch_fused(const StepArgs &a, int precision, int field_kind, int K,
                         long long tiles_e, long long tiles, void *scratch, int order_grid,
                         long long *win, int num_sms, cudaStream_t st)
{
    const bool mixed = precision == QP_MIXED;
    const void *lep = mixed ? fused_kernel_mixed(field_kind) : fused_kernel_fp64(field_kind);
    const void *photons = mixed ? fused_photons_mixed() : fused_photons_fp64();
    if (!lep) return cudaErrorInvalidValue;
    const SpeciesDev &Ph = a.single.sp[2];
    FusedArgs f{};
    f.a = a;
    f.K = K;
    const int key_bits = fused_key_bits(K, tiles, &f.ob);
    f.tiles_e = tiles_e;
    f.tiles = tiles;
    f.fs = fused_scratch(scratch, Ph.present ? Ph.cap : 0, order_grid, key_bits);
    f.win = win;
    void *args[] = {(void *)&f};
    const long long resident = (long long)num_sms * 32;
    const unsigned grid = (unsigned)(tiles < resident ? (tiles > 0 ? tiles : 1) : resident);
    cudaError_t e = cudaMemsetAsync(f.fs.alloc, 0, sizeof(long long), st);
    if (e == cudaSuccess) e = cudaLaunchKernel(lep, dim3(grid), dim3(32), args, 0, st);
    if (e == cudaSuccess) e = launch_fused_order(Ph, scratch, order_grid, key_bits, win, a.status, st);
    const long long cap = Ph.present ? Ph.cap : 0;
    if (e == cudaSuccess && cap > 0) {
        long long pb = (cap + 255) / 256;
        if (pb > (long long)num_sms * 8) pb = (long long)num_sms * 8;
        e = cudaLaunchKernel(photons, dim3((unsigned)pb), dim3(256), args, 0, st);
    }
    return e;
}

cudaError_t launch_init_tau(double *tau, int64_t first, int64_t count, int64_t id_base,
                            int64_t id_split, int64_t id_append, uint64_t seed, int species,
                            cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    int64_t blocks = (count + kDiagTile - 1) / kDiagTile;
    if (blocks > 4096) blocks = 4096;
    k_init_tau<<<(int)blocks, kDiagTile, 0, st>>>(tau, first, count, id_base, id_split,
                                                  id_append, seed, species);
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

// -------------------------------------------------------------------- pulse refill

// One launch: each block fills a tile of 32 columns x kPulseRows rows.  Its
// column factors (for the E_y and the B_z staggering) and row radii go to
// shared memory first: E = A exp(-c r^2) cos(phi + kappa r^2) with
// A = a0 (1 + q^2)^(-1/4) exp(-2 ln2 eta^2/tau^2), c = 1/(w0^2 (1 + q^2)),
// kappa = xi / (2 (xi^2 + zr^2)), phi = -eta - atan(q)/2.  Only eta and the
// phase reduction modulo 2 pi are FP64 (the phase is hundreds of radians);
// the factors and the nodes are FP32.
constexpr int kPulseRows = 64;

__global__ void __launch_bounds__(256) k_pulse_fill(Pulse2DDev p, int64_t nx, int64_t ny,
                                                    double dx, double dy, double x0, double y0,
                                                    double t, float *ey, float *bz)
{
    __shared__ float4 s_col[64];
    __shared__ float s_r2[kPulseRows];
    const int tid = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * kPulseRows;
    if (tid < 64) {
        const int s = tid >> 5;  // 0: E_y column, 1: B_z column (half a cell further)
        const int64_t i = i0 + (tid & 31);
        const double xi = x0 + ((double)i + 0.5 * s) * dx - p.x_focus;
        const double eta = (t - p.t_focus) - xi;
        const float zr = (float)(0.5 * p.w0 * p.w0);
        const float xf = (float)xi, ef = (float)eta;
        const float q = xf / zr, wr2 = 1.0f + q * q;
        const float tau = (float)p.tau_fwhm;
        const float A = (float)p.a0 * rsqrtf(sqrtf(wr2)) *
                        expf(-1.3862943611198906f * ef * ef / (tau * tau));
        // -eta reduced modulo 2 pi in FP64, then the Gouy phase
        const double red = -eta - 6.283185307179586477 * rint(-eta * 0.15915494309189533577);
        const float phi = (float)red - 0.5f * atanf(q);
        s_col[tid] = make_float4(A, 1.0f / ((float)(p.w0 * p.w0) * wr2),
                                 xf / (2.0f * (xf * xf + zr * zr)), phi);
    } else if (tid < 64 + kPulseRows) {
        const int64_t j = j0 + (tid - 64);
        const double r = y0 + ((double)j + 0.5) * dy - p.y_axis;
        s_r2[tid - 64] = (float)(r * r);
    }
    __syncthreads();
    const int c = tid & 31;
    const int64_t i = i0 + c;
    if (i >= nx) return;
    const float4 e = s_col[c], b = s_col[32 + c];
    for (int r = tid >> 5; r < kPulseRows; r += 8) {
        const int64_t j = j0 + r;
        if (j >= ny) break;
        const float r2 = s_r2[r];
        const int64_t k = j * nx + i;
        ey[k] = e.x * expf(-e.y * r2) * cosf(fmaf(e.z, r2, e.w));
        bz[k] = b.x * expf(-b.y * r2) * cosf(fmaf(b.z, r2, b.w));
    }
}

cudaError_t launch_pulse_fill(const Pulse2DDev &p, int64_t nx, int64_t ny, double dx, double dy,
                              double x0, double y0, double t, float *ey, float *bz,
                              cudaStream_t st)
{
    if (nx <= 0 || ny <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((nx + 31) / 32), (unsigned)((ny + kPulseRows - 1) / kPulseRows));
    k_pulse_fill<<<grid, 256, 0, st>>>(p, nx, ny, dx, dy, x0, y0, t, ey, bz);
    return cudaGetLastError();
}

}  // namespace qp
