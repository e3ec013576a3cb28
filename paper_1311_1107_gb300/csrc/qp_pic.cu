// PIC coupling around the QED step on a 2D Yee grid (qp_yee_advance_b,
// qp_yee_advance_e, qp_deposit_current): the paper's QED step runs inside
// a PIC code (section 3); these are the field solver and the current
// deposition a 2D PIC cycle needs around it.
//
// Grid: six float components, ny rows of nx values, staggered as the
// step's field gather reads them: Ex (i+1/2, j), Ey (i, j+1/2), Ez (i, j),
// Bx (i, j+1/2), By (i+1/2, j), Bz (i+1/2, j+1/2); values outside the grid
// are 0.  Normalised units (c = 1): dB/dt = -curl E, dE/dt = curl B - J, J in
// units of e n_c c.  One thread a node; every node's update reads its own
// value and neighbours of the other field only, so both updates run in
// place.  FP32 arithmetic (the grid is FP32).
#include <cuda_runtime.h>
#include <stdint.h>

#include "qp_df.h"
#include "qp_kernels.h"

namespace qp {
namespace {

constexpr int kPicBlock = 256;

__device__ __forceinline__ float at(const float *a, int64_t nx, int64_t ny, int64_t i, int64_t j)
{
    return (i < 0 || j < 0 || i >= nx || j >= ny) ? 0.0f : a[j * nx + i];
}

// Nodes by rows: blockIdx.y strides over the rows, the threads of blockIdx.x
// over the columns (no index division).
__global__ void __launch_bounds__(kPicBlock) k_yee_b(YeeGrid g, float idx, float idy, float dtb)
{
    for (int64_t j = blockIdx.y; j < g.ny; j += gridDim.y)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.nx;
             i += (int64_t)gridDim.x * blockDim.x) {
            const int64_t k = j * g.nx + i;
            const float ez = g.f[2][k];
            const float dEz_dy = (at(g.f[2], g.nx, g.ny, i, j + 1) - ez) * idy;
            const float dEz_dx = (at(g.f[2], g.nx, g.ny, i + 1, j) - ez) * idx;
            const float dEy_dx = (at(g.f[1], g.nx, g.ny, i + 1, j) - g.f[1][k]) * idx;
            const float dEx_dy = (at(g.f[0], g.nx, g.ny, i, j + 1) - g.f[0][k]) * idy;
            g.f[3][k] -= dtb * dEz_dy;
            g.f[4][k] += dtb * dEz_dx;
            g.f[5][k] -= dtb * (dEy_dx - dEx_dy);
        }
}

__global__ void __launch_bounds__(kPicBlock) k_yee_e(YeeGrid g, float idx, float idy,
                                                     const float *jx, const float *jy,
                                                     const float *jz, float dt)
{
    for (int64_t j = blockIdx.y; j < g.ny; j += gridDim.y)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.nx;
             i += (int64_t)gridDim.x * blockDim.x) {
            const int64_t k = j * g.nx + i;
            const float bz = g.f[5][k];
            const float dBz_dy = (bz - at(g.f[5], g.nx, g.ny, i, j - 1)) * idy;
            const float dBz_dx = (bz - at(g.f[5], g.nx, g.ny, i - 1, j)) * idx;
            const float dBy_dx = (g.f[4][k] - at(g.f[4], g.nx, g.ny, i - 1, j)) * idx;
            const float dBx_dy = (g.f[3][k] - at(g.f[3], g.nx, g.ny, i, j - 1)) * idy;
            g.f[0][k] += dt * (dBz_dy - (jx ? jx[k] : 0.0f));
            g.f[1][k] += dt * (-dBz_dx - (jy ? jy[k] : 0.0f));
            g.f[2][k] += dt * (dBy_dx - dBx_dy - (jz ? jz[k] : 0.0f));
        }
}

// The same updates four nodes a thread (x = 4 q .. 4 q + 3 of a row) with
// 16-byte loads and stores, for grids whose rows are whole float4s (nx a
// multiple of 4, arrays 16-byte aligned); the arithmetic of each node is
// k_yee_b's and k_yee_e's.  The neighbour past the four (x + 4 for B, x - 1
// for E) is one scalar load.
__device__ __forceinline__ float4 ld4(const float *a, int64_t k)
{
    return *reinterpret_cast<const float4 *>(a + k);
}

__global__ void __launch_bounds__(kPicBlock) k_yee_b4(YeeGrid g, float idx, float idy, float dtb)
{
    const int64_t nq = g.nx / 4;
    for (int64_t j = blockIdx.y; j < g.ny; j += gridDim.y)
        for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq;
             q += (int64_t)gridDim.x * blockDim.x) {
            const int64_t k = j * g.nx + 4 * q;
            const bool up = j + 1 < g.ny, right = 4 * q + 4 < g.nx;
            const float4 ez = ld4(g.f[2], k), ey = ld4(g.f[1], k), ex = ld4(g.f[0], k);
            const float4 ezu = up ? ld4(g.f[2], k + g.nx) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 exu = up ? ld4(g.f[0], k + g.nx) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float ezr = right ? g.f[2][k + 4] : 0.0f, eyr = right ? g.f[1][k + 4] : 0.0f;
            float4 bx = ld4(g.f[3], k), by = ld4(g.f[4], k), bz = ld4(g.f[5], k);
            const float vez[5] = {ez.x, ez.y, ez.z, ez.w, ezr};
            const float vey[5] = {ey.x, ey.y, ey.z, ey.w, eyr};
            const float vezu[4] = {ezu.x, ezu.y, ezu.z, ezu.w};
            const float vex[4] = {ex.x, ex.y, ex.z, ex.w}, vexu[4] = {exu.x, exu.y, exu.z, exu.w};
            float *pbx = &bx.x, *pby = &by.x, *pbz = &bz.x;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float dEz_dy = (vezu[c] - vez[c]) * idy;
                const float dEz_dx = (vez[c + 1] - vez[c]) * idx;
                const float dEy_dx = (vey[c + 1] - vey[c]) * idx;
                const float dEx_dy = (vexu[c] - vex[c]) * idy;
                pbx[c] -= dtb * dEz_dy;
                pby[c] += dtb * dEz_dx;
                pbz[c] -= dtb * (dEy_dx - dEx_dy);
            }
            *reinterpret_cast<float4 *>(g.f[3] + k) = bx;
            *reinterpret_cast<float4 *>(g.f[4] + k) = by;
            *reinterpret_cast<float4 *>(g.f[5] + k) = bz;
        }
}

__global__ void __launch_bounds__(kPicBlock) k_yee_e4(YeeGrid g, float idx, float idy,
                                                      const float *jx, const float *jy,
                                                      const float *jz, float dt)
{
    const int64_t nq = g.nx / 4;
    for (int64_t j = blockIdx.y; j < g.ny; j += gridDim.y)
        for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq;
             q += (int64_t)gridDim.x * blockDim.x) {
            const int64_t k = j * g.nx + 4 * q;
            const bool down = j > 0, left = q > 0;
            const float4 bz = ld4(g.f[5], k), by = ld4(g.f[4], k), bx = ld4(g.f[3], k);
            const float4 bzd = down ? ld4(g.f[5], k - g.nx) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 bxd = down ? ld4(g.f[3], k - g.nx) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float bzl = left ? g.f[5][k - 1] : 0.0f, byl = left ? g.f[4][k - 1] : 0.0f;
            const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 cx = jx ? ld4(jx, k) : z4, cy = jy ? ld4(jy, k) : z4,
                         cz = jz ? ld4(jz, k) : z4;
            float4 ex = ld4(g.f[0], k), ey = ld4(g.f[1], k), ez = ld4(g.f[2], k);
            const float vbz[5] = {bzl, bz.x, bz.y, bz.z, bz.w};
            const float vby[5] = {byl, by.x, by.y, by.z, by.w};
            const float vbzd[4] = {bzd.x, bzd.y, bzd.z, bzd.w};
            const float vbx[4] = {bx.x, bx.y, bx.z, bx.w}, vbxd[4] = {bxd.x, bxd.y, bxd.z, bxd.w};
            const float vjx[4] = {cx.x, cx.y, cx.z, cx.w}, vjy[4] = {cy.x, cy.y, cy.z, cy.w},
                        vjz[4] = {cz.x, cz.y, cz.z, cz.w};
            float *pex = &ex.x, *pey = &ey.x, *pez = &ez.x;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float dBz_dy = (vbz[c + 1] - vbzd[c]) * idy;
                const float dBz_dx = (vbz[c + 1] - vbz[c]) * idx;
                const float dBy_dx = (vby[c + 1] - vby[c]) * idx;
                const float dBx_dy = (vbx[c] - vbxd[c]) * idy;
                pex[c] += dt * (dBz_dy - vjx[c]);
                pey[c] += dt * (-dBz_dx - vjy[c]);
                pez[c] += dt * (dBy_dx - dBx_dy - vjz[c]);
            }
            *reinterpret_cast<float4 *>(g.f[0] + k) = ex;
            *reinterpret_cast<float4 *>(g.f[1] + k) = ey;
            *reinterpret_cast<float4 *>(g.f[2] + k) = ez;
        }
}

// One thread a particle: q w v / (dx dy) spread with the linear weights of
// each component's staggering at the mid-step position x - v dt/2 (after a
// step: x^(n+1) and v^(n+1/2)).  FP32 atomic sums (their order varies).
// Constants of the deposition: FP32, with the grid's 1/dx, 1/dy and
// x0/dx, y0/dy as float pairs (hi + lo) so that the cell coordinate of a
// position keeps double-float precision without an FP64 instruction.
struct DepositConsts {
    float q_area;                    // q / (dx dy)
    float idx_hi, idx_lo, idy_hi, idy_lo;
    float x0s_hi, x0s_lo, y0s_hi, y0s_lo;
    float hdt_x, hdt_y;              // dt / (2 dx), dt / (2 dy)
};

// Cell and in-cell fraction of a double-float cell coordinate (the fraction
// in [0, 1) from the pair's two parts).
__device__ __forceinline__ float cell_of(df2 a, float &frac)
{
    float f = floorf(a.hi);
    float r = (a.hi - f) + a.lo;
    if (r < 0.0f) {
        r += 1.0f;
        f -= 1.0f;
    }
    if (r >= 1.0f) {
        r -= 1.0f;
        f += 1.0f;
    }
    frac = r;
    return f;
}

// J += q w v at the mid-step position x - v dt/2, linear weights on each
// component's staggered nodes (Jx at i+1/2, Jy at j+1/2, Jz at the node).
// The FP64 state is read as double-float positions and nearest-float
// momenta and weights by integer instructions (qp_df.h): no instruction
// runs on the FP64 pipe.
__global__ void __launch_bounds__(kPicBlock) k_deposit(SpeciesDev S, DepositConsts c, YeeGrid g,
                                                       float *jx, float *jy, float *jz,
                                                       int *status)
{
    long long n = *((volatile long long *)S.n_live);
    if (n < 0 || n > S.cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) raise_status(status, QP_ERR_INVALID_ARG);
        n = n < 0 ? 0 : S.cap;
    }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    float *J[3] = {jx, jy, jz};
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        const double xd = S.x[p], yd = S.y[p], uxd = S.ux[p], uyd = S.uy[p], uzd = S.uz[p],
                     wd = S.w[p];
        const float ux = hi_d(uxd), uy = hi_d(uyd), uz = hi_d(uzd);
        const float ig = rsqrtf(1.0f + ux * ux + uy * uy + uz * uz);
        const float v[3] = {ux * ig, uy * ig, uz * ig};
        // mid-step position in cells
        const df2 gx = df_add_f(df_sub(df_mul(split_d(xd), {c.idx_hi, c.idx_lo}),
                                       {c.x0s_hi, c.x0s_lo}),
                                -c.hdt_x * v[0]);
        const df2 gy = df_add_f(df_sub(df_mul(split_d(yd), {c.idy_hi, c.idy_lo}),
                                       {c.y0s_hi, c.y0s_lo}),
                                -c.hdt_y * v[1]);
        const float a = c.q_area * hi_d(wd);
        float fx0, fy0, fxh, fyh;
        const float fi0 = cell_of(gx, fx0), fj0 = cell_of(gy, fy0);
        const float fih = cell_of(df_add_f(gx, -0.5f), fxh), fjh = cell_of(df_add_f(gy, -0.5f), fyh);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            // Jx: x - 1/2 in cells; Jy: y - 1/2; Jz: the node itself
            const float fi = k == 0 ? fih : fi0, fj = k == 1 ? fjh : fj0;
            const float fx = k == 0 ? fxh : fx0, fy = k == 1 ? fyh : fy0;
            if (!(fi >= -1.0f && fj >= -1.0f && fi < (float)g.nx && fj < (float)g.ny)) continue;
            const int64_t i = (int64_t)fi, j = (int64_t)fj;
            const float av = a * v[k];
            if (av == 0.0f) continue;
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int64_t ii = i + e, jj = j + b;
                    if (ii < 0 || jj < 0 || ii >= g.nx || jj >= g.ny) continue;
                    const float wgt = (e ? fx : 1.0f - fx) * (b ? fy : 1.0f - fy);
                    atomicAdd(&J[k][jj * g.nx + ii], av * wgt);
                }
        }
    }
}

// Blocks of the node kernels: enough column blocks for a row, rows over
// blockIdx.y (a grid of about 8 blocks an SM; each block strides over rows).
dim3 node_grid(const YeeGrid &g, int num_sms)
{
    int64_t bx = (g.nx + kPicBlock - 1) / kPicBlock;
    if (bx > 64) bx = 64;
    if (bx < 1) bx = 1;
    int64_t by = (int64_t)num_sms * 8 / bx;
    if (by > g.ny) by = g.ny;
    if (by > 65535) by = 65535;
    return dim3((unsigned)bx, (unsigned)(by > 0 ? by : 1));
}

dim3 quad_grid(const YeeGrid &g, int num_sms)
{
    YeeGrid q = g;
    q.nx = g.nx / 4;
    return node_grid(q, num_sms);
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0u; }

// Rows of whole float4s: nx a multiple of 4 and every array 16-byte aligned.
bool quads(const YeeGrid &g, const float *jx = nullptr, const float *jy = nullptr,
           const float *jz = nullptr)
{
    if (g.nx % 4 != 0) return false;
    for (int c = 0; c < 6; ++c)
        if (!aligned16(g.f[c])) return false;
    return aligned16(jx) && aligned16(jy) && aligned16(jz);
}

int grid_blocks(int64_t n, int num_sms)
{
    int64_t b = (n + kPicBlock - 1) / kPicBlock;
    const int64_t cap = (int64_t)num_sms * 8;
    if (b > cap) b = cap;
    return (int)(b > 0 ? b : 1);
}

}  // namespace

cudaError_t launch_yee_b(const YeeGrid &g, double dtb, int num_sms, cudaStream_t st)
{
    // 1/dx and 1/dy once, as each node would form them (FP64 quotient to float)
    const float idx = (float)(1.0 / g.dx), idy = (float)(1.0 / g.dy);
    if (quads(g))
        k_yee_b4<<<quad_grid(g, num_sms), kPicBlock, 0, st>>>(g, idx, idy, (float)dtb);
    else
        k_yee_b<<<node_grid(g, num_sms), kPicBlock, 0, st>>>(g, idx, idy, (float)dtb);
    return cudaGetLastError();
}

cudaError_t launch_yee_e(const YeeGrid &g, const float *jx, const float *jy, const float *jz,
                         double dt, int num_sms, cudaStream_t st)
{
    const float idx = (float)(1.0 / g.dx), idy = (float)(1.0 / g.dy);
    if (quads(g, jx, jy, jz))
        k_yee_e4<<<quad_grid(g, num_sms), kPicBlock, 0, st>>>(g, idx, idy, jx, jy, jz,
                                                              (float)dt);
    else
        k_yee_e<<<node_grid(g, num_sms), kPicBlock, 0, st>>>(g, idx, idy, jx, jy, jz,
                                                             (float)dt);
    return cudaGetLastError();
}

cudaError_t launch_deposit(const SpeciesDev &S, double q, double dt, const YeeGrid &g, float *jx,
                           float *jy, float *jz, int *status, int num_sms, cudaStream_t st)
{
    DepositConsts c;
    const double idx = 1.0 / g.dx, idy = 1.0 / g.dy, x0s = g.x0 * idx, y0s = g.y0 * idy;
    auto split = [](double v, float &hi, float &lo) {
        hi = (float)v;
        lo = (float)(v - (double)hi);
    };
    c.q_area = (float)(q / (g.dx * g.dy));
    split(idx, c.idx_hi, c.idx_lo);
    split(idy, c.idy_hi, c.idy_lo);
    split(x0s, c.x0s_hi, c.x0s_lo);
    split(y0s, c.y0s_hi, c.y0s_lo);
    c.hdt_x = (float)(0.5 * dt * idx);
    c.hdt_y = (float)(0.5 * dt * idy);
    k_deposit<<<grid_blocks(S.cap, num_sms), kPicBlock, 0, st>>>(S, c, g, jx, jy, jz, status);
    return cudaGetLastError();
}

}  // namespace qp
