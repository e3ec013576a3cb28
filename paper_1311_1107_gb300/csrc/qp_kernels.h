// Launch wrappers of the libqedpic kernels (defined in qp_kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "qp_device.cuh"

namespace qp {

cudaError_t launch_step(const StepArgs &a, int precision, int field_kind, bool batch, int grid,
                        cudaStream_t st);
int step_blocks_per_sm(int precision, int field_kind, bool batch);
// per-precision instantiations of the step kernel (qp_step_fp64.cu, qp_step_mixed.cu)
const void *step_kernel_fp64(int field_kind, bool batch);
const void *step_kernel_mixed(int field_kind, bool batch);
size_t step_smem_fp64();
size_t step_smem_mixed();
size_t step_smem_bytes(int precision);
// Fused steps (qp_step_fused): one window of K steps of the single problem
// a.single (its time set for the window's first step).  The physics pass
// stages each new photon at a provisional index (arrival order) with its
// order key (step, emitter, emission index); launch_fused_order
// (qp_coalesce.cu, on the coalescence scratch) sorts the keys; the photon
// pass moves the window's photons and writes the new ones at their slots in
// the order of K separate steps.  win: [0] photons at the window start,
// [1] photons it stored, [2] photons it staged (all it emitted up to the
// capacity; those past the free slots in key order are dropped, as K
// separate steps drop them).
struct FusedScratch {
    double *stage[8];               // x y z ux uy uz tau w of the new photons
    unsigned long long *rkeys;      // order key of each provisional photon
    unsigned short *moves_new;      // steps left to each provisional photon
    long long *alloc;               // provisional indices taken
    const unsigned *order;          // provisional index of each slot (sorted)
    const unsigned long long *sorted_keys;  // their keys
};
FusedScratch fused_scratch(void *scratch, int64_t photon_cap, int grid, int key_bits);
cudaError_t launch_fused_order(const SpeciesDev &Ph, void *scratch, int grid, int key_bits,
                               long long *win, int *status, cudaStream_t st);
// Bits of the order key of a window of K steps over `tiles` lepton tiles.
int fused_key_bits(int K, long long tiles, int *ordinal_bits);
cudaError_t launch_fused(const StepArgs &a, int precision, int field_kind, int K,
                         long long tiles_e, long long tiles, void *scratch, int order_grid,
                         long long *win, int num_sms, cudaStream_t st);
const void *fused_kernel_fp64(int field_kind);
const void *fused_kernel_mixed(int field_kind);
const void *fused_photons_fp64();
const void *fused_photons_mixed();
cudaError_t launch_init_tau(double *tau, int64_t first, int64_t count, int64_t id_base,
                            int64_t id_split, int64_t id_append, uint64_t seed, int species,
                            cudaStream_t st);
cudaError_t launch_diag(const SpeciesDev &S, int is_photon, double *partials, int nblocks,
                        double *out, cudaStream_t st);
cudaError_t launch_wait_selftest(unsigned long long *words, unsigned spin_limit, int *status,
                                 cudaStream_t st);

// A 2D Yee grid (qp_pic.cu): six float components, ny rows of nx values.
struct YeeGrid {
    float *f[6];  // Ex Ey Ez Bx By Bz
    int64_t nx, ny;
    double dx, dy, x0, y0;
};
cudaError_t launch_yee_b(const YeeGrid &g, double dtb, int num_sms, cudaStream_t st);
cudaError_t launch_yee_e(const YeeGrid &g, const float *jx, const float *jy, const float *jz,
                         double dt, int num_sms, cudaStream_t st);
cudaError_t launch_deposit(const SpeciesDev &S, double q, double dt, const YeeGrid &g, float *jx,
                           float *jy, float *jz, int *status, int num_sms, cudaStream_t st);
// Stable sort of a species' live slots by cell of g (qp_coalesce.cu; the
// coalescence scratch, stats as there).
cudaError_t launch_sort_cells(const SpeciesDev &S, const YeeGrid &g, void *scratch, int grid,
                              long long *stats, int *status, cudaStream_t st);

// Compaction / coalescence of a photon species (qp_coalesce.cu): scratch
// bytes for `cap` slots and `grid` blocks, and the stream-ordered pipeline
// (P = NULL: compaction only).  stats: 4 device int64 (groups merged,
// photons merged, slots before, slots after).
size_t coalesce_scratch_bytes(int64_t cap, int grid);
cudaError_t launch_coalesce(const SpeciesDev &S, const qp_coalesce_params *P, void *scratch,
                            int grid, long long *stats, int *status, cudaStream_t st);

// Refill of a 2D Yee grid's E_y and B_z with the 2D Gaussian pulse at time t
// (qp_fill_yee2d): one launch, no scratch.
struct Pulse2DDev {
    double a0, w0, tau_fwhm, x_focus, t_focus, y_axis;
};
cudaError_t launch_pulse_fill(const Pulse2DDev &p, int64_t nx, int64_t ny, double dx, double dy,
                              double x0, double y0, double t, float *ey, float *bz,
                              cudaStream_t st);

constexpr int kDiagBlocks = 256;
constexpr int kDiagWords = 8 + QP_HIST_BINS;  // scalars + histogram per block

}  // namespace qp
