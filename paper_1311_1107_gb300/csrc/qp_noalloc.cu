// Allocation-free diagnostics (qp_diagnostics_noalloc): the fixed-order
// species reduction of qp_diagnostics with its scratch in a static device
// array instead of context memory, for callers that cannot allocate.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "qedpic.h"
#include "qp_kernels.h"

namespace {

// One partial row per 256-slot tile, then the final row.
constexpr size_t kScratchWords = (size_t)(QP_NOALLOC_MAX_TILES + 1) * qp::kDiagWords;
static __device__ __align__(256) double g_noalloc_scratch[kScratchWords];

// Device address of the array, looked up once per device with that device
// current (in host code the symbol is only a host-side stand-in, never an
// address a kernel may be given).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch[kMaxDevices] = {nullptr};

int scratch_for_device(int dev, double **out)
{
    if (dev < 0 || dev >= kMaxDevices) return QP_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return QP_ERR_CUDA;
        g_scratch[dev] = (double *)p;
    }
    *out = g_scratch[dev];
    return QP_OK;
}

// The device that owns the species' buffers (its live counter), else the
// current device.
int owning_device(const qp_species_desc *d, int current)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, d->n_live) != cudaSuccess) {
        (void)cudaGetLastError();  // a host pointer is not an error to keep
        return current;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged ? at.device
                                                                                : current;
}

// Makes `dev` current for the life of the guard and restores the caller's
// device afterwards.
struct DeviceSwitch {
    int prev = -1;
    bool ok = true;
    DeviceSwitch(int dev, int current) : prev(current)
    {
        if (dev != current) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceSwitch()
    {
        int now = -1;
        if (cudaGetDevice(&now) == cudaSuccess && now != prev) (void)cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" int qp_diagnostics_noalloc(const qp_species_desc *d, qp_diag *out, void *stream)
{
    if (!d || !out) return QP_ERR_INVALID_ARG;
    if (d->kind < QP_ELECTRON || d->kind > QP_PHOTON || (d->dims != 2 && d->dims != 3) ||
        d->capacity < 0 || !d->n_live)
        return QP_ERR_INVALID_ARG;
    if (d->capacity > (int64_t)QP_NOALLOC_MAX_SLOTS) return QP_ERR_INVALID_ARG;
    if (d->capacity > 0 && (!d->x || !d->y || !d->ux || !d->uy || !d->uz || !d->tau || !d->w))
        return QP_ERR_INVALID_ARG;
    int current = -1;
    if (cudaGetDevice(&current) != cudaSuccess) return QP_ERR_CUDA;
    const int dev = owning_device(d, current);
    DeviceSwitch guard(dev, current);
    if (!guard.ok) return QP_ERR_CUDA;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cap) != cudaSuccess) return QP_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return QP_ERR_INVALID_ARG;  // it synchronises
    double *scratch = nullptr;
    int st = scratch_for_device(dev, &scratch);
    if (st != QP_OK) return st;

    qp::SpeciesDev S{};
    S.x = d->x;
    S.y = d->y;
    S.z = d->dims == 3 ? d->z : nullptr;
    S.ux = d->ux;
    S.uy = d->uy;
    S.uz = d->uz;
    S.tau = d->tau;
    S.w = d->w;
    S.chi = d->chi;
    S.nemit = d->nemit;
    S.n_live = d->n_live;
    S.cap = d->capacity;
    S.present = 1;
    // one block per tile: every partial row read by the final pass is
    // written by this call (tiles past the live count write zeros)
    int tiles = (int)((d->capacity + qp::kDiagTile - 1) / qp::kDiagTile);
    if (tiles < 1) tiles = 1;
    double *partials = scratch;
    double *fin = scratch + (size_t)QP_NOALLOC_MAX_TILES * qp::kDiagWords;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = qp::launch_diag(S, d->kind == QP_PHOTON, partials, tiles, fin, s);
    double h[qp::kDiagWords];
    int64_t n_live = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, fin, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&n_live, d->n_live, sizeof(n_live), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? QP_ERR_OOM : QP_ERR_CUDA;
    memset(out, 0, sizeof(*out));
    out->n_live = n_live;
    out->n_alive = (int64_t)llround(h[0]);
    out->weight = h[1];
    out->energy = h[2];
    out->px = h[3];
    out->py = h[4];
    out->pz = h[5];
    out->chi_mean = (d->chi && h[1] > 0.0) ? h[6] / h[1] : 0.0;
    for (int k = 0; k < QP_HIST_BINS; ++k) out->hist[k] = h[8 + k];
    return QP_OK;
}
