// C ABI of libqedpic: context, species registry, argument checks, launches.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>
#include <new>
#include <vector>

#include "qedpic.h"
#include "qp_internal.h"
#include "qp_kernels.h"

namespace {

constexpr int kMaxSpecies = 4096;
// Bound of every look-back wait (iterations of a ~64 ns sleep): about a
// second, far above the time any predecessor tile needs.
constexpr unsigned kSpinLimit = 1u << 24;

struct SpeciesRec {
    qp_species_desc d;
    bool live = false;
};

// FP64 tables are built once per process and shared by every context.
std::mutex g_tab_mu;
qp::HostTables *g_host_tables = nullptr;

const qp::HostTables *host_tables()
{
    std::lock_guard<std::mutex> lk(g_tab_mu);
    if (!g_host_tables) {
        qp::HostTables *t = new (std::nothrow) qp::HostTables;
        if (!t) return nullptr;
        qp::build_tables_host(t);
        g_host_tables = t;
    }
    return g_host_tables;
}

}  // namespace

struct qp_ctx {
    int device = 0;
    int num_sms = 1;
    double lambda_m = 0.0;
    qp::Units U{};
    // tables: FP64 H Gs Ts Cg Cp, then FP32 copies in the same order
    double *d_tab64 = nullptr;
    float *d_tab32 = nullptr;
    unsigned char *d_guide = nullptr; // guide tables of the CDF rows (emission, pair)
    qp::DevStats *d_stats = nullptr;  // [kMaxSpecies]
    qp::StepCtl *d_ctl = nullptr;     // ticket, done, epoch of qp_step launches
    long long *d_pending = nullptr;   // [3] new live counts of a qp_step launch
    int *d_status = nullptr;
    unsigned long long *d_chain = nullptr;  // lepton chain then photon chain
    size_t chain_words = 0;           // words per chain
    double *d_diag = nullptr;         // partials + final
    double *d_stash = nullptr;        // append records of qp_step launches
    size_t stash_blocks = 0;          // blocks the stash is sized for
    void *d_fuse = nullptr;           // scratch of qp_step_fused
    size_t fuse_bytes = 0;
    void *d_coal = nullptr;           // scratch of qp_coalesce_photons
    size_t coal_bytes = 0;
    long long *d_coal_stats = nullptr;  // [4] of the last coalescence
    long long *h_counts = nullptr;    // [3] pinned: live counts of qp_step_host
    std::vector<SpeciesRec> species;
    int grid_cache[2][2][5];          // [batch][precision][field] blocks per SM, 0 = unknown
    // kernel timing (qp_profile_*): event pool and (kernel, start event) records
    bool profiling = false;
    std::vector<cudaEvent_t> events;
    size_t events_used = 0;
    std::vector<int> records;         // kernel id per recorded pair
};

namespace {

// device layout: H Gs Ts rows of kNRatePad entries, then the CDF rows
constexpr size_t kTabRate = 3 * (size_t)qp::kNRatePad;
constexpr size_t kTabCdf = 2 * (size_t)qp::kNCdf * qp::kNNode;
constexpr size_t kTabWords = kTabRate + kTabCdf;
// FP32 layout: the rate rows, the CDF rows and their complements as float
// pairs (4 kTabCdf floats), then e^(-s_j) at the 2 x kNNode logit nodes
constexpr size_t kTab32 = kTabRate + 4 * kTabCdf + 2 * (size_t)qp::kNNode;

constexpr size_t kGuideHalf = (size_t)qp::kNCdf * qp::kGuideBuckets;

// Guide tables of one CDF table (kNCdf rows of kNNode nodes): [half][row][bucket].
// Lower half, bucket m of xi in (0, 1/2]: the last node j <= 254 with C_j
// below the bucket's lower edge; upper half, bucket m of eta = 1 - xi: the
// last node with 1 - C_j above the bucket's upper edge (0 if none).  The
// margins keep every entry at or before the node a search would find.
void build_guides(const double *rows, unsigned char *g)
{
    for (int r = 0; r < qp::kNCdf; ++r) {
        const double *C = rows + (size_t)r * qp::kNNode;
        for (int m = 0; m < qp::kGuideBuckets; ++m) {
            const int e = -1 - (m >> 2), k = m & 3;
            const double lo_edge = ldexp(1.0 + k / 4.0, e), hi_edge = ldexp(1.0 + (k + 1) / 4.0, e);
            int gl = 0, gu = 0;
            for (int j = 0; j < qp::kNNode - 1; ++j) {
                if (C[j] < lo_edge * (1.0 - 1e-9)) gl = j;
                if (1.0 - C[j] > hi_edge * (1.0 + 1e-9)) gu = j;
            }
            g[(size_t)r * qp::kGuideBuckets + m] = (unsigned char)gl;
            g[kGuideHalf + (size_t)r * qp::kGuideBuckets + m] = (unsigned char)gu;
        }
    }
}

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return QP_OK;
    if (e == cudaErrorMemoryAllocation) return QP_ERR_OOM;
    return QP_ERR_CUDA;
}

void release(qp_ctx *c)
{
    if (!c) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    cudaFree(c->d_tab64);
    cudaFree(c->d_tab32);
    cudaFree(c->d_guide);
    cudaFree(c->d_stats);
    cudaFree(c->d_ctl);
    cudaFree(c->d_pending);
    cudaFree(c->d_status);
    cudaFree(c->d_chain);
    cudaFree(c->d_diag);
    cudaFree(c->d_stash);
    cudaFree(c->d_coal);
    cudaFree(c->d_coal_stats);
    cudaFree(c->d_fuse);
    cudaFreeHost(c->h_counts);
    if (prev >= 0) cudaSetDevice(prev);
    delete c;
}

// RAII switch to the context's device for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

bool valid_handle(const qp_ctx *c, int32_t h)
{
    return c && h >= 0 && (size_t)h < c->species.size() && c->species[h].live;
}

// Make the look-back scratch large enough for `words` tiles per chain.
int ensure_chain(qp_ctx *c, size_t words)
{
    if (words <= c->chain_words) return QP_OK;
    unsigned long long *p = nullptr;
    cudaError_t e = cudaMalloc(&p, 2 * words * sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaMemset(p, 0, 2 * words * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        cudaFree(p);
        return cuda_status(e);
    }
    cudaFree(c->d_chain);
    c->d_chain = p;
    c->chain_words = words;
    return QP_OK;
}

size_t tiles_of(int64_t cap) { return (size_t)((cap + qp::kTile - 1) / qp::kTile); }

// Bytes of the append-record stash of `blocks` resident blocks (kStashBufs
// buffers of kStashFields x kTile doubles each).
size_t stash_bytes(size_t blocks)
{
    return blocks * qp::kStashBufs * (size_t)qp::kStashFieldsHost * qp::kTile * sizeof(double);
}

// Next free event of the profiling pool (grown on demand).
cudaError_t next_event(qp_ctx *c, cudaEvent_t *ev)
{
    if (c->events_used == c->events.size()) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        c->events.push_back(e);
    }
    *ev = c->events[c->events_used++];
    return cudaSuccess;
}

// Launch one kernel of a step, bracketed by events when profiling.
template <class F>
cudaError_t timed(qp_ctx *c, int kernel_id, cudaStream_t st, F launch)
{
    if (!c->profiling) return launch();
    cudaEvent_t a, b;
    cudaError_t e = next_event(c, &a);
    if (e == cudaSuccess) e = next_event(c, &b);
    if (e == cudaSuccess) e = cudaEventRecord(a, st);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) c->records.push_back(kernel_id);
    return e;
}

qp::SpeciesDev species_dev(const qp_ctx *c, int32_t h)
{
    qp::SpeciesDev s{};
    if (!valid_handle(c, h)) return s;
    const qp_species_desc &d = c->species[h].d;
    s.x = d.x;
    s.y = d.y;
    s.z = d.dims == 3 ? d.z : nullptr;
    s.ux = d.ux;
    s.uy = d.uy;
    s.uz = d.uz;
    s.tau = d.tau;
    s.w = d.w;
    s.chi = d.chi;
    s.nemit = d.nemit;
    s.n_live = d.n_live;
    s.cap = d.capacity;
    s.id_base = d.id_base;
    s.id_split = d.id_split;
    s.id_append = d.id_append;
    s.present = 1;
    s.slot_stats = h;
    return s;
}

}  // namespace

extern "C" {

const char *qp_status_string(int status)
{
    switch (status) {
    case QP_OK: return "QP_OK";
    case QP_WARN_BUFFER_FULL: return "QP_WARN_BUFFER_FULL";
    case QP_WARN_TABLE_CLAMPED: return "QP_WARN_TABLE_CLAMPED";
    case QP_ERR_INVALID_ARG: return "QP_ERR_INVALID_ARG";
    case QP_ERR_CUDA: return "QP_ERR_CUDA";
    case QP_ERR_OOM: return "QP_ERR_OOM";
    case QP_ERR_NOT_INITIALIZED: return "QP_ERR_NOT_INITIALIZED";
    case QP_ERR_TIMEOUT: return "QP_ERR_TIMEOUT";
    default: return "QP_UNKNOWN_STATUS";
    }
}

int qp_init_tables(const qp_table_params *p, qp_ctx **out_ctx)
{
    if (!out_ctx) return QP_ERR_INVALID_ARG;
    *out_ctx = nullptr;
    if (!p || !(p->lambda_m > 0.0) || !isfinite(p->lambda_m) || p->device < 0 || p->reserved != 0)
        return QP_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || p->device >= ndev) return QP_ERR_CUDA;
    const qp::HostTables *T = host_tables();
    if (!T) return QP_ERR_OOM;

    qp_ctx *c = new (std::nothrow) qp_ctx;
    if (!c) return QP_ERR_OOM;
    memset(c->grid_cache, 0, sizeof(c->grid_cache));
    c->device = p->device;
    c->lambda_m = p->lambda_m;
    qp::units_for_wavelength(p->lambda_m, &c->U);
    DeviceGuard g(c->device);
    if (!g.ok) {
        delete c;
        return QP_ERR_CUDA;
    }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (c->num_sms < 1) c->num_sms = 1;

    std::vector<double> h64(kTabWords, 0.0);
    std::vector<float> h32(kTab32);
    memcpy(h64.data(), T->H, sizeof(T->H));
    memcpy(h64.data() + qp::kNRatePad, T->Gs, sizeof(T->Gs));
    memcpy(h64.data() + 2 * qp::kNRatePad, T->Ts, sizeof(T->Ts));
    memcpy(h64.data() + kTabRate, T->Cg, sizeof(T->Cg));
    memcpy(h64.data() + kTabRate + qp::kNCdf * qp::kNNode, T->Cp, sizeof(T->Cp));
    for (size_t k = 0; k < kTabRate; ++k) h32[k] = (float)h64[k];
    // CDF rows (emission then pair) as hi + lo pairs, then their complements
    for (size_t k = 0; k < kTabCdf; ++k) {
        const double c = h64[kTabRate + k], q = 1.0 - c;
        const float ch = (float)c, qh = (float)q;
        h32[kTabRate + 2 * k] = ch;
        h32[kTabRate + 2 * k + 1] = (float)(c - (double)ch);
        h32[kTabRate + 2 * kTabCdf + 2 * k] = qh;
        h32[kTabRate + 2 * kTabCdf + 2 * k + 1] = (float)(q - (double)qh);
    }
    // e^(-s_j) at the logit nodes of the emission and pair rows
    for (int j = 0; j < qp::kNNode; ++j) {
        h32[kTabRate + 4 * kTabCdf + j] =
            (float)exp(-(qp::kSgMin + qp::kSgSpan * j / (qp::kNNode - 1)));
        h32[kTabRate + 4 * kTabCdf + qp::kNNode + j] =
            (float)exp(-(qp::kSpMin + qp::kSpSpan * j / (qp::kNNode - 1)));
    }

    cudaError_t e = cudaSuccess;
#define QP_TRY(x)                    \
    do {                             \
        e = (x);                     \
        if (e != cudaSuccess) {      \
            release(c);              \
            return cuda_status(e);   \
        }                            \
    } while (0)
    std::vector<unsigned char> guide(4 * kGuideHalf);
    build_guides(T->Cg, guide.data());
    build_guides(T->Cp, guide.data() + 2 * kGuideHalf);
    QP_TRY(cudaMalloc(&c->d_guide, guide.size()));
    QP_TRY(cudaMemcpy(c->d_guide, guide.data(), guide.size(), cudaMemcpyHostToDevice));
    QP_TRY(cudaMalloc(&c->d_tab64, kTabWords * sizeof(double)));
    QP_TRY(cudaMalloc(&c->d_tab32, kTab32 * sizeof(float)));
    QP_TRY(cudaMemcpy(c->d_tab64, h64.data(), kTabWords * sizeof(double), cudaMemcpyHostToDevice));
    QP_TRY(cudaMemcpy(c->d_tab32, h32.data(), kTab32 * sizeof(float),
                      cudaMemcpyHostToDevice));
    QP_TRY(cudaMalloc(&c->d_stats, kMaxSpecies * sizeof(qp::DevStats)));
    QP_TRY(cudaMemset(c->d_stats, 0, kMaxSpecies * sizeof(qp::DevStats)));
    QP_TRY(cudaMalloc(&c->d_ctl, sizeof(qp::StepCtl)));
    QP_TRY(cudaMemset(c->d_ctl, 0, sizeof(qp::StepCtl)));
    QP_TRY(cudaMalloc(&c->d_pending, 4 * sizeof(long long)));
    QP_TRY(cudaMemset(c->d_pending, 0, 4 * sizeof(long long)));
    QP_TRY(cudaMalloc(&c->d_status, sizeof(int)));
    QP_TRY(cudaMemset(c->d_status, 0, sizeof(int)));
    QP_TRY(cudaMalloc(&c->d_diag, (qp::kDiagBlocks + 1) * qp::kDiagWords * sizeof(double)));
#undef QP_TRY
    int st = ensure_chain(c, 16);
    if (st != QP_OK) {
        release(c);
        return st;
    }
    *out_ctx = c;
    return QP_OK;
}

int qp_destroy(qp_ctx *ctx)
{
    release(ctx);
    return QP_OK;
}

int qp_create_species(qp_ctx *ctx, const qp_species_desc *d, int32_t *out_handle)
{
    if (!ctx) return QP_ERR_NOT_INITIALIZED;
    if (!d || !out_handle) return QP_ERR_INVALID_ARG;
    if (d->kind < QP_ELECTRON || d->kind > QP_PHOTON) return QP_ERR_INVALID_ARG;
    if (d->dims != 2 && d->dims != 3) return QP_ERR_INVALID_ARG;
    if (d->capacity < 0 || !d->n_live || d->id_base < 0) return QP_ERR_INVALID_ARG;
    if (d->id_split < 0 || (d->id_split > 0 && d->id_append < 0)) return QP_ERR_INVALID_ARG;
    if (d->dims == 2 && d->z) return QP_ERR_INVALID_ARG;
    if (d->capacity > 0 && (!d->x || !d->y || !d->ux || !d->uy || !d->uz || !d->tau || !d->w ||
                            (d->dims == 3 && !d->z)))
        return QP_ERR_INVALID_ARG;
    // a free record (of a destroyed species) is reused; its counter block is
    // cleared by qp_reset_counters or qp_batch_set
    size_t h = 0;
    while (h < ctx->species.size() && ctx->species[h].live) ++h;
    if (h >= (size_t)kMaxSpecies) return QP_ERR_INVALID_ARG;
    SpeciesRec r;
    r.d = *d;
    r.live = true;
    if (h == ctx->species.size())
        ctx->species.push_back(r);
    else
        ctx->species[h] = r;
    *out_handle = (int32_t)h;
    return QP_OK;
}

int qp_destroy_species(qp_ctx *ctx, int32_t handle)
{
    if (!ctx) return QP_ERR_NOT_INITIALIZED;
    if (!valid_handle(ctx, handle)) return QP_ERR_NOT_INITIALIZED;
    ctx->species[handle].live = false;
    return QP_OK;
}

int qp_init_optical_depth(qp_ctx *ctx, int32_t handle, uint64_t seed, int64_t first,
                          int64_t count, void *stream)
{
    if (!ctx) return QP_ERR_NOT_INITIALIZED;
    if (!valid_handle(ctx, handle)) return QP_ERR_NOT_INITIALIZED;
    const qp_species_desc &d = ctx->species[handle].d;
    if (first < 0 || count < 0 || first + count > d.capacity) return QP_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return QP_ERR_CUDA;
    return cuda_status(qp::launch_init_tau(d.tau, first, count, d.id_base, d.id_split,
                                           d.id_append, seed, d.kind, (cudaStream_t)stream));
}

// Slots [first, first + count) of a species' FP64 arrays between the device
// and a host block (array k at byte k * host_pitch; slot j at byte 8 j of
// its row); the caller has checked the range and made the device current.
static cudaError_t copy_slots(const qp_species_desc &d, void *host, int64_t host_pitch,
                              int64_t first, int64_t count, int32_t to_device, cudaStream_t st,
                              bool skip_weight = false)
{
    if (count == 0) return cudaSuccess;
    double *arr[8];
    int na = 0;
    arr[na++] = d.x;
    arr[na++] = d.y;
    if (d.dims == 3) arr[na++] = d.z;
    arr[na++] = d.ux;
    arr[na++] = d.uy;
    arr[na++] = d.uz;
    arr[na++] = d.tau;
    arr[na++] = d.w;
    if (skip_weight) --na;  // the weight is the last row
    const size_t width = (size_t)count * sizeof(double);
    char *h0 = (char *)host + (size_t)first * sizeof(double);
    // device arrays at a constant pitch (one allocation): one strided copy
    const ptrdiff_t dpitch = (char *)arr[1] - (char *)arr[0];
    bool strided = dpitch >= (ptrdiff_t)width;
    for (int k = 2; k < na && strided; ++k) strided = (char *)arr[k] - (char *)arr[k - 1] == dpitch;
    cudaError_t e = cudaSuccess;
    if (strided) {
        double *d0 = arr[0] + first;
        e = to_device ? cudaMemcpy2DAsync(d0, (size_t)dpitch, h0, (size_t)host_pitch, width,
                                          (size_t)na, cudaMemcpyHostToDevice, st)
                      : cudaMemcpy2DAsync(h0, (size_t)host_pitch, d0, (size_t)dpitch, width,
                                          (size_t)na, cudaMemcpyDeviceToHost, st);
    } else {
        for (int k = 0; k < na && e == cudaSuccess; ++k) {
            char *h = h0 + (size_t)k * (size_t)host_pitch;
            e = to_device ? cudaMemcpyAsync(arr[k] + first, h, width, cudaMemcpyHostToDevice, st)
                          : cudaMemcpyAsync(h, arr[k] + first, width, cudaMemcpyDeviceToHost, st);
        }
    }
    return e;
}

int qp_species_copy(qp_ctx *ctx, int32_t handle, void *host, int64_t host_pitch, int64_t count,
                    int32_t to_device, void *stream)
{
    if (!ctx) return QP_ERR_NOT_INITIALIZED;
    if (!valid_handle(ctx, handle)) return QP_ERR_NOT_INITIALIZED;
    const qp_species_desc &d = ctx->species[handle].d;
    if (!host || count < 0 || count > d.capacity || host_pitch < 8 * count || host_pitch % 8)
        return QP_ERR_INVALID_ARG;
    if (count == 0) return QP_OK;
    DeviceGuard g(ctx->device);
    if (!g.ok) return QP_ERR_CUDA;
    return cuda_status(copy_slots(d, host, host_pitch, 0, count, to_device, (cudaStream_t)stream));
}

namespace {
int build_problem(const qp_ctx *ctx, const qp_step_params *s, qp::Problem &P);
}

int qp_step_host(qp_ctx *ctx, const qp_step_params *s, qp_host_state *st, void *stream)
{
    if (!ctx) return QP_ERR_NOT_INITIALIZED;
    if (!s || !st) return QP_ERR_INVALID_ARG;
    {
        // what qp_step would reject, before anything is copied
        qp::Problem check{};
        const int v = build_problem(ctx, s, check);
        if (v != QP_OK) return v;
    }
    const int32_t hs[3] = {s->electron, s->positron, s->photon};
    for (int k = 0; k < 3; ++k) {
        if (hs[k] == -1) continue;
        if (!valid_handle(ctx, hs[k])) return QP_ERR_NOT_INITIALIZED;
        const qp_species_desc &d = ctx->species[hs[k]].d;
        if (!st[k].host || st[k].count < 0 || st[k].count > d.capacity ||
            st[k].pitch < 8 * d.capacity || st[k].pitch % 8)
            return QP_ERR_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    if (!g.ok) return QP_ERR_CUDA;
    if (!ctx->h_counts) {
        cudaError_t e = cudaMallocHost((void **)&ctx->h_counts, 3 * sizeof(long long));
        if (e != cudaSuccess) return cuda_status(e);
    }
    const cudaStream_t cs = (cudaStream_t)stream;
    long long *hc = ctx->h_counts;
    // every return leaves no copy of the pinned counts pending (an error
    // after something was enqueued synchronises first)
    auto fail = [&](int r) {
        (void)cudaStreamSynchronize(cs);
        return r;
    };
    // the three live counters side by side in device memory (as a
    // Simulation keeps them): one copy each way instead of three
    bool adjacent = hs[0] != -1 && hs[1] != -1 && hs[2] != -1;
    for (int k = 1; k < 3 && adjacent; ++k)
        adjacent = ctx->species[hs[k]].d.n_live == ctx->species[hs[0]].d.n_live + k;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 3; ++k) {
        if (hs[k] == -1) continue;
        const qp_species_desc &d = ctx->species[hs[k]].d;
        hc[k] = st[k].count;
        e = copy_slots(d, st[k].host, st[k].pitch, 0, st[k].count, 1, cs);
        if (e != cudaSuccess) return fail(cuda_status(e));
        if (!adjacent)
            e = cudaMemcpyAsync(d.n_live, hc + k, sizeof(long long), cudaMemcpyHostToDevice, cs);
        if (e != cudaSuccess) return fail(cuda_status(e));
    }
    if (adjacent)
        e = cudaMemcpyAsync(ctx->species[hs[0]].d.n_live, hc, 3 * sizeof(long long),
                            cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) return fail(cuda_status(e));
    const int st_step = qp_step(ctx, s, stream);
    if (st_step < 0) return fail(st_step);
    // a step never lowers a live count (decayed photons keep their slots):
    // the slots live before it go back at once, behind the step on the
    // stream, without their weights (a step writes the weights of appended
    // particles only, so the host's are current); the appended slots, all
    // rows, wait for the new counts
    for (int k = 0; k < 3; ++k) {
        if (hs[k] == -1) continue;
        const qp_species_desc &d = ctx->species[hs[k]].d;
        e = copy_slots(d, st[k].host, st[k].pitch, 0, st[k].count, 0, cs, true);
        if (e != cudaSuccess) return fail(cuda_status(e));
        if (!adjacent)
            e = cudaMemcpyAsync(hc + k, d.n_live, sizeof(long long), cudaMemcpyDeviceToHost, cs);
        if (e != cudaSuccess) return fail(cuda_status(e));
    }
    if (adjacent)
        e = cudaMemcpyAsync(hc, ctx->species[hs[0]].d.n_live, 3 * sizeof(long long),
                            cudaMemcpyDeviceToHost, cs);
    if (e != cudaSuccess) return fail(cuda_status(e));
    e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return cuda_status(e);
    bool more = false;
    for (int k = 0; k < 3; ++k) {
        if (hs[k] == -1) continue;
        const qp_species_desc &d = ctx->species[hs[k]].d;
        const long long before = st[k].count, after = hc[k];
        if (after < before || after > d.capacity) return fail(QP_ERR_CUDA);  // not a step's counts
        st[k].count = after;
        if (after > before) {
            e = copy_slots(d, st[k].host, st[k].pitch, before, after - before, 0, cs);
            if (e != cudaSuccess) return fail(cuda_status(e));
            more = true;
        }
    }
    if (more) {
        e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return st_step;
}

namespace {

// Checks of a step description (everything but the species' precision and
// field kind, which the caller compares) and the problem it defines: species,
// field, constants; scratch, control words and time are set by the caller.
int build_problem(const qp_ctx *ctx, const qp_step_params *s, qp::Problem &P)
{
    if (!(s->dt > 0.0) || !isfinite(s->dt) || s->n_steps < 0 || s->step < 0)
        return QP_ERR_INVALID_ARG;
    if (s->precision != QP_FP64 && s->precision != QP_MIXED) return QP_ERR_INVALID_ARG;
    if (s->max_emissions < 1 || s->max_emissions > QP_MAX_EMISSIONS) return QP_ERR_INVALID_ARG;
    if (!(s->chi_threshold >= 0.0) || !(s->photon_min_gamma >= 0.0)) return QP_ERR_INVALID_ARG;
    const qp_field &f = s->field;
    if (f.kind < QP_FIELD_NONE || f.kind > QP_FIELD_UNIFORM_B) return QP_ERR_INVALID_ARG;
    if (f.kind == QP_FIELD_GAUSSIAN && (!(f.w0 > 0.0) || !(f.tau_fwhm > 0.0)))
        return QP_ERR_INVALID_ARG;
    if (f.kind == QP_FIELD_YEE2D) {
        // node indices are 32-bit: nx * ny (plus a row) must stay below 2^31
        if (f.nx < 1 || f.ny < 1 || f.nx > (1 << 24) || f.ny > (1 << 24) || !(f.dx > 0.0) ||
            !(f.dy > 0.0) || (f.nx + 2) * (f.ny + 2) >= ((int64_t)1 << 31))
            return QP_ERR_INVALID_ARG;
        for (int k = 0; k < 6; ++k)
            if (!f.yee[k]) return QP_ERR_INVALID_ARG;
    }
    const int32_t hs[3] = {s->electron, s->positron, s->photon};
    const int kinds[3] = {QP_ELECTRON, QP_POSITRON, QP_PHOTON};
    for (int k = 0; k < 3; ++k) {
        if (hs[k] == -1) continue;
        if (!valid_handle(ctx, hs[k])) return QP_ERR_NOT_INITIALIZED;
        if (ctx->species[hs[k]].d.kind != kinds[k]) return QP_ERR_INVALID_ARG;
    }

    P = qp::Problem{};
    for (int k = 0; k < 3; ++k)
        if (hs[k] != -1) P.sp[k] = species_dev(ctx, hs[k]);
    P.f.kind = f.kind;
    P.f.a0 = f.a0;
    P.f.w0 = f.w0;
    P.f.tau_fwhm = f.tau_fwhm;
    P.f.x_focus = f.x_focus;
    P.f.t_focus = f.t_focus;
    P.f.b0 = f.b0;
    for (int k = 0; k < 6; ++k) P.f.yee[k] = f.yee[k];
    P.f.nx = f.nx;
    P.f.ny = f.ny;
    P.f.dx = f.dx;
    P.f.dy = f.dy;
    P.f.x0 = f.x0;
    P.f.y0 = f.y0;
    if (f.kind == QP_FIELD_YEE2D) {
        P.f.inv_dx = 1.0 / f.dx;
        P.f.inv_dy = 1.0 / f.dy;
        P.f.x0s = f.x0 / f.dx;
        P.f.y0s = f.y0 / f.dy;
    }
    P.dt = s->dt;
    P.step = (uint64_t)s->step;
    P.seed = s->seed;
    P.chi_th = s->chi_threshold;
    P.gmin = s->photon_min_gamma;
    P.pairs = s->pairs ? 1 : 0;
    P.max_emit = s->max_emissions;
    // constants of the mixed path (FP32, or double-float pairs split here)
    auto hi_of = [](double v) { return (float)v; };
    auto lo_of = [](double v) { return (float)(v - (double)(float)v); };
    qp::MixedConsts &m = P.mc;
    m.xf_hi = hi_of(f.x_focus);
    m.xf_lo = lo_of(f.x_focus);
    if (f.kind == QP_FIELD_YEE2D) {
        m.idx_hi = hi_of(P.f.inv_dx);
        m.idx_lo = lo_of(P.f.inv_dx);
        m.idy_hi = hi_of(P.f.inv_dy);
        m.idy_lo = lo_of(P.f.inv_dy);
        m.x0s_hi = hi_of(P.f.x0s);
        m.x0s_lo = lo_of(P.f.x0s);
        m.y0s_hi = hi_of(P.f.y0s);
        m.y0s_lo = lo_of(P.f.y0s);
        m.nxf = (float)f.nx;
        m.nyf = (float)f.ny;
    }
    m.h[0] = (float)(-0.5 * s->dt);
    m.h[1] = (float)(0.5 * s->dt);
    m.dt = (float)s->dt;
    m.C_rate = (float)ctx->U.C_rate;
    m.inv_aS = (float)(1.0 / ctx->U.a_S);
    m.inv_aS_lo = (float)(1.0 / ctx->U.a_S - (double)m.inv_aS);
    m.tau0w = (float)ctx->U.tau0w;
    m.chi_th = (float)s->chi_threshold;
    m.gmin = (float)s->photon_min_gamma;
    m.a0 = (float)f.a0;
    m.b0 = (float)f.b0;
    if (f.kind == QP_FIELD_GAUSSIAN) {
        const double zr = 0.5 * f.w0 * f.w0;
        m.zr = (float)zr;
        m.inv_zr = (float)(1.0 / zr);
        m.inv_w0sq = (float)(1.0 / (f.w0 * f.w0));
        m.k_env = (float)(2.0 * 0.6931471805599453 / (f.tau_fwhm * f.tau_fwhm));
    }
    return QP_OK;
}

// Context-wide launch arguments: tables, counters, status, units.
void fill_globals(const qp_ctx *ctx, qp::StepArgs &a)
{
    const size_t R = qp::kNRatePad, CC = (size_t)qp::kNCdf * qp::kNNode;
    a.tab.H = ctx->d_tab64;
    a.tab.Gs = ctx->d_tab64 + R;
    a.tab.Ts = ctx->d_tab64 + 2 * R;
    a.tab.Cg = ctx->d_tab64 + 3 * R;
    a.tab.Cp = ctx->d_tab64 + 3 * R + CC;
    a.tab.Hf = ctx->d_tab32;
    a.tab.Gsf = ctx->d_tab32 + R;
    a.tab.Tsf = ctx->d_tab32 + 2 * R;
    const float2 *c2 = reinterpret_cast<const float2 *>(ctx->d_tab32 + kTabRate);
    a.tab.Cg2 = c2;
    a.tab.Cp2 = c2 + CC;
    a.tab.Qg2 = c2 + 2 * CC;
    a.tab.Qp2 = c2 + 3 * CC;
    a.tab.Eg = ctx->d_tab32 + kTabRate + 4 * kTabCdf;
    a.tab.Ep = a.tab.Eg + qp::kNNode;
    a.tab.Gg = ctx->d_guide;
    a.tab.Gp = ctx->d_guide + 2 * kGuideHalf;
    a.stats = ctx->d_stats;
    a.status = ctx->d_status;
    a.a_S = ctx->U.a_S;
    a.C_rate = ctx->U.C_rate;
    a.tau0w = ctx->U.tau0w;
    a.spin_limit = kSpinLimit;
}

int blocks_per_sm(qp_ctx *ctx, int precision, int field_kind, bool batch)
{
    const int prec = precision == QP_MIXED ? 1 : 0;
    int &bpsm = ctx->grid_cache[batch ? 1 : 0][prec][field_kind];
    if (!bpsm) bpsm = qp::step_blocks_per_sm(precision, field_kind, batch);
    return bpsm;
}

// Time of step `step` and the FP32 / double-float time constants of the
// mixed path (the kernel of a batch computes the same values on the device).
void set_time_host(qp::Problem &P, int64_t step)
{
    P.step = (uint64_t)step;
    P.t = (double)step * P.dt;
    const double tr = P.t - P.f.t_focus;
    P.mc.t_hi = (float)P.t;
    P.mc.t_lo = (float)(P.t - (double)P.mc.t_hi);
    P.mc.tr_hi = (float)tr;
    P.mc.tr_lo = (float)(tr - (double)P.mc.tr_hi);
}

// Look-back words of a problem's two chains: lepton tiles, photon tiles.
void chain_words_of(const qp_ctx *ctx, const qp_step_params *s, size_t &lep, size_t &pho)
{
    auto cap = [&](int32_t h) { return h == -1 ? (int64_t)0 : ctx->species[h].d.capacity; };
    lep = tiles_of(cap(s->electron)) + tiles_of(cap(s->positron)) + 4;
    pho = tiles_of(cap(s->photon)) + 4;
}

}  // namespace

int qp_step(qp_ctx *ctx, const qp_step_params *s, void *stream)
{
    if (!ctx) return QP_ERR_NOT_INITIALIZED;
    if (!s) return QP_ERR_INVALID_ARG;
    qp::StepArgs a{};
    int st = build_problem(ctx, s, a.single);
    if (st != QP_OK) return st;
    if (s->n_steps == 0) return QP_OK;
    DeviceGuard g(ctx->device);
    if (!g.ok) return QP_ERR_CUDA;
    size_t lep = 0, pho = 0;
    chain_words_of(ctx, s, lep, pho);
    st = ensure_chain(ctx, lep > pho ? lep : pho);
    if (st != QP_OK) return st;
    fill_globals(ctx, a);
    a.ctl = ctx->d_ctl;
    a.n_problems = 0;
    a.problems = nullptr;
    qp::Problem &P = a.single;
    P.lep_words = ctx->d_chain;
    P.pho_words = ctx->d_chain + ctx->chain_words;
    P.pending = ctx->d_pending;
    P.device_step = 0;

    // persistent grid: resident blocks, never more than the tiles the
    // species' capacities allow
    const int bpsm = blocks_per_sm(ctx, s->precision, s->field.kind, false);
    int64_t cap_tiles = 0;
    const int32_t hs[3] = {s->electron, s->positron, s->photon};
    for (int k = 0; k < 3; ++k)
        if (hs[k] != -1) cap_tiles += (int64_t)tiles_of(ctx->species[hs[k]].d.capacity);
    const int64_t resident = (int64_t)bpsm * ctx->num_sms;
    const int grid = (int)(cap_tiles < resident ? (cap_tiles > 0 ? cap_tiles : 1) : resident);
    if ((size_t)grid > ctx->stash_blocks) {
        // grows once, to the resident grid (an allocation, synchronous)
        double *p = nullptr;
        cudaError_t e = cudaMalloc(&p, stash_bytes((size_t)resident));
        if (e != cudaSuccess) return cuda_status(e);
        cudaFree(ctx->d_stash);
        ctx->d_stash = p;
        ctx->stash_blocks = (size_t)resident;
    }
    a.stash = ctx->d_stash;
    cudaStream_t cs = (cudaStream_t)stream;
    for (int32_t k = 0; k < s->n_steps; ++k) {
        set_time_host(P, s->step + k);
        cudaError_t e = timed(ctx, 0, cs, [&] {
            return qp::launch_step(a, s->precision, s->field.kind, false, grid, cs);
        });
        if (e != cudaSuccess) return cuda_status(e);
    }
    return QP_OK;
}

// ------------------------------------------------------------------ batches

struct qp_batch {
    qp_ctx *ctx = nullptr;
    int max = 0, precision = 0, field_kind = 0, grid = 1;
    qp::Problem *d_table = nullptr;   // [max]
    long long *d_step = nullptr;      // [max] next step of each problem
    long long *d_left = nullptr;      // [max] launches still to run (0 = idle slot)
    long long *d_pending = nullptr;   // [max][3]
    long long *d_work = nullptr;      // [max] live slots stepped so far
    double *d_stash = nullptr;        // append records of the batch's launches
    qp::StepCtl *d_ctl = nullptr;
    // pinned staging of the descriptors copied by qp_batch_set; entry k is
    // reused only after the copy that read it has completed (its event)
    qp::Problem *h_stage = nullptr;   // [2 max]
    long long *h_stage_ctl = nullptr; // [2 max][2]: first step, steps
    std::vector<cudaEvent_t> stage_ev;
    int stage_next = 0;
};

namespace {

void batch_release(qp_batch *b)
{
    if (!b) return;
    DeviceGuard g(b->ctx->device);
    for (cudaEvent_t e : b->stage_ev)
        if (e) cudaEventDestroy(e);
    cudaFree(b->d_table);
    cudaFree(b->d_step);
    cudaFree(b->d_left);
    cudaFree(b->d_pending);
    cudaFree(b->d_work);
    cudaFree(b->d_stash);
    cudaFree(b->d_ctl);
    cudaFreeHost(b->h_stage);
    cudaFreeHost(b->h_stage_ctl);
    delete b;
}

}  // namespace

int qp_batch_create(qp_ctx *ctx, int32_t max_problems, int32_t precision, int32_t field_kind,
                    qp_batch **out)
{
    if (!ctx) return QP_ERR_NOT_INITIALIZED;
    if (!out || max_problems < 1 || max_problems > QP_MAX_BATCH) return QP_ERR_INVALID_ARG;
    if (precision != QP_FP64 && precision != QP_MIXED) return QP_ERR_INVALID_ARG;
    if (field_kind < QP_FIELD_NONE || field_kind > QP_FIELD_UNIFORM_B) return QP_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return QP_ERR_CUDA;
    qp_batch *b = new (std::nothrow) qp_batch;
    if (!b) return QP_ERR_OOM;
    b->ctx = ctx;
    b->max = max_problems;
    b->precision = precision;
    b->field_kind = field_kind;
    b->grid = blocks_per_sm(ctx, precision, field_kind, true) * ctx->num_sms;
    const size_t n = (size_t)max_problems;
    cudaError_t e = cudaSuccess;
#define QP_TRY(x)                    \
    do {                             \
        e = (x);                     \
        if (e != cudaSuccess) {      \
            batch_release(b);        \
            return cuda_status(e);   \
        }                            \
    } while (0)
    QP_TRY(cudaMalloc(&b->d_table, n * sizeof(qp::Problem)));
    QP_TRY(cudaMemset(b->d_table, 0, n * sizeof(qp::Problem)));
    QP_TRY(cudaMalloc(&b->d_step, n * sizeof(long long)));
    QP_TRY(cudaMemset(b->d_step, 0, n * sizeof(long long)));
    QP_TRY(cudaMalloc(&b->d_left, n * sizeof(long long)));
    QP_TRY(cudaMemset(b->d_left, 0, n * sizeof(long long)));
    QP_TRY(cudaMalloc(&b->d_pending, 3 * n * sizeof(long long)));
    QP_TRY(cudaMemset(b->d_pending, 0, 3 * n * sizeof(long long)));
    QP_TRY(cudaMalloc(&b->d_stash, stash_bytes((size_t)b->grid)));
    QP_TRY(cudaMalloc(&b->d_work, n * sizeof(long long)));
    QP_TRY(cudaMemset(b->d_work, 0, n * sizeof(long long)));
    QP_TRY(cudaMalloc(&b->d_ctl, sizeof(qp::StepCtl)));
    QP_TRY(cudaMemset(b->d_ctl, 0, sizeof(qp::StepCtl)));
    QP_TRY(cudaMallocHost(&b->h_stage, 2 * n * sizeof(qp::Problem)));
    QP_TRY(cudaMallocHost(&b->h_stage_ctl, 4 * n * sizeof(long long)));
    b->stage_ev.assign(2 * n, nullptr);
    for (size_t k = 0; k < 2 * n; ++k)
        QP_TRY(cudaEventCreateWithFlags(&b->stage_ev[k], cudaEventDisableTiming));
    // empty slots hold a zeroed problem whose launch counter points at d_left
    for (size_t k = 0; k < n; ++k) {
        qp::Problem P{};
        P.device_step = 1;
        P.left_ctr = b->d_left + k;
        P.step_ctr = b->d_step + k;
        P.pending = b->d_pending + 3 * k;
        P.work_ctr = b->d_work + k;
        P.dt = 1.0;
        QP_TRY(cudaMemcpy(b->d_table + k, &P, sizeof(P), cudaMemcpyHostToDevice));
    }
    QP_TRY(cudaDeviceSynchronize());
#undef QP_TRY
    *out = b;
    return QP_OK;
}

int qp_batch_destroy(qp_batch *b)
{
    if (!b) return QP_ERR_NOT_INITIALIZED;
    {
        DeviceGuard g(b->ctx->device);
        cudaDeviceSynchronize();
    }
    batch_release(b);
    return QP_OK;
}

int qp_batch_scratch_words(qp_ctx *ctx, const qp_step_params *s, int64_t *words)
{
    if (!ctx) return QP_ERR_NOT_INITIALIZED;
    if (!s || !words) return QP_ERR_INVALID_ARG;
    qp::Problem P;
    const int st = build_problem(ctx, s, P);
    if (st != QP_OK) return st;
    size_t lep = 0, pho = 0;
    chain_words_of(ctx, s, lep, pho);
    *words = (int64_t)(lep + pho);
    return QP_OK;
}

int qp_batch_set(qp_batch *b, int32_t slot, const qp_step_params *s, uint64_t *scratch,
                 int64_t scratch_words, void *stream)
{
    if (!b) return QP_ERR_NOT_INITIALIZED;
    if (!s || slot < 0 || slot >= b->max || !scratch) return QP_ERR_INVALID_ARG;
    if (s->precision != b->precision || s->field.kind != b->field_kind) return QP_ERR_INVALID_ARG;
    qp_ctx *ctx = b->ctx;
    qp::Problem P;
    int st = build_problem(ctx, s, P);
    if (st != QP_OK) return st;
    size_t lep = 0, pho = 0;
    chain_words_of(ctx, s, lep, pho);
    if (scratch_words < (int64_t)(lep + pho)) return QP_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return QP_ERR_CUDA;
    P.lep_words = (unsigned long long *)scratch;
    P.pho_words = (unsigned long long *)scratch + lep;
    P.pending = b->d_pending + 3 * (size_t)slot;
    P.step_ctr = b->d_step + slot;
    P.left_ctr = b->d_left + slot;
    P.work_ctr = b->d_work + slot;
    P.device_step = 1;
    cudaStream_t cs = (cudaStream_t)stream;
    const int k = b->stage_next;
    b->stage_next = (k + 1) % (2 * b->max);
    cudaError_t e = cudaEventSynchronize(b->stage_ev[k]);  // the entry's last copy is done
    if (e != cudaSuccess) return cuda_status(e);
    b->h_stage[k] = P;
    b->h_stage_ctl[2 * k] = s->step;
    b->h_stage_ctl[2 * k + 1] = s->n_steps;
    const int32_t hs[3] = {s->electron, s->positron, s->photon};
    for (int q = 0; q < 3 && e == cudaSuccess; ++q)
        if (hs[q] != -1) e = cudaMemsetAsync(ctx->d_stats + hs[q], 0, sizeof(qp::DevStats), cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch, 0, (lep + pho) * sizeof(uint64_t), cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_work + slot, 0, sizeof(long long), cs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_table + slot, &b->h_stage[k], sizeof(qp::Problem),
                            cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_step + slot, &b->h_stage_ctl[2 * k], sizeof(long long),
                            cudaMemcpyHostToDevice, cs);
    // activation last: the slot is stepped from the next launch on
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_left + slot, &b->h_stage_ctl[2 * k + 1], sizeof(long long),
                            cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaEventRecord(b->stage_ev[k], cs);
    return cuda_status(e);
}

int qp_batch_clear(qp_batch *b, int32_t slot, void *stream)
{
    if (!b) return QP_ERR_NOT_INITIALIZED;
    if (slot < 0 || slot >= b->max) return QP_ERR_INVALID_ARG;
    DeviceGuard g(b->ctx->device);
    if (!g.ok) return QP_ERR_CUDA;
    return cuda_status(
        cudaMemsetAsync(b->d_left + slot, 0, sizeof(long long), (cudaStream_t)stream));
}

int qp_batch_step(qp_batch *b, int32_t n_launches, void *stream)
{
    if (!b) return QP_ERR_NOT_INITIALIZED;
    if (n_launches < 0) return QP_ERR_INVALID_ARG;
    DeviceGuard g(b->ctx->device);
    if (!g.ok) return QP_ERR_CUDA;
    qp::StepArgs a{};
    fill_globals(b->ctx, a);
    a.ctl = b->d_ctl;
    a.n_problems = b->max;
    a.problems = b->d_table;
    a.stash = b->d_stash;
    cudaStream_t cs = (cudaStream_t)stream;
    for (int32_t k = 0; k < n_launches; ++k) {
        cudaError_t e = timed(b->ctx, 0, cs, [&] {
            return qp::launch_step(a, b->precision, b->field_kind, true, b->grid, cs);
        });
        if (e != cudaSuccess) return cuda_status(e);
    }
    return QP_OK;
}

int qp_batch_progress(qp_batch *b, int64_t *steps_left, int64_t *next_step, int64_t *work,
                      void *stream)
{
    if (!b) return QP_ERR_NOT_INITIALIZED;
    if (!steps_left) return QP_ERR_INVALID_ARG;
    DeviceGuard g(b->ctx->device);
    if (!g.ok) return QP_ERR_CUDA;
    cudaStream_t cs = (cudaStream_t)stream;
    const size_t bytes = (size_t)b->max * sizeof(long long);
    cudaError_t e = cudaMemcpyAsync(steps_left, b->d_left, bytes, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess && next_step)
        e = cudaMemcpyAsync(next_step, b->d_step, bytes, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess && work)
        e = cudaMemcpyAsync(work, b->d_work, bytes, cudaMemcpyDeviceToHost, cs);
    return cuda_status(e);
}

int qp_diagnostics(qp_ctx *ctx, int32_t handle, qp_diag *out, void *stream)
{
    if (!ctx) return QP_ERR_NOT_INITIALIZED;
    if (!out) return QP_ERR_INVALID_ARG;
    if (!valid_handle(ctx, handle)) return QP_ERR_NOT_INITIALIZED;
    DeviceGuard g(ctx->device);
    if (!g.ok) return QP_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const qp_species_desc &d = ctx->species[handle].d;
    qp::SpeciesDev S = species_dev(ctx, handle);
    double *partials = ctx->d_diag;
    double *fin = ctx->d_diag + (size_t)qp::kDiagBlocks * qp::kDiagWords;
    cudaError_t e = qp::launch_diag(S, d.kind == QP_PHOTON, partials, qp::kDiagBlocks, fin, st);
    if (e != cudaSuccess) return cuda_status(e);
    double h[qp::kDiagWords];
    qp::DevStats ds;
    int64_t n_live = 0;
    int status = 0;
    if ((e = cudaMemcpyAsync(h, fin, sizeof(h), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&ds, ctx->d_stats + handle, sizeof(ds), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(&n_live, d.n_live, sizeof(n_live), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(&status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_status(e);
    memset(out, 0, sizeof(*out));
    out->n_live = n_live;
    out->n_alive = (int64_t)llround(h[0]);
    out->weight = h[1];
    out->energy = h[2];
    out->px = h[3];
    out->py = h[4];
    out->pz = h[5];
    out->chi_mean = (d.chi && h[1] > 0.0) ? h[6] / h[1] : 0.0;
    for (int k = 0; k < QP_HIST_BINS; ++k) out->hist[k] = h[8 + k];
    out->n_emit = (int64_t)ds.n_emit;
    out->n_photon = (int64_t)ds.n_photon;
    out->n_photon_drop = (int64_t)ds.n_photon_drop;
    out->n_subthreshold = (int64_t)ds.n_subthreshold;
    out->n_pair = (int64_t)ds.n_pair;
    out->n_pair_drop = (int64_t)ds.n_pair_drop;
    out->n_saturated = (int64_t)ds.n_saturated;
    out->n_clamped = (int64_t)ds.n_clamped;
    out->n_continuous = (int64_t)ds.n_continuous;
    out->e_subthreshold = ds.e_subthreshold;
    out->e_dropped = ds.e_dropped;
    out->status = status;
    return status;
}

int qp_step_fused(qp_ctx *ctx, const qp_step_params *s, int32_t fuse, void *stream)
{
    if (!ctx) return QP_ERR_NOT_INITIALIZED;
    if (!s || fuse < 1 || s->pairs) return QP_ERR_INVALID_ARG;
    qp::StepArgs a{};
    int st = build_problem(ctx, s, a.single);
    if (st != QP_OK) return st;
    if (s->n_steps == 0) return QP_OK;
    DeviceGuard g(ctx->device);
    if (!g.ok) return QP_ERR_CUDA;
    cudaStream_t cs = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(cs, &cap) != cudaSuccess) return QP_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return QP_ERR_INVALID_ARG;  // it synchronises
    // the lepton counts (they do not change without pairs): read once
    long long n[2] = {0, 0};
    const int32_t hs[2] = {s->electron, s->positron};
    for (int k = 0; k < 2; ++k) {
        if (hs[k] == -1) continue;
        const qp_species_desc &d = ctx->species[hs[k]].d;
        cudaError_t e = cudaMemcpyAsync(&n[k], d.n_live, sizeof(long long),
                                        cudaMemcpyDeviceToHost, cs);
        if (e != cudaSuccess) return cuda_status(e);
    }
    cudaError_t e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return cuda_status(e);
    for (int k = 0; k < 2; ++k) {
        const int64_t cap = hs[k] == -1 ? 0 : ctx->species[hs[k]].d.capacity;
        if (n[k] < 0 || n[k] > cap) return QP_ERR_INVALID_ARG;
    }
    const long long tiles_e = (n[0] + 31) / 32, tiles = tiles_e + (n[1] + 31) / 32;
    const int K = fuse < s->n_steps ? fuse : s->n_steps;
    if (K > 65535) return QP_ERR_INVALID_ARG;
    const int64_t cap_g = s->photon == -1 ? 0 : ctx->species[s->photon].d.capacity;
    // the photon order sorts 32-bit indices on keys of at most 64 bits
    if (cap_g >= (int64_t)0xFFFFFFFFll || qp::fused_key_bits(K, tiles, nullptr) > 64)
        return QP_ERR_INVALID_ARG;
    const int order_grid = 2 * ctx->num_sms;
    const size_t sort_bytes = (qp::coalesce_scratch_bytes(cap_g, order_grid) + 255) / 256 * 256;
    const size_t bytes = sort_bytes + 256;
    if (bytes > ctx->fuse_bytes) {
        void *p = nullptr;
        e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) return cuda_status(e);
        cudaFree(ctx->d_fuse);
        ctx->d_fuse = p;
        ctx->fuse_bytes = bytes;
    }
    // the window counts after the sort scratch
    long long *win = (long long *)((char *)ctx->d_fuse + sort_bytes);
    fill_globals(ctx, a);
    a.ctl = ctx->d_ctl;
    qp::Problem &P = a.single;
    P.pending = ctx->d_pending;
    P.device_step = 0;
    for (int32_t w0 = 0; w0 < s->n_steps; w0 += K) {
        const int Kw = s->n_steps - w0 < K ? s->n_steps - w0 : K;
        set_time_host(P, s->step + w0);
        e = timed(ctx, 0, cs, [&] {
            return qp::launch_fused(a, s->precision, s->field.kind, Kw, tiles_e, tiles,
                                    ctx->d_fuse, order_grid, win, ctx->num_sms, cs);
        });
        if (e != cudaSuccess) return cuda_status(e);
    }
    return QP_OK;
}

int qp_fill_yee2d(qp_ctx *ctx, const qp_pulse2d *p, const qp_field *grid, double t, void *stream)
{
    if (!ctx) return QP_ERR_NOT_INITIALIZED;
    if (!p || !grid || grid->kind != QP_FIELD_YEE2D || !grid->yee[1] || !grid->yee[5] ||
        grid->nx <= 0 || grid->ny <= 0 || !(grid->dx > 0.0) || !(grid->dy > 0.0) ||
        !(p->w0 > 0.0) || !(p->tau_fwhm > 0.0) || !isfinite(t))
        return QP_ERR_INVALID_ARG;
    if (grid->ny > (int64_t)64 * 65535)  // rows of 64 per block in grid.y
        return QP_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return QP_ERR_CUDA;
    const qp::Pulse2DDev pd{p->a0, p->w0, p->tau_fwhm, p->x_focus, p->t_focus, p->y_axis};
    return cuda_status(qp::launch_pulse_fill(pd, grid->nx, grid->ny, grid->dx, grid->dy,
                                             grid->x0, grid->y0, t, (float *)grid->yee[1],
                                             (float *)grid->yee[5], (cudaStream_t)stream));
}

// A full 2D Yee grid (all six components) as the PIC kernels take it.
static bool yee_grid_of(const qp_field *f, qp::YeeGrid &g)
{
    if (!f || f->kind != QP_FIELD_YEE2D || f->nx <= 0 || f->ny <= 0 || !(f->dx > 0.0) ||
        !(f->dy > 0.0) || !isfinite(f->x0) || !isfinite(f->y0))
        return false;
    for (int c = 0; c < 6; ++c) {
        if (!f->yee[c]) return false;
        g.f[c] = (float *)f->yee[c];
    }
    g.nx = f->nx;
    g.ny = f->ny;
    g.dx = f->dx;
    g.dy = f->dy;
    g.x0 = f->x0;
    g.y0 = f->y0;
    return true;
}

int qp_yee_advance_b(qp_ctx *ctx, const qp_field *grid, double dtb, void *stream)
{
    if (!ctx) return QP_ERR_NOT_INITIALIZED;
    qp::YeeGrid g{};
    if (!yee_grid_of(grid, g) || !isfinite(dtb)) return QP_ERR_INVALID_ARG;
    DeviceGuard d(ctx->device);
    if (!d.ok) return QP_ERR_CUDA;
    return cuda_status(qp::launch_yee_b(g, dtb, ctx->num_sms, (cudaStream_t)stream));
}

int qp_yee_advance_e(qp_ctx *ctx, const qp_field *grid, const float *jx, const float *jy,
                     const float *jz, double dt, void *stream)
{
    if (!ctx) return QP_ERR_NOT_INITIALIZED;
    qp::YeeGrid g{};
    if (!yee_grid_of(grid, g) || !isfinite(dt)) return QP_ERR_INVALID_ARG;
    DeviceGuard d(ctx->device);
    if (!d.ok) return QP_ERR_CUDA;
    return cuda_status(qp::launch_yee_e(g, jx, jy, jz, dt, ctx->num_sms, (cudaStream_t)stream));
}

int qp_deposit_current(qp_ctx *ctx, int32_t handle, const qp_field *grid, float *jx, float *jy,
                       float *jz, double dt, void *stream)
{
    if (!ctx) return QP_ERR_NOT_INITIALIZED;
    if (!valid_handle(ctx, handle)) return QP_ERR_NOT_INITIALIZED;
    const qp_species_desc &sd = ctx->species[handle].d;
    qp::YeeGrid g{};
    if (sd.kind == QP_PHOTON || !yee_grid_of(grid, g) || !jx || !jy || !jz || !isfinite(dt))
        return QP_ERR_INVALID_ARG;
    DeviceGuard d(ctx->device);
    if (!d.ok) return QP_ERR_CUDA;
    const double q = sd.kind == QP_ELECTRON ? -1.0 : 1.0;
    return cuda_status(qp::launch_deposit(species_dev(ctx, handle), q, dt, g, jx, jy, jz,
                                          ctx->d_status, ctx->num_sms, (cudaStream_t)stream));
}

int qp_sort_species(qp_ctx *ctx, int32_t handle, const qp_field *grid, void *stream)
{
    if (!ctx) return QP_ERR_NOT_INITIALIZED;
    if (!valid_handle(ctx, handle)) return QP_ERR_NOT_INITIALIZED;
    const qp_species_desc &sd = ctx->species[handle].d;
    qp::YeeGrid g{};
    if (!yee_grid_of(grid, g) || sd.capacity >= (int64_t)0xFFFFFFFFll) return QP_ERR_INVALID_ARG;
    if ((double)g.nx * (double)g.ny > 9.0e18) return QP_ERR_INVALID_ARG;
    DeviceGuard d(ctx->device);
    if (!d.ok) return QP_ERR_CUDA;
    const int grid_blocks = 2 * ctx->num_sms;
    const size_t bytes = qp::coalesce_scratch_bytes(sd.capacity, grid_blocks);
    if (bytes > ctx->coal_bytes) {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) return cuda_status(e);
        cudaFree(ctx->d_coal);
        ctx->d_coal = p;
        ctx->coal_bytes = bytes;
    }
    if (!ctx->d_coal_stats) {
        cudaError_t e = cudaMalloc(&ctx->d_coal_stats, 4 * sizeof(long long));
        if (e != cudaSuccess) return cuda_status(e);
    }
    return cuda_status(qp::launch_sort_cells(species_dev(ctx, handle), g, ctx->d_coal,
                                             grid_blocks, ctx->d_coal_stats, ctx->d_status,
                                             (cudaStream_t)stream));
}

static bool pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

int qp_coalesce_photons(qp_ctx *ctx, int32_t handle, const qp_coalesce_params *P,
                        qp_coalesce_stats *out, void *stream)
{
    if (!ctx) return QP_ERR_NOT_INITIALIZED;
    if (!valid_handle(ctx, handle)) return QP_ERR_NOT_INITIALIZED;
    const qp_species_desc &d = ctx->species[handle].d;
    if (d.kind != QP_PHOTON || d.capacity >= (int64_t)0xFFFFFFFFll) return QP_ERR_INVALID_ARG;
    if (P) {
        if (P->min_group < 3 || (P->max_group != 0 && P->max_group < P->min_group) ||
            !pow2_in(P->energy_bins_per_octave, 1, 64) ||
            !pow2_in(P->direction_bins, 1, 64) || !(P->dx > 0.0) || !(P->dy > 0.0) ||
            (d.dims == 3 && !(P->dz > 0.0)) || P->nx < 1 || P->ny < 1 || P->nz < 1 ||
            (d.dims == 2 && P->nz != 1) || !isfinite(P->x0) || !isfinite(P->y0) ||
            !isfinite(P->z0))
            return QP_ERR_INVALID_ARG;
        // the key space (cells x 2048 E x 6 D^2) must stay below 2^63
        const double space = (double)P->nx * (double)P->ny * (double)P->nz * 2048.0 *
                             P->energy_bins_per_octave * 6.0 * P->direction_bins *
                             P->direction_bins;
        if (!(space < 9.2e18)) return QP_ERR_INVALID_ARG;
    }
    DeviceGuard g(ctx->device);
    if (!g.ok) return QP_ERR_CUDA;
    const int grid = 2 * ctx->num_sms;
    const size_t bytes = qp::coalesce_scratch_bytes(d.capacity, grid);
    if (bytes > ctx->coal_bytes) {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) return cuda_status(e);
        cudaFree(ctx->d_coal);
        ctx->d_coal = p;
        ctx->coal_bytes = bytes;
    }
    if (!ctx->d_coal_stats) {
        cudaError_t e = cudaMalloc(&ctx->d_coal_stats, 4 * sizeof(long long));
        if (e != cudaSuccess) return cuda_status(e);
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = qp::launch_coalesce(species_dev(ctx, handle), P, ctx->d_coal, grid,
                                        ctx->d_coal_stats, ctx->d_status, st);
    if (e != cudaSuccess) return cuda_status(e);
    if (out) {
        long long h[4];
        e = cudaMemcpyAsync(h, ctx->d_coal_stats, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_status(e);
        out->groups_merged = h[0];
        out->photons_merged = h[1];
        out->n_before = h[2];
        out->n_after = h[3];
    }
    return QP_OK;
}

int qp_compact_photons(qp_ctx *ctx, int32_t handle, qp_coalesce_stats *out, void *stream)
{
    return qp_coalesce_photons(ctx, handle, nullptr, out, stream);
}

int qp_export_tables(qp_ctx *ctx, qp_tables_export *out)
{
    if (!ctx) return QP_ERR_NOT_INITIALIZED;
    if (!out) return QP_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return QP_ERR_CUDA;
    std::vector<double> h(kTabWords);
    cudaError_t e = cudaMemcpy(h.data(), ctx->d_tab64, kTabWords * sizeof(double),
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e);
    memcpy(out->H, h.data(), sizeof(out->H));
    memcpy(out->Gs, h.data() + qp::kNRatePad, sizeof(out->Gs));
    memcpy(out->Ts, h.data() + 2 * qp::kNRatePad, sizeof(out->Ts));
    memcpy(out->Cg, h.data() + kTabRate, sizeof(out->Cg));
    memcpy(out->Cp, h.data() + kTabRate + qp::kNCdf * qp::kNNode, sizeof(out->Cp));
    out->a_S = ctx->U.a_S;
    out->C_rate = ctx->U.C_rate;
    out->tau0w = ctx->U.tau0w;
    return QP_OK;
}

int qp_reset_counters(qp_ctx *ctx, int32_t handle)
{
    if (!ctx) return QP_ERR_NOT_INITIALIZED;
    if (!valid_handle(ctx, handle)) return QP_ERR_NOT_INITIALIZED;
    DeviceGuard g(ctx->device);
    if (!g.ok) return QP_ERR_CUDA;
    cudaError_t e = cudaMemset(ctx->d_stats + handle, 0, sizeof(qp::DevStats));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return cuda_status(e);
}

int qp_profile_enable(qp_ctx *ctx, int enable)
{
    if (!ctx) return QP_ERR_NOT_INITIALIZED;
    ctx->profiling = enable != 0;
    ctx->events_used = 0;
    ctx->records.clear();
    return QP_OK;
}

int qp_profile_read(qp_ctx *ctx, double ms[3], int64_t launches[3])
{
    if (!ctx) return QP_ERR_NOT_INITIALIZED;
    if (!ms || !launches) return QP_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return QP_ERR_CUDA;
    for (int k = 0; k < 3; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
    }
    for (size_t r = 0; r < ctx->records.size(); ++r) {
        cudaEvent_t a = ctx->events[2 * r], b = ctx->events[2 * r + 1];
        cudaError_t e = cudaEventSynchronize(b);
        float t = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
        if (e != cudaSuccess) return cuda_status(e);
        ms[ctx->records[r]] += t;
        launches[ctx->records[r]] += 1;
    }
    return QP_OK;
}

int qp_selftest_wait_timeout(qp_ctx *ctx, uint32_t spin_limit)
{
    if (!ctx) return QP_ERR_NOT_INITIALIZED;
    DeviceGuard g(ctx->device);
    if (!g.ok) return QP_ERR_CUDA;
    cudaError_t e = cudaMemset(ctx->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_chain, 0, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = qp::launch_wait_selftest(ctx->d_chain, spin_limit, ctx->d_status, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int status = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(int));
    // the test wrote look-back words with a made-up epoch: clear them
    if (e == cudaSuccess) e = cudaMemset(ctx->d_chain, 0, 2 * sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_status(e);
    return status;
}

}  // extern "C"
