/*
 * qedpic.h -- C ABI of the GB300 QED particle-step library (libqedpic.so).
 *
 * The library advances super-particles (electrons, positrons, photons) of a
 * particle-in-cell simulation through one or more steps of the radiative and
 * QED model of Lobet et al., "Modeling of radiative and quantum
 * electrodynamics effects in PIC simulations of ultra-relativistic
 * laser-plasma interaction" (arXiv:1311.1107):
 *   - field gather (analytic laser, constant B, or a fixed 2D Yee grid);
 *   - Boris push of the Lorentz force, with Sokolov radiation damping below a
 *     quantum-parameter threshold (section 3, Eq. 4 and Eq. 5);
 *   - Lorentz-invariant quantum parameters chi_e, chi_gamma (section 2, Eq. 1);
 *   - optical-depth decrement against tabulated nonlinear-Compton and
 *     Breit-Wheeler rates (Eq. 2, Eq. 3, Eq. 6);
 *   - inverse-CDF sampling of photon and pair energies (Eq. 7), collinear
 *     recoil (Eq. 8), pair creation at the photon position (section 3);
 *   - deterministic, slot-ordered append of new photons, electrons and
 *     positrons to caller-owned device buffers.
 *
 * Conventions
 *   - Every function returns an int status: QP_OK (0), a warning (> 0) or an
 *     error (< 0).  qp_status_string() names it.
 *   - All particle arrays and counters are DEVICE pointers owned by the
 *     caller; the library never frees caller memory.  Tables, scan scratch
 *     and status flags are owned by the context.
 *   - Streams are passed as `void *` holding a cudaStream_t (NULL = legacy
 *     default stream).  qp_step and qp_init_optical_depth are asynchronous on
 *     that stream; qp_diagnostics synchronises it.
 *   - Units are normalised at the context's reference wavelength lambda:
 *     time in 1/omega (omega = 2 pi c / lambda), length in c/omega, momentum
 *     u = p/(m c), E in m c omega / e, B in m omega / e.  One laser period is
 *     2 pi.
 *   - Storage is FP64 structure-of-arrays, one array per component, each at
 *     least `capacity` elements, 8-byte aligned (256-byte alignment gives the
 *     best coalescing).  Slot i of every array belongs to particle i; slots
 *     [0, *n_live) are live.  A photon with tau < 0 has decayed into a pair
 *     and is skipped; leptons are never removed.
 *   - Random numbers come from Philox4x32-10 keyed by (seed) with counter
 *     (slot, step, species/purpose/emission index), so results do not depend
 *     on the launch configuration and a run can be resumed at any step.
 */
#ifndef QEDPIC_H
#define QEDPIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define QP_OK 0
#define QP_WARN_BUFFER_FULL 1      /* particles dropped: an append buffer is full   */
#define QP_WARN_TABLE_CLAMPED 2    /* chi above the table range (2^10) was clamped  */
#define QP_ERR_INVALID_ARG (-1)    /* rejected before anything was enqueued         */
#define QP_ERR_CUDA (-2)           /* a CUDA runtime call failed                    */
#define QP_ERR_OOM (-3)            /* device allocation failed                      */
#define QP_ERR_NOT_INITIALIZED (-4)/* NULL or destroyed context, unknown handle     */
#define QP_ERR_TIMEOUT (-5)        /* a bounded device-side wait gave up            */

/* ---- enumerations ------------------------------------------------------ */
enum { QP_ELECTRON = 0, QP_POSITRON = 1, QP_PHOTON = 2 };
enum { QP_FP64 = 0, QP_MIXED = 1 };
enum {
    QP_FIELD_NONE = 0,      /* E = B = 0                                         */
    QP_FIELD_PLANE = 1,     /* E_y = B_z = a0 cos(t - x)                         */
    QP_FIELD_GAUSSIAN = 2,  /* paraxial Gaussian pulse along +x, polarised y     */
    QP_FIELD_YEE2D = 3,     /* fixed FP32 Yee grid, linear interpolation         */
    QP_FIELD_UNIFORM_B = 4  /* B = b0 z^ (the paper's section 4 test)            */
};
#define QP_MAX_EMISSIONS 8  /* upper bound of qp_step_params.max_emissions     */
#define QP_MAX_BATCH 64     /* problems (independent runs) per batch            */
#define QP_STEP_TILE 128    /* slots per tile of qp_step (one look-back word)   */
#define QP_HIST_BINS 64     /* diagnostic spectrum bins in log10(gamma)        */
#define QP_HIST_LOG10_MIN (-1.0)
#define QP_HIST_LOG10_MAX (5.0)

typedef struct qp_ctx qp_ctx;

/* ---- qp_init_tables ---------------------------------------------------- */
typedef struct {
    double lambda_m;   /* reference wavelength [m] that fixes the units (> 0) */
    int32_t device;    /* CUDA device ordinal the context lives on            */
    int32_t reserved;  /* must be 0                                           */
} qp_table_params;

/*
 * Create a context on `p->device`: build, in FP64 on the host, the tables of
 * the rates and CDFs that Eq. 2 and Eq. 3 define, and upload FP64 and FP32
 * copies.  Grids (a specification shared with the test oracle):
 *   rate tables  H(chi)=int_0^1 F_gamma du, G(chi)/chi with
 *                G=int_0^1 u F_gamma du (Eq. 5), T(chi) exp(8/(3 chi)) with
 *                T=int_0^1 F_pm dv, at chi_j = 2^(-14+j/32)(1+(j mod 32)/32),
 *                j = 0..768, linear interpolation in chi;
 *   CDF tables   Eq. 7 rows at chi_j = 2^(-14+j/4)(1+(j mod 4)/4), j = 0..96,
 *                on 256 logit nodes of u (-30..20) and of v (-20..20).
 * Also allocates the context's scan scratch and status flags.
 * Returns QP_ERR_INVALID_ARG for bad arguments, QP_ERR_CUDA / QP_ERR_OOM on
 * device failure (nothing is leaked; *out_ctx is left NULL).
 */
int qp_init_tables(const qp_table_params *p, qp_ctx **out_ctx);

/* Release everything the context owns (not the caller's buffers).  Safe on
 * NULL.  The caller must make sure no step is still running on its streams. */
int qp_destroy(qp_ctx *ctx);

/* ---- qp_create_species ------------------------------------------------- */
typedef struct {
    int32_t kind;       /* QP_ELECTRON, QP_POSITRON or QP_PHOTON                 */
    int32_t dims;       /* 3 (x, y, z) or 2 (x, y; z must be NULL)               */
    int64_t capacity;   /* slots in every array below (>= 0)                     */
    double *x, *y, *z;  /* positions                                             */
    double *ux, *uy, *uz; /* momenta p/(m c); photons: |u| = gamma_gamma         */
    double *tau;        /* remaining optical depth (tau_f - tau of Eq. 6)        */
    double *w;          /* super-particle weight                                 */
    double *chi;        /* optional (may be NULL): chi of the particle's last
                           step (chi_e, or chi_gamma for photons above 2 m c^2)  */
    int32_t *nemit;     /* optional (may be NULL): events caused by the particle,
                           accumulated over steps (emissions of a lepton, stored
                           or not; 1 for a photon that decayed into a pair);
                           set to 0 for particles the library appends          */
    int64_t *n_live;    /* device counter of live slots; the library updates it
                           when it appends; the caller sets its initial value    */
    int64_t id_base;    /* particle id of slot 0 (>= 0): slot i is particle
                           id_base + i, the counter of its random streams.  A
                           population split over GPUs keeps every particle's
                           draws when each part gets the id of its first slot */
    int64_t id_split;   /* 0: every slot i is particle id_base + i.  > 0: only
                           slots below id_split are; slot i >= id_split is
                           particle id_append + (i - id_split).  A part of a
                           split population gives the particles it appends ids
                           no other part uses (slots past its own primaries
                           would otherwise take the next part's ids and share
                           their random streams)                            */
    int64_t id_append;  /* id of slot id_split when id_split > 0 (>= 0)      */
} qp_species_desc;

/*
 * Register a species' caller-owned device buffers with the context
 * (super-particles of section 3: weight, position, momentum) and return a
 * handle (>= 0).  Nothing is copied or enqueued.  QP_ERR_INVALID_ARG if a
 * required pointer is NULL, dims is not 2 or 3, or z is given for dims 2.
 */
int qp_create_species(qp_ctx *ctx, const qp_species_desc *d, int32_t *out_handle);

/*
 * Draw the final optical depth tau_f = -log(xi), xi in ]0,1] (section 3,
 * after Eq. 6), for slots [first, first + count) of a species, from the
 * Philox stream (seed, slot, purpose "initial").  Asynchronous on `stream`.
 */
int qp_init_optical_depth(qp_ctx *ctx, int32_t handle, uint64_t seed, int64_t first,
                          int64_t count, void *stream);

/*
 * Copy slots [0, count) of a species' FP64 state between its device arrays
 * and a host block: array k of (x, y, [z if dims == 3], ux, uy, uz, tau, w)
 * starts at byte k * host_pitch of `host` (host_pitch >= 8 count, a
 * multiple of 8).  to_device != 0 copies host -> device, else device ->
 * host.  Asynchronous on `stream` (pinned host memory lets it overlap); one
 * strided copy when the device arrays lie at a constant pitch in that order,
 * else one copy per array.  The live count is not touched.  Returns
 * QP_ERR_INVALID_ARG for a null host pointer, a count outside [0, capacity]
 * or a pitch too small.  No counterpart in the paper: host I/O of the state.
 */
int qp_species_copy(qp_ctx *ctx, int32_t handle, void *host, int64_t host_pitch, int64_t count,
                    int32_t to_device, void *stream);

/* ---- qp_step ----------------------------------------------------------- */
typedef struct {
    int32_t kind;         /* QP_FIELD_*                                         */
    int32_t reserved;
    double a0;            /* PLANE, GAUSSIAN: peak normalised amplitude           */
    double w0;            /* GAUSSIAN: waist (1/e field radius at focus)          */
    double tau_fwhm;      /* GAUSSIAN: FWHM duration of the intensity             */
    double x_focus;       /* GAUSSIAN: focal plane                                */
    double t_focus;       /* GAUSSIAN: time the envelope peak crosses x_focus     */
    double b0;            /* UNIFORM_B: B_z                                       */
    const float *yee[6];  /* YEE2D: device Ex Ey Ez Bx By Bz, ny rows of nx values;
                             staggering Ex(i+1/2,j) Ey(i,j+1/2) Ez(i,j)
                             Bx(i,j+1/2) By(i+1/2,j) Bz(i+1/2,j+1/2)              */
    int64_t nx, ny;       /* YEE2D: nodes per row, rows                           */
    double dx, dy;        /* YEE2D: cell size                                     */
    double x0, y0;        /* YEE2D: position of node (0,0)                        */
} qp_field;

typedef struct {
    qp_field field;
    double dt;               /* time step (> 0)                                   */
    int64_t step;            /* index n of the first step; fields at t = n dt     */
    int32_t n_steps;         /* steps to run (>= 0)                               */
    int32_t precision;       /* QP_FP64 or QP_MIXED                               */
    uint64_t seed;           /* Philox key                                        */
    double chi_threshold;    /* Sokolov (continuous) regime below, MC above      */
    double photon_min_gamma; /* super-photons stored only above this energy (2)  */
    int32_t pairs;           /* 1 = photons above 2 m c^2 may create pairs        */
    int32_t max_emissions;   /* 1..QP_MAX_EMISSIONS emissions per particle-step   */
    int32_t electron;        /* species handles, -1 = absent                      */
    int32_t positron;
    int32_t photon;
    int32_t reserved;
} qp_step_params;

/*
 * Advance the species named in `s` by s->n_steps steps, asynchronously on
 * `stream`.  Per step n, in this order:
 *   electrons then positrons, slots [0, n_live at the start of the step):
 *     gather E, B at x^n, t^n; Boris u^(n-1/2) -> u^(n+1/2); chi_e (Eq. 1);
 *     chi_e < chi_threshold: Sokolov damping (Eq. 4, P_rad of Eq. 5);
 *     otherwise tau -= W dt (Eq. 6) with a residual-time sub-loop: on
 *     tau <= W dt an emission at chi_gamma = u chi_e with u from Eq. 7,
 *     collinear recoil (Eq. 8), a super-photon appended if gamma_gamma >
 *     photon_min_gamma, tau = -log(xi), and the rest of the step continues;
 *     x^(n+1) = x^n + (v + delta_v) dt.
 *   photons existing at the start of the step (tau >= 0): chi_gamma (Eq. 1);
 *     above 2 m c^2 with pairs on, tau -= W_pm dt; on decay the photon gets
 *     tau = -1 and an electron and a positron are appended at its position
 *     with v = chi_-/chi_gamma from the pair CDF; otherwise x += c k^ dt.
 * Appended particles fill slots [n_live, ...) in the order of their parent's
 * slot (then emission index); photons emitted by electrons precede those of
 * positrons.  Particles that do not fit are counted as dropped and their
 * energy recorded; the step still completes.  The first step with species
 * larger than any stepped before grows the context's look-back scratch (one
 * allocation, synchronous); otherwise no allocation, no host synchronisation,
 * no host reads: the call can then be captured in a CUDA graph.  Each step
 * is one launch of the step kernel over every resident block of the GPU; on
 * the mixed path it is a cooperative launch, which starts only once all its
 * blocks fit on the GPU (kernels of other streams that hold SMs finish
 * first).
 * Returns QP_ERR_INVALID_ARG (nothing enqueued) for bad parameters, a
 * missing photon species while species emit, or a YEE2D grid with a NULL
 * component; QP_ERR_CUDA if a launch fails.  Overflow, table clamping and
 * wait time-outs are reported by the next qp_diagnostics.
 */
int qp_step(qp_ctx *ctx, const qp_step_params *s, void *stream);

/* One species' state in host memory, for qp_step_host. */
typedef struct qp_host_state {
    void *host;      /* block: array k of (x, y, [z if dims == 3], ux, uy, uz, tau, w)
                        at byte k * pitch; pinned memory copies fastest            */
    int64_t pitch;   /* bytes between arrays: >= 8 * capacity, a multiple of 8     */
    int64_t count;   /* in: live slots to step; out: live slots after the steps    */
} qp_host_state;

/*
 * qp_step for a caller whose state lives in host memory: for each species
 * named in s (electron, positron, photon: st[0..2]; entries of absent
 * species are ignored), slots [0, st[k].count) are copied from st[k].host
 * to the device arrays and the live count set; s->n_steps steps run as
 * qp_step runs them; the new live counts are read back into st[k].count and
 * slots [0, count) are copied back into st[k].host (the slots live before
 * the steps as soon as they are done, every array but the weights, which a
 * step writes for appended particles only: a step never lowers a live
 * count, since decayed photons keep their slots; the appended ones, every
 * array, once the counts are read).  The call synchronises `stream` once, or twice
 * when the steps appended particles, and returns when the host blocks hold
 * the result.  Per-particle event
 * counts and chi are left on the device (qp_diagnostics).  Returns what
 * qp_step returns, or QP_ERR_INVALID_ARG (nothing enqueued) for st == NULL,
 * a null host block, a count outside [0, capacity] or a pitch below 8 *
 * capacity.  No counterpart in the paper: the host I/O of qp_species_copy
 * and a step in one call, so that a step of host-resident state costs one
 * call of the library.
 */
int qp_step_host(qp_ctx *ctx, const qp_step_params *s, qp_host_state *st, void *stream);

/*
 * Fused steps: the s->n_steps steps of qp_step, `fuse` steps per launch
 * window, every lepton held in registers from the first step of a window to
 * its last (the data-parallel step has nothing to exchange between
 * particles when the fields are given: analytic fields, or a Yee grid that
 * stays fixed over the call).  Requires s->pairs == 0: leptons then never
 * change in number and photons only move.  The results are those of
 * qp_step with the same parameters, bit for bit: the same per-particle
 * arithmetic, photons in the same slots (step, then emitter slot, then
 * emission index), the same counters.  A window is one physics pass (each
 * new photon staged at a provisional index with its order key: step,
 * emitter, emission index), a radix sort of those keys, and the motion of
 * the window's photons, one thread a slot (those that existed at its start
 * over K steps, the new ones gathered into key order and moved over the
 * steps left after their birth).  Photons past the free slots are dropped
 * in key order, as separate steps drop them, while one window emits no more
 * photons than the photon capacity; beyond that the counters and leptons
 * still agree but the surviving photons may differ (QP_WARN_BUFFER_FULL in
 * both cases).  The call reads the live lepton counts to the host once (it
 * synchronises `stream`) and grows the context's scratch (about 110 bytes
 * per photon slot; an allocation).  Windows hold at most 65535 steps; the
 * photon capacity stays below 2^32.  QP_ERR_INVALID_ARG (nothing enqueued)
 * for pairs on, fuse < 1, a stream being captured, or what qp_step rejects.
 */
int qp_step_fused(qp_ctx *ctx, const qp_step_params *s, int32_t fuse, void *stream);

/* ---- batches: several independent runs in shared launches --------------
 *
 * A batch is a device table of up to max_problems independent problems
 * (runs), each with its own species, field parameters, seed, first step and
 * number of steps, all of one precision and field kind.  One launch takes one
 * step of every active problem (the same arithmetic as qp_step, tile by tile,
 * so a problem's results do not depend on what else is in the batch); each
 * problem's step counter lives on the device and advances with every launch,
 * and a problem becomes idle by itself when its steps are done.  The table
 * is read by the kernel at every launch, so problems can be set and cleared
 * between launches without touching a captured CUDA graph of qp_batch_step.
 * This is the batching layer of a serving loop (requests = problems).
 */
typedef struct qp_batch qp_batch;

/* Allocate a batch (device table, counters, pinned staging) for problems of
 * one precision (QP_FP64 / QP_MIXED) and field kind.  Synchronous.
 * QP_ERR_INVALID_ARG unless 1 <= max_problems <= QP_MAX_BATCH. */
int qp_batch_create(qp_ctx *ctx, int32_t max_problems, int32_t precision, int32_t field_kind,
                    qp_batch **out);

/* Release the batch (waits for the device first).  The context must outlive
 * its batches. */
int qp_batch_destroy(qp_batch *b);

/* Look-back scratch a problem needs: 64-bit words, from the capacities of
 * the species named in s (one word per QP_STEP_TILE slots of each chain,
 * plus a few). */
int qp_batch_scratch_words(qp_ctx *ctx, const qp_step_params *s, int64_t *words);

/*
 * Put a problem in slot `slot`: species handles, field, dt, seed, chi
 * threshold, photon cut, pairs and max emissions as for qp_step; s->step is
 * its first step index and s->n_steps the launches it takes part in.
 * `scratch` is caller-owned device memory of at least qp_batch_scratch_words
 * words, used by this problem alone until it is done or cleared.  Enqueued on
 * `stream` (the stream of the batch's launches): clears the scratch and the
 * species' counters, copies the descriptor, and activates the slot last, so
 * the problem is stepped from the next launch on.  The host side returns
 * without waiting for the device (staging buffers are reused only after
 * their copy completed).  QP_ERR_INVALID_ARG for a bad slot, a precision or
 * field kind other than the batch's, too little scratch, or what qp_step
 * rejects.  The species' initial state (positions, momenta, optical depths,
 * live counts) must be in place, in stream order, before the next launch.
 */
int qp_batch_set(qp_batch *b, int32_t slot, const qp_step_params *s, uint64_t *scratch,
                 int64_t scratch_words, void *stream);

/* Deactivate a slot (stream-ordered): it takes no part in later launches. */
int qp_batch_clear(qp_batch *b, int32_t slot, void *stream);

/* Enqueue n_launches launches; each takes one step of every active problem
 * and advances its step counter.  No allocation, no host synchronisation:
 * capturable in a CUDA graph, and a captured graph stays valid while the
 * batch's problems change. */
int qp_batch_step(qp_batch *b, int32_t n_launches, void *stream);

/* Enqueue copies of every slot's remaining launches (0 = idle or done) and,
 * where the pointers are not NULL, of its next step index and of the live
 * slots (all three species) stepped since it was set, into caller-owned host
 * arrays of max_problems entries (pinned memory for an asynchronous copy);
 * valid once the stream has reached this point. */
int qp_batch_progress(qp_batch *b, int64_t *steps_left, int64_t *next_step, int64_t *work,
                      void *stream);

/* Free a species handle (host-side registry only; the caller still owns
 * the buffers).  A later qp_create_species may reuse the handle. */
int qp_destroy_species(qp_ctx *ctx, int32_t handle);

/* ---- qp_diagnostics ---------------------------------------------------- */
typedef struct {
    int64_t n_live;          /* live slots                                         */
    int64_t n_alive;         /* slots with tau >= 0                                */
    double weight;           /* sum w over alive slots                             */
    double energy;           /* sum w gamma (leptons) or w |u| (photons), m c^2    */
    double px, py, pz;       /* sum w u                                            */
    double chi_mean;         /* w-weighted mean chi (0 if no chi array)            */
    double hist[QP_HIST_BINS]; /* w-weighted histogram of log10(gamma) over
                                  [QP_HIST_LOG10_MIN, QP_HIST_LOG10_MAX); out-of-
                                  range values go to the first / last bin          */
    /* counters accumulated by qp_step since the species was created, for the
       events this species caused (emissions for leptons, pairs for photons) */
    int64_t n_emit;          /* emission events                                    */
    int64_t n_photon;        /* super-photons appended                             */
    int64_t n_photon_drop;   /* super-photons that did not fit                     */
    int64_t n_subthreshold;  /* emissions below photon_min_gamma                   */
    int64_t n_pair;          /* pair events                                        */
    int64_t n_pair_drop;     /* pairs that did not fit                             */
    int64_t n_saturated;     /* particle-steps that reached max_emissions          */
    int64_t n_clamped;       /* particle-steps with chi above the table range      */
    int64_t n_continuous;    /* particle-steps in the Sokolov regime               */
    double e_subthreshold;   /* sum w gamma_gamma of photons below the cut         */
    double e_dropped;        /* sum w gamma of particles that did not fit          */
    int32_t status;          /* sticky context status (QP_OK or the first error
                                or warning raised on the device)                   */
    int32_t reserved;
} qp_diag;

/*
 * Reduce a species' state in a fixed order (the result does not depend on
 * the launch or on timing) into `out`, on `stream`, and synchronise it.
 * These are the quantities of the paper's Fig. 1 and Fig. 2 captions: total
 * energy, number (weight), mean quantum parameter and energy spectrum.  The
 * returned status is out->status when the call itself succeeded.
 */
int qp_diagnostics(qp_ctx *ctx, int32_t handle, qp_diag *out, void *stream);

/* ---- qp_export_tables -------------------------------------------------- */
#define QP_NRATE 769
#define QP_NCDF 97
#define QP_NNODE 256
typedef struct {
    double H[QP_NRATE];             /* H(chi_j)                                  */
    double Gs[QP_NRATE];            /* G(chi_j) / chi_j                          */
    double Ts[QP_NRATE];            /* T(chi_j) exp(8/(3 chi_j)), 0 below 2^-8    */
    double Cg[QP_NCDF * QP_NNODE];  /* emission CDF rows (Eq. 7)                  */
    double Cp[QP_NCDF * QP_NNODE];  /* pair CDF rows                              */
    double a_S;                     /* Schwinger field in normalised units        */
    double C_rate;                  /* alpha / (sqrt(3) pi tau_c omega)           */
    double tau0w;                   /* Sokolov tau_0 in units of 1/omega          */
} qp_tables_export;

/* Copy the context's FP64 tables and unit constants to host memory `out`
 * (caller-owned).  Synchronous. */
int qp_export_tables(qp_ctx *ctx, qp_tables_export *out);

/* ---- refill of a 2D Yee grid from the analytic pulse ----------------------- */

/* A 2D paraxial Gaussian pulse along +x, polarised along y (normalised
 * units; not in the paper: the laser of the foil workload):
 *   xi = x - x_focus, eta = (t - t_focus) - xi, zr = w0^2/2, q = xi/zr,
 *   E_y = B_z = a0 (1 + q^2)^(-1/4) exp(-r^2/(w0^2 (1 + q^2)) - 2 ln2 eta^2/tau^2)
 *               cos(-eta + r^2 xi/(2 (xi^2 + zr^2)) - atan(q)/2),  r = y - y_axis. */
typedef struct {
    double a0, w0, tau_fwhm, x_focus, t_focus, y_axis;
} qp_pulse2d;

/*
 * Per-step refill of a 2D Yee grid's fields from the pulse at time t (the
 * fields a fixed snapshot freezes: the refill lets them follow the pulse
 * across the target; the PIC context of the paper's section 3).  Writes E_y
 * at (x0 + i dx, y0 + (j + 1/2) dy) and B_z at (x0 + (i + 1/2) dx, y0 +
 * (j + 1/2) dy) of `grid` (kind QP_FIELD_YEE2D; its yee[1] and yee[5] are
 * written through, the other components are not touched).  One launch:
 * each block forms the x-dependent factors of its 32 columns (amplitude,
 * envelope, Gouy phase and curvature; the phase reduced modulo 2 pi in
 * FP64) and the radii of its 64 rows, then its nodes in FP32: every node is
 * within ~1e-6 of a0 of the FP64 formula rounded to float.  Give the step
 * that follows t = n dt, as the particle step evaluates its fields at that
 * time.  Stream-ordered, no allocation.  QP_ERR_INVALID_ARG for a grid of
 * another kind, missing E_y/B_z pointers or a non-positive size.
 */
int qp_fill_yee2d(qp_ctx *ctx, const qp_pulse2d *p, const qp_field *grid, double t, void *stream);

/* ---- PIC coupling: 2D Yee Maxwell solver, current deposition, sorting ----
 *
 * The paper's QED step runs inside a PIC code (section 3, CALDER); these
 * calls are the rest of a 2D PIC cycle around qp_step on a QP_FIELD_YEE2D
 * grid (the grid qp_step gathers from; all six component pointers must be
 * set and are written through).  Staggering as for the gather: Ex (i+1/2,
 * j), Ey (i, j+1/2), Ez (i, j), Bx (i, j+1/2), By (i+1/2, j), Bz (i+1/2,
 * j+1/2); fields outside the grid are taken as 0.  Normalised units (c = 1):
 * dB/dt = -curl E, dE/dt = curl B - J, J in units of e n_c c (n in units of
 * the reference density n_c, the weights of the foil workload's electrons
 * being n dx dy / ppc).  FP32 arithmetic on the FP32 grid; one thread a node
 * or a particle; stream-ordered, no allocation (the sort excepted).  A cycle
 * with E^n and B^(n-1/2) stored:
 *   qp_yee_advance_b(dt/2)   B^(n-1/2) -> B^n
 *   qp_step                  particles pushed in E^n, B^n
 *   J = 0; qp_deposit_current for electrons and positrons: J^(n+1/2)
 *   qp_yee_advance_b(dt/2)   B^n -> B^(n+1/2)
 *   qp_yee_advance_e(dt, J)  E^n -> E^(n+1)
 * QP_ERR_INVALID_ARG for a grid of another kind or with a missing component.
 */

/* B -= dtb curl E on the grid, in place. */
int qp_yee_advance_b(qp_ctx *ctx, const qp_field *grid, double dtb, void *stream);

/* E += dt (curl B - J) on the grid, in place; jx, jy, jz: device float
 * arrays of ny rows of nx values on E's staggering, or NULL (no current). */
int qp_yee_advance_e(qp_ctx *ctx, const qp_field *grid, const float *jx, const float *jy,
                     const float *jz, double dt, void *stream);

/* Adds the current of a lepton species' live slots to jx, jy, jz (device
 * float arrays on E's staggering, ny rows of nx, caller-owned; the caller
 * zeroes them): each particle gives q w v / (dx dy) (q = -1 for electrons,
 * +1 for positrons) with the linear weights of each component's staggering
 * at its mid-step position x - v dt/2 (after qp_step: x^(n+1), v^(n+1/2)).
 * Direct deposition, not charge-conserving; float atomics, so the last bits
 * of a sum vary from run to run.  QP_ERR_INVALID_ARG for a photon species. */
int qp_deposit_current(qp_ctx *ctx, int32_t handle, const qp_field *grid, float *jx, float *jy,
                       float *jz, double dt, void *stream);

/* Stable sort of a species' live slots by the grid cell that holds them
 * (row-major: floor((y - y0)/dy) nx + floor((x - x0)/dx); particles outside
 * the grid after every cell, in slot order): every array moves with its
 * particle, so the gather of the next steps reads the grid cell by cell.
 * Slots are renumbered: later draws follow the new slots.  The first call
 * for a capacity allocates the context's scratch (as qp_coalesce_photons;
 * not during a stream capture).  Capacity below 2^32 slots. */
int qp_sort_species(qp_ctx *ctx, int32_t handle, const qp_field *grid, void *stream);

/* ---- super-photon compaction and coalescence ---------------------------- */

/* Grid and bins of qp_coalesce_photons.  A live photon belongs to the group
 * of (cell, energy bin, direction bin):
 *   cell        floor((x - x0) (1/dx)), floor((y - y0) (1/dy)), floor((z - z0) (1/dz))
 *               (z cell 0 for dims 2), each in [0, n); photons outside the
 *               box are never merged;
 *   energy bin  the binary exponent of |u| and its leading log2(E) mantissa
 *               bits (E = energy_bins_per_octave bins per octave, linear in
 *               |u| within the octave);
 *   direction   the dominant axis of u with its sign (a face of a cube) and
 *               the two other components times 1/|dominant component|, each
 *               in D = direction_bins bins over [-1, 1].
 * Every decision is an exact FP64 operation or a bit extraction, so the CPU
 * oracle forms the same groups. */
typedef struct {
    double x0, y0, z0;      /* corner of the grid (normalised length)            */
    double dx, dy, dz;      /* cell sizes (> 0; dz unused for dims 2)            */
    int64_t nx, ny, nz;     /* cells per axis (>= 1; nz = 1 for dims 2)          */
    int32_t energy_bins_per_octave; /* E: a power of two, 1..64                  */
    int32_t direction_bins; /* D: a power of two, 1..64                          */
    int32_t min_group;      /* groups of at least this many photons merge (>= 3) */
    int32_t max_group;      /* a larger group merges in runs of max_group photons
                               (slot order; a last run below min_group is kept);
                               0: 256; else >= min_group                         */
    uint64_t seed;          /* key of the merged photons' optical-depth draws    */
    int64_t step;           /* step counter of those draws                       */
} qp_coalesce_params;

typedef struct {
    int64_t groups_merged;  /* groups replaced by two photons                    */
    int64_t photons_merged; /* photons in those groups                           */
    int64_t n_before;       /* live slots before (decayed photons included)      */
    int64_t n_after;        /* live slots after                                  */
} qp_coalesce_stats;

/*
 * Coalescence of super-photons (section 3, last paragraph: a coalescence of
 * super-photons conserving energy and momentum; the paper gives no
 * algorithm).  Every group (see qp_coalesce_params) of at least min_group
 * live photons is replaced by two photons of weight W/2 each, energy E/W
 * each and momenta P/W +- d, where W, E and P are the group's total
 * weight, energy (sum w |u|) and momentum (sum w u), d is perpendicular to P
 * with |P/W|^2 + |d|^2 = (E/W)^2 and lies in the plane of P and the group's
 * first photon (lowest slot; if that one is parallel to P, the coordinate
 * axis least aligned with P); both sit at the group's weighted mean
 * position and draw fresh optical depths -log(xi) from the Philox stream
 * (seed; photon species, purpose 5, the first photon's particle id, step,
 * k = 0, 1).  A group of more than max_group photons merges in runs of
 * max_group (its members in slot order), each run as a group of its own;
 * a run whose momentum vanishes is kept as it is.  W, E and P
 * of every group are conserved to rounding and both photons are massless.
 * Decayed photons (tau < 0) are removed.  The survivors keep their slot
 * order, a merged pair taking its group's first slot; their chi and nemit
 * go with them (0 for a merged pair).  Slots are renumbered, so a photon's
 * later draws follow its new slot (particle id rule of qp_species_desc).
 * `P` = NULL: compaction only (decayed photons removed, nothing merged).
 * Photon species only, capacity below 2^32 slots.  Stream-ordered on
 * `stream`; the live count is read and rewritten on the device.  The first
 * call for a capacity allocates the context's scratch (about 105 bytes per
 * slot: sort keys, offsets and staging arrays; not during a stream capture).
 * `out` (host, may be NULL): if given, the call synchronises `stream` and
 * fills it.  QP_ERR_INVALID_ARG for bad parameters or a non-photon species;
 * a live count outside [0, capacity] raises the sticky status.
 */
int qp_coalesce_photons(qp_ctx *ctx, int32_t handle, const qp_coalesce_params *P,
                        qp_coalesce_stats *out, void *stream);

/* Compaction of decayed photons: qp_coalesce_photons with P = NULL. */
int qp_compact_photons(qp_ctx *ctx, int32_t handle, qp_coalesce_stats *out, void *stream);

/*
 * Allocation-free diagnostics, for callers that cannot allocate device
 * memory: a host application whose device memory is owned by its own pool
 * allocator (a cudaMalloc behind the pool's back would take memory the pool
 * has budgeted, or fail once the pool has reserved it all).
 * It needs no context: the caller passes the species' buffers (`d`, device
 * pointers as for qp_create_species) and a host `out`, and gets the same
 * state reductions as qp_diagnostics (n_live, n_alive, weight, energy,
 * momentum, chi_mean, hist; equal to within rounding, the partition of the
 * sums differs).  The event counters and `status` are context data and come
 * back as 0.
 * Scratch is a static device array of the library sized for
 * QP_NOALLOC_MAX_TILES tiles of 256 slots (QP_NOALLOC_MAX_SLOTS slots, about
 * 2.4 MB), which every GPU that loads the library holds until the process
 * exits.  A species whose capacity exceeds QP_NOALLOC_MAX_SLOTS is rejected
 * with QP_ERR_INVALID_ARG before anything is enqueued.  The call runs on the
 * device that owns `d->n_live` (made current for the call, the caller's
 * current device restored before it returns); `stream` must belong to that
 * device.  The first call on a device looks the array up on that device
 * (make it before any stream capture).  Every call overwrites the part of
 * the array it reads, but all calls share it: calls that overlap on the GPU
 * (other streams, no ordering between them) race and return wrong results.
 * The result is copied to host memory and `stream` is synchronised before
 * the call returns: a stream being captured is refused with
 * QP_ERR_INVALID_ARG (nothing enqueued).
 * The paper has no counterpart: this is plumbing of the library.
 */
#define QP_NOALLOC_MAX_TILES 4096
#define QP_NOALLOC_MAX_SLOTS (QP_NOALLOC_MAX_TILES * 256)
int qp_diagnostics_noalloc(const qp_species_desc *d, qp_diag *out, void *stream);

/* Reset the species' event counters and the context's sticky status. */
int qp_reset_counters(qp_ctx *ctx, int32_t handle);

/*
 * Kernel timing for benchmarks.  While enabled, qp_step and qp_batch_step
 * bracket each launch of the fused step kernel (one launch per step) with CUDA
 * events recorded on the step's stream (events are owned by the context;
 * enabling clears earlier records).  qp_profile_read synchronises on the
 * recorded events and returns in ms[0] the summed device time in ms and in
 * launches[0] the number of launches; entries 1 and 2 are reserved and read
 * as 0.  No counterpart in the paper.
 */
int qp_profile_enable(qp_ctx *ctx, int enable);
int qp_profile_read(qp_ctx *ctx, double ms[3], int64_t launches[3]);

/*
 * Self-test of the device-side failure detection: one look-back wait on a
 * predecessor tile that never publishes, bounded by `spin_limit` sleeps of
 * about 64 ns.  Returns the status the device raised (QP_ERR_TIMEOUT when the
 * bound works) and clears the context's sticky status.  Synchronous; the
 * context stays usable.  No counterpart in the paper (it tests the library).
 */
int qp_selftest_wait_timeout(qp_ctx *ctx, uint32_t spin_limit);

/* Static, NUL-terminated name of a status code. */
const char *qp_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* QEDPIC_H */
