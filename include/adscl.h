/*
 * adscl.h -- C ABI of the B300 (sm_103a) solver for spherically symmetric scalar-field
 * collapse in AdS4: the Einstein-Klein-Gordon system in the variables Phi, Pi, A, delta of
 * Liebling & Khanna, arXiv:1706.07413, Sec. II, Eqs. (metric), (eq:phi)-(eq:delta).
 *
 * The solver evolves batches of independent instances ("instances" = one radial grid and its
 * fields each) by the method of lines: 4th-order centred differences, Kreiss-Oliger
 * dissipation and classic RK4, with the two constraints (eq:aprime) and (eq:delta) solved on
 * the GPU inside every RK stage.  Grid of one instance: x_i = i h, i = 0..N-1,
 * h = pi / (2 (N - 1)), so x_0 = 0 and x_{N-1} = pi/2.
 *
 * Conventions shared by every entry point:
 *  - Fields of a batch are packed instance after instance: instance b occupies the N_b
 *    doubles starting at offset sum_{c<b} N_c ("packed layout").
 *  - The caller owns every buffer it passes.  The library owns its device state and copies
 *    in and out on the context's stream.
 *  - ptr_is_device = 1: the pointers are device pointers and the call is asynchronous on the
 *    context's stream.  ptr_is_device = 0: host pointers; the call returns after the stream
 *    has finished the work.
 *  - No entry point throws or aborts.  Each returns an adscl_status; on failure the context
 *    keeps a message readable with adscl_last_error.  Per-instance outcomes (collapse,
 *    non-finite fields) are reported in inst_status and the call itself returns ADSCL_OK.
 *  - A context is not thread-safe: one host thread at a time.
 */
#ifndef ADSCL_H
#define ADSCL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct adscl_ctx adscl_ctx; /* opaque, owned by the library */

/* time-stepping schemes (adscl_config.scheme) */
enum { ADSCL_SCHEME_RK4 = 0, ADSCL_SCHEME_EVOLVED_A_RK3 = 1, ADSCL_SCHEME_EVOLVED_A_RK2 = 2,
       ADSCL_SCHEME_FIXED_METRIC_RK3 = 3 };

typedef enum {
    ADSCL_OK = 0,
    ADSCL_EINVAL = 1,       /* bad argument or configuration; nothing was launched */
    ADSCL_ENOMEM = 2,       /* a device or host allocation failed */
    ADSCL_ECUDA = 3,        /* a CUDA runtime call failed (message names it) */
    ADSCL_ETIMEOUT = 4,     /* a bounded device-side wait ran out */
    ADSCL_ENONFINITE = 5,   /* input fields contain NaN or Inf */
    ADSCL_EUNSUPPORTED = 6, /* valid request the library does not provide */
    ADSCL_ECAPACITY = 7     /* request larger than the fixed capacity of adscl_evolve_noalloc */
} adscl_status;

typedef enum {
    ADSCL_INST_RUNNING = 0,   /* can be evolved further */
    ADSCL_INST_DONE = 1,      /* reached the requested time in the last adscl_evolve call */
    ADSCL_INST_COLLAPSED = 2, /* min_x A fell below the collapse threshold (Sec. II) */
    ADSCL_INST_NONFINITE = 3, /* a slice produced NaN or Inf; the instance stopped */
    ADSCL_INST_TIMEOUT = 4    /* a bounded device wait gave up for this instance */
} adscl_inst_status;

typedef struct {
    int32_t num_instances;       /* B >= 1 */
    const int32_t *N;            /* host array of B grid sizes; each N >= 17 with (N - 1) a
                                    multiple of 8 and N <= adscl_max_points() */
    double cfl;                  /* lambda: dt <= lambda h; 0 selects 0.5 */
    double ko_sigma;             /* Kreiss-Oliger strength sigma >= 0 (not in the paper) */
    double collapse_threshold;   /* theta: an instance collapses when min A < theta (the paper
                                    uses 0.01, Sec. II) */
    double out_dt;               /* cadence D: dt = D / ceil(D / (lambda h)) so that steps land
                                    on multiples of D; 0 selects 1.0 */
    int32_t spec_J;              /* number of modes of the spectrum diagnostic (<= 64); 0 = 64 */
    int32_t ckpt_every;          /* adjoint checkpoint interval in steps; 0 = 256 */
    int64_t max_device_iters;    /* iteration limit of any device-side wait; 0 = default */
    int32_t device;              /* CUDA device ordinal */
    int32_t one_per_launch;      /* 0: all instances in one persistent launch;
                                    1: one kernel launch per instance (comparison mode) */
    int32_t chunk_steps;         /* RK4 steps of one instance per scheduling unit of the
                                    persistent launch (instances migrate between SMs at chunk
                                    boundaries); 0 = 16 */
    int32_t direct_launch;       /* 0: adscl_evolve replays a cached CUDA graph of its launches
                                    (recaptured each call on a private stream, updated in
                                    place); 1: it issues the launches one by one */
    int32_t scheme;              /* ADSCL_SCHEME_*: 0 = classic RK4 with A integrated from
                                    Eq. (eq:aprime) at every stage (default); 1 / 2 = the
                                    paper's production variant (Sec. II): A evolved with
                                    Eq. (eq:adot), SSP Runge-Kutta of order 3 / 2; 3 = A = 1 and
                                    delta = 0 held fixed (the paper's Table II case, the linear
                                    wave equation on AdS4), SSP-RK3 */
    int32_t a_reint_every;       /* schemes 1, 2: re-integrate A from Eq. (eq:aprime) on slices
                                    whose step index is a multiple of this (0: never; the
                                    initial slice always takes the constraint solution) */
    int32_t adjoint_ctas;        /* CTAs per instance of the adjoint kernel (adscl_grad): 1, 2 (a
                                    thread-block cluster), or 0 = 2 when the batch has at most
                                    half as many instances as the GPU has SMs, else 1 */
    int32_t adjoint_stage_buffers; /* most checkpoint segments whose stages adscl_grad keeps in
                                    device memory at once: 0 = as many as fit (all segments:
                                    the forward pass stores every stage and nothing is
                                    recomputed; else segments recomputed from checkpoints, see
                                    adscl_grad: 2 buffers let the adjoint kernel's
                                    recomputation of one segment run beside the backward sweep
                                    of the next; else 1) */
    void *stream;                /* cudaStream_t for all work; NULL = the legacy default stream */
    int32_t spectrum_chunks;     /* tensor-core spectrum: 64-point K chunks per FP32
                                    accumulation run (one CTA task); 0 = 1, the most accurate
                                    (see adscl_spectrum for the error bound) */
} adscl_config;

/* Largest grid size N one instance may use with this library: 65537 (the paper's Table II
 * grid).  Grids up to 4097 run on one CTA (one SM) per instance by default, larger ones on a
 * thread-block cluster of 2, 4, 8 or 16 CTAs sharing the instance through distributed shared
 * memory (16 CTAs, for N > 32769, is a non-portable cluster size: on a device that cannot place
 * such a cluster, adscl_create returns ADSCL_EUNSUPPORTED for those grids).  adscl_autotune and
 * adscl_set_shape may also choose a 9-CTA cluster (P = 8, NT = 512) for 73 <= N <= 36865, also
 * non-portable: on a B300 15 such clusters are co-resident (135 SMs) against 15 of 8 CTAs. */
int32_t adscl_max_points(void);

/* Create a context: validates cfg (ADSCL_EINVAL before any allocation or launch), builds the
 * geometry tables of every distinct N, allocates the device state.  *out receives the
 * context, or NULL on failure. */
adscl_status adscl_create(const adscl_config *cfg, adscl_ctx **out);

/* Set the initial slice t = 0 of every instance from packed Phi(x,0), Pi(x,0) and solve the
 * constraints (eq:aprime), (eq:delta) for A and delta on it (Sec. II: initial data are the two
 * scalar-field functions, the metric functions follow from the constraints).  The boundary values Phi(0) = Phi(pi/2) = Pi(pi/2) = 0 are
 * imposed.  Resets every instance to step 0 with status RUNNING (or COLLAPSED at t = 0 if
 * min A already lies below the threshold).  ADSCL_ENONFINITE if an input is NaN/Inf. */
adscl_status adscl_set_initial(adscl_ctx *ctx, const double *Phi, const double *Pi, int ptr_is_device);

/* Same, with Phi(x,0) = 0 and Pi(x,0) = sum_{j<K} a_j e_j(x), e_j the AdS4 normal modes
 * (Sec. II builds initial data from sums of these modes).  a: B x K row-major,
 * K <= 64. */
adscl_status adscl_set_initial_modes(adscl_ctx *ctx, const double *a, int32_t K, int ptr_is_device);

/* Evolve every RUNNING instance until t >= t_end (its step count n with n dt >= t_end - 1e-9 dt)
 * or until it collapses (min A < theta; Sec. II) or turns non-finite.  Outputs, each of
 * length B (any may be NULL): t_reached (time of the last slice), t_collapse (linear
 * interpolation of min A across theta, +inf if none), mass (the paper's mass M = int tan^2 x A
 * rho dx of the last slice: m(pi/2) of the mass function under ADSCL_SCHEME_RK4, the composite
 * Simpson rule on the nodes under the evolved-A schemes), inst_status (adscl_inst_status).
 * The launches (queue set-up, the persistent kernels, the gather of the outputs) run as one
 * CUDA graph launch on the context's stream unless cfg.direct_launch is set.  If the caller is
 * capturing the context's stream, they are issued directly so that the caller's graph records
 * them (with ptr_is_device = 1 the call is then capturable; a replay evolves to the same
 * t_end). */
adscl_status adscl_evolve(adscl_ctx *ctx, double t_end, double *t_reached, double *t_collapse,
                          double *mass, int32_t *inst_status, int ptr_is_device);

/* adscl_evolve for a context of ONE instance under ADSCL_SCHEME_FIXED_METRIC_RK3 (the paper's
 * Table II case, Sec. IV: A = 1 and delta = 0 held fixed, Eqs. (eq:phi), (eq:pi) with SSP-RK3),
 * spread over the whole GPU: one cooperative launch of ceil(N / 500) CTAs of 512 threads, each
 * owning 500 grid nodes and forming the three Runge-Kutta stages of a step on them and on a
 * 9-node halo, meeting at one grid-wide barrier per step (adscl_evolve gives one instance at
 * most one 16-CTA cluster).  Same discretisation and readings as adscl_evolve, so
 * the slices agree with it to rounding; same outputs and per-instance statuses (length 1),
 * same step counter and slice diagnostics (mass: the composite Simpson rule), so calls of the
 * two may follow each other.  The barrier waits are bounded by cfg.max_device_iters: if one
 * runs out the instance is reported TIMEOUT (and a synchronous call returns ADSCL_ETIMEOUT).
 * Scratch of 2 N + ceil(N / 500) doubles is allocated at the first call and kept by the context.
 * The launch is issued directly on the context's stream; not for use inside a stream capture
 * (ADSCL_EUNSUPPORTED).  ADSCL_EUNSUPPORTED also for contexts of more than one instance, other
 * schemes, or a grid whose CTAs do not fit one cooperative launch (N above 500 x the SM count). */
adscl_status adscl_evolve_wide(adscl_ctx *ctx, double t_end, double *t_reached, double *t_collapse,
                               double *mass, int32_t *inst_status, int ptr_is_device);

/* Mode-energy spectrum of every instance's current slice (Sec. II: the evolving solution is
 * projected onto the normal modes to follow the energy in each): E_j = Pi_j^2 + Phi_j^2/omega_j^2,
 * Pi_j = (sqrt(A) Pi, e_j), Phi_j = (sqrt(A) Phi, e_j'), (u, w) = int_0^{pi/2} u w tan^2 x dx by
 * the trapezoid rule on the grid, e_j the AdS4 normal modes (omega_j = 3 + 2j), j < J <= 64.
 * Output E: B x J row-major.  A is recomputed from the current slice (no state change).
 * precision: ADSCL_PREC_FP64 (FP64 CUDA cores), ADSCL_PREC_BF16X3 or ADSCL_PREC_TF32X3: the
 * projections on the tensor cores (tcgen05) with each operand split into a rounded high part
 * and a rounded remainder (BF16 or TF32), three products hi*hi + hi*lo + lo*hi, hi*hi and the
 * two corrections accumulated in FP32 in separate accumulators over runs of
 * cfg.spectrum_chunks x 64 grid points, partial sums added in FP64.  Accuracy (derived, M the
 * mass of the slice): max_j |E_j - E_j(FP64)| <= 2 eps M with
 * eps = 3 2^-2p (1 + 2^-p) + c n 2^-23 (1 + 2^{1-p}), p = 8 (BF16) or 11 (TF32) bits, n = 4
 * (BF16) or 8 (TF32) MMA instructions per 64 points, c = spectrum_chunks: at c = 1,
 * 9.3e-5 M (BF16x3) and 3.4e-6 M (TF32x3).  Small E_j are not relatively accurate.
 * ADSCL_ETIMEOUT if a bounded wait of the tensor-core kernel ran out (host pointers only). */
enum { ADSCL_PREC_FP64 = 0, ADSCL_PREC_BF16X3 = 1, ADSCL_PREC_TF32X3 = 2 };
adscl_status adscl_spectrum(adscl_ctx *ctx, int32_t J, int precision, double *E, int ptr_is_device);

/* Two of the three quantities the two-time-framework (TTF) equations conserve, from the mode
 * energies E_j (j < J) of every instance's current slice (Sec. II: the normal-mode decomposition
 * provides the conserved quantities of the TTF formalism; the temperature quoted for the
 * quasi-periodic data after Eq. (eq:approxQP) is their ratio):
 *   ttf[3b + 0] = E = sum_{j<J} E_j          (total energy; equals the mass M as J grows),
 *   ttf[3b + 1] = N = sum_{j<J} E_j / omega_j (particle number, omega_j = 3 + 2j),
 *   ttf[3b + 2] = T = E / N                   (temperature),
 * summed in order of j in FP64 from the E_j of adscl_spectrum with the same J and precision
 * (an instance with no energy in these modes, e.g. static AdS, gets E = N = 0 and T = NaN).
 * The third conserved quantity, the TTF Hamiltonian, needs interaction coefficients that the
 * paper does not give; it is not provided.  E: optional (NULL or B x J), receives the mode
 * energies.  Errors as adscl_spectrum. */
adscl_status adscl_ttf(adscl_ctx *ctx, int32_t J, int precision, double *ttf, double *E, int ptr_is_device);

/* Track the spectrum in time (Sec. II: the evolving solution is decomposed into normal modes at
 * any time): for k = 0 .. n_snap-1, evolve to t_k = t_first + k cadence exactly as adscl_evolve
 * does (per-instance stop at collapse), then take the mode energies (adscl_spectrum) and the TTF
 * quantities (adscl_ttf) of every instance's current slice.  Outputs (each optional, row k of
 * snapshot k): t_hist (n_snap x B) the time of the slice each instance is on (an instance that
 * collapsed stays on its last slice), ttf_hist (n_snap x B x 3), E_hist (n_snap x B x J).  Steps
 * land on the snapshot times when cadence is a multiple of the context's out_dt.  With host
 * pointers the history is gathered in a temporary device buffer, copied once at the end, and
 * the call reports ADSCL_ETIMEOUT if a device wait ran out (as adscl_evolve). */
adscl_status adscl_track(adscl_ctx *ctx, double t_first, double cadence, int32_t n_snap, int32_t J,
                         int precision, double *t_hist, double *ttf_hist, double *E_hist,
                         int ptr_is_device);

/* Discrete-adjoint gradient of the mode-energy drift functional (Sec. II spectrum; the
 * functional and the adjoint are not in the paper):  for every instance, with
 * Pi(x,0) = sum_{k<K} a_k e_k(x), Phi(x,0) = 0 (a: B x K row-major, K <= 64),
 *   J = sum_{j<spec_J} (E_j(T) - E_j(0))^2,
 * evolved without the collapse stop for n = ceil(T/dt) RK4 steps (the same n for every
 * instance; N <= 8193, above 4097 on 2-CTA clusters of the adjoint kernel, so adjoint_ctas
 * must then be 0 or 2).  Outputs J_out (B) and dJda (B x K).  The steps are cut into segments of
 * ckpt_every; every stage of a segment is stored in device memory (B * ckpt_every * 24 * N
 * doubles per segment) and swept backwards through the exact transpose of the discrete step
 * (constraint scans included).  When every segment's stages fit (adjoint_stage_buffers), the
 * forward pass stores them all; otherwise it keeps (Phi, Pi) at the segment starts, stores the
 * stages of as many last segments as fit and recomputes each earlier segment once before its
 * sweep (adscl_adjoint_storage reports the buffers and the recomputed segments).  The
 * recording runs in the evolution kernel itself (a variant that records every stage) when the
 * context's kernel shapes give the batch at least one CTA per SM, directly or with a small
 * batch's one-CTA shapes split over 2- or 4-CTA clusters for the gradient's own evolutions (see
 * adscl_autotune); else in the adjoint kernel's recomputation.  Replaces the context's state by
 * the final slice (step index n). */
adscl_status adscl_grad(adscl_ctx *ctx, const double *a, int32_t K, double T, double *J_out,
                        double *dJda, int ptr_is_device);

/* Copy out one instance's current slice: Phi, Pi and the constraint solution A, delta on it
 * (each length N_inst; any may be NULL). */
adscl_status adscl_get_state(adscl_ctx *ctx, int32_t inst, double *Phi, double *Pi, double *A,
                             double *delta, int ptr_is_device);

/* Replace one instance's slice by host arrays Phi, Pi at step index `step` (time step*dt);
 * its status becomes RUNNING and the constraints are re-solved. */
adscl_status adscl_set_state(adscl_ctx *ctx, int32_t inst, const double *Phi, const double *Pi,
                             int64_t step);

/* Per-instance time step dt and current step index (host outputs, length B, may be NULL). */
adscl_status adscl_get_clock(adscl_ctx *ctx, double *dt, int64_t *step);

/* Stage storage of adscl_grad (host outputs, each may be NULL): the device bytes the context
 * holds for stage records (kept between calls, freed by adscl_destroy), the number of segment
 * buffers in them, and for the last adscl_grad call its number of checkpoint segments and how
 * many of them were recomputed from their checkpoints (0 when every stage was stored by the
 * forward pass).  All zero before the first adscl_grad.  No device work. */
adscl_status adscl_adjoint_storage(adscl_ctx *ctx, int64_t *bytes, int32_t *buffers, int64_t *segments,
                                   int64_t *recomputed);

/* Autotuner (classic RK4 scheme): for every grid size N of the context, time each kernel shape
 * that fits N -- P grid nodes per thread, NT threads per CTA (so 512 / NT CTAs per SM), CL CTAs
 * (a thread-block cluster) per instance -- on the context's own instances of that N for
 * max(trial_steps, 4 chunk_steps) RK4 steps (trial_steps 0 = 8; at least four scheduling
 * chunks, so that the queue's load balancing shows) from their current slices, keep the fastest,
 * and restore the
 * state (the call changes no instance's slice -- Phi, Pi and, under the evolved-A schemes, A --
 * step or status).  With one grid size the two fastest shapes are timed again over
 * four times the trial length and the faster one is kept.  With several grid sizes, which run
 * concurrently in a batch, the per-size choice is kept only if the whole batch (timed over that
 * longer window) is more than 1 % faster with it than with the default shapes.  Results are
 * cached for the process by (GPU name, SM count, scheme, the batch's grid sizes with their
 * instance counts, and floor(2 log2) of the instances of each size still running): a cached entry
 * is reused without timing or touching the state, and calling this again after collapses have
 * thinned a batch re-tunes for the smaller number of running instances.
 * Synchronous.  The evolved-A and fixed-metric kernels are built for the shapes (8, 512, 1/2/4/8/16),
 * (8, 256, 2) and (8, 128, 2).
 * Different shapes associate the radial scans differently, so results agree with the default
 * shape to rounding, not bit for bit. */
adscl_status adscl_autotune(adscl_ctx *ctx, int32_t trial_steps);

/* The kernel shape (P, NT, CL) instance `inst` runs with (any output may be NULL). */
adscl_status adscl_get_shape(adscl_ctx *ctx, int32_t inst, int32_t *P, int32_t *NT, int32_t *CL);

/* Run every instance of grid size N with shape (P, NT, CL); ADSCL_EINVAL if the library is not
 * built with that shape, it does not fit N, or no instance has that N. */
adscl_status adscl_set_shape(adscl_ctx *ctx, int32_t N, int32_t P, int32_t NT, int32_t CL);

/* Kernel launches issued by this context since creation (for launch accounting). */
int64_t adscl_launch_count(const adscl_ctx *ctx);

/* Measured FP64 throughput of `device` in TFLOP/s (a fused multiply-add counts 2 flops):
 * independent FMA chains on every SM, best of three timed launches on `stream` (a
 * cudaStream_t or NULL).  It is the ceiling of the FP64-bound evolution kernels. */
adscl_status adscl_probe_fp64(int32_t device, void *stream, double *tflops);

/* The solver's e^{-x} (Tang's table-driven method, used for F = A e^{-delta}) on n host
 * values x >= 0, written to host y; exposed so that it can be checked against a reference exp.
 * Synchronous; allocates its own device buffers. */
adscl_status adscl_exp_neg(int32_t device, const double *x, double *y, int64_t n);

/* The same with the argument in units of ln2/256: y = e^{-X ln2/256} for n host values X >= 0.
 * This is the form the evolution kernels use (they accumulate delta in these units, which makes
 * the argument reduction exact without a two-term ln2).  Synchronous; allocates its own device
 * buffers. */
adscl_status adscl_exp_neg_scaled(int32_t device, const double *X, double *y, int64_t n);

/* ---- evolution without device allocation ----------------------------------------------
 * The paper has no counterpart of this entry point; it exists for callers of the library.
 *
 * adscl_evolve_noalloc runs the same computation as adscl_create + adscl_set_initial +
 * adscl_evolve(t_end) (+ adscl_get_state for the fields) for one batch of B instances of one
 * grid size N, but allocates no device memory at all.  It is meant for callers that cannot
 * allocate: programs that give the whole GPU memory to their own pool when they start and
 * forbid allocations outside it, code in latency-critical loops that cannot afford the
 * device-wide synchronisation of cudaMalloc/cudaFree, and plug-ins running inside another
 * framework that owns every allocation.
 *
 * The caller provides, as device pointers: Phi and Pi (packed B x N doubles; on entry the
 * initial slice Phi(x,0), Pi(x,0); on return the slice at t_reached), and four outputs of
 * length B (t_reached, t_collapse, mass, inst_status) with the meaning of adscl_evolve.
 * cfl, ko_sigma and collapse_threshold as in adscl_config (out_dt is 1).  N must satisfy the
 * same rule as adscl_config.N: N >= 17 with (N - 1) a multiple of 8 (so N = 1003 is refused
 * with ADSCL_EINVAL, N = 1025 is accepted).  All other working storage is one fixed array in
 * device memory that the library holds on every GPU where it is loaded (about 1.3 MB, until the
 * process exits), hence the limits: B <= 64 instances, N <= 4097, B * N <= 65552 (16 instances
 * of N = 4097); larger requests return ADSCL_ECAPACITY.
 *
 * Every argument check (ADSCL_EINVAL, ADSCL_ECAPACITY) happens before anything is queued: a
 * refused call leaves Phi, Pi and the outputs untouched.  ADSCL_EINVAL covers a null pointer,
 * a bad device ordinal, N outside the rule above, cfl outside (0, 2], ko_sigma outside
 * [0, 10), a non-finite threshold, and t_end negative, non-finite or so long that the step
 * count overflows the 32-bit work queue (beyond about 2^27 / B RK4 steps).
 *
 * Differences from the allocating path: the geometry tables are computed on the device with
 * CUDA's sin, cos and tan (adscl_create computes them on the host with the C library), so the
 * two paths can differ in the last bit of a table entry and the fields agree to rounding rather
 * than bit for bit.  An instance whose initial slice holds NaN or Inf (adscl_set_initial
 * rejects such a batch with ADSCL_ENONFINITE) is reported here with inst_status
 * ADSCL_INST_NONFINITE at t_reached = 0, and the other instances evolve normally.
 *
 * The work is queued on `stream` (a cudaStream_t, NULL = legacy default) and the call returns
 * without waiting; read the outputs after synchronising that stream.  The first call on a
 * device also looks up the fixed array's device address and sets the kernel's shared-memory
 * attribute; make that first call before any stream capture.  Every call uses the same fixed
 * array (the previous call's contents stay in it until overwritten; each call re-initialises
 * what it needs), so calls whose GPU work overlaps -- on two streams, or from two threads --
 * race with each other: serialise them.  Returns ADSCL_EINVAL for bad arguments and
 * ADSCL_ECUDA if a CUDA call fails. */
#define ADSCL_NOALLOC_MAX_INSTANCES 64
#define ADSCL_NOALLOC_MAX_POINTS 65552
adscl_status adscl_evolve_noalloc(int32_t device, void *stream, int32_t B, int32_t N,
                                  double *Phi, double *Pi, double t_end, double cfl,
                                  double ko_sigma, double collapse_threshold, double *t_reached,
                                  double *t_collapse, double *mass, int32_t *inst_status);

/* Message of the last failure on this context ("" if none).  Valid until the next call. */
const char *adscl_last_error(const adscl_ctx *ctx);

/* Free every resource of the context (NULL is ignored). */
void adscl_destroy(adscl_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* ADSCL_H */
