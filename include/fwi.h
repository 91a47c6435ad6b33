/*
 * fwi.h -- C ABI of the GB300 acoustic full-waveform-inversion solver.
 *
 * The library solves the acoustic wave equation of Sec. 2.4, Eq. 10 of the
 * Stride paper (arXiv 2110.03345) without attenuation,
 *     (1/vp^2) p_tt = rho div(rho^-1 grad p) + s,
 * with a second-order leapfrog in time, 8th- or 10th-order central stencils
 * in space, a sponge absorbing layer and off-grid (bi-/tri-linear) sources
 * and receivers (Sec. 2.4, last paragraphs).  It returns receiver traces
 * (forward modelling, Sec. 3.1) and the L2 trace misfit with its gradient
 * with respect to the squared slowness m = 1/vp^2, computed by the
 * adjoint-state method of Sec. 2.2, Eqs. 5-9 on the discrete scheme (one
 * forward and one adjoint propagation per shot, Sec. 3.2).  For the
 * inversion loop around the gradient (Sec. 2.3, Sec. 3.2) it also provides
 * the per-block low-pass of wavelets and traces (fwi_lowpass) and the
 * gradient-descent update of vp (fwi_vp_update).
 *
 * Conventions shared by every call:
 *  - Arrays are C order, the LAST axis fastest: 2D fields are [ny][nx],
 *    3D fields are [nz][ny][nx].  Coordinates are given in the same axis
 *    order (slowest first), in metres, with node i of axis d at i*spacing[d].
 *  - "device" pointers are CUDA global memory visible to the plan's device;
 *    "host" pointers are ordinary CPU memory.  The caller owns every array
 *    passed in; the library never frees or retains them after a call returns.
 *  - Fields are FP32; the misfit is accumulated in FP64.
 *  - Every call returns a status; nothing aborts.  fwi_last_error() gives a
 *    message for the last failing call on the calling thread.
 *  - Work is enqueued on the plan's CUDA stream.  fwi_forward and
 *    fwi_gradient synchronise that stream once after validating the model and
 *    again before they return (results are complete, the misfit is a host
 *    value, and non-finite results are reported).
 */
#ifndef FWI_H
#define FWI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FWI_OK = 0,
    FWI_ERR_INVALID_ARG = 1,  /* bad sizes, pointers, coordinates or options */
    FWI_ERR_UNSTABLE_CFL = 2, /* dt above 0.95 x the leapfrog stability limit */
    FWI_ERR_BUDGET = 3,       /* workspace does not fit the plan's HBM budget */
    FWI_ERR_CUDA = 4,         /* a CUDA runtime call failed */
    FWI_ERR_NONFINITE = 5,    /* the model or the result holds Inf/NaN */
    FWI_ERR_TIMEOUT = 6,      /* a bounded device wait gave up */
    FWI_ERR_UNSUPPORTED = 7   /* valid request the library does not implement */
} fwi_status;

/* Regular grid and spatial discretisation (Sec. 2.3 Listing 5, Sec. 2.4). */
typedef struct {
    int ndim;           /* 2 or 3 */
    int64_t shape[3];   /* points per axis, slowest first; unused entries ignored */
    double spacing[3];  /* metres per axis, same order */
    int order;          /* spatial order: 8 or 10 (stencil radius 4 or 5) */
    int sponge;         /* sponge width in points on every face, >= 0, < shape/2 */
    double c_ref;       /* sponge reference speed (m/s); <= 0: the maximum vp of
                           the first model the plan sees, then kept fixed */
} fwi_grid;

/* Medium (Sec. 2.3 Listing 6): sound speed, optional density and optional
 * power-law attenuation (the eta d/dt (-lap)^(y/2) p term of Eq. 10, Sec. 2.4,
 * eta = -2 alpha0 vp^(y-1)).  Zero-initialise the fields you do not use. */
typedef struct {
    const float* vp;    /* device [N], N = prod(shape): the sound speed in m/s, or
                           the squared slowness m = 1/vp^2 in s^2/m^2 when
                           param = FWI_PARAM_M; > 0 and finite */
    const float* rho;   /* device [N] kg/m^3, > 0; NULL selects constant density */
    int param;          /* FWI_PARAM_VP (0) or FWI_PARAM_M (1) */
    const float* alpha0; /* device [N] attenuation coefficient alpha0 >= 0, or NULL
                            for none: nepers/m for att_power 0 (frequency
                            independent), nepers/m per (rad/s)^2 for att_power 2;
                            held fixed (not differentiated) */
    int att_power;      /* y: 0 (damping alpha0 vp dt added to the sponge term of the
                           update) or 2 (2 alpha0 vp times the backward difference
                           in time of the Laplacian); ignored when alpha0 is NULL */
} fwi_model;

#define FWI_PARAM_VP 0
#define FWI_PARAM_M 1

/* Acquisition geometry (Sec. 2.3 Listings 7-8): nshots shots, each with nsrc
 * point sources; nrec receivers shared by every shot.  Points must lie inside
 * the grid: 0 <= x_d <= (shape[d]-1)*spacing[d].  The wavelet and trace
 * arrays of one call must each hold fewer than 2^31 samples
 * (nshots*nsrc*nt, nshots*nrec*nt); larger requests are split over calls. */
typedef struct {
    int nshots;               /* >= 1 */
    int nsrc;                 /* sources per shot, >= 1 */
    int nrec;                 /* receivers, 1 .. 2^20 */
    const double* src_xyz;    /* host [nshots][nsrc][ndim] metres */
    const double* rec_xyz;    /* host [nrec][ndim] metres */
} fwi_geometry;

typedef struct fwi_plan fwi_plan;

/* Execution options; zero-initialise and set what you need.  Every field has
 * a default chosen by the plan when left at 0. */
typedef struct {
    int batch;          /* shots propagated concurrently (0: largest the budget allows) */
    int ckpt_every;     /* gradient: 0 = full history if it fits, else sqrt(2 nt)
                           checkpoints; > 0 forces checkpoints every ckpt_every
                           steps; -1 forces the full history */
    int tile;           /* kernel variant: 0 = default; 2D: 1-4 shared-memory staged,
                           one shot per CTA; 5-8 TMA-staged, shots looped inside
                           a CTA (same four tile shapes); 3D: 1-4 shared-memory
                           staged, 5-8 TMA plane ring (32 x points per CTA row),
                           9-12 TMA plane ring with two x points per thread (64);
                           the TMA families give bit-identical results */
    int profile;        /* n > 0: time every n-th stencil launch with CUDA events
                           (1: every launch); 0: no events */
    int use_graphs;     /* reserved, must be 0 (consecutive steps overlap through
                           programmatic dependent launch; whole runs of uneven
                           problems are graphs in fwi_batch_*) */
    int shots_per_cta;  /* 2D TMA variants: shots per CTA (0: chosen from the SM count; 3D: 1) */
    int time_order;     /* 0 or 2: second-order leapfrog; 4: the fourth-order-in-time
                           modified-equation scheme (Sec. 2.4 states the paper's
                           solver is fourth order in time): per step
                           F = k w + k (L(k w) + s^{n+1} - 2 s^n + s^{n-1}) / 12,
                           w = L u^n + s^n, (1+a) u^{n+1} = 2u^n - (1-a) u^{n-1} + F;
                           stable to sqrt(3) x the leapfrog's CFL limit */
    int interp;         /* off-grid sources and receivers: FWI_INTERP_LINEAR (0) or
                           FWI_INTERP_SINC (1), see fwi_point_weights */
    int boundary;       /* absorbing boundary over the grid's sponge width (Sec. 2.4):
                           0 the sponge; 1 a perfectly matched layer (unsplit,
                           second-order form of the coordinate stretching
                           d_j -> d_j / (1 + z_j / p) with the sponge's damping
                           profile z_j per axis, auxiliary fields phi_j and, in
                           3D, the time integral q of u; leapfrog without
                           attenuation; the density must be constant over the
                           layer and the stencil reach next to it) */
} fwi_options;

/* Counters of the last forward/gradient call on a plan. */
typedef struct {
    int batch;                  /* shots per launch used */
    int ckpt_every;             /* 0 = full history, else checkpoint interval */
    int tile;                   /* tile variant used */
    size_t workspace_bytes;     /* device bytes held by the plan */
    int64_t launches;           /* kernels launched by the last call */
    int64_t updates;            /* grid-point updates in the last call (all kernels) */
    int64_t fwd_launches;       /* forward stencil launches (incl. recompute) */
    int64_t adj_launches;       /* adjoint stencil launches */
    double fwd_ms;              /* summed CUDA-event time of the timed forward stencil launches */
    double adj_ms;              /* same for adjoint stencil launches */
    int64_t fwd_points;         /* grid points (interior) x shots of every forward launch, summed */
    int64_t adj_points;
    int64_t fwd_timed;          /* forward launches that carried events (profile option) */
    int64_t adj_timed;
} fwi_stats;

/* Create a plan for one grid and time axis (nt samples of step dt seconds).
 * The plan holds the device workspace, allocated on first use and kept
 * within hbm_budget_bytes (0: 90% of the free device memory at creation).
 * stream: a cudaStream_t (NULL = legacy default stream) the plan enqueues on.
 * Errors: FWI_ERR_INVALID_ARG for a bad grid (including one whose padded
 * field would hold 2^31 floats or more, in-field offsets being 32-bit, or
 * whose second-fastest axis exceeds 524280 points, the CTA grid's y limit),
 * nt < 1 or dt <= 0. */
fwi_status fwi_plan_create(fwi_plan** plan, const fwi_grid* grid, int nt, double dt,
                           size_t hbm_budget_bytes, void* stream);

/* Set execution options (see fwi_options).  Takes effect on the next call.
 * Errors: FWI_ERR_INVALID_ARG (NULL, negative batch), FWI_ERR_UNSUPPORTED
 * (use_graphs != 0); a tile variant out of range is reported by the next call. */
fwi_status fwi_plan_set_options(fwi_plan* plan, const fwi_options* opt);

/* Counters of the last call. */
fwi_status fwi_plan_stats(const fwi_plan* plan, fwi_stats* out);

/* Device bytes one forward (gradient = 0) or gradient (gradient = 1) call
 * with this geometry would hold, at the batch and checkpoint policy the plan
 * would choose.  No device work. */
fwi_status fwi_plan_estimate(const fwi_plan* plan, const fwi_geometry* geom, int gradient,
                             size_t* bytes);

/* Release the workspace and the plan.  NULL is ignored. */
void fwi_plan_destroy(fwi_plan* plan);

/* Forward modelling (Sec. 2.4; Sec. 3.2 Listing 13 `pde(wavelets, vp)`).
 *   wavelet: device [nshots][nsrc][nt] source time functions q^n.
 *   traces:  device [nshots][nrec][nt] output, d^n = P u^n, n = 0..nt-1.
 * nt and dt must equal the plan's (they are repeated for checking).
 * u^0 = u^-1 = 0; step n injects q^n and produces u^{n+1}; d^0 = 0. */
fwi_status fwi_forward(fwi_plan* plan, const fwi_model* model, const fwi_geometry* geom,
                       const float* wavelet, int nt, double dt, float* traces);

/* Misfit and gradient (Sec. 2.2 Eqs. 5-9; Sec. 3.2 Listing 13 `loss`,
 * `fun.adjoint()`).
 *   observed:   device [nshots][nrec][nt] observed data d_obs.
 *   misfit:     host out, J = 1/2 sum_shots sum_rec sum_n (d - d_obs)^2.
 *   grad_m:     device [N] out (overwritten), dJ/dm with m = 1/vp^2, summed
 *               over shots, defined on the whole grid (sponge included).
 *   traces_opt: device [nshots][nrec][nt] out for the modelled traces, or NULL.
 * The paper's vp.grad follows as -2 grad_m / vp^3. */
fwi_status fwi_gradient(fwi_plan* plan, const fwi_model* model, const fwi_geometry* geom,
                        const float* wavelet, const float* observed, double* misfit,
                        float* grad_m, float* traces_opt);

/* The gradient of fwi_gradient split in its two halves, for reverse-mode
 * automatic differentiation (Sec. 2.2: a forward evaluation that records what
 * the adjoint needs, then the adjoint sweep).
 *
 * fwi_misfit_forward runs the forward propagation of every shot, computes the
 * misfit (host out) and optionally the traces, and keeps in the plan what the
 * adjoint needs: for every shot either the history h^n or, when that does not
 * fit the budget (or ckpt_every > 0), checkpoints (u^n, u^{n-1}) every K
 * steps (default K = ceil(sqrt(2 nt))), plus the residual traces.  The
 * model, wavelet and observed device arrays must stay allocated and unchanged
 * until fwi_misfit_backward; any other call on the plan drops the state.
 *
 * fwi_misfit_backward runs the adjoint propagation of those shots with the
 * imaging condition, recomputing each checkpoint segment forward first, and
 * writes grad_m as fwi_gradient does.  It can be called once per forward. */
fwi_status fwi_misfit_forward(fwi_plan* plan, const fwi_model* model, const fwi_geometry* geom,
                              const float* wavelet, const float* observed, double* misfit,
                              float* traces_opt);
fwi_status fwi_misfit_backward(fwi_plan* plan, float* grad_m);

/* fwi_misfit_backward with an optional second output: the gradient of the
 * misfit with respect to the source wavelets,
 *   grad_wavelet[s][i][n] = dJ/dq_{s,i}^n,   device [nshots][nsrc][nt] out,
 * i.e. the adjoint field of each shot sampled at its sources with the
 * injection weights / cell volume (the transpose of the source injection of
 * Sec. 2.4; with the wavelets as the linear input of the forward map
 * F: q -> traces, this is F* applied to the residual, the operator of the
 * adjoint-state method of Sec. 2.2, Eqs. 7-9, for the wavelet variable).
 * dJ/dq^{nt-1} is 0 (the last sample reaches no trace).  Either output may be
 * NULL, not both.  Errors: as fwi_misfit_backward, FWI_ERR_BUDGET when the
 * per-step source samples (nt x batch x nsrc floats) cannot be allocated. */
fwi_status fwi_misfit_backward_ex(fwi_plan* plan, float* grad_m, float* grad_wavelet);

/* ---- Uneven batches (many independent problems in one CUDA graph) ---- */

/* One independent problem of a batch: its own grid, time axis, model,
 * geometry, wavelets (device [nshots][nsrc][nt]) and traces (device out
 * [nshots][nrec][nt]); the arrays follow fwi_forward.  A gradient problem
 * (Sec. 2.2, as fwi_gradient) also gives observed (device [nshots][nrec][nt]),
 * grad_m (device out, N floats, dJ/dm with m = 1/vp^2) and misfit (host out,
 * J, written by fwi_batch_run); traces may then be NULL.  A forward problem
 * leaves observed, grad_m and misfit NULL.  The problems of one batch are all
 * forward or all gradient problems. */
typedef struct {
    fwi_grid grid;
    int nt;
    double dt;
    fwi_model model;
    fwi_geometry geom;
    const float* wavelet;
    float* traces;
    const float* observed;
    float* grad_m;
    double* misfit;
} fwi_problem;

typedef struct {
    int problems;
    int64_t units;       /* (problem, tile, shot) work units of one step */
    int64_t launches;    /* kernel launches (graph nodes) of one run */
    int64_t updates;     /* grid-point updates of one run */
    double run_ms;       /* device time of the last fwi_batch_run */
    int shots_per_cta;   /* the largest shot group of one CTA in the batch's launches */
    int checkpointed;    /* gradient batches: problems run with checkpoints (their
                            full history did not fit the budget left to them) */
} fwi_batch_stats;

typedef struct fwi_batch fwi_batch;

/* Prepare a batch of 2D problems that share the stencil order and density
 * mode but differ in grid, time axis, shot count and geometry (the shot-level
 * parallelism of Sec. 2.5 / 3.3, applied to independent problems on one
 * GPU).  Each problem's model is validated (CFL) and prepared, its tables
 * built and its workspace allocated (all its shots at once; the total must
 * fit hbm_budget_bytes, 0 = free memory).  Every time step of every problem
 * then runs in ONE launch of a multi-problem kernel per step (units =
 * problem x tile x shot; problems that have finished drop out), and with
 * use_graph = 1 the whole sequence, including the final sampling and trace
 * transposition, is captured once into a CUDA graph.  opt (or NULL) selects
 * the kernel variant (tile, shots_per_cta; 2D TMA variants 5-8 or variant 1)
 * for every problem.  A gradient batch runs each problem's gradient as
 * fwi_gradient does (all its shots at once; the full wavefield history when
 * it fits the budget left, else sqrt(nt) checkpoints), each problem on its
 * own stream forked from the batch's: with use_graph = 1 the graph holds one
 * independent branch per problem, which the GPU runs concurrently.  Unless
 * opt fixes shots_per_cta, a gradient batch sizes the shot groups for the
 * batch as a whole (the largest S <= 6 whose CTAs over all its problems make
 * four waves of two per SM), not per problem.  The problem arrays must stay
 * valid until fwi_batch_destroy. */
fwi_status fwi_batch_create(fwi_batch** batch, int nprob, const fwi_problem* probs,
                            const fwi_options* opt, size_t hbm_budget_bytes, void* stream,
                            int use_graph);
/* Run the batch (one graph launch); synchronises the stream. */
fwi_status fwi_batch_run(fwi_batch* batch);
fwi_status fwi_batch_stats_get(const fwi_batch* batch, fwi_batch_stats* out);
void fwi_batch_destroy(fwi_batch* batch);

/* Size of the fixed device scratch used by fwi_forward_noalloc (64 MiB). */
#define FWI_NOALLOC_SCRATCH_BYTES (64u << 20)

/* Forward modelling that allocates no device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- a service that reserves its device memory at start-up and must
 * not allocate while serving, a plugin whose host application owns the
 * device allocator, or code that must avoid the implicit synchronisation of
 * cudaMalloc/cudaFree.  It computes what fwi_forward computes (same kernels,
 * same results), without a plan: the workspace lives in one static device
 * array of FWI_NOALLOC_SCRATCH_BYTES that every device loading this library
 * holds until the process exits.
 *   grid, nt, dt: as for fwi_plan_create (the sponge reference speed c_ref
 *     <= 0 takes the maximum vp of this call's model).
 *   model, geom, wavelet, traces: as for fwi_forward; the caller allocates the
 *     inputs and the output.  Shots run in batches that fit the scratch.
 *   stream: cudaStream_t to enqueue on; the call synchronises it before
 *     returning.
 * The call runs on the current device; every device array must live there
 * (FWI_ERR_INVALID_ARG otherwise).  The first call on a device looks up the
 * scratch address (once per device, with that device current).  The address
 * is kept for the life of the process, so the entry point must not be used on
 * a device after a cudaDeviceReset of it.  All calls share the scratch and keep the last
 * call's contents, so calls that overlap on the GPU race; each call clears
 * what must start at zero, and returns only when its own work on the scratch
 * has finished, on success and on error.
 * Errors: FWI_ERR_BUDGET (with the required and available sizes in
 * fwi_last_error) when one shot of the grid does not fit the scratch, plus
 * the errors of fwi_plan_create and fwi_forward. */
fwi_status fwi_forward_noalloc(const fwi_grid* grid, int nt, double dt, const fwi_model* model,
                               const fwi_geometry* geom, const float* wavelet, float* traces,
                               void* stream);

/* Message describing the last error on the calling thread ("" if none). */
const char* fwi_last_error(void);

/* Device bytes that plan workspaces can still take on the current device:
 * free device memory plus the part of the default stream-ordered pool that
 * freed plans left reserved but unused (the default budget of a new plan is
 * 0.9 of this).  Host utility, no counterpart in the paper.  Errors:
 * FWI_ERR_INVALID_ARG (NULL), FWI_ERR_CUDA (no device). */
fwi_status fwi_mem_available(size_t* bytes);

/* Self-check of the bounded device wait that guards the step kernels' TMA
 * pipelines (a wait on a copy that never lands gives up, flags the step and
 * the call returns FWI_ERR_TIMEOUT instead of hanging the GPU): one thread on
 * the current device waits, with a limit of `polls` polls, on an mbarrier
 * phase that nothing completes.  Returns FWI_ERR_TIMEOUT when the wait gave
 * up and the flag reached the host, which is the expected outcome; the
 * device stays usable.  Host utility, no counterpart in the paper.  Errors:
 * FWI_ERR_INVALID_ARG (polls outside [1, 2^22]), FWI_ERR_CUDA. */
fwi_status fwi_check_bounded_wait(unsigned int polls);

/* ------------------------------------------------------------------------
 * The inversion loop around the gradient (Sec. 2.3: a gradient-descent
 * optimiser steps the model after each gradient; Sec. 3.2: blocks of
 * increasing frequency, each iteration on a random subset of the shots, the
 * wavelets and traces processed for the block's upper frequency).  The loop
 * itself is host code; these are its two device steps besides fwi_gradient.
 * ------------------------------------------------------------------------ */

#define FWI_LOWPASS_MAX_HALF_WIDTH 2048

/* Zero-phase low-pass of rows of samples, gathered by shot: the processing
 * of wavelets and observed traces for a frequency block with upper
 * frequency f_max.
 *   out[i][r][n] = sum_{j=-M}^{M} h_j in[ids[i]][r][n - j], in = 0 outside
 *   0 <= n < nt, with h_j proportional to sinc(2 f_max dt j) times the Hann
 *   window 0.5 (1 + cos(pi j / (M + 1))), scaled so that sum_j h_j = 1
 *   (gain 1 at zero frequency, 1/2 at f_max; M >= 3 / (f_max dt) keeps the
 *   pass band below 0.7 f_max within 1% and the stop band above 1.5 f_max
 *   below 0.25%).
 *   in:  device [n_in][rows][nt] (wavelets: rows = nsrc; traces: rows = nrec).
 *   ids: host [n_ids], each in [0, n_in); repeats allowed.
 *   out: device [n_ids][rows][nt], must not overlap in.
 *   half_width M in [0, FWI_LOWPASS_MAX_HALF_WIDTH] (0 copies the rows).
 * Enqueued on `stream` (a cudaStream_t, NULL = legacy default stream); no
 * synchronisation.  The taps are evaluated in FP32 on the device and the
 * sums accumulate in FP32 in the order j = -M..M.  Errors:
 * FWI_ERR_INVALID_ARG (sizes, NULL arrays, ids, half_width, dt or f_max not
 * positive, overlap, rows > 65535), FWI_ERR_CUDA. */
fwi_status fwi_lowpass(const float* in, int n_in, int rows, int nt, const int* ids, int n_ids,
                       double dt, double f_max, int half_width, float* out, void* stream);

/* One gradient-descent step on the sound speed (Sec. 2.3), normalised so
 * that the largest change of any point is `step`:
 *   d_i = mask_i * (-2 grad_m_i / vp_i^3)     (dJ/dvp from dJ/dm, m = 1/vp^2)
 *   s = max_i |d_i|
 *   vp_i <- min(max(vp_i - step * d_i / s, vp_min), vp_max)
 * vp is left unchanged when s = 0; when any d_i is Inf or NaN every vp_i
 * becomes NaN (the next propagation then reports FWI_ERR_NONFINITE).
 *   vp:     device [n] in/out, positive.
 *   grad_m: device [n], dJ/dm as written by fwi_gradient.
 *   mask:   device [n] weights (0 freezes a point) or NULL for all ones.
 *   work:   device scratch of at least 4 bytes (overwritten).
 * Enqueued on `stream`; no synchronisation.  FP32; the maximum is exact and
 * independent of scheduling.  Errors: FWI_ERR_INVALID_ARG (n < 0, NULL
 * arrays, step < 0 or not finite, vp_min > vp_max), FWI_ERR_CUDA. */
fwi_status fwi_vp_update(float* vp, const float* grad_m, const float* mask, long long n,
                         float step, float vp_min, float vp_max, float* work, void* stream);

/* Interpolation weights of one off-grid point (Sec. 2.4: bi-/tri-linear or
 * high-order sinc interpolation of sources and receivers).  Host utility, no
 * device work.
 *   FWI_INTERP_LINEAR: the 2^ndim bi-/tri-linear corners the solver uses
 *     (sources spread w / cell volume, receivers sample with w).
 *   FWI_INTERP_SINC: Kaiser-windowed sinc, per axis the 2r nodes
 *     floor(x)-r+1 .. floor(x)+r (x in grid units) weighted by
 *     I0(b sqrt(1 - (d/r)^2)) / I0(b) * sin(pi d) / (pi d), d = node - x,
 *     r = FWI_SINC_RADIUS, b = FWI_SINC_KAISER_B (the window that minimises
 *     the largest error of interpolating cosines down to 4 points per
 *     wavelength, 1.3e-3); the point's weights are the products over the
 *     axes, (2r)^ndim nodes, the slowest axis varying slowest.  The solver
 *     injects and samples with these weights when fwi_options.interp is
 *     FWI_INTERP_SINC.
 *   xyz:     host [ndim] metres, slowest axis first, inside the grid (sinc:
 *            at least r - 1 nodes inside every face).
 *   nodes:   host out [cap][ndim] grid indices, slowest axis first.
 *   weights: host out [cap].
 *   count:   out, the number of nodes (set even when cap is too small).
 * Errors: FWI_ERR_INVALID_ARG (grid, NULL, interp, point outside or too close
 * to a face, cap below count). */
#define FWI_INTERP_LINEAR 0
#define FWI_INTERP_SINC 1
#define FWI_SINC_RADIUS 4
#define FWI_SINC_KAISER_B 6.31
fwi_status fwi_point_weights(const fwi_grid* grid, const double* xyz, int interp,
                             int64_t* nodes, double* weights, int cap, int* count);

/* Leapfrog stability limit of c*dt/h for this order and dimension:
 * 2/sqrt(ndim * lambda_max), lambda_max = |sum_j (-1)^j w2_j| of the
 * second-derivative stencil.  Returns a negative value for bad input. */
double fwi_cfl_limit(int ndim, int order);

#ifdef __cplusplus
}
#endif

#endif /* FWI_H */
