/*
 * qlbm.h - C ABI of a GB300 (sm_103a) solver for the finite-difference
 * Enskog-Shakhov lattice Boltzmann model of S. Busuioc, "Quadrature-based
 * Lattice Boltzmann model for non-equilibrium dense gas flows"
 * (arXiv:2211.16933).
 *
 * The model evolves the two reduced distributions phi_k(x, t), theta_k(x, t)
 * of Sec. II.C on the Q-point full-range Gauss-Hermite velocity set of
 * Sec. II.D, with Eq. (evolution_lb):
 *   d_t psi_k + p_k d_x psi_k = -(psi_k - psi_S;k)/tau + J1_k,  psi in {phi, theta},
 * advanced by the third-order TVD Runge-Kutta scheme of App. A.1 (Eq. rk3),
 * with WENO-5 advection (App. A.2) and 6th-order central gradients (App. A.3).
 *
 * Units are the nondimensional ones of Sec. II.A: m = k_B = T_ref = 1.
 *
 * Conventions for every entry point:
 *   - Returns a ql_status; nothing is thrown across the ABI.  On an error other
 *     than QL_OK, ql_last_error() describes it.
 *   - Pointers named "host" are caller-owned host memory; the library copies
 *     from or into them before returning.  Pointers named "device" are
 *     caller-owned device memory on the context's device.
 *   - The context owns its device buffers and frees them in ql_destroy.
 *   - Work is queued on the stream given at creation; only ql_step returns
 *     before its work is done.  Calls on one context are not thread-safe.
 *   - Non-physical states (n <= 0, T <= 0 or a non-finite moment in any
 *     interior cell) raise a device error word that the next synchronising
 *     call (ql_sync, ql_moments, ql_get_state, ql_totals) reports as
 *     QL_ENONPHYSICAL.
 */
#ifndef QLBM_H
#define QLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ql_ctx ql_ctx; /* opaque, library-owned */

typedef enum {
    QL_OK = 0,
    QL_EINVAL = 1,        /* invalid argument or unsupported combination */
    QL_ENOMEM = 2,        /* device or host allocation failed */
    QL_ECUDA = 3,         /* a CUDA runtime call failed */
    QL_ENONPHYSICAL = 4,  /* n <= 0, T <= 0 or non-finite moments in a cell */
    QL_ETIMEOUT = 5,      /* a bounded device wait ran out */
    QL_EUNSUPPORTED = 6   /* a velocity-set size this build has no kernel for */
} ql_status;

enum { QL_FP64 = 0, QL_FP32 = 1 };              /* arithmetic of the state and its update */
enum { QL_SUMS_DFP32 = 0, QL_SUMS_FP64 = 1 };   /* FP32 mode: per-cell conserved sums */
enum { QL_LAUNCH_AUTO = 0, QL_LAUNCH_STAGES = 1, QL_LAUNCH_RUN = 2 }; /* how ql_step launches (ql_opts.launch) */
enum { QL_BC_PERIODIC = 0, QL_BC_FIXED = 1 };   /* boundary of the 1D domain */
enum { QL_INIT_SOUND = 0, QL_INIT_RIEMANN = 1, QL_INIT_SHOCK = 2, QL_INIT_FIELDS = 3 };
enum { QL_PR_CONST = 0, QL_PR_DENSE = 1 };
/* Contact value of the pair correlation function (Sec. II.A): chi_SET of the
 * local density (Eq. chi), or chi_RET-FM, chi_SET of the density averaged over
 * a ball of radius sigma (Eq. chi_ret). */
enum { QL_CHI_SET = 0, QL_CHI_RET_FM = 1 };
/* Largest number of cells on each side that the chi_RET-FM ball may reach
 * (sigma / dx < QL_FM_MAX_HALFWIDTH + 1/2). */
#define QL_FM_MAX_HALFWIDTH 256

/* Velocity set, Sec. II.D: the Q roots p_k of the probabilists' Hermite
 * polynomial He_Q with weights w_k = Q!/He_{Q+1}(p_k)^2 (kind 0 is the only
 * kind).  Tiled kernels exist for Q in {8, 16, 20, 24, 32, 40} (the batched
 * form: {8, 16, 24, 32}); any other even Q up to 200 (the paper's
 * near-ballistic runs use 200) runs on a generic FP64 path whose per-cell
 * work grows as Q^2: FP64 only (chi_SET or chi_RET-FM), for domains of the
 * paper's sizes (hundreds to thousands of cells). */
typedef struct {
    int32_t Q;
    int32_t kind;
} ql_velset;

/* Uniform grid of nx cells of width dx = length/nx, centres x_i = (i+1/2) dx,
 * and the time step dt (> 0) of Eq. (rk3). */
typedef struct {
    int64_t nx;
    double length;
    double dt;
} ql_grid;

/* Boundary: QL_BC_PERIODIC, or QL_BC_FIXED, where three ghost cells on each
 * side hold the discrete equilibrium of fixed states for the whole run (the
 * far field of the initial state, or ql_init.ghost for QL_INIT_FIELDS). */
typedef struct {
    int32_t kind;
    int32_t pad_;
} ql_bc;

/* Initial macroscopic state; the distributions start as its discrete
 * equilibrium, phi_k = n g_k[u, T] and theta_k = 2 T n g_k of Eq. (feq).
 *   QL_INIT_SOUND   prm = {rho0, T0, A}: rho = rho0 (1 + A cos(2 pi x/L)),
 *                   u = 0, T such that the pressure P = rho T (1 + b rho chi)
 *                   is uniform (Sec. IV.A, delta P = 0).  Needs periodic bc.
 *   QL_INIT_RIEMANN prm = {rhoL, uL, TL, rhoR, uR, TR}: two states split at
 *                   x = L/2 (the Sod tube of Eq. shock_init).
 *   QL_INIT_SHOCK   prm = {rho1, T1, M, width}: standing normal shock, the
 *                   upstream state moving at u1 = M c_s(rho1, T1) and the
 *                   downstream state from the Rankine-Hugoniot relations of
 *                   Eq. (rankine_hugoniot) with the dense equation of state,
 *                   joined by a tanh of the given width centred at L/2.
 *   QL_INIT_FIELDS  rho, u, T: host arrays of nx doubles; with QL_BC_FIXED,
 *                   ghost: host array of 6 (rho, u, T) triples for cells
 *                   -3, -2, -1, nx, nx+1, nx+2 in that order. */
typedef struct {
    int32_t kind;
    int32_t pad_;
    double prm[8];
    const double *rho, *u, *T;
    const double *ghost;
} ql_init;

/* Device allocator hooks (for example a PyTorch caching allocator); when alloc
 * is NULL the library calls cudaMalloc/cudaFree. */
typedef void *(*ql_alloc_fn)(size_t bytes, void *user);
typedef void (*ql_free_fn)(void *ptr, void *user);

/* Options.
 *   precision  QL_FP64: state, update and sums in FP64.
 *              QL_FP32: state and update in FP32; the per-cell
 *              conserved-moment sums (mass, momentum, energy) as `sums` says;
 *              the domain totals in FP64.
 *   sums       FP32 only.  QL_SUMS_DFP32 (0, default): the per-cell conserved
 *              sums are combined, and u and T derived, in double-FP32 (about
 *              48 significant bits).  QL_SUMS_FP64: in FP64, as are the
 *              per-cell sums behind the domain totals of ql_totals and
 *              ql_moments.  FP32 products are summed over groups of 8 velocity
 *              pairs in FP32 first in either mode.
 *   pr_mode    QL_PR_CONST uses pr_const; QL_PR_DENSE the Prandtl number of
 *              the dense gas as a function of b rho chi (Sec. II.B).
 *   enskog     1 adds the simplified-Enskog term J1 of Eq. (j1_expanded);
 *              0 leaves it out (b rho chi still sets tau and Pr).
 *   chi_mode   QL_CHI_SET or QL_CHI_RET_FM.  With QL_CHI_RET_FM, chi of
 *              every cell is chi_SET of nbar, the density averaged over the
 *              ball of radius sigma around the cell centre (for fields that
 *              depend on x only: nbar = 3/(4 sigma^3) int n(x+s)(sigma^2-s^2)
 *              ds over |s| < sigma, cells constant over their width); it
 *              enters b rho chi, tau, Pr and J1, and d ln chi is the 6th-order
 *              difference of ln chi.  Beyond the domain the density continues
 *              periodically, or (fixed bc) as that of ghost cell -3 / nx + 2.
 *              The output pressure keeps chi_SET of the local density.
 *   rho_ref    density at which the denseness E_l is given; the local reduced
 *              density is eta = eta0 rho / rho_ref.
 *   fault      0 normally.  1 (for failure-detection tests of the caller's
 *              error handling, tiled velocity sets only): the stage kernels
 *              arm their tile-staging barrier but issue no copies, so each
 *              CTA's bounded wait gives up (no copy is in flight, nothing
 *              faults) and the next synchronising call returns QL_ECUDA
 *              ("gave up waiting"); the state is left as it was.
 *   launch     How ql_step launches the stages of FP32 chi_SET solvers of the
 *              tiled velocity sets (Q = 8, 16, 20, 24, 32, 40); other solvers
 *              always launch per stage.  QL_LAUNCH_STAGES: one launch per
 *              Runge-Kutta stage (ql_step of several steps replays a recorded
 *              step).  QL_LAUNCH_RUN: each ql_step call is one launch of
 *              (stage, tile) work items (several for runs of more than
 *              2^31 - 1 of them), a tile's stage starting once the previous
 *              stage of it and of its neighbours has completed, so that
 *              consecutive stages and steps overlap.  QL_LAUNCH_AUTO (0,
 *              default): QL_LAUNCH_RUN for domains of one to eight times as
 *              many tiles (248 cells each) as the GPU holds CTAs at once, where
 *              a stage's last wave of CTAs leaves much of the GPU idle, and
 *              QL_LAUNCH_STAGES otherwise.  Results are the same bit for bit.
 *   stream     cudaStream_t for all work, NULL for the legacy default stream. */
typedef struct {
    int32_t precision;
    int32_t pr_mode;
    int32_t enskog;
    int32_t device;
    int32_t chi_mode;
    int32_t fault;
    int32_t sums;
    int32_t launch;
    double pr_const;
    double rho_ref;
    void *stream;
    ql_alloc_fn alloc;
    ql_free_fn free;
    void *alloc_user;
} ql_opts;

/* Creates a solver (Secs. II.B-II.D).
 *   denseness  E_l = sigma/l > 0 at rho_ref (Sec. II.B), which fixes the
 *              reduced density eta0 through E_l = 6 sqrt(2) eta0 chi(eta0).
 *   kn         l0/L > 0, l0 the Enskog mean free path at rho_ref; with E_l it
 *              fixes sigma = E_l l0 and so tau = sigma g[eta] (Eq. tau_sigma).
 * Errors: QL_EINVAL (bad sizes, dt <= 0, eta0 out of range, init kind needs
 * another bc, bad chi_mode), QL_EUNSUPPORTED (Q; a chi_RET-FM ball reaching
 * more than QL_FM_MAX_HALFWIDTH cells), QL_ENOMEM, QL_ECUDA.  On error *out is
 * NULL. */
ql_status ql_create(const ql_velset *vs, const ql_grid *grid, double denseness, double kn,
                    const ql_bc *bc, const ql_init *init, const ql_opts *opts, ql_ctx **out);

/* Queues nsteps >= 0 steps of Eq. (rk3): three fused stage kernels per step,
 * each computing moments, equilibrium, Shakhov targets, J1, WENO-5 fluxes and
 * the Runge-Kutta combination for every (cell, velocity).  Asynchronous.  With
 * nsteps > 1 the first call records one step as a CUDA graph (on a stream the
 * context creates) and every step replays it, with results bitwise those of
 * single steps; if recording fails the launches are issued one by one. */
ql_status ql_step(ql_ctx *ctx, int64_t nsteps);

/* Waits for the context's stream and reports the device error word. */
ql_status ql_sync(ql_ctx *ctx);

/* Macroscopic fields of Sec. II.D per cell, computed on the device in FP64:
 * rho, u, T, P = n T (1 + b rho chi) (Sec. II.B), q, Pxx = sum xi^2 phi.
 * Each output is a host array of nx doubles or NULL; totals (host, 3 doubles
 * or NULL) gets the domain sums of mass, momentum and energy times dx.
 * Synchronises. */
ql_status ql_moments(ql_ctx *ctx, double *rho, double *u, double *T, double *P, double *q,
                     double *Pxx, double *totals);

/* Domain totals only (host, 3 doubles), FP64.  Synchronises. */
ql_status ql_totals(ql_ctx *ctx, double *totals);

/* Copies the state to host arrays phi, theta of nx*Q doubles, cell-major
 * (phi[i*Q + k]), converting FP32 states to double.  Synchronises. */
ql_status ql_get_state(ql_ctx *ctx, double *phi, double *theta);

/* Replaces the state from host arrays laid out as in ql_get_state (rounded
 * to FP32 for QL_FP32 contexts).  Ghost cells are refreshed. */
ql_status ql_set_state(ql_ctx *ctx, const double *phi, const double *theta);

/* Re-initialises the state from host macroscopic fields rho, u, T (nx
 * doubles each) as the discrete equilibrium, like QL_INIT_FIELDS.  Fixed
 * ghost cells keep their states. */
ql_status ql_load_fields(ql_ctx *ctx, const double *rho, const double *u, const double *T);

/* Evaluates the right-hand side L[psi] of Eq. (cast) for the current state
 * into host arrays Lphi, Ltheta (nx*Q doubles, cell-major).  Synchronises. */
ql_status ql_rhs(ql_ctx *ctx, double *Lphi, double *Ltheta);

/* Device view of the current state for callers that keep data on the GPU:
 * the state is Q rows, one per velocity k (ascending p_k), of pairs
 * (phi_k, theta_k); *psi points at cell 0 of row 0 and cell i of row k is
 * pair (*psi)[k * row_stride + i].  A pair is two doubles for QL_FP64 and two
 * floats for QL_FP32.  Valid until the next ql_step returns and the stream has
 * run it.  The view is for reading: with chi_RET-FM the solver keeps the
 * averaged densities of the state it last wrote, so a state changed through
 * this pointer must be loaded again with ql_set_state. */
ql_status ql_state_device(ql_ctx *ctx, void **psi, int64_t *row_stride);

/* Numbers fixed at creation: out[0] = eta0, out[1] = chi(eta0),
 * out[2] = sigma, out[3] = dx, out[4] = dt, out[5] = max |p_k|,
 * out[6..6+Q) = p_k, out[6+Q..6+2Q) = w_k.  out holds 6 + 2Q doubles. */
ql_status ql_info(const ql_ctx *ctx, double *out);

/* How ql_step launches (no counterpart in the paper; for timing tools):
 * *steps_per_launch = the most steps one launch of the whole-run kernel covers
 * (ql_opts.launch), or 0 when the solver launches one kernel per Runge-Kutta
 * stage.  QL_EINVAL for a null argument. */
ql_status ql_launch_info(const ql_ctx *ctx, int64_t *steps_per_launch);

/* ---- Batched form -------------------------------------------------------- */

/* Many independent domains (for example sound waves and shocks of different
 * size, velocity set, denseness and Mach number) advanced together: each
 * Runge-Kutta stage is one persistent kernel launch over a list of (instance,
 * tile) work items, and ql_batch_run captures a whole run in one CUDA graph. */
typedef struct ql_batch ql_batch; /* opaque, library-owned */

/* One instance: the arguments of ql_create, with its own gas options
 * (pr_mode, enskog, pr_const, rho_ref and chi_mode as in ql_opts; chi_mode
 * QL_CHI_RET_FM takes chi of each cell from the ball-averaged density, Eq.
 * (chi_ret), with the same limit on the ball's half-width). */
typedef struct {
    ql_velset vs;
    ql_grid grid;
    double denseness;
    double kn;
    ql_bc bc;
    ql_init init;
    int32_t pr_mode;
    int32_t enskog;
    double pr_const;
    double rho_ref;
    int32_t chi_mode;
    int32_t pad_;
} ql_instance;

/* Creates a batch of n >= 1 instances (host array inst; the initial-field
 * arrays it points to are read before return).  Each instance uses chi_SET or
 * chi_RET-FM (its chi_mode); with chi_RET-FM every stage is followed by one
 * batched ball-average launch over those instances.  From
 * opts only precision, sums, device, stream and the allocator hooks are used; with stream NULL the batch
 * creates its own stream (a CUDA graph cannot be captured on the legacy
 * default stream).  Errors as for ql_create, naming the first bad instance. */
ql_status ql_batch_create(const ql_instance *inst, int64_t n, const ql_opts *opts, ql_batch **out);

/* Picks the CTA shape (warps per CTA, 8 or 4) and the grid by timing
 * trial_launches >= 1 launches of the first stage for each candidate (the
 * first stage leaves the state unchanged): one CTA per work item, which the
 * batch starts with (*ctas_per_sm = 0), or a persistent grid of ctas_per_sm
 * CTAs per SM walking the work list.  Every choice gives the same results.
 * Outputs may be NULL.  Synchronises. */
ql_status ql_batch_tune(ql_batch *b, int32_t trial_launches, int32_t *warps, int32_t *ctas_per_sm);

/* Sets the CTA shape and grid that ql_batch_tune would pick: warps per CTA (8
 * or 4) and ctas_per_sm (0: one CTA per work item; else a persistent grid of
 * that many CTAs per SM, at most what an SM holds).  QL_EINVAL otherwise. */
ql_status ql_batch_set_shape(ql_batch *b, int32_t warps, int32_t ctas_per_sm);

/* Queues nsteps steps of Eq. (rk3) for every instance as one CUDA graph
 * launch (3 nsteps persistent stage kernels; the graph is rebuilt only when
 * nsteps or the tuned shape changes).  Asynchronous. */
ql_status ql_batch_run(ql_batch *b, int64_t nsteps);

/* Waits for the batch's stream; flags (host, n words, or NULL) receives each
 * instance's error word.  QL_ENONPHYSICAL if any instance went non-physical. */
ql_status ql_batch_sync(ql_batch *b, uint32_t *flags);

/* ql_moments for instance i (0 <= i < n); arrays of that instance's nx. */
ql_status ql_batch_moments(ql_batch *b, int64_t i, double *rho, double *u, double *T, double *P, double *q,
                           double *Pxx, double *totals);

/* Amplitude of density mode m of every instance (Sec. IV.A: the projection
 * (2/nx) sum_j rho_j cos(2 pi m x_j / L) used to follow a sound wave), written
 * as n doubles to the device array out (caller-owned).  Asynchronous on the
 * batch's stream.  QL_EINVAL for a null batch or out, or m < 0. */
ql_status ql_batch_project(ql_batch *b, int32_t mode, double *out);

/* Fields of every instance on the device, averaged over blocks of nx/ncoarse
 * cells (ncoarse must divide every instance's nx; ncoarse = nx gives the
 * fields themselves): out (device, f64, n * 5 * ncoarse) holds, for instance
 * i, rows rho, u, T, q, Pxx (Sec. II.D) of ncoarse values at offset
 * i * 5 * ncoarse.  One launch; asynchronous. */
ql_status ql_batch_fields(ql_batch *b, int32_t ncoarse, double *out);

/* ql_get_state for instance i. */
ql_status ql_batch_get_state(ql_batch *b, int64_t i, double *phi, double *theta);

/* out (host, 6 doubles) = {n, sum of nx Q (updates per step), warps per CTA,
 * persistent CTAs, bytes per state arena, SM count}. */
ql_status ql_batch_info(const ql_batch *b, double *out);

ql_status ql_batch_destroy(ql_batch *b);
const char *ql_batch_last_error(const ql_batch *b);

/* ---- Learned coarse-grid closure (not in the paper) ----------------------- */

/* A 1D convolutional network that corrects moment fields computed on a coarse
 * grid: layers convolutions of kernel size ksize over `positions` cells, width
 * hidden channels, ReLU between layers, in_channels input features and
 * out_channels outputs per cell.  BF16 weights and activations with FP32
 * accumulation on the tensor cores; FP32 master weights trained by Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8).  Inputs are normalised as
 * (x - in_shift) / in_scale, outputs are out_scale times the network output.
 * This build supports ksize 5, width 64, in_channels and out_channels <= 8. */
typedef struct ql_closure ql_closure; /* opaque, library-owned */
typedef struct {
    int32_t in_channels;
    int32_t out_channels;
    int32_t width;
    int32_t layers;
    int32_t ksize;
    int32_t positions;
    int32_t max_batch;
    int32_t pad_;
    uint64_t seed; /* seeded He-uniform initial weights, zero biases */
    float in_shift[8], in_scale[8], out_scale[8];
} ql_closure_desc;

ql_status ql_closure_create(const ql_closure_desc *desc, const ql_opts *opts, ql_closure **out);

/* Device arrays: x [B][positions][in_channels] f32, y [B][positions][out_channels]
 * f32 (physical units), periodic [B] int32 (nonzero: periodic padding at the
 * ends, zero: the end values are replicated).  1 <= B <= max_batch.  Asynchronous on the stream. */
ql_status ql_closure_forward(ql_closure *c, const float *x, const int32_t *periodic, int64_t B, float *y);

/* Mean squared error between the network and the targets y / out_scale, and its
 * gradient for every parameter.  loss (host) and grad (host, count floats from
 * ql_closure_params) may be NULL; either one synchronises. */
ql_status ql_closure_gradients(ql_closure *c, const float *x, const float *y, const int32_t *periodic,
                               int64_t B, float *loss, float *grad);

/* One Adam step on the mean squared error of the batch, learning rate lr. */
ql_status ql_closure_train_step(ql_closure *c, const float *x, const float *y, const int32_t *periodic,
                                int64_t B, float lr, float *loss);

/* nsteps Adam steps on mini-batches drawn on the device (the training loop of
 * the learned closure without a host round trip per step).  x [n][positions]
 * [in_channels], y [n][positions][out_channels] and periodic [n] hold the whole
 * training set on the device; perm (device, nsteps * B int32) lists the samples
 * of step s at perm[s B .. s B + B - 1]; lr (host, nsteps floats) the learning
 * rate of each step; losses (device, nsteps floats, may be NULL) receives the
 * mean squared error of each step's batch before its update.  The same
 * arithmetic as nsteps calls of ql_closure_train_step on the gathered batches.
 * Synchronises once at the end; an index of perm outside [0, n) returns
 * QL_EINVAL (sample 0 is used in its place, nothing is read out of bounds). */
ql_status ql_closure_train_steps(ql_closure *c, const float *x, const float *y, const int32_t *periodic,
                                 int64_t n, const int32_t *perm, int64_t nsteps, int64_t B, const float *lr,
                                 float *losses);

/* Parameter vector (f32, host): for each layer W[cout][ksize][cin] then
 * bias[cout], channels padded to 16 (padding stays zero).  get and set may be
 * NULL; count (may be NULL) receives the length.  Synchronises. */
ql_status ql_closure_params(ql_closure *c, float *get, const float *set, int64_t *count);

ql_status ql_closure_destroy(ql_closure *c);
const char *ql_closure_last_error(const ql_closure *c);

/* ---- Stepping without allocation ----------------------------------------- */

/* Largest scratch ql_step_noalloc uses, in bytes. */
#define QL_NOALLOC_MAX_BYTES (64u * 1024u * 1024u)

/* Advances a caller-owned state by nsteps steps, like ql_step, without
 * allocating any device memory.  The paper has no counterpart: this
 * entry point exists for callers that must not call cudaMalloc, for example
 * code that runs under a memory budget another framework has already reserved
 * (where an allocation can fail) or inside a latency-critical loop (where
 * cudaMalloc can synchronise the whole device).
 *   psi         device, caller-owned: the state in the layout ql_state_device
 *               reports (Q rows of row_stride (phi, theta) pairs; psi points at
 *               cell 0 of row 0 and cell i of row k is pair k * row_stride + i),
 *               for -4 <= i < nx + 4: the 4 ghost columns on each side hold the
 *               periodic images or the fixed boundary states (kept).  psi - 4
 *               pairs must be 16-byte aligned.  Advanced in place.
 *   row_stride  pairs per row, at least (nx + 264 + 31) / 32 * 32 (the stride
 *               ql_state_device reports for a context of the same nx); rows
 *               start 16-byte aligned, so in FP32 it must be even.
 *   The other arguments are those of ql_create; from opts only precision,
 *   sums, pr_mode, enskog, device, pr_const, rho_ref, stream and chi_mode are
 *   used, and chi_mode must be QL_CHI_SET (QL_EUNSUPPORTED otherwise: chi_RET-FM
 *   needs per-cell density buffers).
 * The two intermediate stage buffers and the error word live in one fixed
 * scratch array of QL_NOALLOC_MAX_BYTES that every GPU loading this library
 * holds until the process exits; a state whose two stage buffers (2 Q
 * row_stride pairs) do not fit is rejected with QL_EINVAL before any device
 * work.  Every call shares that array and finds the previous call's contents
 * there (the error word is cleared on entry), so calls that overlap on the GPU
 * (other threads, other streams) race and must be serialised by the caller.
 * The first call on a device also uploads the kernel tables and looks up the
 * scratch address on that device; make that first call before any stream
 * capture.  Every call synchronises the stream: it returns after the stream
 * has run the steps and the error word has been read back.  Errors:
 * QL_EINVAL, QL_EUNSUPPORTED, QL_ECUDA, QL_ENONPHYSICAL; ql_last_error(NULL)
 * describes them. */
ql_status ql_step_noalloc(const ql_velset *vs, const ql_grid *grid, double denseness, double kn,
                          const ql_bc *bc, const ql_opts *opts, void *psi, int64_t row_stride,
                          int64_t nsteps);

/* ---- Host-only helpers (no GPU needed), FP64 ---------------------------- */

/* Velocity set of Sec. II.D: p (ascending) and w (summing to 1), each a host
 * array of Q doubles; 1 <= Q <= 200.  QL_EINVAL if Q is out of range. */
ql_status ql_velocity_set(int32_t Q, double *p, double *w);

/* Reduced density eta0 with E_l = 6 sqrt(2) eta0 chi_SET(eta0) (Sec. II.B,
 * Eq. chi), for 0 <= E_l <= E_l(0.49).  QL_EINVAL outside that range. */
ql_status ql_eta_of_denseness(double denseness, double *eta0);

/* Squared adiabatic sound speed of the dense gas, Eq. (sw_cs) with the
 * equation of state P = rho T (1 + b rho chi) and c_V = 3/2, at density rho
 * and temperature T, for eta = eta0 rho / rho_ref. */
double ql_sound_speed2(double eta0, double rho_ref, double rho, double T);

/* Linear modes of a sound wave of wave number k on the uniform state
 * (rho, T) of a model with these parameters (Sec. IV.A, Eqs. sw_cs and
 * sw_coeff), from the transport coefficients the kinetic model carries:
 * mu = tau P_i (Sec. II.B), lambda = (5/2) mu / Pr, the bulk viscosity of Eq.
 * (bulk_viscosity) as a fraction of Eq. (viscosity), c_V = 3/2 and the
 * equation of state P = rho T (1 + b rho chi):
 *   alpha_t = lambda k^2 / (rho c_P),
 *   alpha_a = k^2 / (2 rho) [4 mu / 3 + mu_v + (gamma - 1) lambda / c_P].
 * out (host, 5 doubles) = {c_s, alpha_a, alpha_a with mu_v = 0, alpha_t,
 * gamma}.  A density perturbation started with no pressure perturbation
 * evolves as rho~(t) = rho~(0) [(1 - 1/gamma) exp(-alpha_t t) + (1/gamma)
 * exp(-alpha_a t) cos(k c_s t)] (Eq. sw_solution).  QL_EINVAL on bad input. */
ql_status ql_sound_modes(double denseness, double kn, double length, double rho_ref, int32_t pr_mode,
                         double pr_const, double rho, double T, double k, double *out);

/* Standing normal shock of Mach number mach > 1 into (rho1, T1), Eq.
 * (rankine_hugoniot) with the dense equation of state: out (host, 4 doubles)
 * = {u1, rho2, u2, T2}.  QL_EINVAL if no compressive solution exists. */
ql_status ql_rankine_hugoniot(double eta0, double rho_ref, double rho1, double T1, double mach,
                              double *out);

/* Inviscid limit of the dense-gas shock tube, Sec. IV.B ("Inviscid limit"),
 * Eqs. (euler), (euler_xi), (sod_sol), (rankine_hugoniot): the exact solution
 * of the Euler equations with P = rho T (1 + 4 eta chi_SET(eta)), eta =
 * eta0 rho / rho_ref and internal energy e = (3/2) rho T, for a left state
 * (left[0] = rho, left[1] = T) and a right state (right[0], right[1]), both at
 * rest, with the left pressure above the right: a left-facing rarefaction, a
 * contact and a right-facing shock.  The energy relation across the shock is
 * taken with -e_R xi_s on its right-hand side, as energy conservation across
 * a shock moving into gas at rest requires (the printed relation has +e_R xi_s).
 * waves (host, 9 doubles; may be NULL) = {P_c, u_c, rho1, T1, rho2, T2,
 * xi_head, xi_tail, xi_shock}: star pressure and velocity, the states left (1)
 * and right (2) of the contact, the speeds of the fan's head and tail and of
 * the shock.  For i < n, rho[i], u[i], T[i] at the similarity variable xi[i] =
 * (x - x0) / t (host arrays; may be NULL when n = 0).  Runs on the host; no
 * device memory.  QL_EINVAL on invalid states or a left pressure not above the
 * right. */
ql_status ql_riemann_exact(double eta0, double rho_ref, const double *left, const double *right, double *waves,
                           int64_t n, const double *xi, double *rho, double *u, double *T);

/* Frees the context and its device buffers (waits for its stream). */
ql_status ql_destroy(ql_ctx *ctx);

/* Last error message of ctx, or of the last failed ql_create when ctx is
 * NULL.  The string lives until the next call on that context. */
const char *ql_last_error(const ql_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* QLBM_H */
