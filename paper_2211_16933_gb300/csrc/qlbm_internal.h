// Internal interface between the C ABI (qlbm_api.cu) and the per-precision
// kernel translation units (fdlb_f32.cu, fdlb_f64.cu).  Not installed.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "qlbm.h"

#ifdef __CUDACC__
#define QL_HD __host__ __device__
#else
#define QL_HD
#endif

namespace qlbm {

// Velocity-set sizes with compiled single-domain kernels (Q = 20 is the
// paper's set for sigma = 0.1, Q = 40 a near-ballistic one), and the subset
// the batched form compiles.
constexpr int kNumQ = 6;
constexpr int kQList[kNumQ] = {8, 16, 20, 24, 32, 40};
constexpr int kMaxQ = 40;
// Other even sizes up to kLargeMaxQ (the paper's near-ballistic runs use 200)
// run on the generic FP64 path of fdlb_lq.cuh.
constexpr int kLargeMaxQ = 200;
constexpr int kNumBatchQ = 4;
constexpr int kBatchQList[kNumBatchQ] = {8, 16, 24, 32};
constexpr int kBatchMaxQ = 32;

// CTA geometry of the stage kernel.  A CTA stages kSeg consecutive cells of
// every (component, velocity) row in shared memory: kTile cells it updates
// plus kHalo cells on each side (the WENO-5 and 6th-order stencils reach 3).
// Each warp updates 31 cells; its lane 0 computes the flux on the warp's
// left face.
constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;
constexpr int kTile = 31 * kWarps;
constexpr int kHalo = 4;
constexpr int kSeg = kTile + 2 * kHalo;
static_assert(kSeg == kThreads, "one staged cell per thread in the moment phase");

// Row layout of a state buffer: Q rows, one per velocity k, each of `stride`
// pairs (phi_k, theta_k) of the working precision; cell i (-kHalo <= i <
// nx + kHalo) of row k sits at pair k * stride + kHalo + i.  stride covers
// every staged segment of the last tile and is a multiple of 32 pairs.
inline int64_t num_tiles(int64_t nx) { return (nx + kTile - 1) / kTile; }
// Any tile of at most 248 cells staged from any start i0 < nx stays inside the
// row: (i0 + tile + 2 kHalo) - (-kHalo) <= nx + 256 + kHalo.
inline int64_t row_stride(int64_t nx) { return (nx + 256 + 2 * kHalo + 31) / 32 * 32; }

// Per-Q constant tables, built on the host in FP64 and stored per precision.
//   p[k], p2[k] = p^2, p3[k] = p^3: velocities, ascending
//   G[k][l] = w_k He_l(p_k) / sqrt(l!)    (normalised Hermite basis)
//   ca[l] = 1/sqrt(l), cb[l] = sqrt((l-1)/l)  (l >= 2), for the recurrence of
//   the normalised equilibrium coefficients c^_l = c_l sqrt(l!):
//   c^_0 = 1, c^_1 = u, c^_l = ca[l] u c^_{l-1} + cb[l] (T-1) c^_{l-2}.
// The stage kernels' constant-bank copy rescales G[k][l] by 1/sqrt(l!) and
// holds l - 1 in cb[l] (upload_tables_f32/f64).
QL_HD constexpr int tab_size(int Q) { return Q * Q + 5 * Q; }
QL_HD constexpr int tab_offset(int Q)
{
    // tables of the sizes in kQList, in ascending order
    return (Q > 8 ? tab_size(8) : 0) + (Q > 16 ? tab_size(16) : 0) + (Q > 20 ? tab_size(20) : 0) +
           (Q > 24 ? tab_size(24) : 0) + (Q > 32 ? tab_size(32) : 0) + (Q > 40 ? tab_size(40) : 0);
}
constexpr int kTabTotal = tab_offset(1 << 30);
struct TabView {
    int p, p2, p3, G, ca, cb;
};
QL_HD constexpr TabView tab_view(int Q)
{
    return TabView{tab_offset(Q), tab_offset(Q) + Q, tab_offset(Q) + 2 * Q, tab_offset(Q) + 3 * Q,
                   tab_offset(Q) + 3 * Q + Q * Q, tab_offset(Q) + 4 * Q + Q * Q};
}

struct StageArgs {
    const void *in;    // stage input psi^(s-1)
    const void *base;  // psi^n (read by stages 2 and 3)
    void *out;         // stage output (or L[psi] for stage 0)
    int64_t nx;
    int64_t stride;
    double inv_dx, dt;
    double eta0, inv_rho_ref, tau_pref, pr_const;
    int pr_mode, enskog, periodic;
    int fault;      // 1: arm the staging barrier without issuing the copies (failure-detection tests)
    int sums64;     // FP32: 1 combines the per-cell conserved sums in FP64, 0 in double-FP32
    int vsplit;     // FP64: CTAs per tile, each updating a contiguous range of the velocity pairs (>= 1)
    unsigned *err;  // device error word; bit 0: non-physical cell, bit 1: a TMA staging wait gave up,
                    // bit 2: a persistent run gave up waiting for a neighbouring tile
    // chi_RET-FM only (else null): nbar of every column of the stage input
    // (nx + 2 kHalo values of the working precision), and the density of
    // every interior cell of the stage output, written by the kernel.
    const void *nbar;
    void *nout;
};

// A run of steps in one launch (FP32, chi_SET, tiled velocity sets): CTA b
// takes tile b mod ntiles of stage b / ntiles of the run (stage g is
// Runge-Kutta stage g mod 3 + 1 of step g / 3).  st[p][s] are the arguments of
// stage s + 1 of the steps whose psi^n sits in the buffer of parity p (0: the
// run's first step).  done[i] counts the stages tile i has completed, modulo
// 2^32, over all runs of the solver; each is g0 at launch.
struct RunArgs {
    StageArgs st[2][3];
    int64_t ntiles;
    unsigned *done;
    unsigned g0;
};

// chi_RET-FM: nbar of every column (cells -kHalo .. nx+kHalo-1) from the
// interior densities n, as the weighted sum over offsets -W .. W (weights K,
// FP64); beyond the interior the density continues periodically or, fixed bc,
// as ghost[0..2] (cells -3..-1) and ghost[3..5] (cells nx..nx+2), cells
// further out taking the value of cell -3 / nx + 2.
struct FmArgs {
    const void *n;
    void *nbar;
    const double *K;
    int64_t nx;
    int W, periodic;
    double ghost[6];
};

// Batched form: instances packed in three arenas (psi^n, psi^(1), psi^(2)),
// instance rows starting at pair offset `off` in each.
struct BatchInstance {
    int64_t nx, stride, off;
    double inv_dx, dt, eta0, inv_rho_ref, tau_pref, pr_const;
    int32_t Q, pr_mode, enskog, periodic;
    // chi_RET-FM (ret != 0): the instance's densities and nbar sit at column
    // offset noff of the batch's density and nbar arrays (stride values each),
    // its ball weights K_-W .. K_W at koff of the weight array (W = fm_w), and
    // ghost_n holds the fixed-bc ghost densities as FmArgs::ghost
    int64_t noff, koff;
    int32_t ret, fm_w;
    double ghost_n[6];
};
struct BatchArgs {
    const BatchInstance *inst;
    const int2 *work;  // (instance, tile) items
    int64_t nwork;
    void *arena[3];
    unsigned *err;  // one error word per instance
    int sums64;     // FP32: per-cell conserved sums in FP64 (else double-FP32)
    // chi_RET-FM work lists: densities of the stage's output, and nbar
    void *n, *nbar;
};
// Threads (columns) per block of the ball-average kernels.
constexpr int kFmThreads = 256;
// Ball averages of the chi_RET-FM instances of a batch: one CTA per work item
// (instance, block of kFmThreads columns), as fdlb_fm_kernel per instance.
struct BatchFmArgs {
    const BatchInstance *inst;
    const int2 *work;
    int64_t nwork;
    const void *n;
    void *nbar;
    const double *K;
};
// Tile shapes the batched kernels are compiled for (warps per CTA).
constexpr int kBatchWarps[2] = {8, 4};

// Uploads all tables (kTabTotal doubles, laid out by tab_view) to the
// current device, rounded to the precision of the translation unit.
cudaError_t upload_tables_f32(const double *all);
cudaError_t upload_tables_f64(const double *all);

// The tables of every compiled velocity set (qlbm_api.cu): built on the host
// once per process and uploaded once per device, under one lock, with that
// device current.  Every entry point that launches tiled kernels calls it.
// On failure returns false with a message in err.  host_tables() (kTabTotal
// doubles) is valid after a successful call.
bool ensure_device_tables(int device, std::string &err);
const double *host_tables();

// stage: 0 writes L[psi] into out, 1..3 are the stages of Eq. (rk3).
cudaError_t launch_stage_f32(int Q, int stage, const StageArgs &a, cudaStream_t s);
cudaError_t launch_stage_f64(int Q, int stage, const StageArgs &a, cudaStream_t s);
// A run of `steps` steps as one launch (RunArgs) of at most kRunMaxTickets
// CTAs; false from run_supported_f32 for velocity sets without it.
constexpr int64_t kRunMaxTickets = (int64_t(1) << 31) - 1;
cudaError_t launch_run_f32(int Q, const RunArgs &r, int64_t steps, cudaStream_t s);
bool run_supported_f32(int Q);
// CTAs of the run kernel the current device holds at once (0 if the query fails).
int64_t run_resident_f32(int Q);

// psi = discrete equilibrium of (rho, u, T) given for cells -kHalo .. nx+kHalo-1
// (device arrays of nx + 2 kHalo doubles); interior and ghost columns.
// tab64: the FP64 tables (kTabTotal doubles, device memory).
cudaError_t launch_init_f32(int Q, const double *rho, const double *u, const double *T, void *psi,
                            int64_t nx, int64_t stride, const double *tab64, cudaStream_t s);
cudaError_t launch_init_f64(int Q, const double *rho, const double *u, const double *T, void *psi,
                            int64_t nx, int64_t stride, const double *tab64, cudaStream_t s);

// Copies the kHalo cells next to each end into the ghost columns of the
// other end (periodic images), all Q rows.
cudaError_t launch_periodic_ghosts_f32(int Q, void *psi, int64_t nx, int64_t stride, cudaStream_t s);
// Density sum_k phi_k of every interior cell of a state (chi_RET-FM).
cudaError_t launch_density_f32(int Q, const void *psi, int64_t nx, int64_t stride, void *n, cudaStream_t s);
cudaError_t launch_density_f64(int Q, const void *psi, int64_t nx, int64_t stride, void *n, cudaStream_t s);
cudaError_t launch_fm_f32(const FmArgs &a, cudaStream_t s);
cudaError_t launch_fm_f64(const FmArgs &a, cudaStream_t s);
cudaError_t launch_periodic_ghosts_f64(int Q, void *psi, int64_t nx, int64_t stride, cudaStream_t s);

// Output fields in FP64 per interior cell and per-block partial totals.
struct MomentArgs {
    const void *psi;
    int64_t nx, stride;
    double eta0, inv_rho_ref, dx;
    double *rho, *u, *T, *P, *q, *Pxx;  // each nx doubles (device), any may be null
    double *partial;                    // [nblocks][3] (device)
    unsigned *err;
    int sums64;  // FP32 state: per-cell sums in FP64 (else double-FP32)
};
constexpr int kMomThreads = 256;
inline int64_t moment_blocks(int64_t nx) { return (nx + kMomThreads - 1) / kMomThreads; }
// Generic-Q FP64 path (velocity sets without compiled kernels).  Per stage:
// cell moments of every column, per-cell collision coefficients, then one
// thread per (cell, velocity) for fluxes, equilibrium and update.  tab holds
// tab_view(Q) with offset 0; mom 6 x (nx + 2 kHalo) doubles (n, u, T, q, ln n,
// ln T); coef 9 x nx doubles.
struct LqArgs {
    const void *in;
    const void *base;
    void *out;
    int64_t nx, stride;
    int Q, periodic, pr_mode, enskog;
    double inv_dx, dt, eta0, inv_rho_ref, tau_pref, pr_const;
    const double *tab;
    double *mom, *coef;
    unsigned *err;
};
cudaError_t launch_lq_stage(int stage, const LqArgs &a, cudaStream_t s);
cudaError_t launch_lq_init(int Q, const double *rho, const double *u, const double *T, void *psi, int64_t nx,
                           int64_t stride, const double *tab, cudaStream_t s);
cudaError_t launch_lq_moments(int Q, const MomentArgs &a, const double *tab, cudaStream_t s);

// One batched stage over the work list: `grid` persistent CTAs of `warps`
// warps (8 or 4; the work list must be built for the same tile width).
// One launch over the work items of the instances with velocity-set size Q.
cudaError_t launch_batch_stage_f32(int Q, int stage, int warps, int grid, const BatchArgs &b, cudaStream_t s);
cudaError_t launch_batch_stage_f64(int Q, int stage, int warps, int grid, const BatchArgs &b, cudaStream_t s);
// The chi_RET-FM form (8-warp tiles; b.n and b.nbar set), then the batched
// ball average of its output densities (max_w: the largest W of the list).
cudaError_t launch_batch_stage_ret_f32(int Q, int stage, int grid, const BatchArgs &b, cudaStream_t s);
cudaError_t launch_batch_stage_ret_f64(int Q, int stage, int grid, const BatchArgs &b, cudaStream_t s);
cudaError_t launch_batch_fm_f32(const BatchFmArgs &a, int max_w, cudaStream_t s);
cudaError_t launch_batch_fm_f64(const BatchFmArgs &a, int max_w, cudaStream_t s);
// Resident CTAs per SM of the batched kernel (occupancy calculator).
int batch_ctas_per_sm_f32(int stage, int warps);
int batch_ctas_per_sm_f64(int stage, int warps);

cudaError_t launch_moments_f32(int Q, const MomentArgs &a, const double *tab64, cudaStream_t s);
cudaError_t launch_moments_f64(int Q, const MomentArgs &a, const double *tab64, cudaStream_t s);
// totals[3] = fixed-order sum of partial[nblocks][3]
cudaError_t launch_reduce_totals(const double *partial, int64_t nblocks, double *totals, cudaStream_t s);

}  // namespace qlbm
