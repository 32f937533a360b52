// C ABI of the solver (include/qlbm.h): context, buffers, launches, copies.
#include <cuda_runtime.h>
#include <errno.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#include <algorithm>
#include <mutex>
#include <memory>
#include <string>
#include <vector>

#include "../../include/qlbm.h"
#include "../../include/qlbm_io.h"
#include "qlbm_host.h"
#include "qlbm_internal.h"
#include "qlbm_lq.h"

using namespace qlbm;

struct ql_ctx {
    int Q = 0, precision = 0, pr_mode = 0, enskog = 1, periodic = 1, device = 0, fault = 0;
    int sums64 = 0;  // FP32: per-cell conserved sums in FP64 (QL_SUMS_FP64) instead of double-FP32
    int64_t nx = 0, stride = 0;
    double L = 0, dx = 0, dt = 0, El = 0, kn = 0, pr_const = 2.0 / 3.0, rho_ref = 1.0;
    double eta0 = 0, chi0 = 1, sigma = 0, tau_pref = 0;
    std::vector<double> p, w;  // velocity set (Q)
    // velocity sets without compiled tiled kernels run on the generic FP64 path
    bool lq = false;
    double *d_lqtab = nullptr, *d_lqmom = nullptr, *d_lqcoef = nullptr;
    cudaStream_t stream = nullptr;
    ql_alloc_fn alloc = nullptr;
    ql_free_fn free_fn = nullptr;
    void *alloc_user = nullptr;
    size_t elem = 8;
    // psi^n is buf[cur] (cur 0 or 1); a step's stages write psi^(1) into
    // buf[1 - cur], psi^(2) into buf[2] and, on the tiled path, psi^(n+1) into
    // buf[1 - cur] again (an in-place last stage, which reads and rewrites the
    // same lines, ran about 3 % slower), after which cur flips
    void *buf[3] = {nullptr, nullptr, nullptr};
    int cur = 0;
    double *d_fields = nullptr;   // 6 * nx output fields
    double *d_init = nullptr;     // 3 * (nx + 2 kHalo) initial fields
    double *d_partial = nullptr;  // moment_blocks(nx) * 3
    double *d_totals = nullptr;   // 3
    double *d_tab64 = nullptr;    // kTabTotal
    unsigned *d_err = nullptr;
    std::vector<double> ghost_state;  // (rho, u, T) of the 2 kHalo ghost columns, fixed bc
    // chi_RET-FM (Eq. chi_ret): ball half-width in cells, weights, interior
    // densities of the latest stage output, and nbar of every column
    int chi_mode = QL_CHI_SET, fm_w = 0;
    double *d_fmk = nullptr;  // 2 fm_w + 1
    void *d_n = nullptr;      // nx values of the working precision
    void *d_nbar = nullptr;   // stride values (columns -kHalo .. ; the tail past nx + kHalo unused)
    // ql_step of more than one step replays a recorded step, one recording per
    // value of cur (its launches read only buffers fixed for the context's lifetime)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t step_graph[2] = {nullptr, nullptr};
    bool step_graph_failed = false;
    int64_t steps = 0;  // steps advanced (restart files carry it)
    // FP32 chi_SET on the tiled path: ql_step may launch whole runs of steps
    // (ql_opts.launch) with per-tile counts of completed stages in d_done,
    // run_stages stages counted modulo 2^32 so far
    int launch = QL_LAUNCH_AUTO;
    unsigned *d_done = nullptr;
    unsigned run_stages = 0;
    std::string err;
};

static std::string g_create_error;
static std::mutex g_mutex;
static bool g_tables_ready[64] = {};
static double g_tab[kTabTotal];
static bool g_tab_built = false;

namespace qlbm {
void set_global_error(const std::string &msg) { g_create_error = msg; }

// The kernel tables of every compiled velocity set: built on the host once per
// process, uploaded once per device (the current one must be `device`).  All
// entry points that launch tiled kernels share this one flag per device.
static bool host_tables_locked(std::string &err)
{
    if (!g_tab_built) {
        if (!build_tables(g_tab)) {
            err = "velocity-set construction failed";
            return false;
        }
        g_tab_built = true;
    }
    return true;
}

bool ensure_device_tables(int device, std::string &err)
{
    std::lock_guard<std::mutex> lk(g_mutex);
    if (!host_tables_locked(err)) return false;
    if (!g_tables_ready[device & 63]) {
        cudaError_t e = upload_tables_f32(g_tab);
        if (e == cudaSuccess) e = upload_tables_f64(g_tab);
        if (e != cudaSuccess) {
            err = std::string("table upload: ") + cudaGetErrorString(e);
            return false;
        }
        g_tables_ready[device & 63] = true;
    }
    return true;
}

const double *host_tables() { return g_tab; }
}  // namespace qlbm

static ql_status fail(ql_ctx *c, ql_status st, const std::string &msg)
{
    if (c) c->err = msg; else g_create_error = msg;
    return st;
}

static ql_status cuda_fail(ql_ctx *c, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? QL_ENOMEM : QL_ECUDA, m);
}

#define QL_CUDA(ctx, call)                                  \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

static void *dev_alloc(ql_ctx *c, size_t bytes)
{
    if (c->alloc) return c->alloc(bytes, c->alloc_user);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    return p;
}

static void dev_free(ql_ctx *c, void *p)
{
    if (!p) return;
    if (c->free_fn) c->free_fn(p, c->alloc_user);
    else cudaFree(p);
}

static FmArgs fm_args(ql_ctx *c);

// The buffer holding the current state psi^n, and the one the next step's
// first and last stages write.
static void *state_buf(ql_ctx *c) { return c->buf[c->cur]; }
static void *other_buf(ql_ctx *c) { return c->buf[1 - c->cur]; }
// Whether a step ends in the other buffer (the tiled path; the generic large-Q
// path keeps psi^n in place).
static bool rotates(const ql_ctx *c) { return !c->lq; }

// Arguments of one stage on the tiled path (chi_SET; stage() adds the chi_RET-FM buffers).
static StageArgs stage_args(const ql_ctx *c, const void *in, const void *base, void *out)
{
    StageArgs a;
    a.in = in;
    a.base = base;
    a.out = out;
    a.nx = c->nx;
    a.stride = c->stride;
    a.inv_dx = 1.0 / c->dx;
    a.dt = c->dt;
    a.eta0 = c->eta0;
    a.inv_rho_ref = 1.0 / c->rho_ref;
    a.tau_pref = c->tau_pref;
    a.pr_const = c->pr_const;
    a.pr_mode = c->pr_mode;
    a.enskog = c->enskog;
    a.periodic = c->periodic;
    a.fault = c->fault;
    a.sums64 = c->sums64;
    a.vsplit = 1;
    a.err = c->d_err;
    a.nbar = nullptr;
    a.nout = nullptr;
    return a;
}

static cudaError_t stage(ql_ctx *c, int s, const void *in, const void *base, void *out)
{
    if (c->lq) {
        LqArgs l;
        l.in = in;
        l.base = base;
        l.out = out;
        l.nx = c->nx;
        l.stride = c->stride;
        l.Q = c->Q;
        l.periodic = c->periodic;
        l.pr_mode = c->pr_mode;
        l.enskog = c->enskog;
        l.inv_dx = 1.0 / c->dx;
        l.dt = c->dt;
        l.eta0 = c->eta0;
        l.inv_rho_ref = 1.0 / c->rho_ref;
        l.tau_pref = c->tau_pref;
        l.pr_const = c->pr_const;
        l.tab = c->d_lqtab;
        l.mom = c->d_lqmom;
        l.coef = c->d_lqcoef;
        l.err = c->d_err;
        if (c->chi_mode == QL_CHI_RET_FM) {
            // each stage averages the densities of its own input (its moments kernel writes them)
            FmArgs f = fm_args(c);
            f.n = c->d_lqmom + kHalo;
            return launch_lq_stage_ret(s, l, f, c->stream);
        }
        return launch_lq_stage(s, l, c->stream);
    }
    StageArgs a = stage_args(c, in, base, out);  // the launcher picks the FP64 split
    const bool ret = c->chi_mode == QL_CHI_RET_FM;
    a.nbar = ret ? c->d_nbar : nullptr;
    a.nout = ret && s != 0 ? c->d_n : nullptr;
    return c->precision == QL_FP32 ? launch_stage_f32(c->Q, s, a, c->stream)
                                   : launch_stage_f64(c->Q, s, a, c->stream);
}

// chi_RET-FM: ball-average arguments, densities from d_n.
static FmArgs fm_args(ql_ctx *c)
{
    FmArgs f;
    f.n = c->d_n;
    f.nbar = c->d_nbar;
    f.K = c->d_fmk;
    f.nx = c->nx;
    f.W = c->fm_w;
    f.periodic = c->periodic;
    for (int g = 0; g < 6; ++g) f.ghost[g] = 0.0;
    if (!c->periodic && !c->ghost_state.empty())
        for (int g = 0; g < 3; ++g) {
            f.ghost[g] = c->ghost_state[3 * (g + 1)];      // cells -3..-1: columns 1..3
            f.ghost[3 + g] = c->ghost_state[3 * (kHalo + g)];  // cells nx..nx+2
        }
    return f;
}

// chi_RET-FM: nbar of every column from the densities in d_n.
static cudaError_t fm_average(ql_ctx *c)
{
    const FmArgs f = fm_args(c);
    return c->precision == QL_FP32 ? launch_fm_f32(f, c->stream) : launch_fm_f64(f, c->stream);
}

// chi_RET-FM: densities of the current state psi^n, then nbar (the generic
// large-Q path forms nbar inside each stage instead).
static cudaError_t refresh_nbar(ql_ctx *c)
{
    if (c->chi_mode != QL_CHI_RET_FM || c->lq) return cudaSuccess;
    cudaError_t e = c->precision == QL_FP32 ? launch_density_f32(c->Q, state_buf(c), c->nx, c->stride, c->d_n, c->stream)
                                            : launch_density_f64(c->Q, state_buf(c), c->nx, c->stride, c->d_n, c->stream);
    return e == cudaSuccess ? fm_average(c) : e;
}

static ql_status check_err_word(ql_ctx *c)
{
    unsigned h = 0;
    QL_CUDA(c, cudaMemcpyAsync(&h, c->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    QL_CUDA(c, cudaStreamSynchronize(c->stream));
    if (h & 2u) return fail(c, QL_ECUDA, "a stage kernel gave up waiting for its tile's TMA copies");
    if (h & 4u) return fail(c, QL_ECUDA, "a run gave up waiting for a neighbouring tile's previous stage");
    if (h & 1u) return fail(c, QL_ENONPHYSICAL, "non-physical state: n <= 0, T <= 0 or non-finite moments");
    return QL_OK;
}

static ql_status upload_fields_and_init(ql_ctx *c, const double *rho, const double *u, const double *T)
{
    const int64_t ncol = c->nx + 2 * kHalo;
    std::vector<double> h(3 * ncol);
    memcpy(h.data(), rho, sizeof(double) * ncol);
    memcpy(h.data() + ncol, u, sizeof(double) * ncol);
    memcpy(h.data() + 2 * ncol, T, sizeof(double) * ncol);
    QL_CUDA(c, cudaMemcpyAsync(c->d_init, h.data(), sizeof(double) * 3 * ncol, cudaMemcpyHostToDevice, c->stream));
    cudaError_t e = c->lq ? launch_lq_init(c->Q, c->d_init, c->d_init + ncol, c->d_init + 2 * ncol, state_buf(c), c->nx,
                                           c->stride, c->d_lqtab, c->stream)
                    : c->precision == QL_FP32
                        ? launch_init_f32(c->Q, c->d_init, c->d_init + ncol, c->d_init + 2 * ncol, state_buf(c), c->nx,
                                          c->stride, c->d_tab64, c->stream)
                        : launch_init_f64(c->Q, c->d_init, c->d_init + ncol, c->d_init + 2 * ncol, state_buf(c), c->nx,
                                          c->stride, c->d_tab64, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
    QL_CUDA(c, cudaStreamSynchronize(c->stream));  // h goes out of scope
    return QL_OK;
}

static void destroy_buffers(ql_ctx *c)
{
    for (auto &g : c->step_graph)
        if (g) cudaGraphExecDestroy(g);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    c->step_graph[0] = c->step_graph[1] = nullptr;
    c->cap_stream = nullptr;
    for (int b = 0; b < 3; ++b) dev_free(c, c->buf[b]);
    dev_free(c, c->d_fields);
    dev_free(c, c->d_init);
    dev_free(c, c->d_partial);
    dev_free(c, c->d_totals);
    dev_free(c, c->d_tab64);
    dev_free(c, c->d_err);
    dev_free(c, c->d_done);
    dev_free(c, c->d_fmk);
    dev_free(c, c->d_n);
    dev_free(c, c->d_nbar);
    dev_free(c, c->d_lqtab);
    dev_free(c, c->d_lqmom);
    dev_free(c, c->d_lqcoef);
}

extern "C" {

ql_status ql_create(const ql_velset *vs, const ql_grid *grid, double denseness, double kn, const ql_bc *bc,
                    const ql_init *init, const ql_opts *opts, ql_ctx **out)
{
    if (out) *out = nullptr;
    if (!vs || !grid || !bc || !init || !opts || !out) return fail(nullptr, QL_EINVAL, "null argument");
    bool qok = false;
    for (int j = 0; j < kNumQ; ++j) qok |= vs->Q == kQList[j];
    if (vs->kind != 0) return fail(nullptr, QL_EINVAL, "velocity set kind must be 0 (Gauss-Hermite)");
    const bool lq = !qok && vs->Q >= 2 && vs->Q <= kLargeMaxQ && vs->Q % 2 == 0;
    if (!qok && !lq) return fail(nullptr, QL_EUNSUPPORTED, "Q must be even and at most 200");
    if (lq && opts->precision != QL_FP64)
        return fail(nullptr, QL_EUNSUPPORTED, "velocity sets other than 8, 16, 20, 24, 32, 40 run in FP64 only");
    if (grid->nx < 8 || grid->nx > (int64_t(1) << 31)) return fail(nullptr, QL_EINVAL, "nx must be in [8, 2^31]");
    if (!(grid->length > 0) || !(grid->dt > 0)) return fail(nullptr, QL_EINVAL, "length and dt must be > 0");
    if (!(denseness > 0) || !(kn > 0)) return fail(nullptr, QL_EINVAL, "denseness and kn must be > 0");
    if (bc->kind != QL_BC_PERIODIC && bc->kind != QL_BC_FIXED) return fail(nullptr, QL_EINVAL, "bad bc kind");
    if (opts->precision != QL_FP32 && opts->precision != QL_FP64) return fail(nullptr, QL_EINVAL, "bad precision");
    if (!(opts->rho_ref > 0)) return fail(nullptr, QL_EINVAL, "rho_ref must be > 0");
    if (opts->pr_mode == QL_PR_CONST && !(opts->pr_const > 0)) return fail(nullptr, QL_EINVAL, "pr_const must be > 0");
    if (opts->chi_mode != QL_CHI_SET && opts->chi_mode != QL_CHI_RET_FM) return fail(nullptr, QL_EINVAL, "bad chi_mode");
    if (opts->fault != 0 && opts->fault != 1) return fail(nullptr, QL_EINVAL, "bad fault (0 or 1)");
    if (opts->sums != QL_SUMS_DFP32 && opts->sums != QL_SUMS_FP64) return fail(nullptr, QL_EINVAL, "bad sums");
    if (opts->launch != QL_LAUNCH_AUTO && opts->launch != QL_LAUNCH_STAGES && opts->launch != QL_LAUNCH_RUN)
        return fail(nullptr, QL_EINVAL, "bad launch (QL_LAUNCH_AUTO, QL_LAUNCH_STAGES or QL_LAUNCH_RUN)");

    ql_ctx *c = new ql_ctx();
    c->chi_mode = opts->chi_mode;
    c->fault = opts->fault;
    c->launch = opts->launch;
    c->sums64 = opts->precision == QL_FP32 && opts->sums == QL_SUMS_FP64;
    c->lq = lq;
    c->Q = vs->Q;
    c->precision = opts->precision;
    c->pr_mode = opts->pr_mode;
    c->enskog = opts->enskog ? 1 : 0;
    c->periodic = bc->kind == QL_BC_PERIODIC;
    c->device = opts->device;
    c->nx = grid->nx;
    c->L = grid->length;
    c->dx = grid->length / double(grid->nx);
    c->dt = grid->dt;
    c->El = denseness;
    c->kn = kn;
    c->pr_const = opts->pr_const;
    c->rho_ref = opts->rho_ref;
    c->stream = static_cast<cudaStream_t>(opts->stream);
    c->alloc = opts->alloc;
    c->free_fn = opts->free;
    c->alloc_user = opts->alloc_user;
    c->elem = c->precision == QL_FP32 ? 8 : 16;  // one (phi, theta) pair
    c->stride = row_stride(c->nx);

    auto bail = [&](ql_status st, const std::string &m) {
        destroy_buffers(c);
        delete c;
        return fail(nullptr, st, m);
    };

    if (!eta_of_denseness(denseness, &c->eta0)) return bail(QL_EINVAL, "denseness out of range (eta0 >= 0.49)");
    c->chi0 = chi_set(c->eta0);
    // sigma = E_l l0 with l0 = Kn L; tau = (5 sqrt(2 pi)/16) Kn L chi0 / (rho^ chi sqrt T) (1 + 0.8 Y + ...)
    c->sigma = denseness * kn * grid->length;
    if (c->chi_mode == QL_CHI_RET_FM) {
        c->fm_w = fm_halfwidth(c->dx, c->sigma);
        if (c->fm_w > QL_FM_MAX_HALFWIDTH)
            return bail(QL_EUNSUPPORTED, "the chi_RET-FM ball reaches " + std::to_string(c->fm_w) +
                                             " cells on each side; at most QL_FM_MAX_HALFWIDTH are supported");
    }
    c->tau_pref = tau_prefactor(kn, grid->length, c->eta0);
    {
        std::lock_guard<std::mutex> lk(g_mutex);
        std::string terr;
        if (!host_tables_locked(terr)) return bail(QL_EINVAL, terr);
    }
    c->p.assign(c->Q, 0.0);
    c->w.assign(c->Q, 0.0);
    std::vector<double> lqtab;
    if (c->lq) {
        lqtab.assign(size_t(c->Q) * c->Q + 5 * size_t(c->Q), 0.0);
        if (!build_table_q(c->Q, lqtab.data())) return bail(QL_EINVAL, "velocity-set construction failed");
        for (int k = 0; k < c->Q; ++k) {
            c->p[k] = lqtab[k];
            c->w[k] = lqtab[3 * size_t(c->Q) + size_t(k) * c->Q];  // w_k h_0 = w_k
        }
    } else {
        const TabView tv = tab_view(c->Q);
        for (int k = 0; k < c->Q; ++k) {
            c->p[k] = g_tab[tv.p + k];
            c->w[k] = g_tab[tv.G + k * c->Q];  // w_k h_0 = w_k
        }
    }

    // initial fields on the host, ghost columns included
    const int64_t ncol = c->nx + 2 * kHalo;
    std::vector<double> rho(ncol), u(ncol), T(ncol);
    if (!initial_fields(init->kind, init->prm, c->nx, c->L, c->periodic, c->eta0, c->rho_ref, init->rho, init->u,
                        init->T, init->ghost, kHalo, rho.data(), u.data(), T.data()))
        return bail(QL_EINVAL, "invalid initial state for this init kind / boundary");

    // device set-up
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return bail(QL_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    {
        std::string terr;
        if (!ensure_device_tables(c->device, terr)) return bail(QL_ECUDA, terr);
    }
    const size_t state_bytes = size_t(c->Q) * size_t(c->stride) * c->elem;
    for (int b = 0; b < 3; ++b) {
        c->buf[b] = dev_alloc(c, state_bytes);
        if (!c->buf[b]) return bail(QL_ENOMEM, "state buffer allocation failed");
    }
    c->d_fields = static_cast<double *>(dev_alloc(c, sizeof(double) * 6 * c->nx));
    c->d_init = static_cast<double *>(dev_alloc(c, sizeof(double) * 3 * ncol));
    c->d_partial = static_cast<double *>(dev_alloc(c, sizeof(double) * 3 * moment_blocks(c->nx)));
    c->d_totals = static_cast<double *>(dev_alloc(c, sizeof(double) * 4));
    c->d_tab64 = static_cast<double *>(dev_alloc(c, sizeof(double) * kTabTotal));
    c->d_err = static_cast<unsigned *>(dev_alloc(c, 256));
    if (!c->d_fields || !c->d_init || !c->d_partial || !c->d_totals || !c->d_tab64 || !c->d_err)
        return bail(QL_ENOMEM, "work buffer allocation failed");
    if (!c->lq && c->precision == QL_FP32 && run_supported_f32(c->Q)) {
        const size_t bytes = sizeof(unsigned) * size_t(num_tiles(c->nx));
        c->d_done = static_cast<unsigned *>(dev_alloc(c, bytes));
        if (!c->d_done) return bail(QL_ENOMEM, "run counter allocation failed");
        e = cudaMemsetAsync(c->d_done, 0, bytes, c->stream);
        if (e != cudaSuccess) return bail(QL_ECUDA, std::string("run counters: ") + cudaGetErrorString(e));
    }
    if (c->lq) {
        c->d_lqtab = static_cast<double *>(dev_alloc(c, sizeof(double) * lqtab.size()));
        c->d_lqmom = static_cast<double *>(dev_alloc(c, sizeof(double) * 6 * ncol));
        c->d_lqcoef = static_cast<double *>(dev_alloc(c, sizeof(double) * 9 * c->nx));
        if (!c->d_lqtab || !c->d_lqmom || !c->d_lqcoef) return bail(QL_ENOMEM, "large-Q buffer allocation failed");
        e = cudaMemcpyAsync(c->d_lqtab, lqtab.data(), sizeof(double) * lqtab.size(), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // lqtab goes out of scope
        if (e != cudaSuccess) return bail(QL_ECUDA, std::string("large-Q tables: ") + cudaGetErrorString(e));
    }
    if (c->chi_mode == QL_CHI_RET_FM) {
        const size_t real = c->precision == QL_FP32 ? 4 : 8;
        c->d_fmk = static_cast<double *>(dev_alloc(c, sizeof(double) * (2 * c->fm_w + 1)));
        c->d_n = dev_alloc(c, real * c->nx);
        c->d_nbar = dev_alloc(c, real * c->stride);
        if (!c->d_fmk || !c->d_n || !c->d_nbar) return bail(QL_ENOMEM, "chi_RET-FM buffer allocation failed");
        std::vector<double> K(2 * c->fm_w + 1);
        fm_weights(c->dx, c->sigma, c->fm_w, K.data());
        e = cudaMemcpyAsync(c->d_fmk, K.data(), sizeof(double) * K.size(), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->d_nbar, 0, real * c->stride, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // K goes out of scope
        if (e != cudaSuccess) return bail(QL_ECUDA, std::string("chi_RET-FM set-up: ") + cudaGetErrorString(e));
    }
    e = cudaMemcpyAsync(c->d_tab64, g_tab, sizeof(double) * kTabTotal, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, 256, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->buf[0], 0, state_bytes, c->stream);
    if (e != cudaSuccess) return bail(QL_ECUDA, std::string("set-up copy: ") + cudaGetErrorString(e));
    ql_status st = upload_fields_and_init(c, rho.data(), u.data(), T.data());
    if (st != QL_OK) {
        std::string m = c->err;
        return bail(st, m);
    }
    // the other buffers start as copies so their ghost columns hold the fixed
    // states (a step may leave psi^n in buf[1]; cur is 0 here)
    for (int b = 1; b < 3 && e == cudaSuccess; ++b)
        e = cudaMemcpyAsync(c->buf[b], c->buf[0], state_bytes, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return bail(QL_ECUDA, std::string("set-up: ") + cudaGetErrorString(e));
    if (!c->periodic) {
        c->ghost_state.assign(3 * 2 * kHalo, 0.0);
        for (int g = 0; g < 2 * kHalo; ++g) {
            const int64_t col = g < kHalo ? g : c->nx + g;
            c->ghost_state[3 * g] = rho[col];
            c->ghost_state[3 * g + 1] = u[col];
            c->ghost_state[3 * g + 2] = T[col];
        }
    }
    e = refresh_nbar(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return bail(QL_ECUDA, std::string("chi_RET-FM set-up: ") + cudaGetErrorString(e));
    *out = c;
    return QL_OK;
}

// One step of Eq. (rk3) on c->stream from psi^n in buf[cur]: three stages and,
// with chi_RET-FM on the tiled path, the ball average after each (each tiled
// stage also writes the densities of its output, from which nbar for the next
// stage is averaged).  The caller flips cur afterwards when the step rotates.
static cudaError_t enqueue_step(ql_ctx *c, int cur)
{
    const bool ret = c->chi_mode == QL_CHI_RET_FM && !c->lq;
    void *S = c->buf[cur], *T1 = c->buf[1 - cur], *T2 = c->buf[2];
    cudaError_t e = stage(c, 1, S, S, T1);
    if (e == cudaSuccess && ret) e = fm_average(c);
    if (e == cudaSuccess) e = stage(c, 2, T1, S, T2);
    if (e == cudaSuccess && ret) e = fm_average(c);
    if (e == cudaSuccess) e = stage(c, 3, T2, S, rotates(c) ? T1 : S);
    if (e == cudaSuccess && ret) e = fm_average(c);
    return e;
}

// Records the step from buf[cur] as a CUDA graph, on a stream of the context's
// own (the caller's may be the legacy default stream, which cannot be
// recorded).  A recording that fails leaves the steps to plain launches.
static void record_step_graph(ql_ctx *c, int cur)
{
    if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        c->cap_stream = nullptr;
        c->step_graph_failed = true;
        (void)cudaGetLastError();
        return;
    }
    cudaStream_t user = c->stream;
    c->stream = c->cap_stream;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        e = enqueue_step(c, cur);
        const cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
        if (e == cudaSuccess) e = e2;
    }
    c->stream = user;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->step_graph[cur], g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->step_graph[cur] = nullptr;
        c->step_graph_failed = true;
        (void)cudaGetLastError();
    }
}

// FP32 chi_SET solvers on the tiled path may run whole runs of steps as single
// launches (fdlb_run_kernel): always with QL_LAUNCH_RUN, and with
// QL_LAUNCH_AUTO for domains of 1 to kRunAutoWaves times as many tiles as the
// GPU holds CTAs.  Measured on the Sod tube, Q = 32, against per-stage
// launches: 0.70x the step time at 2^17 cells (1.2 waves of CTAs per stage),
// 0.92x at 2^19 (4.6 waves), 1.02x at 2^21 (18.5 waves), 1.04x at 2^22; 1.10x
// at 2^13 and 2^15 (fewer tiles than CTA slots).  Never with fault.
constexpr int64_t kRunAutoWaves = 8;
static bool runs_whole(const ql_ctx *c)
{
    if (!c->d_done || c->chi_mode != QL_CHI_SET || c->fault || c->launch == QL_LAUNCH_STAGES) return false;
    const int64_t n = num_tiles(c->nx);
    if (3 * n > kRunMaxTickets) return false;  // not even one step fits one launch
    if (c->launch == QL_LAUNCH_RUN) return true;
    const int64_t resident = run_resident_f32(c->Q);
    return resident > 0 && n >= resident && n <= kRunAutoWaves * resident;
}

// nsteps steps as launches of fdlb_run_kernel (each at most kRunMaxTickets
// (stage, tile) tickets), rotating the buffers as the step-by-step path does.
static int64_t run_steps_per_launch(const ql_ctx *c)
{
    return std::max<int64_t>(1, kRunMaxTickets / (3 * num_tiles(c->nx)));
}

static ql_status run_steps(ql_ctx *c, int64_t nsteps)
{
    const int64_t N = num_tiles(c->nx);
    const int64_t per_launch = run_steps_per_launch(c);
    while (nsteps > 0) {
        const int64_t k = std::min(nsteps, per_launch);
        RunArgs r;
        for (int p = 0; p < 2; ++p) {
            const int cur = c->cur ^ p;
            void *S = c->buf[cur], *T1 = c->buf[1 - cur], *T2 = c->buf[2];
            r.st[p][0] = stage_args(c, S, S, T1);
            r.st[p][1] = stage_args(c, T1, S, T2);
            r.st[p][2] = stage_args(c, T2, S, T1);
        }
        r.ntiles = N;
        r.done = c->d_done;
        r.g0 = c->run_stages;
        const cudaError_t e = launch_run_f32(c->Q, r, k, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "run kernel launch");
        c->run_stages += unsigned(3 * k);
        if (k & 1) c->cur = 1 - c->cur;
        c->steps += k;
        nsteps -= k;
    }
    return QL_OK;
}

ql_status ql_step(ql_ctx *c, int64_t nsteps)
{
    if (!c || nsteps < 0) return fail(c, QL_EINVAL, "bad arguments to ql_step");
    if (runs_whole(c)) return run_steps(c, nsteps);
    // several steps replay a recorded step: one graph launch per step instead
    // of three to six kernel launches, which matters where launches are slow
    const bool rot = rotates(c);
    if (nsteps > 1 && !c->step_graph_failed) {
        if (!c->step_graph[c->cur]) record_step_graph(c, c->cur);
        if (rot && !c->step_graph_failed && !c->step_graph[1 - c->cur]) record_step_graph(c, 1 - c->cur);
    }
    const bool replay = nsteps > 1 && !c->step_graph_failed;
    for (int64_t s = 0; s < nsteps; ++s) {
        const cudaError_t e = replay ? cudaGraphLaunch(c->step_graph[c->cur], c->stream) : enqueue_step(c, c->cur);
        if (e != cudaSuccess) return cuda_fail(c, e, "stage kernel launch");
        if (rot) c->cur = 1 - c->cur;
        c->steps += 1;
    }
    return QL_OK;
}

ql_status ql_sync(ql_ctx *c)
{
    if (!c) return fail(c, QL_EINVAL, "null context");
    return check_err_word(c);
}

static ql_status run_moments(ql_ctx *c, bool fields)
{
    MomentArgs a;
    a.psi = state_buf(c);
    a.nx = c->nx;
    a.stride = c->stride;
    a.eta0 = c->eta0;
    a.inv_rho_ref = 1.0 / c->rho_ref;
    a.dx = c->dx;
    double *f = c->d_fields;
    a.rho = fields ? f : nullptr;
    a.u = fields ? f + c->nx : nullptr;
    a.T = fields ? f + 2 * c->nx : nullptr;
    a.P = fields ? f + 3 * c->nx : nullptr;
    a.q = fields ? f + 4 * c->nx : nullptr;
    a.Pxx = fields ? f + 5 * c->nx : nullptr;
    a.partial = c->d_partial;
    a.err = c->d_err;
    a.sums64 = c->sums64;
    cudaError_t e = c->lq                      ? launch_lq_moments(c->Q, a, c->d_lqtab, c->stream)
                    : c->precision == QL_FP32 ? launch_moments_f32(c->Q, a, c->d_tab64, c->stream)
                                              : launch_moments_f64(c->Q, a, c->d_tab64, c->stream);
    if (e == cudaSuccess) e = launch_reduce_totals(c->d_partial, moment_blocks(c->nx), c->d_totals, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "moments kernel");
    return QL_OK;
}

ql_status ql_moments(ql_ctx *c, double *rho, double *u, double *T, double *P, double *q, double *Pxx,
                     double *totals)
{
    if (!c) return fail(c, QL_EINVAL, "null context");
    ql_status st = run_moments(c, true);
    if (st != QL_OK) return st;
    double *outs[6] = {rho, u, T, P, q, Pxx};
    for (int j = 0; j < 6; ++j)
        if (outs[j])
            QL_CUDA(c, cudaMemcpyAsync(outs[j], c->d_fields + j * c->nx, sizeof(double) * c->nx,
                                       cudaMemcpyDeviceToHost, c->stream));
    if (totals)
        QL_CUDA(c, cudaMemcpyAsync(totals, c->d_totals, sizeof(double) * 3, cudaMemcpyDeviceToHost, c->stream));
    return check_err_word(c);
}

ql_status ql_totals(ql_ctx *c, double *totals)
{
    if (!c || !totals) return fail(c, QL_EINVAL, "bad arguments to ql_totals");
    ql_status st = run_moments(c, false);
    if (st != QL_OK) return st;
    QL_CUDA(c, cudaMemcpyAsync(totals, c->d_totals, sizeof(double) * 3, cudaMemcpyDeviceToHost, c->stream));
    return check_err_word(c);
}

// rows [Q][nx] of (phi, theta) pairs of buffer b <-> cell-major host arrays of doubles
static ql_status download_rows(ql_ctx *c, const void *dev, double *phi, double *theta)
{
    const int Q = c->Q;
    const int64_t nx = c->nx;
    std::vector<unsigned char> h(size_t(Q) * nx * c->elem);
    QL_CUDA(c, cudaMemcpy2DAsync(h.data(), nx * c->elem, static_cast<const unsigned char *>(dev) + kHalo * c->elem,
                                 c->stride * c->elem, nx * c->elem, Q, cudaMemcpyDeviceToHost, c->stream));
    QL_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < Q; ++k) {
        for (int64_t i = 0; i < nx; ++i) {
            const size_t src = 2 * (size_t(k) * nx + i);
            double f, t;
            if (c->precision == QL_FP32) {
                f = double(reinterpret_cast<const float *>(h.data())[src]);
                t = double(reinterpret_cast<const float *>(h.data())[src + 1]);
            } else {
                f = reinterpret_cast<const double *>(h.data())[src];
                t = reinterpret_cast<const double *>(h.data())[src + 1];
            }
            if (phi) phi[i * Q + k] = f;
            if (theta) theta[i * Q + k] = t;
        }
    }
    return QL_OK;
}

ql_status ql_get_state(ql_ctx *c, double *phi, double *theta)
{
    if (!c) return fail(c, QL_EINVAL, "null context");
    ql_status st = download_rows(c, state_buf(c), phi, theta);
    if (st != QL_OK) return st;
    return check_err_word(c);
}

ql_status ql_set_state(ql_ctx *c, const double *phi, const double *theta)
{
    if (!c || !phi || !theta) return fail(c, QL_EINVAL, "bad arguments to ql_set_state");
    const int Q = c->Q;
    const int64_t nx = c->nx;
    std::vector<unsigned char> h(size_t(Q) * nx * c->elem);
    for (int k = 0; k < Q; ++k) {
        for (int64_t i = 0; i < nx; ++i) {
            const size_t dst = 2 * (size_t(k) * nx + i);
            if (c->precision == QL_FP32) {
                reinterpret_cast<float *>(h.data())[dst] = float(phi[i * Q + k]);
                reinterpret_cast<float *>(h.data())[dst + 1] = float(theta[i * Q + k]);
            } else {
                reinterpret_cast<double *>(h.data())[dst] = phi[i * Q + k];
                reinterpret_cast<double *>(h.data())[dst + 1] = theta[i * Q + k];
            }
        }
    }
    QL_CUDA(c, cudaMemcpy2DAsync(static_cast<unsigned char *>(state_buf(c)) + kHalo * c->elem, c->stride * c->elem,
                                 h.data(), nx * c->elem, nx * c->elem, Q, cudaMemcpyHostToDevice, c->stream));
    if (c->periodic) {
        cudaError_t e = c->precision == QL_FP32 ? launch_periodic_ghosts_f32(Q, state_buf(c), nx, c->stride, c->stream)
                                                : launch_periodic_ghosts_f64(Q, state_buf(c), nx, c->stride, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "ghost kernel");
    }
    QL_CUDA(c, refresh_nbar(c));
    QL_CUDA(c, cudaStreamSynchronize(c->stream));
    return QL_OK;
}

ql_status ql_load_fields(ql_ctx *c, const double *rho, const double *u, const double *T)
{
    if (!c || !rho || !u || !T) return fail(c, QL_EINVAL, "bad arguments to ql_load_fields");
    const int64_t nx = c->nx, ncol = nx + 2 * kHalo;
    // interior columns straight from the caller's arrays (DMA when they are pinned)
    const double *src[3] = {rho, u, T};
    for (int f = 0; f < 3; ++f)
        QL_CUDA(c, cudaMemcpyAsync(c->d_init + f * ncol + kHalo, src[f], sizeof(double) * nx, cudaMemcpyHostToDevice,
                                   c->stream));
    // ghost columns: periodic images, or the fixed states kept from creation
    double gh[3][2 * kHalo];
    for (int g = 0; g < 2 * kHalo; ++g) {
        for (int f = 0; f < 3; ++f) {
            if (c->periodic) {
                const int64_t cell = g < kHalo ? nx - kHalo + g : g - kHalo;
                gh[f][g] = src[f][cell];
            } else {
                gh[f][g] = c->ghost_state[3 * g + f];
            }
        }
    }
    for (int f = 0; f < 3; ++f) {
        QL_CUDA(c, cudaMemcpyAsync(c->d_init + f * ncol, gh[f], sizeof(double) * kHalo, cudaMemcpyHostToDevice,
                                   c->stream));
        QL_CUDA(c, cudaMemcpyAsync(c->d_init + f * ncol + kHalo + nx, gh[f] + kHalo, sizeof(double) * kHalo,
                                   cudaMemcpyHostToDevice, c->stream));
    }
    cudaError_t e = c->lq ? launch_lq_init(c->Q, c->d_init, c->d_init + ncol, c->d_init + 2 * ncol, state_buf(c), nx,
                                           c->stride, c->d_lqtab, c->stream)
                    : c->precision == QL_FP32
                        ? launch_init_f32(c->Q, c->d_init, c->d_init + ncol, c->d_init + 2 * ncol, state_buf(c), nx,
                                          c->stride, c->d_tab64, c->stream)
                        : launch_init_f64(c->Q, c->d_init, c->d_init + ncol, c->d_init + 2 * ncol, state_buf(c), nx,
                                          c->stride, c->d_tab64, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
    QL_CUDA(c, refresh_nbar(c));
    QL_CUDA(c, cudaStreamSynchronize(c->stream));
    return QL_OK;
}

ql_status ql_rhs(ql_ctx *c, double *Lphi, double *Ltheta)
{
    if (!c) return fail(c, QL_EINVAL, "null context");
    cudaError_t e = stage(c, 0, state_buf(c), state_buf(c), other_buf(c));
    if (e != cudaSuccess) return cuda_fail(c, e, "stage kernel launch");
    ql_status st = download_rows(c, other_buf(c), Lphi, Ltheta);
    if (st != QL_OK) return st;
    return check_err_word(c);
}

ql_status ql_state_device(ql_ctx *c, void **phi, int64_t *row_stride)
{
    if (!c || !phi || !row_stride) return fail(c, QL_EINVAL, "bad arguments to ql_state_device");
    *phi = static_cast<unsigned char *>(state_buf(c)) + kHalo * c->elem;
    *row_stride = c->stride;
    return QL_OK;
}

ql_status ql_info(const ql_ctx *c, double *out)
{
    if (!c || !out) return QL_EINVAL;
    out[0] = c->eta0;
    out[1] = c->chi0;
    out[2] = c->sigma;
    out[3] = c->dx;
    out[4] = c->dt;
    double pm = 0;
    for (int k = 0; k < c->Q; ++k) pm = fmax(pm, fabs(c->p[k]));
    out[5] = pm;
    for (int k = 0; k < c->Q; ++k) {
        out[6 + k] = c->p[k];
        out[6 + c->Q + k] = c->w[k];
    }
    return QL_OK;
}

ql_status ql_launch_info(const ql_ctx *c, int64_t *steps_per_launch)
{
    if (!c || !steps_per_launch) return QL_EINVAL;
    *steps_per_launch = runs_whole(c) ? run_steps_per_launch(c) : 0;
    return QL_OK;
}

ql_status ql_destroy(ql_ctx *c)
{
    if (!c) return QL_OK;
    cudaStreamSynchronize(c->stream);
    destroy_buffers(c);
    delete c;
    return QL_OK;
}

const char *ql_last_error(const ql_ctx *c) { return c ? c->err.c_str() : g_create_error.c_str(); }

ql_status ql_velocity_set(int32_t Q, double *p, double *w)
{
    if (!p || !w || !gh_quadrature(Q, p, w)) return fail(nullptr, QL_EINVAL, "velocity set: Q out of range");
    return QL_OK;
}

ql_status ql_eta_of_denseness(double denseness, double *eta0)
{
    if (!eta0 || !eta_of_denseness(denseness, eta0)) return fail(nullptr, QL_EINVAL, "denseness out of range");
    return QL_OK;
}

double ql_sound_speed2(double eta0, double rho_ref, double rho, double T)
{
    return sound_speed2(eta0, rho_ref, rho, T);
}

ql_status ql_sound_modes(double denseness, double kn, double length, double rho_ref, int32_t pr_mode,
                         double pr_const, double rho, double T, double k, double *out)
{
    if (!out || !sound_modes(denseness, kn, length, rho_ref, pr_mode, pr_const, rho, T, k, out))
        return fail(nullptr, QL_EINVAL, "bad arguments to ql_sound_modes");
    return QL_OK;
}

ql_status ql_rankine_hugoniot(double eta0, double rho_ref, double rho1, double T1, double mach, double *out)
{
    if (!out || !rankine_hugoniot(eta0, rho_ref, rho1, T1, mach, out))
        return fail(nullptr, QL_EINVAL, "no compressive Rankine-Hugoniot solution");
    return QL_OK;
}

ql_status ql_riemann_exact(double eta0, double rho_ref, const double *left, const double *right, double *waves,
                           int64_t n, const double *xi, double *rho, double *u, double *T)
{
    if (!left || !right || n < 0 || (n > 0 && (!xi || !rho || !u || !T)) || !(eta0 >= 0.0) || !(eta0 < 0.5) ||
        !(rho_ref > 0.0))
        return fail(nullptr, QL_EINVAL, "bad arguments to ql_riemann_exact");
    std::unique_ptr<RiemannWaves> w(new RiemannWaves());
    if (!riemann_solve(eta0, rho_ref, left[0], left[1], right[0], right[1], w.get()))
        return fail(nullptr, QL_EINVAL, "no rarefaction-contact-shock solution for these states");
    if (waves) {
        const double v[9] = {w->P_c, w->u_c, w->rho1, w->T1, w->rho2, w->T2, w->xi_head, w->xi_tail, w->xi_shock};
        for (int k = 0; k < 9; ++k) waves[k] = v[k];
    }
    for (int64_t i = 0; i < n; ++i) riemann_sample(*w, xi[i], &rho[i], &u[i], &T[i]);
    return QL_OK;
}


// ---------------------------------------------------------------------------
// Restart files: a text header (first line and one JSON line) and the state.

static const char kCkptMagic[] = "qlbm-checkpoint 1";

static bool host_little_endian()
{
    const uint32_t one = 1;
    unsigned char b;
    memcpy(&b, &one, 1);
    return b == 1;
}

// Value after "key": in a one-line JSON object written by ql_save.
static const char *json_value(const std::string &h, const char *key)
{
    const std::string k = std::string("\"") + key + "\":";
    const size_t at = h.find(k);
    if (at == std::string::npos) return nullptr;
    const char *v = h.c_str() + at + k.size();
    while (*v == ' ') ++v;
    return v;
}

static bool json_double(const std::string &h, const char *key, double *out)
{
    const char *v = json_value(h, key);
    if (!v) return false;
    char *end = nullptr;
    *out = strtod(v, &end);
    return end != v && isfinite(*out);
}

static bool json_int(const std::string &h, const char *key, int64_t *out)
{
    const char *v = json_value(h, key);
    if (!v) return false;
    char *end = nullptr;
    *out = strtoll(v, &end, 10);
    return end != v && (*end == ',' || *end == '}' || *end == ' ');
}

static bool json_string(const std::string &h, const char *key, std::string *out)
{
    const char *v = json_value(h, key);
    if (!v || *v != '"') return false;
    const char *e = strchr(v + 1, '"');
    if (!e) return false;
    out->assign(v + 1, e);
    return true;
}

// Parses the header of an open restart file; leaves f at the state.
static ql_status read_header(FILE *f, ql_checkpoint_info *in, std::string *why)
{
    if (!host_little_endian()) {
        *why = "restart files are little-endian; this host is not";
        return QL_EUNSUPPORTED;
    }
    char line[64];
    if (!fgets(line, sizeof line, f) || strncmp(line, kCkptMagic, strlen(kCkptMagic)) != 0 ||
        line[strlen(kCkptMagic)] != '\n') {
        *why = "not a restart file (first line)";
        return QL_EINVAL;
    }
    std::string h;
    for (int ch; (ch = fgetc(f)) != EOF && ch != '\n';) {
        h.push_back(char(ch));
        if (h.size() > (1u << 16)) break;
    }
    if (h.empty() || h.front() != '{' || h.back() != '}') {
        *why = "malformed header line";
        return QL_EINVAL;
    }
    memset(in, 0, sizeof *in);
    int64_t Q = 0, prm = 0, ens = 0, chi = 0;
    std::string bc, prec, order;
    bool ok = json_int(h, "Q", &Q) && json_int(h, "nx", &in->nx) && json_double(h, "length", &in->length) &&
              json_double(h, "dt", &in->dt) && json_double(h, "denseness", &in->denseness) &&
              json_double(h, "kn", &in->kn) && json_string(h, "bc", &bc) && json_string(h, "precision", &prec) &&
              json_int(h, "pr_mode", &prm) && json_double(h, "pr_const", &in->pr_const) &&
              json_int(h, "enskog", &ens) && json_double(h, "rho_ref", &in->rho_ref) &&
              json_int(h, "chi_mode", &chi) && json_int(h, "steps", &in->steps) &&
              json_string(h, "byte_order", &order);
    ok = ok && (bc == "periodic" || bc == "fixed") && (prec == "fp64" || prec == "fp32") && order == "little";
    ok = ok && Q >= 2 && Q <= kLargeMaxQ && in->nx >= 1 && in->nx <= (int64_t(1) << 31) && in->steps >= 0;
    const char *g = json_value(h, "ghost");
    ok = ok && g && *g == '[';
    if (ok) {
        ++g;
        for (int j = 0; j < 18 && ok; ++j) {
            while (*g == ' ' || *g == ',') ++g;
            char *end = nullptr;
            in->ghost[j] = strtod(g, &end);
            ok = end != g && isfinite(in->ghost[j]);
            g = end;
        }
        while (ok && *g == ' ') ++g;
        ok = ok && *g == ']';
    }
    if (!ok) {
        *why = "missing or malformed header field";
        return QL_EINVAL;
    }
    in->Q = int32_t(Q);
    in->bc_kind = bc == "fixed" ? QL_BC_FIXED : QL_BC_PERIODIC;
    in->precision = prec == "fp32" ? QL_FP32 : QL_FP64;
    in->pr_mode = int32_t(prm);
    in->enskog = int32_t(ens);
    in->chi_mode = int32_t(chi);
    // the rest of the file is exactly the two state arrays
    const long at = ftell(f);
    if (at < 0 || fseek(f, 0, SEEK_END) != 0) {
        *why = "cannot seek in the file";
        return QL_EINVAL;
    }
    const long end = ftell(f);
    const double want = 2.0 * double(in->nx) * double(Q) * sizeof(double);
    if (end < 0 || double(end - at) != want || fseek(f, at, SEEK_SET) != 0) {
        *why = "state size does not match nx and Q";
        return QL_EINVAL;
    }
    return QL_OK;
}

ql_status ql_step_count(const ql_ctx *c, int64_t *steps)
{
    if (!c || !steps) return fail(nullptr, QL_EINVAL, "null argument to ql_step_count");
    *steps = c->steps;
    return QL_OK;
}

ql_status ql_save(ql_ctx *c, const char *path)
{
    if (!c || !path) return fail(c, QL_EINVAL, "null argument to ql_save");
    const size_t n = size_t(c->nx) * size_t(c->Q);
    std::vector<double> phi, theta;
    try {
        phi.resize(n);
        theta.resize(n);
    } catch (...) {
        return fail(c, QL_ENOMEM, "host buffers for ql_save");
    }
    ql_status st = ql_get_state(c, phi.data(), theta.data());
    if (st != QL_OK) return st;
    double ghost[18] = {};
    if (!c->periodic && c->ghost_state.size() >= size_t(3 * 2 * kHalo))
        for (int g = 0; g < 3; ++g)
            for (int v = 0; v < 3; ++v) {
                ghost[3 * g + v] = c->ghost_state[3 * (g + 1) + v];          // cells -3..-1
                ghost[9 + 3 * g + v] = c->ghost_state[3 * (kHalo + g) + v];  // cells nx..nx+2
            }
    std::string h = "{";
    char b[96];
    auto num = [&](const char *k, double v, bool last = false) {
        snprintf(b, sizeof b, "\"%s\": %.17g%s", k, v, last ? "" : ", ");
        h += b;
    };
    auto integer = [&](const char *k, int64_t v) {
        snprintf(b, sizeof b, "\"%s\": %lld, ", k, (long long)v);
        h += b;
    };
    integer("Q", c->Q);
    integer("nx", c->nx);
    num("length", c->L);
    num("dt", c->dt);
    num("denseness", c->El);
    num("kn", c->kn);
    h += std::string("\"bc\": \"") + (c->periodic ? "periodic" : "fixed") + "\", ";
    h += std::string("\"precision\": \"") + (c->precision == QL_FP32 ? "fp32" : "fp64") + "\", ";
    integer("pr_mode", c->pr_mode);
    num("pr_const", c->pr_const);
    integer("enskog", c->enskog);
    num("rho_ref", c->rho_ref);
    integer("chi_mode", c->chi_mode);
    integer("steps", c->steps);
    num("time", double(c->steps) * c->dt);
    h += "\"ghost\": [";
    for (int j = 0; j < 18; ++j) {
        snprintf(b, sizeof b, "%.17g%s", ghost[j], j < 17 ? ", " : "");
        h += b;
    }
    h += "], \"byte_order\": \"little\"}";
    const std::string tmp = std::string(path) + ".tmp" + std::to_string(long(getpid()));
    FILE *f = fopen(tmp.c_str(), "wb");
    if (!f) return fail(c, QL_EINVAL, std::string("cannot write ") + tmp + ": " + strerror(errno));
    bool ok = fprintf(f, "%s\n%s\n", kCkptMagic, h.c_str()) > 0 && fwrite(phi.data(), sizeof(double), n, f) == n &&
              fwrite(theta.data(), sizeof(double), n, f) == n;
    ok = (fclose(f) == 0) && ok;
    if (!ok || rename(tmp.c_str(), path) != 0) {
        const std::string why = strerror(errno);
        remove(tmp.c_str());
        return fail(c, QL_EINVAL, std::string("cannot write ") + path + ": " + why);
    }
    return QL_OK;
}

ql_status ql_checkpoint_read_info(const char *path, ql_checkpoint_info *info)
{
    if (!path || !info) return fail(nullptr, QL_EINVAL, "null argument to ql_checkpoint_read_info");
    FILE *f = fopen(path, "rb");
    if (!f) return fail(nullptr, QL_EINVAL, std::string("cannot open ") + path + ": " + strerror(errno));
    std::string why;
    const ql_status st = read_header(f, info, &why);
    fclose(f);
    return st == QL_OK ? QL_OK : fail(nullptr, st, std::string(path) + ": " + why);
}

ql_status ql_load(const char *path, const ql_opts *opts, ql_ctx **out)
{
    if (out) *out = nullptr;
    if (!path || !out) return fail(nullptr, QL_EINVAL, "null argument to ql_load");
    FILE *f = fopen(path, "rb");
    if (!f) return fail(nullptr, QL_EINVAL, std::string("cannot open ") + path + ": " + strerror(errno));
    ql_checkpoint_info in;
    std::string why;
    ql_status st = read_header(f, &in, &why);
    if (st != QL_OK) {
        fclose(f);
        return fail(nullptr, st, std::string(path) + ": " + why);
    }
    const size_t n = size_t(in.nx) * size_t(in.Q);
    std::vector<double> phi, theta;
    try {
        phi.resize(n);
        theta.resize(n);
    } catch (...) {
        fclose(f);
        return fail(nullptr, QL_ENOMEM, "host buffers for ql_load");
    }
    const bool got = fread(phi.data(), sizeof(double), n, f) == n && fread(theta.data(), sizeof(double), n, f) == n;
    fclose(f);
    if (!got) return fail(nullptr, QL_EINVAL, std::string(path) + ": short state");
    // re-create from uniform fields and the stored fixed states (which set the
    // ghost cells exactly as at the original creation), then load the state
    ql_velset vs = {in.Q, 0};
    ql_grid grid = {in.nx, in.length, in.dt};
    ql_bc bc = {in.bc_kind, 0};
    std::vector<double> r(size_t(in.nx), in.rho_ref), u(size_t(in.nx), 0.0), T(size_t(in.nx), 1.0);
    ql_init init;
    memset(&init, 0, sizeof init);
    init.kind = QL_INIT_FIELDS;
    init.rho = r.data();
    init.u = u.data();
    init.T = T.data();
    init.ghost = in.bc_kind == QL_BC_FIXED ? in.ghost : nullptr;
    ql_opts o;
    memset(&o, 0, sizeof o);
    if (opts) o = *opts;
    o.precision = in.precision;
    o.pr_mode = in.pr_mode;
    o.enskog = in.enskog;
    o.chi_mode = in.chi_mode;
    o.pr_const = in.pr_const;
    o.rho_ref = in.rho_ref;
    ql_ctx *c = nullptr;
    st = ql_create(&vs, &grid, in.denseness, in.kn, &bc, &init, &o, &c);
    if (st != QL_OK) return st;
    st = ql_set_state(c, phi.data(), theta.data());
    if (st != QL_OK) {
        const std::string m = c->err;
        ql_destroy(c);
        return fail(nullptr, st, m);
    }
    c->steps = in.steps;
    *out = c;
    return QL_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Fixed-order sum of the per-block partial totals (one block).
__global__ void qlbm_reduce_totals_kernel(const double *__restrict__ partial, int64_t nblocks,
                                          double *__restrict__ totals)
{
    __shared__ double red[3][256];
    double s[3] = {0, 0, 0};
    for (int64_t b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int c = 0; c < 3; ++c) s[c] += partial[b * 3 + c];
    for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = s[c];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 3) totals[threadIdx.x] = red[threadIdx.x][0];
}

namespace qlbm {
cudaError_t launch_reduce_totals(const double *partial, int64_t nblocks, double *totals, cudaStream_t s)
{
    qlbm_reduce_totals_kernel<<<1, 256, 0, s>>>(partial, nblocks, totals);
    return cudaGetLastError();
}
}  // namespace qlbm
