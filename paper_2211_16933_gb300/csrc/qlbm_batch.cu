// C ABI of the batched form (include/qlbm.h, ql_batch_*): many independent 1D
// domains advanced together by persistent stage kernels over one work list,
// whole runs captured in a CUDA graph, and a tuner for the CTA shape.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <string>
#include <vector>

#include "../../include/qlbm.h"
#include "qlbm_host.h"
#include "qlbm_internal.h"

using namespace qlbm;

struct ql_batch {
    int precision = QL_FP32, device = 0;
    int sums64 = 0;  // FP32: per-cell conserved sums in FP64 (QL_SUMS_FP64)
    int64_t n = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    ql_alloc_fn alloc = nullptr;
    ql_free_fn free_fn = nullptr;
    void *alloc_user = nullptr;
    size_t elem = 8;
    std::vector<BatchInstance> inst;
    std::vector<double> updates;  // nx * Q per instance
    BatchInstance *d_inst = nullptr;
    int2 *d_work[2] = {nullptr, nullptr};  // work lists for kBatchWarps[0], kBatchWarps[1]
    int64_t nwork[2] = {0, 0};
    // each list holds the items of the instances with Q = kBatchQList[g] at [qstart, qstart + qcount)
    int64_t qstart[2][kNumBatchQ] = {}, qcount[2][kNumBatchQ] = {};
    void *arena[3] = {nullptr, nullptr, nullptr};
    size_t arena_bytes = 0;
    unsigned *d_err = nullptr;
    double *d_tab64 = nullptr, *d_fields = nullptr, *d_partial = nullptr, *d_totals = nullptr, *d_init = nullptr;
    int64_t max_nx = 0;
    int warps = 8, grid = 0, sms = 0;
    // chi_RET-FM instances: their (instance, tile) list of 8-warp tiles grouped by
    // velocity set, the (instance, block) list of the ball average, their densities
    // and nbar (Real, stride columns each) and ball weights
    int2 *d_rwork = nullptr, *d_fmwork = nullptr;
    int64_t rstart[kNumBatchQ] = {}, rcount[kNumBatchQ] = {}, nfm = 0;
    int max_w = 0;
    void *d_n = nullptr, *d_nbar = nullptr;
    double *d_fmk = nullptr;
    // A step writes psi^(n+1) into the buffer that held psi^(1) (a last stage
    // writing in place ran about 3 % slower), and arena[0] and arena[1] swap on
    // the host, so that arena[0] always holds the state.  A run recorded as a
    // CUDA graph is kept per buffer order (swapped: arena[0] is the second
    // allocation) and per step count and CTA shape.
    bool swapped = false;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int64_t graph_steps[2] = {-1, -1};
    int graph_warps[2] = {0, 0}, graph_grid[2] = {0, 0};
    std::string err;
};

static std::string g_batch_error;

static ql_status bfail(ql_batch *b, ql_status st, const std::string &m)
{
    if (b) b->err = m; else g_batch_error = m;
    return st;
}

static ql_status bcuda(ql_batch *b, cudaError_t e, const char *what)
{
    return bfail(b, e == cudaErrorMemoryAllocation ? QL_ENOMEM : QL_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define QB_CUDA(b, call)                                   \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return bcuda(b, e_, #call); \
    } while (0)

static void *balloc(ql_batch *b, size_t bytes)
{
    if (b->alloc) return b->alloc(bytes, b->alloc_user);
    void *p = nullptr;
    return cudaMalloc(&p, bytes) == cudaSuccess ? p : nullptr;
}

static void bfree(ql_batch *b, void *p)
{
    if (!p) return;
    if (b->free_fn) b->free_fn(p, b->alloc_user);
    else cudaFree(p);
}

static void batch_release(ql_batch *b)
{
    for (auto &g : b->graph)
        if (g) cudaGraphExecDestroy(g);
    for (int j = 0; j < 3; ++j) bfree(b, b->arena[j]);
    for (int j = 0; j < 2; ++j) bfree(b, b->d_work[j]);
    bfree(b, b->d_inst);
    bfree(b, b->d_err);
    bfree(b, b->d_tab64);
    bfree(b, b->d_fields);
    bfree(b, b->d_partial);
    bfree(b, b->d_totals);
    bfree(b, b->d_init);
    bfree(b, b->d_rwork);
    bfree(b, b->d_fmwork);
    bfree(b, b->d_n);
    bfree(b, b->d_nbar);
    bfree(b, b->d_fmk);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

// nbar of every chi_RET-FM instance from the densities in d_n (one launch).
static cudaError_t launch_fm_all(ql_batch *b)
{
    if (b->nfm == 0) return cudaSuccess;
    BatchFmArgs f;
    f.inst = b->d_inst;
    f.work = b->d_fmwork;
    f.nwork = b->nfm;
    f.n = b->d_n;
    f.nbar = b->d_nbar;
    f.K = b->d_fmk;
    return b->precision == QL_FP32 ? launch_batch_fm_f32(f, b->max_w, b->stream)
                                   : launch_batch_fm_f64(f, b->max_w, b->stream);
}

// One Runge-Kutta stage of every instance: a launch per velocity set present,
// of `grid` CTAs walking the set's work items, or (grid 0) one CTA per item;
// the chi_RET-FM instances in launches of their own (8-warp tiles, one CTA per
// item), then (fm) the ball average of their output densities.  With par = 1
// the stage runs from arena[1] as psi^n (the odd steps of a run: each step
// leaves the state in the other of the first two buffers).
static cudaError_t launch_stage(ql_batch *b, int stage, int warps, int grid, bool fm = true, int par = 0)
{
    void *const order[3] = {b->arena[par], b->arena[1 - par], b->arena[2]};
    const int wi = warps == kBatchWarps[0] ? 0 : 1;
    for (int g = 0; g < kNumBatchQ; ++g) {
        if (b->qcount[wi][g] == 0) continue;
        const int gq = grid > 0 ? grid : int(std::min<int64_t>(b->qcount[wi][g], INT32_MAX));
        BatchArgs a;
        a.inst = b->d_inst;
        a.work = b->d_work[wi] + b->qstart[wi][g];
        a.nwork = b->qcount[wi][g];
        for (int j = 0; j < 3; ++j) a.arena[j] = order[j];
        a.err = b->d_err;
        a.sums64 = b->sums64;
        const cudaError_t e = b->precision == QL_FP32
                                  ? launch_batch_stage_f32(kBatchQList[g], stage, warps, gq, a, b->stream)
                                  : launch_batch_stage_f64(kBatchQList[g], stage, warps, gq, a, b->stream);
        if (e != cudaSuccess) return e;
    }
    for (int g = 0; g < kNumBatchQ; ++g) {
        if (b->rcount[g] == 0) continue;
        BatchArgs a;
        a.inst = b->d_inst;
        a.work = b->d_rwork + b->rstart[g];
        a.nwork = b->rcount[g];
        for (int j = 0; j < 3; ++j) a.arena[j] = order[j];
        a.err = b->d_err;
        a.sums64 = b->sums64;
        a.n = b->d_n;
        a.nbar = b->d_nbar;
        const int gq = int(std::min<int64_t>(b->rcount[g], INT32_MAX));
        const cudaError_t e = b->precision == QL_FP32
                                  ? launch_batch_stage_ret_f32(kBatchQList[g], stage, gq, a, b->stream)
                                  : launch_batch_stage_ret_f64(kBatchQList[g], stage, gq, a, b->stream);
        if (e != cudaSuccess) return e;
    }
    return fm ? launch_fm_all(b) : cudaSuccess;
}

// Fields of every instance averaged over blocks of nx/ncoarse cells:
// out[(i * 5 + f) * ncoarse + c] for f = rho, u, T, q, Pxx.  One thread per
// (instance, coarse cell); moments per fine cell in FP64 (Sec. II.D).
template <typename Real>
__global__ void batch_fields_kernel(const BatchInstance *__restrict__ inst, const void *__restrict__ arena,
                                    const double *__restrict__ tab, int ncoarse, double *__restrict__ out)
{
    using V = typename std::conditional<sizeof(Real) == 4, float2, double2>::type;
    const int i = blockIdx.y;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncoarse) return;
    const BatchInstance I = inst[i];
    const int Q = I.Q;
    int p_off = 0;
    switch (Q) {
    case 8: p_off = tab_view(8).p; break;
    case 16: p_off = tab_view(16).p; break;
    case 24: p_off = tab_view(24).p; break;
    default: p_off = tab_view(32).p; break;
    }
    const V *psi = static_cast<const V *>(arena) + I.off;
    const int64_t f = I.nx / ncoarse;
    double acc[5] = {0, 0, 0, 0, 0};
    for (int64_t j = 0; j < f; ++j) {
        const int64_t cell = int64_t(c) * f + j;
        double S0 = 0, S1 = 0, S2 = 0, S3 = 0, R0 = 0, R1 = 0;
        for (int k = 0; k < Q; ++k) {
            const V v = psi[int64_t(k) * I.stride + kHalo + cell];
            const double ph = double(v.x), th = double(v.y), p = tab[p_off + k];
            S0 += ph;
            S1 += p * ph;
            S2 += p * p * ph;
            S3 += p * p * p * ph;
            R0 += th;
            R1 += p * th;
        }
        const double n = S0, u = S1 / n, c2 = S2 - u * S1;
        acc[0] += n;
        acc[1] += u;
        acc[2] += (c2 + R0) / (3.0 * n);
        acc[3] += 0.5 * (S3 - 3.0 * u * S2 + 2.0 * u * u * S1 + R1 - u * R0);
        acc[4] += c2;
    }
    for (int q = 0; q < 5; ++q) out[(int64_t(i) * 5 + q) * ncoarse + c] = acc[q] / double(f);
}

// Sec. IV.A: amplitude of density mode m of every instance,
//   out[i] = (2 / nx) sum_j rho_j cos(2 pi m x_j / L),  x_j = (j + 1/2) L / nx,
// with rho_j = sum_k phi_k.  One block per instance, FP64 sums, fixed-order
// tree reduction.
constexpr int kProjThreads = 256;
template <typename Real>
__global__ void __launch_bounds__(kProjThreads) batch_project_kernel(const BatchInstance *__restrict__ inst,
                                                                     const void *__restrict__ arena, int mode,
                                                                     double *__restrict__ out)
{
    using V = typename std::conditional<sizeof(Real) == 4, float2, double2>::type;
    __shared__ double red[kProjThreads];
    const int i = blockIdx.x;
    const BatchInstance I = inst[i];
    const V *psi = static_cast<const V *>(arena) + I.off;
    const double w = 2.0 * 3.14159265358979323846 * double(mode) / double(I.nx);
    double acc = 0.0;
    for (int64_t c = threadIdx.x; c < I.nx; c += kProjThreads) {
        double rho = 0.0;
        for (int k = 0; k < I.Q; ++k) rho += double(psi[int64_t(k) * I.stride + kHalo + c].x);
        acc += rho * cos(w * (double(c) + 0.5));
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = kProjThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[i] = 2.0 * red[0] / double(I.nx);
}

static int ctas_per_sm(ql_batch *b, int warps)
{
    int m = 8;
    for (int s = 1; s <= 3; ++s) {
        const int c = b->precision == QL_FP32 ? batch_ctas_per_sm_f32(s, warps) : batch_ctas_per_sm_f64(s, warps);
        m = std::min(m, c);
    }
    return m;
}

extern "C" {

ql_status ql_batch_create(const ql_instance *in, int64_t n, const ql_opts *opts, ql_batch **out)
{
    if (out) *out = nullptr;
    if (!in || n <= 0 || !opts || !out) return bfail(nullptr, QL_EINVAL, "bad arguments to ql_batch_create");
    if (opts->precision != QL_FP32 && opts->precision != QL_FP64) return bfail(nullptr, QL_EINVAL, "bad precision");
    if (opts->sums != QL_SUMS_DFP32 && opts->sums != QL_SUMS_FP64) return bfail(nullptr, QL_EINVAL, "bad sums");
    ql_batch *b = new ql_batch();
    b->precision = opts->precision;
    b->sums64 = opts->precision == QL_FP32 && opts->sums == QL_SUMS_FP64;
    b->device = opts->device;
    b->n = n;
    b->alloc = opts->alloc;
    b->free_fn = opts->free;
    b->alloc_user = opts->alloc_user;
    b->elem = b->precision == QL_FP32 ? 8 : 16;
    auto bail = [&](ql_status st, const std::string &m) {
        batch_release(b);
        delete b;
        return bfail(nullptr, st, m);
    };

    // descriptors and host initial fields
    std::vector<std::vector<double>> fields(n);
    int64_t off = 0, noff = 0;
    std::vector<double> fmk;      // ball weights of the chi_RET-FM instances
    std::vector<int2> fmwork;     // their (instance, block) list
    b->inst.resize(n);
    b->updates.resize(n);
    for (int64_t i = 0; i < n; ++i) {
        const ql_instance &I = in[i];
        bool qok = false;
        for (int j = 0; j < kNumBatchQ; ++j) qok |= I.vs.Q == kBatchQList[j];
        const std::string id = "instance " + std::to_string(i) + ": ";
        if (!qok || I.vs.kind != 0) return bail(QL_EUNSUPPORTED, id + "Q must be one of 8, 16, 24, 32");
        if (I.grid.nx < 8 || I.grid.nx > (int64_t(1) << 31) || !(I.grid.length > 0) || !(I.grid.dt > 0))
            return bail(QL_EINVAL, id + "bad grid");
        if (!(I.denseness > 0) || !(I.kn > 0) || !(I.rho_ref > 0)) return bail(QL_EINVAL, id + "bad gas parameters");
        if (I.bc.kind != QL_BC_PERIODIC && I.bc.kind != QL_BC_FIXED) return bail(QL_EINVAL, id + "bad bc");
        if (I.pr_mode == QL_PR_CONST && !(I.pr_const > 0)) return bail(QL_EINVAL, id + "bad pr_const");
        if (I.chi_mode != QL_CHI_SET && I.chi_mode != QL_CHI_RET_FM) return bail(QL_EINVAL, id + "bad chi_mode");
        double eta0;
        if (!eta_of_denseness(I.denseness, &eta0)) return bail(QL_EINVAL, id + "denseness out of range");
        BatchInstance &D = b->inst[i];
        D.nx = I.grid.nx;
        D.stride = row_stride(D.nx);
        D.off = off;
        off += int64_t(I.vs.Q) * D.stride;
        D.inv_dx = 1.0 / (I.grid.length / double(D.nx));  // as ql_create computes it
        D.dt = I.grid.dt;
        D.eta0 = eta0;
        D.inv_rho_ref = 1.0 / I.rho_ref;
        D.tau_pref = tau_prefactor(I.kn, I.grid.length, eta0);
        D.pr_const = I.pr_const;
        D.Q = I.vs.Q;
        D.pr_mode = I.pr_mode;
        D.enskog = I.enskog ? 1 : 0;
        D.periodic = I.bc.kind == QL_BC_PERIODIC;
        b->updates[i] = double(D.nx) * D.Q;
        b->max_nx = std::max(b->max_nx, D.nx);
        const int64_t ncol = D.nx + 2 * kHalo;
        fields[i].resize(3 * ncol);
        if (!initial_fields(I.init.kind, I.init.prm, D.nx, I.grid.length, D.periodic, eta0, I.rho_ref, I.init.rho,
                            I.init.u, I.init.T, I.init.ghost, kHalo, fields[i].data(), fields[i].data() + ncol,
                            fields[i].data() + 2 * ncol))
            return bail(QL_EINVAL, id + "invalid initial state for this init kind / boundary");
        if (I.chi_mode == QL_CHI_RET_FM) {
            // as ql_create: sigma = E_l Kn L, the ball's half-width in cells, its weights
            const double dx = I.grid.length / double(D.nx), sigma = I.denseness * I.kn * I.grid.length;
            const int W = fm_halfwidth(dx, sigma);
            if (W > QL_FM_MAX_HALFWIDTH)
                return bail(QL_EUNSUPPORTED, id + "the chi_RET-FM ball reaches " + std::to_string(W) +
                                                 " cells on each side; at most QL_FM_MAX_HALFWIDTH are supported");
            D.ret = 1;
            D.fm_w = W;
            D.noff = noff;
            noff += D.stride;
            D.koff = int64_t(fmk.size());
            fmk.resize(fmk.size() + 2 * size_t(W) + 1);
            fm_weights(dx, sigma, W, fmk.data() + D.koff);
            b->max_w = std::max(b->max_w, W);
            // fixed bc: densities of ghost cells -3..-1 (columns 1..3) and nx..nx+2
            for (int g = 0; g < 3; ++g) {
                D.ghost_n[g] = D.periodic ? 0.0 : fields[i][1 + g];
                D.ghost_n[3 + g] = D.periodic ? 0.0 : fields[i][D.nx + kHalo + g];
            }
            const int64_t nb = (ncol + kFmThreads - 1) / kFmThreads;
            for (int64_t k = 0; k < nb; ++k) fmwork.push_back(make_int2(int(i), int(k)));
        }
    }
    // work lists, grouped by velocity set: all tiles of the first instance with
    // Q = kBatchQList[0], then of the next one, ..., then the instances with kBatchQList[1], ...
    // (the chi_SET instances; the chi_RET-FM ones in a list of 8-warp tiles of their own)
    std::vector<int2> work[2], rwork;
    for (int wi = 0; wi < 2; ++wi) {
        const int tile = 31 * kBatchWarps[wi];
        for (int g = 0; g < kNumBatchQ; ++g) {
            b->qstart[wi][g] = int64_t(work[wi].size());
            for (int64_t i = 0; i < n; ++i) {
                if (b->inst[i].Q != kBatchQList[g] || b->inst[i].ret) continue;
                const int64_t nt = (b->inst[i].nx + tile - 1) / tile;
                for (int64_t t = 0; t < nt; ++t) work[wi].push_back(make_int2(int(i), int(t)));
            }
            b->qcount[wi][g] = int64_t(work[wi].size()) - b->qstart[wi][g];
        }
        b->nwork[wi] = int64_t(work[wi].size());
    }
    for (int g = 0; g < kNumBatchQ; ++g) {
        b->rstart[g] = int64_t(rwork.size());
        for (int64_t i = 0; i < n; ++i) {
            if (b->inst[i].Q != kBatchQList[g] || !b->inst[i].ret) continue;
            const int64_t nt = (b->inst[i].nx + 31 * kBatchWarps[0] - 1) / (31 * kBatchWarps[0]);
            for (int64_t t = 0; t < nt; ++t) rwork.push_back(make_int2(int(i), int(t)));
        }
        b->rcount[g] = int64_t(rwork.size()) - b->rstart[g];
    }
    b->nfm = int64_t(fmwork.size());

    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return bail(QL_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    if (opts->stream) {
        b->stream = static_cast<cudaStream_t>(opts->stream);
    } else {
        // graph capture needs a stream other than the legacy default stream
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(QL_ECUDA, std::string("stream: ") + cudaGetErrorString(e));
        b->own_stream = true;
    }
    {
        std::string terr;
        if (!ensure_device_tables(b->device, terr)) return bail(QL_ECUDA, terr);
    }
    const double *tab = host_tables();
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);

    b->arena_bytes = size_t(off) * b->elem;
    for (int j = 0; j < 3; ++j) {
        b->arena[j] = balloc(b, b->arena_bytes);
        if (!b->arena[j]) return bail(QL_ENOMEM, "arena allocation failed");
    }
    b->d_inst = static_cast<BatchInstance *>(balloc(b, sizeof(BatchInstance) * n));
    for (int wi = 0; wi < 2; ++wi) b->d_work[wi] = static_cast<int2 *>(balloc(b, sizeof(int2) * work[wi].size()));
    b->d_err = static_cast<unsigned *>(balloc(b, sizeof(unsigned) * n));
    b->d_tab64 = static_cast<double *>(balloc(b, sizeof(double) * kTabTotal));
    b->d_fields = static_cast<double *>(balloc(b, sizeof(double) * 6 * b->max_nx));
    b->d_partial = static_cast<double *>(balloc(b, sizeof(double) * 3 * moment_blocks(b->max_nx)));
    b->d_totals = static_cast<double *>(balloc(b, sizeof(double) * 4));
    b->d_init = static_cast<double *>(balloc(b, sizeof(double) * 3 * (b->max_nx + 2 * kHalo)));
    if (!b->d_inst || !b->d_work[0] || !b->d_work[1] || !b->d_err || !b->d_tab64 || !b->d_fields || !b->d_partial ||
        !b->d_totals || !b->d_init)
        return bail(QL_ENOMEM, "work buffer allocation failed");
    if (b->nfm > 0) {
        const size_t real = b->elem / 2;
        b->d_rwork = static_cast<int2 *>(balloc(b, sizeof(int2) * rwork.size()));
        b->d_fmwork = static_cast<int2 *>(balloc(b, sizeof(int2) * fmwork.size()));
        b->d_n = balloc(b, real * size_t(noff));
        b->d_nbar = balloc(b, real * size_t(noff));
        b->d_fmk = static_cast<double *>(balloc(b, sizeof(double) * fmk.size()));
        if (!b->d_rwork || !b->d_fmwork || !b->d_n || !b->d_nbar || !b->d_fmk)
            return bail(QL_ENOMEM, "chi_RET-FM buffer allocation failed");
    }
    e = cudaMemcpyAsync(b->d_inst, b->inst.data(), sizeof(BatchInstance) * n, cudaMemcpyHostToDevice, b->stream);
    for (int wi = 0; wi < 2 && e == cudaSuccess; ++wi)
        e = cudaMemcpyAsync(b->d_work[wi], work[wi].data(), sizeof(int2) * work[wi].size(), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, sizeof(unsigned) * n, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_tab64, tab, sizeof(double) * kTabTotal, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->arena[0], 0, b->arena_bytes, b->stream);
    for (int64_t i = 0; i < n && e == cudaSuccess; ++i) {
        const BatchInstance &D = b->inst[i];
        const int64_t ncol = D.nx + 2 * kHalo;
        e = cudaMemcpyAsync(b->d_init, fields[i].data(), sizeof(double) * 3 * ncol, cudaMemcpyHostToDevice, b->stream);
        void *psi = static_cast<unsigned char *>(b->arena[0]) + size_t(D.off) * b->elem;
        if (e == cudaSuccess)
            e = b->precision == QL_FP32 ? launch_init_f32(D.Q, b->d_init, b->d_init + ncol, b->d_init + 2 * ncol, psi,
                                                          D.nx, D.stride, b->d_tab64, b->stream)
                                        : launch_init_f64(D.Q, b->d_init, b->d_init + ncol, b->d_init + 2 * ncol, psi,
                                                          D.nx, D.stride, b->d_tab64, b->stream);
        // d_init is reused by the next instance: wait before overwriting it from the host
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    }
    for (int j = 1; j < 3 && e == cudaSuccess; ++j)
        e = cudaMemcpyAsync(b->arena[j], b->arena[0], b->arena_bytes, cudaMemcpyDeviceToDevice, b->stream);
    if (b->nfm > 0) {
        // chi_RET-FM: work lists, weights, then nbar of the initial states (densities, ball average)
        const size_t real = b->elem / 2;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_rwork, rwork.data(), sizeof(int2) * rwork.size(), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_fmwork, fmwork.data(), sizeof(int2) * fmwork.size(), cudaMemcpyHostToDevice,
                                b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_fmk, fmk.data(), sizeof(double) * fmk.size(), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->d_nbar, 0, real * size_t(noff), b->stream);
        for (int64_t i = 0; i < n && e == cudaSuccess; ++i) {
            const BatchInstance &D = b->inst[i];
            if (!D.ret) continue;
            const void *psi = static_cast<unsigned char *>(b->arena[0]) + size_t(D.off) * b->elem;
            void *dn = static_cast<unsigned char *>(b->d_n) + size_t(D.noff) * real;
            e = b->precision == QL_FP32 ? launch_density_f32(D.Q, psi, D.nx, D.stride, dn, b->stream)
                                        : launch_density_f64(D.Q, psi, D.nx, D.stride, dn, b->stream);
        }
        if (e == cudaSuccess) e = launch_fm_all(b);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bail(QL_ECUDA, std::string("batch set-up: ") + cudaGetErrorString(e));
    b->warps = kBatchWarps[0];
    b->grid = 0;  // one CTA per work item until ql_batch_tune picks otherwise
    *out = b;
    return QL_OK;
}

ql_status ql_batch_tune(ql_batch *b, int32_t trial_launches, int32_t *warps_out, int32_t *ctas_per_sm_out)
{
    if (!b || trial_launches < 1) return bfail(b, QL_EINVAL, "bad arguments to ql_batch_tune");
    cudaEvent_t e0, e1;
    QB_CUDA(b, cudaEventCreate(&e0));
    QB_CUDA(b, cudaEventCreate(&e1));
    float best = 1e30f;
    int bw = b->warps, bg = b->grid;
    for (int wi = 0; wi < 2; ++wi) {
        const int w = kBatchWarps[wi];
        const int cmax = ctas_per_sm(b, w);
        // c = 0: one CTA per work item, the block scheduler filling the SMs
        for (int c = 0; c <= cmax; ++c) {
            const int grid = b->sms * c;
            // stage 1 reads psi^n and writes psi^(1) only, so timing it leaves the state unchanged
            // (with chi_RET-FM it also rewrites the densities, scratch until the next
            // stage's own; nbar is left alone)
            QB_CUDA(b, launch_stage(b, 1, w, grid, false));
            QB_CUDA(b, cudaEventRecord(e0, b->stream));
            for (int r = 0; r < trial_launches; ++r) QB_CUDA(b, launch_stage(b, 1, w, grid, false));
            QB_CUDA(b, cudaEventRecord(e1, b->stream));
            QB_CUDA(b, cudaEventSynchronize(e1));
            float ms = 0;
            QB_CUDA(b, cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                bw = w;
                bg = grid;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->warps = bw;
    b->grid = bg;
    if (warps_out) *warps_out = bw;
    if (ctas_per_sm_out) *ctas_per_sm_out = bg / std::max(1, b->sms);  // 0: one CTA per work item
    return QL_OK;
}

ql_status ql_batch_set_shape(ql_batch *b, int32_t warps, int32_t per_sm)
{
    if (!b || (warps != kBatchWarps[0] && warps != kBatchWarps[1]) || per_sm < 0)
        return bfail(b, QL_EINVAL, "bad arguments to ql_batch_set_shape (warps 8 or 4, ctas_per_sm >= 0)");
    const int cmax = ctas_per_sm(b, warps);
    if (per_sm > cmax)
        return bfail(b, QL_EINVAL, "ctas_per_sm above the " + std::to_string(cmax) + " CTAs an SM holds");
    b->warps = warps;
    b->grid = b->sms * per_sm;
    return QL_OK;
}

ql_status ql_batch_run(ql_batch *b, int64_t nsteps)
{
    if (!b || nsteps < 0) return bfail(b, QL_EINVAL, "bad arguments to ql_batch_run");
    if (nsteps == 0) return QL_OK;
    const int o = b->swapped ? 1 : 0;
    if (!b->graph[o] || b->graph_steps[o] != nsteps || b->graph_warps[o] != b->warps || b->graph_grid[o] != b->grid) {
        if (b->graph[o]) {
            cudaGraphExecDestroy(b->graph[o]);
            b->graph[o] = nullptr;
        }
        QB_CUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        for (int64_t s = 0; s < nsteps && e == cudaSuccess; ++s)
            for (int st = 1; st <= 3 && e == cudaSuccess; ++st)
                e = launch_stage(b, st, b->warps, b->grid, true, int(s & 1));
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return bcuda(b, e != cudaSuccess ? e : e2, "graph capture");
        }
        e = cudaGraphInstantiate(&b->graph[o], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return bcuda(b, e, "graph instantiate");
        b->graph_steps[o] = nsteps;
        b->graph_warps[o] = b->warps;
        b->graph_grid[o] = b->grid;
    }
    QB_CUDA(b, cudaGraphLaunch(b->graph[o], b->stream));
    if (nsteps & 1) {
        std::swap(b->arena[0], b->arena[1]);
        b->swapped = !b->swapped;
    }
    return QL_OK;
}

ql_status ql_batch_sync(ql_batch *b, uint32_t *flags)
{
    if (!b) return bfail(b, QL_EINVAL, "null batch");
    std::vector<unsigned> h(b->n);
    QB_CUDA(b, cudaMemcpyAsync(h.data(), b->d_err, sizeof(unsigned) * b->n, cudaMemcpyDeviceToHost, b->stream));
    QB_CUDA(b, cudaStreamSynchronize(b->stream));
    bool bad = false, gave_up = false;
    for (int64_t i = 0; i < b->n; ++i) {
        if (flags) flags[i] = h[i];
        bad |= (h[i] & 1u) != 0;
        gave_up |= (h[i] & 2u) != 0;
    }
    if (gave_up) return bfail(b, QL_ECUDA, "a stage kernel gave up waiting for its tile's TMA copies");
    if (bad) return bfail(b, QL_ENONPHYSICAL, "non-physical state in at least one instance");
    return QL_OK;
}

ql_status ql_batch_moments(ql_batch *b, int64_t i, double *rho, double *u, double *T, double *P, double *q,
                           double *Pxx, double *totals)
{
    if (!b || i < 0 || i >= b->n) return bfail(b, QL_EINVAL, "bad arguments to ql_batch_moments");
    const BatchInstance &D = b->inst[i];
    MomentArgs a;
    a.psi = static_cast<unsigned char *>(b->arena[0]) + size_t(D.off) * b->elem;
    a.nx = D.nx;
    a.stride = D.stride;
    a.eta0 = D.eta0;
    a.inv_rho_ref = D.inv_rho_ref;
    a.dx = 1.0 / D.inv_dx;
    double *f = b->d_fields;
    a.rho = f;
    a.u = f + D.nx;
    a.T = f + 2 * D.nx;
    a.P = f + 3 * D.nx;
    a.q = f + 4 * D.nx;
    a.Pxx = f + 5 * D.nx;
    a.partial = b->d_partial;
    a.err = b->d_err + i;
    a.sums64 = b->sums64;
    cudaError_t e = b->precision == QL_FP32 ? launch_moments_f32(D.Q, a, b->d_tab64, b->stream)
                                            : launch_moments_f64(D.Q, a, b->d_tab64, b->stream);
    if (e == cudaSuccess) e = launch_reduce_totals(b->d_partial, moment_blocks(D.nx), b->d_totals, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "moments kernel");
    double *outs[6] = {rho, u, T, P, q, Pxx};
    for (int j = 0; j < 6; ++j)
        if (outs[j])
            QB_CUDA(b, cudaMemcpyAsync(outs[j], f + j * D.nx, sizeof(double) * D.nx, cudaMemcpyDeviceToHost, b->stream));
    if (totals) QB_CUDA(b, cudaMemcpyAsync(totals, b->d_totals, sizeof(double) * 3, cudaMemcpyDeviceToHost, b->stream));
    unsigned h = 0;
    QB_CUDA(b, cudaMemcpyAsync(&h, b->d_err + i, sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream));
    QB_CUDA(b, cudaStreamSynchronize(b->stream));
    if (h & 2u) return bfail(b, QL_ECUDA, "a stage kernel gave up waiting for its tile's TMA copies");
    if (h & 1u) return bfail(b, QL_ENONPHYSICAL, "non-physical state in instance " + std::to_string(i));
    return QL_OK;
}

ql_status ql_batch_fields(ql_batch *b, int32_t ncoarse, double *out)
{
    if (!b || ncoarse < 1 || !out) return bfail(b, QL_EINVAL, "bad arguments to ql_batch_fields");
    for (int64_t i = 0; i < b->n; ++i)
        if (b->inst[i].nx % ncoarse != 0)
            return bfail(b, QL_EINVAL, "ncoarse must divide nx of every instance (instance " + std::to_string(i) + ")");
    const dim3 grid(unsigned((ncoarse + 127) / 128), unsigned(b->n));
    if (b->precision == QL_FP32)
        batch_fields_kernel<float><<<grid, 128, 0, b->stream>>>(b->d_inst, b->arena[0], b->d_tab64, ncoarse, out);
    else
        batch_fields_kernel<double><<<grid, 128, 0, b->stream>>>(b->d_inst, b->arena[0], b->d_tab64, ncoarse, out);
    QB_CUDA(b, cudaGetLastError());
    return QL_OK;
}

ql_status ql_batch_project(ql_batch *b, int32_t mode, double *out)
{
    if (!b || !out || mode < 0) return bfail(b, QL_EINVAL, "bad arguments to ql_batch_project");
    if (b->precision == QL_FP32)
        batch_project_kernel<float><<<unsigned(b->n), kProjThreads, 0, b->stream>>>(b->d_inst, b->arena[0], mode, out);
    else
        batch_project_kernel<double><<<unsigned(b->n), kProjThreads, 0, b->stream>>>(b->d_inst, b->arena[0], mode, out);
    QB_CUDA(b, cudaGetLastError());
    return QL_OK;
}

ql_status ql_batch_get_state(ql_batch *b, int64_t i, double *phi, double *theta)
{
    if (!b || i < 0 || i >= b->n) return bfail(b, QL_EINVAL, "bad arguments to ql_batch_get_state");
    const BatchInstance &D = b->inst[i];
    const int Q = D.Q;
    const int64_t nx = D.nx;
    std::vector<unsigned char> h(size_t(Q) * nx * b->elem);
    const unsigned char *src = static_cast<const unsigned char *>(b->arena[0]) + size_t(D.off + kHalo) * b->elem;
    QB_CUDA(b, cudaMemcpy2DAsync(h.data(), nx * b->elem, src, D.stride * b->elem, nx * b->elem, Q,
                                 cudaMemcpyDeviceToHost, b->stream));
    QB_CUDA(b, cudaStreamSynchronize(b->stream));
    for (int k = 0; k < Q; ++k)
        for (int64_t c = 0; c < nx; ++c) {
            const size_t s = 2 * (size_t(k) * nx + c);
            double f, t;
            if (b->precision == QL_FP32) {
                f = reinterpret_cast<const float *>(h.data())[s];
                t = reinterpret_cast<const float *>(h.data())[s + 1];
            } else {
                f = reinterpret_cast<const double *>(h.data())[s];
                t = reinterpret_cast<const double *>(h.data())[s + 1];
            }
            if (phi) phi[c * Q + k] = f;
            if (theta) theta[c * Q + k] = t;
        }
    return QL_OK;
}

ql_status ql_batch_info(const ql_batch *b, double *out)
{
    if (!b || !out) return QL_EINVAL;
    double upd = 0;
    for (double v : b->updates) upd += v;
    out[0] = double(b->n);
    out[1] = upd;
    out[2] = b->warps;
    out[3] = b->grid;
    out[4] = double(b->arena_bytes);
    out[5] = double(b->sms);
    return QL_OK;
}

ql_status ql_batch_destroy(ql_batch *b)
{
    if (!b) return QL_OK;
    cudaStreamSynchronize(b->stream);
    batch_release(b);
    delete b;
    return QL_OK;
}

const char *ql_batch_last_error(const ql_batch *b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

}  // extern "C"
