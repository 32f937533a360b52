// Launchers shared by the per-precision translation units.  Before including
// this file a unit defines QL_REAL (float or double), QL_SUFFIX (f32 or f64)
// and declares `static __constant__ QL_REAL QL_TAB[kTabTotal]`.
#pragma once
#include "fdlb_kernels.cuh"
#include "fdlb_aux.cuh"

#define QL_CAT2(a, b) a##b
#define QL_CAT(a, b) QL_CAT2(a, b)
#define QL_FN(name) QL_CAT(name, QL_SUFFIX)

namespace qlbm {

// The stage kernels' copy of the tables: as built, except that the
// equilibrium rows are G[k][l] / sqrt(l!) = w_k He_l(p_k) / l! and cb[l] holds
// l - 1, for the coefficients d_l = l! c_l of Eq. (g_alpha), whose recurrence
// d_l = u d_{l-1} + (l - 1)(T - 1) d_{l-2} takes one operation less per
// coefficient than that of the normalised c^_l.
cudaError_t QL_FN(upload_tables_)(const double *all)
{
    static QL_REAL host[kTabTotal];
    for (int e = 0; e < kTabTotal; ++e) host[e] = QL_REAL(all[e]);
    for (int j = 0; j < kNumQ; ++j) {
        const int Q = kQList[j];
        const TabView tv = tab_view(Q);
        double isf = 1.0;  // 1 / sqrt(l!)
        for (int l = 0; l < Q; ++l) {
            if (l > 0) isf /= sqrt(double(l));
            for (int k = 0; k < Q; ++k) host[tv.G + k * Q + l] = QL_REAL(all[tv.G + k * Q + l] * isf);
            host[tv.cb + l] = QL_REAL(l >= 2 ? l - 1 : 0);
        }
    }
    return cudaMemcpyToSymbol(QL_TAB, host, sizeof(host));
}

// One CTA per tile; in FP64, a domain of fewer tiles than the GPU holds CTAs
// splits each tile's velocity pairs over up to Q/2 CTAs (FP64 arithmetic, not
// memory, bounds those small domains).  With chi_RET-FM the densities of the
// output then come from a separate pass, in the order the stage sums them.
template <int Q, int STAGE, bool RET>
static cudaError_t stage_q(const StageArgs &a, cudaStream_t s)
{
    constexpr size_t smem = stage_smem_bytes<QL_REAL, Q, kWarps, RET>();
    auto kern = fdlb_stage_kernel<QL_REAL, Q, STAGE, RET>;
    static int resident[64] = {};  // CTAs of this kernel the device holds at once
    int dev = 0;
    cudaGetDevice(&dev);
    if (!resident[dev & 63]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        int per_sm = 0, sms = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        resident[dev & 63] = per_sm * sms > 0 ? per_sm * sms : 1;
    }
    const int64_t nt = num_tiles(a.nx);
    StageArgs b = a;
    b.vsplit = 1;
    if (sizeof(QL_REAL) == 8 && nt < resident[dev & 63]) {
        const int64_t v = resident[dev & 63] / nt;
        b.vsplit = int(v < Q / 2 ? v : Q / 2);
    }
    // programmatic stream serialisation: the launch may overlap the tail of the
    // previous kernel in the stream, which the kernel waits for before its
    // first access to memory
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(nt * b.vsplit));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, b);
    if (e == cudaSuccess && RET && STAGE != 0 && b.vsplit > 1)
        e = QL_FN(launch_density_)(Q, b.out, b.nx, b.stride, b.nout, s);
    return e;
}

template <int Q, bool RET>
static cudaError_t stage_dispatch_ret(int stage, const StageArgs &a, cudaStream_t s)
{
    switch (stage) {
    case 0: return stage_q<Q, 0, RET>(a, s);
    case 1: return stage_q<Q, 1, RET>(a, s);
    case 2: return stage_q<Q, 2, RET>(a, s);
    case 3: return stage_q<Q, 3, RET>(a, s);
    }
    return cudaErrorInvalidValue;
}

// chi_RET-FM kernels when the averaged densities are given (a.nbar, and a.nout
// for stages 1-3), chi_SET kernels otherwise.
template <int Q>
static cudaError_t stage_dispatch(int stage, const StageArgs &a, cudaStream_t s)
{
    if (a.nbar != nullptr) {
        if (stage != 0 && a.nout == nullptr) return cudaErrorInvalidValue;
        return stage_dispatch_ret<Q, true>(stage, a, s);
    }
    return stage_dispatch_ret<Q, false>(stage, a, s);
}

cudaError_t QL_FN(launch_stage_)(int Q, int stage, const StageArgs &a, cudaStream_t s)
{
    switch (Q) {
    case 8: return stage_dispatch<8>(stage, a, s);
    case 16: return stage_dispatch<16>(stage, a, s);
    case 20: return stage_dispatch<20>(stage, a, s);
    case 24: return stage_dispatch<24>(stage, a, s);
    case 32: return stage_dispatch<32>(stage, a, s);
    case 40: return stage_dispatch<40>(stage, a, s);
    }
    return cudaErrorInvalidValue;
}

// ---- batched stages
template <int Q, int STAGE, int WARPS, bool RET = false>
static cudaError_t batch_qsw(int grid, const BatchArgs &b, cudaStream_t s, bool query, int *ctas)
{
    constexpr size_t smem = stage_smem_bytes<QL_REAL, Q, WARPS, RET>();
    auto kern = fdlb_batch_stage_kernel<QL_REAL, Q, STAGE, WARPS, RET>;
    static bool configured[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (!configured[dev & 63]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        configured[dev & 63] = true;
    }
    if (query) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, kern, 32 * WARPS, smem);
    kern<<<dim3(unsigned(grid)), dim3(32 * WARPS), smem, s>>>(b);
    return cudaGetLastError();
}

template <int Q, int WARPS, bool RET = false>
static cudaError_t batch_qw(int stage, int grid, const BatchArgs &b, cudaStream_t s, bool query, int *ctas)
{
    switch (stage) {
    case 1: return batch_qsw<Q, 1, WARPS, RET>(grid, b, s, query, ctas);
    case 2: return batch_qsw<Q, 2, WARPS, RET>(grid, b, s, query, ctas);
    case 3: return batch_qsw<Q, 3, WARPS, RET>(grid, b, s, query, ctas);
    }
    return cudaErrorInvalidValue;
}

template <int WARPS, bool RET = false>
static cudaError_t batch_w(int Q, int stage, int grid, const BatchArgs &b, cudaStream_t s, bool query, int *ctas)
{
    switch (Q) {
    case 8: return batch_qw<8, WARPS, RET>(stage, grid, b, s, query, ctas);
    case 16: return batch_qw<16, WARPS, RET>(stage, grid, b, s, query, ctas);
    case 24: return batch_qw<24, WARPS, RET>(stage, grid, b, s, query, ctas);
    case 32: return batch_qw<32, WARPS, RET>(stage, grid, b, s, query, ctas);
    }
    return cudaErrorInvalidValue;
}

cudaError_t QL_FN(launch_batch_stage_)(int Q, int stage, int warps, int grid, const BatchArgs &b, cudaStream_t s)
{
    if (warps == 8) return batch_w<8>(Q, stage, grid, b, s, false, nullptr);
    if (warps == 4) return batch_w<4>(Q, stage, grid, b, s, false, nullptr);
    return cudaErrorInvalidValue;
}

// Resident CTAs per SM of the largest velocity set's kernel (the most shared memory).
cudaError_t QL_FN(launch_batch_stage_ret_)(int Q, int stage, int grid, const BatchArgs &b, cudaStream_t s)
{
    return batch_w<8, true>(Q, stage, grid, b, s, false, nullptr);
}

cudaError_t QL_FN(launch_batch_fm_)(const BatchFmArgs &a, int max_w, cudaStream_t s)
{
    if (max_w < 0 || max_w > QL_FM_MAX_HALFWIDTH || a.nwork <= 0 || a.nwork > INT32_MAX) return cudaErrorInvalidValue;
    const size_t smem = sizeof(QL_REAL) * (kFmThreads + 4 * size_t(max_w) + 1);
    fdlb_batch_fm_kernel<QL_REAL><<<unsigned(a.nwork), kFmThreads, smem, s>>>(a);
    return cudaGetLastError();
}

int QL_FN(batch_ctas_per_sm_)(int stage, int warps)
{
    int n = 0;
    cudaError_t e = warps == 8 ? batch_w<8>(kBatchMaxQ, stage, 0, BatchArgs{}, nullptr, true, &n)
                               : batch_w<4>(kBatchMaxQ, stage, 0, BatchArgs{}, nullptr, true, &n);
    return e == cudaSuccess ? n : 0;
}

cudaError_t QL_FN(launch_init_)(int Q, const double *rho, const double *u, const double *T, void *psi,
                                int64_t nx, int64_t stride, const double *tab64, cudaStream_t s)
{
    const int64_t n = nx + 2 * kHalo;  // one thread per column
    const unsigned blocks = unsigned((n + 255) / 256);
    P2<QL_REAL> *p = static_cast<P2<QL_REAL> *>(psi);
    switch (Q) {
    case 8: fdlb_init_kernel<QL_REAL, 8><<<blocks, 256, 0, s>>>(rho, u, T, p, nx, stride, tab64); break;
    case 16: fdlb_init_kernel<QL_REAL, 16><<<blocks, 256, 0, s>>>(rho, u, T, p, nx, stride, tab64); break;
    case 20: fdlb_init_kernel<QL_REAL, 20><<<blocks, 256, 0, s>>>(rho, u, T, p, nx, stride, tab64); break;
    case 24: fdlb_init_kernel<QL_REAL, 24><<<blocks, 256, 0, s>>>(rho, u, T, p, nx, stride, tab64); break;
    case 32: fdlb_init_kernel<QL_REAL, 32><<<blocks, 256, 0, s>>>(rho, u, T, p, nx, stride, tab64); break;
    case 40: fdlb_init_kernel<QL_REAL, 40><<<blocks, 256, 0, s>>>(rho, u, T, p, nx, stride, tab64); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t QL_FN(launch_periodic_ghosts_)(int Q, void *psi, int64_t nx, int64_t stride, cudaStream_t s)
{
    P2<QL_REAL> *p = static_cast<P2<QL_REAL> *>(psi);
    fdlb_periodic_ghost_kernel<QL_REAL><<<Q, 32, 0, s>>>(p, nx, stride);
    return cudaGetLastError();
}

cudaError_t QL_FN(launch_density_)(int Q, const void *psi, int64_t nx, int64_t stride, void *n, cudaStream_t s)
{
    const P2<QL_REAL> *p = static_cast<const P2<QL_REAL> *>(psi);
    QL_REAL *out = static_cast<QL_REAL *>(n);
    const unsigned blocks = unsigned((nx + 255) / 256);
    switch (Q) {
    case 8: fdlb_density_kernel<QL_REAL, 8><<<blocks, 256, 0, s>>>(p, nx, stride, out); break;
    case 16: fdlb_density_kernel<QL_REAL, 16><<<blocks, 256, 0, s>>>(p, nx, stride, out); break;
    case 20: fdlb_density_kernel<QL_REAL, 20><<<blocks, 256, 0, s>>>(p, nx, stride, out); break;
    case 24: fdlb_density_kernel<QL_REAL, 24><<<blocks, 256, 0, s>>>(p, nx, stride, out); break;
    case 32: fdlb_density_kernel<QL_REAL, 32><<<blocks, 256, 0, s>>>(p, nx, stride, out); break;
    case 40: fdlb_density_kernel<QL_REAL, 40><<<blocks, 256, 0, s>>>(p, nx, stride, out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t QL_FN(launch_fm_)(const FmArgs &a, cudaStream_t s)
{
    if (a.W < 0 || a.W > QL_FM_MAX_HALFWIDTH) return cudaErrorInvalidValue;
    const size_t smem = sizeof(QL_REAL) * (kFmThreads + 4 * size_t(a.W) + 1);
    const unsigned blocks = unsigned((a.nx + 2 * kHalo + kFmThreads - 1) / kFmThreads);
    fdlb_fm_kernel<QL_REAL><<<blocks, kFmThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t QL_FN(launch_moments_)(int Q, const MomentArgs &a, const double *tab64, cudaStream_t s)
{
    const unsigned blocks = unsigned(moment_blocks(a.nx));
    if constexpr (sizeof(QL_REAL) == 4) {
        if (!a.sums64 && !(a.rho || a.u || a.T || a.P || a.q || a.Pxx)) {  // totals only, double-FP32 sums
            switch (Q) {
            case 8: fdlb_totals_f32_kernel<8><<<blocks, kMomThreads, 0, s>>>(a, tab64); break;
            case 16: fdlb_totals_f32_kernel<16><<<blocks, kMomThreads, 0, s>>>(a, tab64); break;
            case 20: fdlb_totals_f32_kernel<20><<<blocks, kMomThreads, 0, s>>>(a, tab64); break;
            case 24: fdlb_totals_f32_kernel<24><<<blocks, kMomThreads, 0, s>>>(a, tab64); break;
            case 32: fdlb_totals_f32_kernel<32><<<blocks, kMomThreads, 0, s>>>(a, tab64); break;
            case 40: fdlb_totals_f32_kernel<40><<<blocks, kMomThreads, 0, s>>>(a, tab64); break;
            default: return cudaErrorInvalidValue;
            }
            return cudaGetLastError();
        }
    }
    switch (Q) {
    case 8: fdlb_moments_kernel<QL_REAL, 8><<<blocks, kMomThreads, 0, s>>>(a, tab64); break;
    case 16: fdlb_moments_kernel<QL_REAL, 16><<<blocks, kMomThreads, 0, s>>>(a, tab64); break;
    case 20: fdlb_moments_kernel<QL_REAL, 20><<<blocks, kMomThreads, 0, s>>>(a, tab64); break;
    case 24: fdlb_moments_kernel<QL_REAL, 24><<<blocks, kMomThreads, 0, s>>>(a, tab64); break;
    case 32: fdlb_moments_kernel<QL_REAL, 32><<<blocks, kMomThreads, 0, s>>>(a, tab64); break;
    case 40: fdlb_moments_kernel<QL_REAL, 40><<<blocks, kMomThreads, 0, s>>>(a, tab64); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace qlbm
