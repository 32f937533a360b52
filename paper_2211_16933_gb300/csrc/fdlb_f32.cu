// FP32 kernels: state, fluxes and update in FP32; per-cell conserved-moment
// sums combined in double-FP32, domain totals in FP64.
#include "qlbm_internal.h"
namespace qlbm {
// 16-byte aligned: the stage kernels read the table rows as pairs.
static __constant__ __align__(16) float QL_TAB[kTabTotal];
}
#define QL_REAL float
#define QL_SUFFIX f32
#include "fdlb_impl.cuh"

namespace qlbm {
// Per device: the kernel's shared-memory limit set, and the CTAs it holds at once.
template <int Q>
static cudaError_t run_setup(int64_t *resident_out)
{
    constexpr size_t smem = stage_smem_bytes<float, Q, kWarps, false>();
    auto kern = fdlb_run_kernel<Q>;
    static int64_t resident[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (!resident[dev & 63]) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        int per_sm = 0, sms = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        resident[dev & 63] = int64_t(per_sm) * sms;
    }
    if (resident_out) *resident_out = resident[dev & 63];
    return cudaSuccess;
}

// A run of `steps` steps: one CTA per (stage, tile) ticket.
template <int Q>
static cudaError_t run_q(const RunArgs &r, int64_t steps, cudaStream_t s)
{
    constexpr size_t smem = stage_smem_bytes<float, Q, kWarps, false>();
    auto kern = fdlb_run_kernel<Q>;
    const cudaError_t e = run_setup<Q>(nullptr);
    if (e != cudaSuccess) return e;
    const int64_t tickets = 3 * steps * r.ntiles;
    if (tickets <= 0) return cudaSuccess;
    if (tickets > int64_t(kRunMaxTickets)) return cudaErrorInvalidValue;
    // programmatic stream serialisation, as for the stage kernels
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(tickets));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, r);
}

bool run_supported_f32(int Q) { return Q == 8 || Q == 16 || Q == 20 || Q == 24 || Q == 32 || Q == 40; }

int64_t run_resident_f32(int Q)
{
    int64_t n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (Q) {
    case 8: e = run_setup<8>(&n); break;
    case 16: e = run_setup<16>(&n); break;
    case 20: e = run_setup<20>(&n); break;
    case 24: e = run_setup<24>(&n); break;
    case 32: e = run_setup<32>(&n); break;
    case 40: e = run_setup<40>(&n); break;
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_run_f32(int Q, const RunArgs &r, int64_t steps, cudaStream_t s)
{
    switch (Q) {
    case 8: return run_q<8>(r, steps, s);
    case 16: return run_q<16>(r, steps, s);
    case 20: return run_q<20>(r, steps, s);
    case 24: return run_q<24>(r, steps, s);
    case 32: return run_q<32>(r, steps, s);
    case 40: return run_q<40>(r, steps, s);
    }
    return cudaErrorInvalidValue;
}
}  // namespace qlbm
