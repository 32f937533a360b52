// ql_step_noalloc: Runge-Kutta steps of a caller-owned state with no device
// allocation.  The two intermediate stage buffers and the error word live in a
// fixed scratch array that this library reserves in device memory when it is
// loaded, so callers that must not allocate can still advance a state.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>
#include <string>

#include "../../include/qlbm.h"
#include "qlbm_host.h"
#include "qlbm_internal.h"

using namespace qlbm;

// Size of the scratch array (bytes); the largest state this entry point accepts
// has two stage buffers of Q * row_stride pairs within it.
#define QL_NOALLOC_SCRATCH_BYTES size_t(QL_NOALLOC_MAX_BYTES)

namespace qlbm {
void set_global_error(const std::string &msg);  // ql_last_error(NULL), qlbm_api.cu
}

namespace {

// Scratch for every call: a 256-byte header holding the device error word,
// then psi^(1) and psi^(2), each Q rows of row_stride (phi, theta) pairs.  Every
// GPU that loads the library holds this array until the process exits.
constexpr size_t kScratchBytes = size_t(QL_NOALLOC_SCRATCH_BYTES);
constexpr size_t kHeaderBytes = 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct DeviceSetup {
    bool ready = false;
    unsigned char *scratch = nullptr;  // device address of g_noalloc_scratch
};
static DeviceSetup g_setup[64];
static std::mutex g_setup_mutex;
ql_status nfail(ql_status st, const std::string &m)
{
    set_global_error(m);
    return st;
}

// Once per device, with that device current: the kernel tables and the device
// address of the scratch array.  In host code the array's name is only a
// host-side stand-in, so kernels get the address from cudaGetSymbolAddress.
ql_status setup_device(int device, unsigned char **scratch)
{
    std::lock_guard<std::mutex> lk(g_setup_mutex);
    DeviceSetup &d = g_setup[device & 63];
    if (!d.ready) {
        std::string terr;
        if (!ensure_device_tables(device, terr)) return nfail(QL_ECUDA, terr);
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return nfail(QL_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        d.scratch = static_cast<unsigned char *>(p);
        d.ready = true;
    }
    *scratch = d.scratch;
    return QL_OK;
}

}  // namespace

extern "C" {

ql_status ql_step_noalloc(const ql_velset *vs, const ql_grid *grid, double denseness, double kn, const ql_bc *bc,
                          const ql_opts *opts, void *psi, int64_t row_stride, int64_t nsteps)
{
    if (!vs || !grid || !bc || !opts || !psi || nsteps < 0) return nfail(QL_EINVAL, "null argument or nsteps < 0");
    bool qok = false;
    for (int j = 0; j < kNumQ; ++j) qok |= vs->Q == kQList[j];
    if (!qok || vs->kind != 0) return nfail(QL_EUNSUPPORTED, "Q must be one of 8, 16, 20, 24, 32, 40");
    if (grid->nx < 8 || grid->nx > (int64_t(1) << 31) || !(grid->length > 0) || !(grid->dt > 0))
        return nfail(QL_EINVAL, "bad grid");
    if (!(denseness > 0) || !(kn > 0) || !(opts->rho_ref > 0)) return nfail(QL_EINVAL, "bad gas parameters");
    if (bc->kind != QL_BC_PERIODIC && bc->kind != QL_BC_FIXED) return nfail(QL_EINVAL, "bad bc kind");
    if (opts->precision != QL_FP32 && opts->precision != QL_FP64) return nfail(QL_EINVAL, "bad precision");
    if (opts->pr_mode == QL_PR_CONST && !(opts->pr_const > 0)) return nfail(QL_EINVAL, "bad pr_const");
    if (opts->chi_mode != QL_CHI_SET)
        return nfail(QL_EUNSUPPORTED, "ql_step_noalloc supports chi_SET only (chi_RET-FM needs density buffers)");
    if (opts->sums != QL_SUMS_DFP32 && opts->sums != QL_SUMS_FP64) return nfail(QL_EINVAL, "bad sums");
    if (row_stride < qlbm::row_stride(grid->nx))
        return nfail(QL_EINVAL, "row_stride " + std::to_string(row_stride) + " is below the " +
                                    std::to_string(qlbm::row_stride(grid->nx)) + " pairs this nx needs");
    const size_t elem = opts->precision == QL_FP32 ? 8 : 16;
    // the largest row_stride whose two stage buffers fit, checked before any
    // product that could overflow
    if (uint64_t(row_stride) > (kScratchBytes - kHeaderBytes) / (2 * size_t(vs->Q) * elem))
        return nfail(QL_EINVAL, "state of row_stride " + std::to_string(row_stride) + " exceeds the " +
                                    std::to_string(kScratchBytes) + "-byte scratch (two stage buffers)");
    // psi points at cell 0 of row 0; the buffer starts at the first ghost column
    void *rows = static_cast<unsigned char *>(psi) - kHalo * elem;
    if (reinterpret_cast<uintptr_t>(rows) % 16 != 0 || (size_t(row_stride) * elem) % 16 != 0)
        return nfail(QL_EINVAL, "state rows must be 16-byte aligned (FP32: row_stride must be even)");
    const size_t buf = size_t(vs->Q) * size_t(row_stride) * elem;
    if (kHeaderBytes + 2 * buf > kScratchBytes)
        return nfail(QL_EINVAL, "state of " + std::to_string(buf) + " bytes per stage buffer exceeds the " +
                                    std::to_string(kScratchBytes) + "-byte scratch (two stage buffers)");
    double eta0;
    if (!eta_of_denseness(denseness, &eta0)) return nfail(QL_EINVAL, "denseness out of range");

    int prev = 0;
    cudaGetDevice(&prev);
    cudaError_t e = cudaSetDevice(opts->device);
    if (e != cudaSuccess) return nfail(QL_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    unsigned char *scratch = nullptr;
    ql_status st = setup_device(opts->device, &scratch);
    if (st != QL_OK) {
        cudaSetDevice(prev);
        return st;
    }
    cudaStream_t s = static_cast<cudaStream_t>(opts->stream);
    unsigned *err = reinterpret_cast<unsigned *>(scratch);
    unsigned char *B = scratch + kHeaderBytes, *C = B + buf;
    const int64_t nx = grid->nx, pitch = row_stride * int64_t(elem);
    // the scratch keeps the previous call's contents: clear the error word, and
    // give both stage buffers this state's ghost columns (fixed states, or the
    // periodic images that the stage kernels then keep up to date)
    e = cudaMemsetAsync(err, 0, sizeof(unsigned), s);
    const unsigned char *src = static_cast<const unsigned char *>(rows);
    for (unsigned char *dst : {B, C}) {
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(dst, pitch, src, pitch, kHalo * elem, vs->Q, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(dst + (kHalo + nx) * elem, pitch, src + (kHalo + nx) * elem, pitch, kHalo * elem,
                                  vs->Q, cudaMemcpyDeviceToDevice, s);
    }
    StageArgs a;
    a.nx = nx;
    a.stride = row_stride;
    a.inv_dx = 1.0 / (grid->length / double(nx));
    a.dt = grid->dt;
    a.eta0 = eta0;
    a.inv_rho_ref = 1.0 / opts->rho_ref;
    a.tau_pref = tau_prefactor(kn, grid->length, eta0);
    a.pr_const = opts->pr_const;
    a.pr_mode = opts->pr_mode;
    a.enskog = opts->enskog ? 1 : 0;
    a.periodic = bc->kind == QL_BC_PERIODIC;
    a.fault = 0;
    a.sums64 = opts->precision == QL_FP32 && opts->sums == QL_SUMS_FP64;
    a.vsplit = 1;  // the launcher picks the FP64 split
    a.err = err;
    a.nbar = nullptr;
    a.nout = nullptr;
    a.base = rows;
    for (int64_t n = 0; n < nsteps && e == cudaSuccess; ++n) {
        void *ins[3] = {rows, B, C}, *outs[3] = {B, C, rows};
        for (int stg = 1; stg <= 3 && e == cudaSuccess; ++stg) {
            a.in = ins[stg - 1];
            a.out = outs[stg - 1];
            e = opts->precision == QL_FP32 ? launch_stage_f32(vs->Q, stg, a, s) : launch_stage_f64(vs->Q, stg, a, s);
        }
    }
    unsigned h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaSetDevice(prev);
    if (e != cudaSuccess) return nfail(QL_ECUDA, std::string("ql_step_noalloc: ") + cudaGetErrorString(e));
    if (h & 2u) return nfail(QL_ECUDA, "a stage kernel gave up waiting for its tile's TMA copies");
    if (h & 1u) return nfail(QL_ENONPHYSICAL, "non-physical state: n <= 0, T <= 0 or non-finite moments");
    return QL_OK;
}

}  // extern "C"
