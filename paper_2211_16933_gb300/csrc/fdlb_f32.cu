// FP32 kernels: state, fluxes and update in FP32; per-cell conserved-moment
// sums combined in double-FP32, domain totals in FP64.
#include "qlbm_internal.h"
namespace qlbm {
static __constant__ float QL_TAB[kTabTotal];
}
#define QL_REAL float
#define QL_SUFFIX f32
#include "fdlb_impl.cuh"
