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
