// FP64 kernels: everything in FP64.
#include "qlbm_internal.h"
namespace qlbm {
// 16-byte aligned: the stage kernels read the table rows as pairs.
static __constant__ __align__(16) double QL_TAB[kTabTotal];
}
#define QL_REAL double
#define QL_SUFFIX f64
#include "fdlb_impl.cuh"
#include "fdlb_lq.cuh"
