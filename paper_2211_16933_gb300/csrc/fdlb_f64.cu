// FP64 kernels: everything in FP64.
#include "qlbm_internal.h"
namespace qlbm {
static __constant__ double QL_TAB[kTabTotal];
}
#define QL_REAL double
#define QL_SUFFIX f64
#include "fdlb_impl.cuh"
#include "fdlb_lq.cuh"
