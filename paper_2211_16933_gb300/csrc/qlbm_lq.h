// Host interface of the generic-Q FP64 path's chi_RET-FM form (Eq. chi_ret).
#pragma once
#include "qlbm_internal.h"

namespace qlbm {

// One stage with chi_RET-FM: the cell moments of the stage input, then nbar of
// every column averaged over the ball from the densities the moments kernel
// wrote (f.n must be a.mom + kHalo, the interior cells' densities; f.nbar
// receives nx + 2 kHalo doubles), then the collision coefficients with
// chi_SET(nbar) and the 6th-order difference of ln chi_SET(nbar), then the
// update.  Same errors as launch_lq_stage, plus cudaErrorInvalidValue for a
// ball wider than QL_FM_MAX_HALFWIDTH cells.
cudaError_t launch_lq_stage_ret(int stage, const LqArgs &a, const FmArgs &f, cudaStream_t s);

}  // namespace qlbm
