// FP64 Newton series of small grids in one thread-block cluster
// (cluster_f64.cu).
#pragma once
#include "ad_internal.h"

namespace ad {

// Runs the whole FP64 Newton series -- the phi_1 form, or the augmented form
// of two-stage quadrature (a.aug) -- and, with fuse (s == 1 or 2, matching
// a.aug), the whole exponential step, in one cluster launch of up to 16 CTAs
// whose shared memory holds the grid.  Returns 10 when launched, 0 when the
// grid or the request does not fit (the caller then runs the other paths).
// AD_F64_CLUSTER=0 turns it off.
int series_run_cluster(const SeriesArgs& a, cudaStream_t s, const StepFuse* fuse);

}  // namespace ad
