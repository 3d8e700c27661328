// Per-iteration epilogue of the one-launch-per-iteration Newton series
// kernels, shared by the translation units that define such kernels.
#pragma once
#include "tile_f32.cuh"

namespace ad {
namespace {

// Per-iteration epilogue of the Newton series (Section 2): publish the block's
// norm partials; the last block of the launch (ticket, no waiting) reduces all
// partials in block order, applies the stopping rule
//   |d_{m+1}| ||y_{m+1}|| <= tol ||p_{m+1}||  (m+1 >= 2), or the forced count,
// advances m and sets the graph loop condition.  The series always ends: m
// grows by one per launch and the rule stops at max_iters <= kMaxIters.
__device__ void series_finish(const SeriesArgs& a, double sy, double sp) {
  __shared__ unsigned int s_last;
  block_sum2(sy, sp);
  Ctrl* ctrl = a.ctrl;
  if (threadIdx.x == 0) {
    a.partials[2 * blockIdx.x] = sy;
    a.partials[2 * blockIdx.x + 1] = sp;
    __threadfence();
    const unsigned int t = atomicAdd(&ctrl->ticket, 1u);
    s_last = (t == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double ty = 0.0, tp = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    ty += __ldcg(&a.partials[2 * b]);
    tp += __ldcg(&a.partials[2 * b + 1]);
  }
  block_sum2(ty, tp);
  if (threadIdx.x == 0) {
    const int m = ctrl->m;
    const int terms = m + 1;
    const double absd = a.lc[m].absd;
    ctrl->ynorm2 = ty;
    ctrl->pnorm2 = tp;
    ctrl->iters = terms;
    ctrl->err_est = absd;           // the host forms |d| ||y|| / ||p|| from the squares
    const double tol = ctrl->tol;
    int stop = 0;
    if (ctrl->force > 0) {
      stop = terms >= ctrl->force;
    } else if (!isfinite(ty) || !isfinite(tp)) {   // NaN or overflow: give up
      stop = 1;
      ctrl->status = 3;
    } else if (terms >= 2 && (absd * absd) * ty <= (tol * tol) * tp) {   // squared test
      stop = 1;
    } else if (terms >= ctrl->max_iters) {
      stop = 1;
      ctrl->status = 3;
    }
    if (terms >= kMaxIters) stop = 1;               // hard cap, independent of the settings
    if (ctrl->status == 4) stop = 1;                // a bounded wait gave up in this launch
    ctrl->ticket = 0u;
    ctrl->stop = stop;
    ctrl->m = m + 1;
    __threadfence();
    if (a.has_handle)
      cudaGraphSetConditional((cudaGraphConditionalHandle)a.handle, stop ? 0u : 1u);
  }
}

}  // namespace
}  // namespace ad
