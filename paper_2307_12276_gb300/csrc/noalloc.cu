// ad_leja_phi1_noalloc: phi_1(dt A) v for callers that cannot allocate device
// memory.
//
// Some callers may not call cudaMalloc at all: code that runs inside a host
// framework which owns the device heap (and hands out only the buffers it
// manages), code running under a memory budget that forbids allocation
// after start-up, or code on a path where an allocation's implicit device
// synchronisation is not acceptable.  ad_create_operator allocates the
// packed coefficients and the series workspace, so such callers cannot use
// it.  This entry point keeps every scratch buffer it needs (the packed and
// scaled 9-point weights, the two Newton basis vectors, the partial sum, the
// per-iteration Leja scalars, the control block and the norm partials) in one
// file-scope __device__ array of fixed size, so nothing is allocated: the
// caller passes the coefficient fields, the input vector and the output
// vector, all on the device.
//
// Limits and caveats:
//   * at most kNoAllocMaxCells = 65536 cells (for example 256 x 256); larger
//     grids are rejected with AD_ERR_INVALID.  The array occupies about
//     6.4 MB on every GPU that loads the library, until the process exits;
//   * FP64 only, constant advection only, one substep (rho = gamma dt <= 200);
//   * every call shares the array and it keeps the previous call's contents:
//     calls that overlap on the GPU (two streams, two host threads) race on
//     it and must be serialised by the caller;
//   * every call looks up the array's device address on the current device
//     (cudaGetSymbolAddress, which allocates nothing), so the address is
//     never stale, even after the primary context was reset and the module
//     reloaded at another address.  The first call on a device may load the
//     module: make it before any stream capture.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "ad_internal.h"
#include "anidiff.h"
#include "leja_host.h"

namespace {

using namespace ad;

constexpr long long kNoAllocMaxCells = 1LL << 16;
constexpr int kNoAllocMaxBlocks = 152 * 8;   // upper bound of stream_blocks()
constexpr double kNoAllocRhoMax = 200.0;

struct NoAllocScratch {
  double weights[9 * kNoAllocMaxCells];   // packed, then scaled in place to (W - c)/gamma
  double y[2][kNoAllocMaxCells];          // Newton basis ping-pong
  double p[kNoAllocMaxCells];             // partial sum
  double partials[2 * kNoAllocMaxBlocks];
  LejaCoef lc[kMaxIters];
  Ctrl ctrl;
  double scal[4];
};

// The scratch itself.  In host code this name is only a stand-in: host code
// must use the address from cudaGetSymbolAddress (see scratch_on_device).
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

int nfail(int code, const std::string& msg) {
  set_error_message(msg.c_str());   // reported by ad_last_error()
  return code;
}

// Device address of the scratch on the current device, looked up on every
// call: a saved address could outlive the context it belongs to.
int scratch_on_device(NoAllocScratch** out) {
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess || !ptr) {
    cudaGetLastError();
    return nfail(AD_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  }
  *out = static_cast<NoAllocScratch*>(ptr);
  return AD_OK;
}

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

#define NA_CUDA(expr)                                                                    \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      cudaGetLastError();                                                                \
      return nfail(AD_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));     \
    }                                                                                    \
  } while (0)

}  // namespace

extern "C" int ad_leja_phi1_noalloc(const ad_grid* grid, const double* Dxx, const double* Dxy,
                                    const double* Dyy, double ax_c, double ay_c, double alpha,
                                    const double* v, double* out, double dt, double tol,
                                    int force_iters, void* cuda_stream, ad_stats* stats) {
  set_error_message("");
  if (!grid || !Dxx || !Dxy || !Dyy || !v || !out) return nfail(AD_ERR_INVALID, "NULL argument");
  if (grid->nx < 1 || grid->ny < 1) return nfail(AD_ERR_INVALID, "grid: nx, ny must be >= 1");
  const long long n = (long long)grid->nx * grid->ny;
  if (n > kNoAllocMaxCells)
    return nfail(AD_ERR_INVALID, "grid too large for the no-allocation variant: at most 65536 "
                                 "cells (use ad_create_operator + ad_leja_phi1)");
  if (!(grid->x1 > grid->x0) || !(grid->y1 > grid->y0)) return nfail(AD_ERR_INVALID, "grid: empty domain");
  if (grid->bc != AD_BC_PERIODIC && grid->bc != AD_BC_DIRICHLET0) return nfail(AD_ERR_INVALID, "grid: bad bc");
  if (!(dt > 0) || !std::isfinite(dt)) return nfail(AD_ERR_INVALID, "dt must be positive");
  if (force_iters > kMaxIters) return nfail(AD_ERR_INVALID, "force_iters > 500");
  if (force_iters < 0 && !(tol > 0)) return nfail(AD_ERR_INVALID, "tol must be positive");
  if (alpha > 0 || !std::isfinite(alpha)) return nfail(AD_ERR_INVALID, "alpha must be <= 0 (0: Gershgorin)");
  for (const void* p : {(const void*)Dxx, (const void*)Dxy, (const void*)Dyy, (const void*)v, (const void*)out})
    if (!on_device(p)) return nfail(AD_ERR_INVALID, "all arrays must be device pointers");
  cudaGetLastError();

  NoAllocScratch* S = nullptr;
  {
    const int r = scratch_on_device(&S);
    if (r != AD_OK) return r;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  GridDev g{grid->nx, grid->ny, grid->bc, n};
  const double dx = (grid->x1 - grid->x0) / grid->nx, dy = (grid->y1 - grid->y0) / grid->ny;
  const int nb = stream_blocks(n);
  const long long l0 = launch_counter();

  pack_weights_f64(g, dx, dy, Dxx, Dxy, Dyy, nullptr, nullptr, ax_c, ay_c, S->weights, s);
  if (alpha == 0.0) {  // Gershgorin (Section 2)
    gershgorin_partials_f64(g, S->weights, S->partials, nb, s);
    reduce_partials(S->partials, nb, 1, S->scal, s);
    double a = 0.0;
    NA_CUDA(cudaMemcpyAsync(&a, S->scal, sizeof(double), cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaStreamSynchronize(s));
    // the same refusal as ad_spectral_bound: a bound >= 0 defines no Leja interval
    if (!(a < 0.0)) return nfail(AD_ERR_INVALID, "spectral bound is not negative (A == 0?)");
    alpha = a;
  }
  const double c = alpha / 2.0, gamma = -alpha / 4.0;
  if (gamma * dt > kNoAllocRhoMax)
    return nfail(AD_ERR_INVALID, "dt too large for the no-allocation variant "
                                 "(gamma dt > 200): split the step");
  scale_weights_f64(g, S->weights, c, gamma, S->weights, s);   // in place, per element

  // Leja scalars for f(xi) = phi_1((c + gamma xi) dt): host stack only
  const std::vector<double>& xi = leja_points();
  double f[kMaxIters + 1], d[kMaxIters + 1];
  for (int m = 0; m <= kMaxIters; ++m) f[m] = phi1((c + gamma * xi[m]) * dt);
  divided_differences(xi.data(), f, kMaxIters + 1, d);
  LejaCoef hlc[kMaxIters];
  for (int m = 0; m < kMaxIters; ++m)
    hlc[m] = LejaCoef{xi[m], d[m + 1], std::fabs(d[m + 1]), 0.0, 0.0, {0.0, 0.0, 0.0}};
  NA_CUDA(cudaMemcpyAsync(S->lc, hlc, sizeof(hlc), cudaMemcpyHostToDevice, s));

  SeriesArgs a{};
  a.g = g;
  a.prec = 0;
  a.coef = S->weights;
  a.c = c;
  a.gamma = gamma;
  a.y[0] = S->y[0];
  a.y[1] = S->y[1];
  a.p = S->p;
  a.lc = S->lc;
  a.ctrl = &S->ctrl;
  a.partials = S->partials;
  a.nblocks = series_blocks(0, n);
  const int force = force_iters < 0 ? -1 : force_iters;
  series_init(a, v, d[0], force, kMaxIters, tol, s);
  Ctrl hc{};
  if (force != 0) {
    int launched = 0;
    for (;;) {   // host-driven: chunks of iterations, then poll the stop flag
      for (int k = 0; k < 16; ++k) series_iteration(a, s);
      launched += 16;
      NA_CUDA(cudaGetLastError());
      NA_CUDA(cudaMemcpyAsync(&hc, &S->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
      NA_CUDA(cudaStreamSynchronize(s));
      if (hc.stop || launched >= kMaxIters + 16) break;
    }
    if (!hc.stop) return nfail(AD_ERR_TIMEOUT, "Leja series did not reach its stop state");
    hc.err_est = hc.pnorm2 > 0.0 ? hc.err_est * std::sqrt(hc.ynorm2 / hc.pnorm2)
                                 : (hc.ynorm2 > 0.0 ? INFINITY : 0.0);
  }
  axpby(0, n, 1.0, S->p, 0.0, nullptr, out, s);
  NA_CUDA(cudaGetLastError());
  NA_CUDA(cudaStreamSynchronize(s));
  if (stats) {
    *stats = ad_stats{};
    stats->iters = hc.iters;
    stats->matvecs = hc.iters;
    stats->substeps = 1;
    stats->converged = hc.status == 0;
    stats->err_est = hc.err_est;
    stats->alpha = alpha;
    stats->kernel_launches = (int)(launch_counter() - l0);
  }
  if (hc.status != 0) return nfail(AD_ERR_NOT_CONVERGED, "Leja series reached max_iters");
  return AD_OK;
}
