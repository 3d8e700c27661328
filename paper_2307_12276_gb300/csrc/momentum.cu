// Transport with momentum coupling (Eq. cr_full, Section 1) and its Leja
// phi_1 series (Section 2) on the grid (p, y, x).
//
// Eq. cr_full adds to the spatial terms of Eq. anidiff the momentum terms
//   d/dp( p^2 D_pp d/dp(u / p^2) ) - d/dp( (pdot - (p/3) div v) u ) - (1/tau_f + 1/tau_r) u.
// The paper integrates only the two-dimensional equation; the readings here:
//   * np momentum cells with faces P_0 < ... < P_np, centres
//     p_k = sqrt(P_k P_{k+1}), widths dP_k = P_{k+1} - P_k;
//   * D(x, y, p_k) = beta_k D(x, y); the advection a does not depend on p;
//   * D_pp and b = pdot - (p/3) div v at the faces, loss rates per cell;
//   * finite volumes in p, no flux through P_0 and P_np:
//       F_{k+1/2} = P_{k+1}^2 D_pp (u_{k+1}/p_{k+1}^2 - u_k/p_k^2) / (p_{k+1} - p_k)
//       G_{k+1/2} = b (u_k if b >= 0 else u_{k+1})                         (upwind)
//       (A_p u)_k = (F_{k+1/2} - F_{k-1/2} - G_{k+1/2} + G_{k-1/2}) / dP_k - L_k u_k;
//   * unknowns slice-major, index k * n + (j * nx + i).
// So A = blockdiag_k(beta_k A_D + A_a) + M (x) I_n, with A_D and A_a the
// diffusive and advective parts of the 9-point operator of Eq. anidiff
// (packed by pack_weights_f64; the operator is linear in D and a, so the two
// parts pack separately) and M tridiagonal.
//
// Layout: the 9 diffusion weights [9][n] and the 5 non-zero advection weights
// (centre, west, east, south, north) [5][n] are read once per spatial cell
// and reused for all np slices; y, p are [np][n].  A thread owns a spatial
// cell and marches through the slices, keeping y_{k-1}, y_k, y_{k+1} of its
// cell in registers; the 8 spatial neighbours of y_k come through L1/L2.
// Per cell and slice: 16 FP64 operations (21 with advection) and ~32 B of
// DRAM traffic (y_k, p read; y_{k+1} and p written), so the kernel is bound
// by the FP64 pipe like the two-dimensional FP64 kernels.
//
// The series is host driven: chunks of 8 fused iteration launches, then a
// read of the control block; a launch after the stopping one returns at
// once.  The stopping rule and the block-ordered norm sums are those of the
// two-dimensional kernels (series_finish).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "anidiff.h"
#include "ad_internal.h"
#include "leja_host.h"
#include "series_finish.cuh"
#include "sqsum.cuh"

struct ad_momentum_operator;

namespace ad {
namespace {

constexpr int kMomMaxSlices = 1024;
constexpr int kMomChunk = 8;          // iteration launches between control reads

struct MomCoef {       // per momentum slice
  double beta;         // spatial diffusion scale
  double lo, di, up;   // row k of M: coefficients of u_{k-1}, u_k, u_{k+1}
  double slo, sdi, sup;  // Newton operator: lo / gamma, (di - c) / gamma, up / gamma
  double pad;
};

int mfail(int code, const std::string& msg) {
  set_error_message(msg.c_str());
  return code;
}

#define M_CUDA(expr)                                                                     \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      cudaGetLastError();                                                                \
      return mfail(AD_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));    \
    }                                                                                    \
  } while (0)

#define M_TRY(expr)               \
  do {                            \
    int r_ = (expr);              \
    if (r_ != AD_OK) return r_;   \
  } while (0)

// Flat indices of the 9 spatial neighbours in weight-slot order
// (slot = (dj + 1) * 3 + (di + 1)); with zero Dirichlet an out-of-domain slot
// has weight 0 and its index is clamped into the domain.
__device__ __forceinline__ void mom_neighbours(int i, int j, int nx, int ny, int bc, int* o) {
  int im, ip, jm, jp;
  if (bc == 0) {
    im = i ? i - 1 : nx - 1;
    ip = (i + 1 < nx) ? i + 1 : 0;
    jm = j ? j - 1 : ny - 1;
    jp = (j + 1 < ny) ? j + 1 : 0;
  } else {
    im = i ? i - 1 : 0;
    ip = (i + 1 < nx) ? i + 1 : i;
    jm = j ? j - 1 : 0;
    jp = (j + 1 < ny) ? j + 1 : j;
  }
  o[0] = jm * nx + im; o[1] = jm * nx + i; o[2] = jm * nx + ip;
  o[3] = j * nx + im;  o[4] = j * nx + i;  o[5] = j * nx + ip;
  o[6] = jp * nx + im; o[7] = jp * nx + i; o[8] = jp * nx + ip;
}

// advection planes hold slots centre, west, east, south, north
__device__ __constant__ int kAdvSlot[5] = {4, 3, 5, 1, 7};

// beta (sum_9 WD u) + sum_5 WA u at one cell of slice u (u: that slice's base)
template <bool ADV>
__device__ __forceinline__ double mom_spatial(const double* __restrict__ u, const int* o,
                                              const double* wd, const double* wa, double beta,
                                              double uc) {
  double acc = wd[4] * uc;
  acc = fma(wd[0], u[o[0]], acc);
  acc = fma(wd[1], u[o[1]], acc);
  acc = fma(wd[2], u[o[2]], acc);
  acc = fma(wd[3], u[o[3]], acc);
  acc = fma(wd[5], u[o[5]], acc);
  acc = fma(wd[6], u[o[6]], acc);
  acc = fma(wd[7], u[o[7]], acc);
  acc = fma(wd[8], u[o[8]], acc);
  double z = beta * acc;
  if (ADV) {
    z = fma(wa[0], uc, z);
    z = fma(wa[1], u[o[3]], z);
    z = fma(wa[2], u[o[5]], z);
    z = fma(wa[3], u[o[1]], z);
    z = fma(wa[4], u[o[7]], z);
  }
  return z;
}

// out = A u (+ S)
template <bool ADV>
__global__ void mom_apply_k(GridDev g, int np, const double* __restrict__ WD,
                            const double* __restrict__ WA, const MomCoef* __restrict__ mc,
                            const double* __restrict__ u, const double* __restrict__ S,
                            double* __restrict__ out) {
  const long long n = g.n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % g.nx), j = (int)(idx / g.nx);
    int o[9];
    mom_neighbours(i, j, g.nx, g.ny, g.bc, o);
    double wd[9], wa[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int s = 0; s < 9; ++s) wd[s] = WD[s * n + idx];
    if (ADV) {
#pragma unroll
      for (int s = 0; s < 5; ++s) wa[s] = WA[s * n + idx];
    }
    double yp = 0.0, yc = u[idx], yn = np > 1 ? u[n + idx] : 0.0;
    for (int k = 0; k < np; ++k) {
      const double* uk = u + (long long)k * n;
      double z = mom_spatial<ADV>(uk, o, wd, wa, mc[k].beta, yc);
      z = fma(mc[k].lo, yp, z);
      z = fma(mc[k].di, yc, z);
      z = fma(mc[k].up, yn, z);
      if (S) z += S[(long long)k * n + idx];
      out[(long long)k * n + idx] = z;
      yp = yc;
      yc = yn;
      yn = k + 2 < np ? u[(long long)(k + 2) * n + idx] : 0.0;
    }
  }
}

// One fused Newton iteration on all slices: y_{m+1} = ((A - c)/gamma - xi_m) y_m,
// p += d_{m+1} y_{m+1}, norm partials; then the stopping rule (series_finish).
// SQ: the norms' sums of squares on the integer and FP32 pipes (sqsum.cuh),
// two FP64 instructions per unknown fewer; otherwise FP64 FMAs.
template <bool ADV, bool SQ>
__global__ void __launch_bounds__(kThreads) mom_iter_k(SeriesArgs a, int np,
                                                       const double* __restrict__ sWD,
                                                       const double* __restrict__ sWA,
                                                       const MomCoef* __restrict__ mc) {
  extern __shared__ double msm[];            // [4][np]: beta, slo, sdi - xi, sup
  const volatile Ctrl* vc = a.ctrl;
  if (vc->stop) return;
  const int m = vc->m;
  const double xi = a.lc[m].xi, d = a.lc[m].d;
  double* s_beta = msm;
  double* s_lo = msm + np;
  double* s_di = msm + 2 * np;
  double* s_up = msm + 3 * np;
  for (int k = threadIdx.x; k < np; k += blockDim.x) {
    s_beta[k] = mc[k].beta;
    s_lo[k] = mc[k].slo;
    s_di[k] = mc[k].sdi - xi;
    s_up[k] = mc[k].sup;
  }
  __syncthreads();
  const double* __restrict__ yin = static_cast<const double*>(a.y[m & 1]);
  double* __restrict__ yout = static_cast<double*>(a.y[(m + 1) & 1]);
  double* __restrict__ p = static_cast<double*>(a.p);
  const long long n = a.g.n;
  double sy = 0.0, sp = 0.0;
  SqSum qy, qp;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % a.g.nx), j = (int)(idx / a.g.nx);
    int o[9];
    mom_neighbours(i, j, a.g.nx, a.g.ny, a.g.bc, o);
    double wd[9], wa[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int s = 0; s < 9; ++s) wd[s] = sWD[s * n + idx];
    if (ADV) {
#pragma unroll
      for (int s = 0; s < 5; ++s) wa[s] = sWA[s * n + idx];
    }
    double yp = 0.0, yc = yin[idx], yn = np > 1 ? yin[n + idx] : 0.0;
    for (int k = 0; k < np; ++k) {
      const long long base = (long long)k * n;
      double z = mom_spatial<ADV>(yin + base, o, wd, wa, s_beta[k], yc);
      z = fma(s_lo[k], yp, z);
      z = fma(s_di[k], yc, z);
      z = fma(s_up[k], yn, z);
      yout[base + idx] = z;
      const double pv = fma(d, z, p[base + idx]);
      p[base + idx] = pv;
      if (SQ) {
        qy.add(z);
        qp.add(pv);
      } else {
        sy = fma(z, z, sy);
        sp = fma(pv, pv, sp);
      }
      yp = yc;
      yc = yn;
      yn = k + 2 < np ? yin[base + 2 * n + idx] : 0.0;
    }
  }
  if (SQ) {
    sy = qy.value();
    sp = qp.value();
  }
  series_finish(a, sy, sp);
}

// The momentum iteration forms its norms' sums of squares off the FP64 pipe
// unless AD_F64_NORMS=fp64 asks for FP64 FMAs (the rule of the large-grid
// FP64 iteration).
bool mom_int_squares() {
  static const bool on = [] {
    const char* e = getenv("AD_F64_NORMS");
    return !(e && e[0] == 'f');
  }();
  return on;
}

// Gershgorin bound of the coupled operator: min over rows of
// a_ii - sum_{j != i} |a_ij| (spatial slots that reach the same cell merged).
__global__ void mom_gershgorin_k(GridDev g, int np, const double* __restrict__ WD,
                                 const double* __restrict__ WA, const MomCoef* __restrict__ mc,
                                 double* partials) {
  __shared__ double smin[kThreads];
  double mn = 1e308;
  const long long n = g.n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % g.nx), j = (int)(idx / g.nx);
    long long col[9];
    for (int s = 0; s < 9; ++s) {
      const int di = s % 3 - 1, dj = s / 3 - 1;
      int ti = i + di, tj = j + dj;
      if (g.bc == 0) {
        ti = (ti + g.nx) % g.nx;
        tj = (tj + g.ny) % g.ny;
      }
      col[s] = (ti < 0 || tj < 0 || ti >= g.nx || tj >= g.ny) ? -1 : (long long)tj * g.nx + ti;
    }
    for (int k = 0; k < np; ++k) {
      double val[9];
      for (int s = 0; s < 9; ++s) val[s] = mc[k].beta * WD[s * n + idx];
      if (WA)
        for (int q = 0; q < 5; ++q) val[kAdvSlot[q]] += WA[q * n + idx];
      long long c2[9];
      for (int s = 0; s < 9; ++s) c2[s] = col[s];
      for (int s = 0; s < 9; ++s)      // merge slots that reach the same cell
        for (int q = s + 1; q < 9; ++q)
          if (c2[s] >= 0 && c2[q] == c2[s]) { val[s] += val[q]; val[q] = 0.0; c2[q] = -1; }
      double diag = mc[k].di, rad = fabs(mc[k].lo) + fabs(mc[k].up);
      for (int s = 0; s < 9; ++s) {
        if (c2[s] < 0) continue;
        if (c2[s] == idx) diag += val[s]; else rad += fabs(val[s]);
      }
      mn = fmin(mn, diag - rad);
    }
  }
  smin[threadIdx.x] = mn;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = smin[0];
}

__global__ void copy_planes_k(long long n, const double* __restrict__ src, double* __restrict__ dst) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < 5 * n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(idx / n);
    const long long c = idx - q * n;
    dst[idx] = src[kAdvSlot[q] * n + c];
  }
}

// Row k of M from the faces (zero flux through P_0 and P_np).
void momentum_rows(int np, const double* P, const double* dpp, const double* b,
                   const double* loss, std::vector<MomCoef>& rows) {
  rows.assign(np, MomCoef{});
  std::vector<double> pc(np), dP(np);
  for (int k = 0; k < np; ++k) {
    pc[k] = std::sqrt(P[k] * P[k + 1]);
    dP[k] = P[k + 1] - P[k];
  }
  for (int f = 1; f < np; ++f) {        // interior face between cells f - 1 and f
    const int lo = f - 1, hi = f;
    const double K = P[f] * P[f] * dpp[f] / (pc[hi] - pc[lo]);
    const double fh = K / (pc[hi] * pc[hi]), fl = -K / (pc[lo] * pc[lo]);   // F = fh u_hi + fl u_lo
    rows[lo].up += fh / dP[lo];
    rows[lo].di += fl / dP[lo];
    rows[hi].di -= fh / dP[hi];
    rows[hi].lo -= fl / dP[hi];
    if (b[f] >= 0) {                    // G = b u_lo
      rows[lo].di -= b[f] / dP[lo];
      rows[hi].lo += b[f] / dP[hi];
    } else {                            // G = b u_hi
      rows[lo].up -= b[f] / dP[lo];
      rows[hi].di += b[f] / dP[hi];
    }
  }
  for (int k = 0; k < np; ++k) rows[k].di -= loss[k];
}

int blocks_for(long long n) {
  const long long want = (n + kThreads - 1) / kThreads;
  return (int)std::max<long long>(1, std::min<long long>(want, 152LL * 4));
}

}  // namespace
}  // namespace ad

using namespace ad;

struct ad_momentum_operator {
  GridDev g{};
  int np = 0;
  long long N = 0;
  cudaStream_t stream = nullptr;
  bool adv = false;
  double *WD = nullptr, *WA = nullptr, *sWD = nullptr, *sWA = nullptr;
  std::vector<MomCoef> rows;
  MomCoef* mc = nullptr;
  double *y0 = nullptr, *y1 = nullptr, *P = nullptr, *T1 = nullptr, *T2 = nullptr, *T3 = nullptr;
  double* partials = nullptr;
  int nblocks = 1;
  double* dscal = nullptr;
  LejaCoef* lc = nullptr;
  std::vector<LejaCoef> h_lc;
  Ctrl* ctrl = nullptr;
  Ctrl* h_ctrl = nullptr;
  double alpha = 0.0, c = 0.0, gamma = 0.0;
  double rho_max = 200.0;
  int max_iters = kMaxIters;
  double cache_h = -1.0, cache_alpha = 0.0;
  std::vector<double> d_host;
};

namespace {

void free_mop(ad_momentum_operator* op) {
  for (void* p : {(void*)op->WD, (void*)op->WA, (void*)op->sWD, (void*)op->sWA, (void*)op->mc,
                  (void*)op->y0, (void*)op->y1, (void*)op->P, (void*)op->T1, (void*)op->T2,
                  (void*)op->T3, (void*)op->partials, (void*)op->dscal, (void*)op->lc,
                  (void*)op->ctrl})
    if (p) cudaFree(p);
  if (op->h_ctrl) cudaFreeHost(op->h_ctrl);
  delete op;
}

int mop_set_alpha(ad_momentum_operator* op, double alpha) {
  if (!(alpha < 0.0) || !std::isfinite(alpha))
    return mfail(AD_ERR_INVALID, "spectral bound alpha must be finite and negative");
  op->alpha = alpha;
  op->c = alpha / 2.0;          // Section 2: c = alpha/2, gamma = -alpha/4
  op->gamma = -alpha / 4.0;
  const long long n = op->g.n;
  axpby(0, 9 * n, 1.0 / op->gamma, op->WD, 0.0, nullptr, op->sWD, op->stream);
  if (op->adv) axpby(0, 5 * n, 1.0 / op->gamma, op->WA, 0.0, nullptr, op->sWA, op->stream);
  for (MomCoef& r : op->rows) {
    r.slo = r.lo / op->gamma;
    r.sdi = (r.di - op->c) / op->gamma;
    r.sup = r.up / op->gamma;
  }
  M_CUDA(cudaMemcpyAsync(op->mc, op->rows.data(), sizeof(MomCoef) * op->np,
                         cudaMemcpyHostToDevice, op->stream));
  M_CUDA(cudaStreamSynchronize(op->stream));
  return AD_OK;
}

int mop_upload(ad_momentum_operator* op, double h, double* d0) {
  const std::vector<double>& xi = leja_points();
  const int M = kMaxIters + 1;
  if (!(op->cache_h == h && op->cache_alpha == op->alpha)) {
    std::vector<double> f(M);
    for (int m = 0; m < M; ++m) f[m] = phi1((op->c + op->gamma * xi[m]) * h);
    op->d_host.assign(M, 0.0);
    divided_differences(xi.data(), f.data(), M, op->d_host.data());
    op->h_lc.assign(kMaxIters, LejaCoef{});
    for (int m = 0; m < kMaxIters; ++m)
      op->h_lc[m] = LejaCoef{xi[m], op->d_host[m + 1], std::fabs(op->d_host[m + 1]), 0.0, 0.0,
                             {0.0, 0.0, 0.0}};
    M_CUDA(cudaMemcpyAsync(op->lc, op->h_lc.data(), sizeof(LejaCoef) * kMaxIters,
                           cudaMemcpyHostToDevice, op->stream));
    M_CUDA(cudaStreamSynchronize(op->stream));
    op->cache_h = h;
    op->cache_alpha = op->alpha;
  }
  *d0 = op->d_host[0];
  return AD_OK;
}

SeriesArgs mop_args(ad_momentum_operator* op) {
  SeriesArgs a{};
  a.g = op->g;
  a.g.n = op->N;                  // series_init and the vectors span all slices
  a.prec = 0;
  a.y[0] = op->y0;
  a.y[1] = op->y1;
  a.p = op->P;
  a.lc = op->lc;
  a.ctrl = op->ctrl;
  a.partials = op->partials;
  a.nblocks = op->nblocks;
  return a;
}

void mop_apply(ad_momentum_operator* op, const double* u, const double* S, double* out) {
  ++launch_counter();
  if (op->adv)
    mom_apply_k<true><<<op->nblocks, kThreads, 0, op->stream>>>(op->g, op->np, op->WD, op->WA,
                                                                op->mc, u, S, out);
  else
    mom_apply_k<false><<<op->nblocks, kThreads, 0, op->stream>>>(op->g, op->np, op->WD,
                                                                 nullptr, op->mc, u, S, out);
}

// One Newton series from src into op->P; *iters receives its iteration count.
int mop_series(ad_momentum_operator* op, const double* src, double d0, int force, double tol,
               ad_stats* st, int* iters) {
  SeriesArgs a = mop_args(op);
  series_init(a, src, d0, force, op->max_iters, tol, op->stream);
  M_CUDA(cudaGetLastError());
  *iters = 0;
  if (force == 0) return AD_OK;
  a.g.n = op->g.n;                // the iteration kernel strides over spatial cells
  const size_t smem = sizeof(double) * 4 * op->np;
  int launched = 0;
  for (;;) {
    for (int q = 0; q < kMomChunk; ++q) {
      ++launch_counter();
      const double* wa = op->adv ? op->sWA : nullptr;
      if (mom_int_squares()) {
        if (op->adv)
          mom_iter_k<true, true><<<op->nblocks, kThreads, smem, op->stream>>>(a, op->np, op->sWD,
                                                                              wa, op->mc);
        else
          mom_iter_k<false, true><<<op->nblocks, kThreads, smem, op->stream>>>(a, op->np,
                                                                               op->sWD, wa, op->mc);
      } else {
        if (op->adv)
          mom_iter_k<true, false><<<op->nblocks, kThreads, smem, op->stream>>>(a, op->np,
                                                                               op->sWD, wa, op->mc);
        else
          mom_iter_k<false, false><<<op->nblocks, kThreads, smem, op->stream>>>(a, op->np,
                                                                                op->sWD, wa, op->mc);
      }
    }
    launched += kMomChunk;
    M_CUDA(cudaGetLastError());
    M_CUDA(cudaMemcpyAsync(op->h_ctrl, op->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost,
                           op->stream));
    M_CUDA(cudaStreamSynchronize(op->stream));
    if (op->h_ctrl->stop || launched >= kMaxIters + kMomChunk) break;
  }
  if (!op->h_ctrl->stop) return mfail(AD_ERR_TIMEOUT, "Leja series did not reach its stop state");
  const Ctrl& h = *op->h_ctrl;
  const double est = h.pnorm2 > 0.0 ? h.err_est * std::sqrt(h.ynorm2 / h.pnorm2)
                                    : (h.ynorm2 > 0.0 ? INFINITY : 0.0);
  *iters = h.iters;
  if (st) {
    st->iters += h.iters;
    st->matvecs += h.iters;
    st->err_est = std::max(st->err_est, est);
    if (h.status != 0) st->converged = 0;
  }
  return h.status == 0 ? AD_OK : AD_ERR_NOT_CONVERGED;
}

// out = phi_1(dt A) v (substeps: w_{k+1} = w_k + h phi_1(h A)(A w_k + v),
// out = w_K / dt).  v is read before T1..T3 are written and out is written
// last, so v and out may be any of T1..T3 or the caller's vectors.
int mop_phi1(ad_momentum_operator* op, const double* v, double* out, double dt, double tol,
             int force, ad_stats* st) {
  const double rho = op->gamma * dt;
  const int K = rho <= op->rho_max ? 1 : (int)std::ceil(rho / op->rho_max);
  const double h = dt / K;
  double d0;
  M_TRY(mop_upload(op, h, &d0));
  if (st) st->substeps = K;
  const long long N = op->N;
  int status = AD_OK, it = 0;
  if (K == 1) {
    const int r = mop_series(op, v, d0, force, tol, st, &it);
    if (r != AD_OK && r != AD_ERR_NOT_CONVERGED) return r;
    status = r;
    axpby(0, N, 1.0, op->P, 0.0, nullptr, out, op->stream);
  } else {
    axpby(0, N, 1.0, v, 0.0, nullptr, op->T1, op->stream);
    axpby(0, N, 0.0, nullptr, 0.0, nullptr, op->T2, op->stream);
    for (int k = 0; k < K; ++k) {
      const double* rhs = op->T1;
      if (k > 0) {
        mop_apply(op, op->T2, op->T1, op->T3);      // A w + v
        rhs = op->T3;
        if (st) st->matvecs += 1;
      }
      const int r = mop_series(op, rhs, d0, force, tol, st, &it);
      if (r != AD_OK && r != AD_ERR_NOT_CONVERGED) return r;
      if (r != AD_OK) status = r;
      axpby(0, N, 1.0, op->T2, h, op->P, op->T2, op->stream);
    }
    axpby(0, N, 1.0 / dt, op->T2, 0.0, nullptr, out, op->stream);
  }
  M_CUDA(cudaGetLastError());
  return status;
}

bool dev_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

int ad_create_momentum_operator(const ad_grid* grid, const ad_momentum* mom, const double* Dxx,
                                const double* Dxy, const double* Dyy, double ax, double ay,
                                void* cuda_stream, ad_momentum_operator** out) {
  set_error_message("");
  cudaGetLastError();
  if (!out) return mfail(AD_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!grid || !mom || !Dxx || !Dxy || !Dyy) return mfail(AD_ERR_INVALID, "NULL argument");
  if (grid->nx < 1 || grid->ny < 1) return mfail(AD_ERR_INVALID, "grid: nx, ny must be >= 1");
  if (!(grid->x1 > grid->x0) || !(grid->y1 > grid->y0))
    return mfail(AD_ERR_INVALID, "grid: empty domain");
  if (grid->bc != AD_BC_PERIODIC && grid->bc != AD_BC_DIRICHLET0)
    return mfail(AD_ERR_INVALID, "grid: unknown boundary condition");
  const int np = mom->np;
  if (np < 1 || np > kMomMaxSlices) return mfail(AD_ERR_INVALID, "np must be in [1, 1024]");
  if (!mom->P || !mom->beta || !mom->dpp || !mom->b || !mom->loss)
    return mfail(AD_ERR_INVALID, "momentum arrays must not be NULL");
  for (int k = 0; k < np; ++k) {
    if (!(mom->P[k + 1] > mom->P[k]) || !(mom->P[k] > 0.0))
      return mfail(AD_ERR_INVALID, "momentum faces must be positive and increasing");
    if (!(mom->beta[k] >= 0.0) || !std::isfinite(mom->beta[k]) || !std::isfinite(mom->loss[k]))
      return mfail(AD_ERR_INVALID, "beta must be finite and >= 0, loss finite");
  }
  for (int f = 0; f <= np; ++f)
    if (!std::isfinite(mom->dpp[f]) || !(mom->dpp[f] >= 0.0) || !std::isfinite(mom->b[f]))
      return mfail(AD_ERR_INVALID, "D_pp must be finite and >= 0, b finite");
  if (!std::isfinite(ax) || !std::isfinite(ay)) return mfail(AD_ERR_INVALID, "advection not finite");
  const long long n = (long long)grid->nx * grid->ny;
  if (n * np > (1LL << 31) - 1) return mfail(AD_ERR_INVALID, "grid x momentum cells: too many");
  for (const void* p : {(const void*)Dxx, (const void*)Dxy, (const void*)Dyy})
    if (!dev_ptr(p)) return mfail(AD_ERR_INVALID, "D fields must be device pointers");

  ad_momentum_operator* op = new ad_momentum_operator();
  op->g = GridDev{grid->nx, grid->ny, grid->bc, n};
  op->np = np;
  op->N = n * np;
  op->stream = (cudaStream_t)cuda_stream;
  op->adv = ax != 0.0 || ay != 0.0;
  op->nblocks = blocks_for(n);
  bool ok = true;
  auto alloc = [&](void** p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) { cudaGetLastError(); ok = false; }
  };
  const size_t vb = sizeof(double) * (size_t)op->N;
  alloc((void**)&op->WD, sizeof(double) * 9 * n);
  alloc((void**)&op->sWD, sizeof(double) * 9 * n);
  if (op->adv) {
    alloc((void**)&op->WA, sizeof(double) * 5 * n);
    alloc((void**)&op->sWA, sizeof(double) * 5 * n);
  }
  alloc((void**)&op->mc, sizeof(MomCoef) * np);
  for (double** v : {&op->y0, &op->y1, &op->P, &op->T1, &op->T2, &op->T3}) alloc((void**)v, vb);
  alloc((void**)&op->partials, sizeof(double) * 2 * op->nblocks);
  alloc((void**)&op->dscal, sizeof(double) * 4);
  alloc((void**)&op->lc, sizeof(LejaCoef) * kMaxIters);
  alloc((void**)&op->ctrl, sizeof(Ctrl));
  if (ok && cudaMallocHost((void**)&op->h_ctrl, sizeof(Ctrl)) != cudaSuccess) {
    cudaGetLastError();
    ok = false;
  }
  if (!ok) {
    free_mop(op);
    return mfail(AD_ERR_NOMEM, "device allocation failed");
  }
  cudaMemsetAsync(op->ctrl, 0, sizeof(Ctrl), op->stream);
  const double dx = (grid->x1 - grid->x0) / grid->nx, dy = (grid->y1 - grid->y0) / grid->ny;
  // diffusion weights (a = 0); advection weights (D = 0) packed as 9 planes in
  // scratch, of which the 5 non-zero ones are kept
  pack_weights_f64(op->g, dx, dy, Dxx, Dxy, Dyy, nullptr, nullptr, 0.0, 0.0, op->WD, op->stream);
  if (op->adv) {
    double* tmp = nullptr;          // 9 planes + one zero field
    if (cudaMalloc((void**)&tmp, sizeof(double) * 10 * n) != cudaSuccess) {
      cudaGetLastError();
      free_mop(op);
      return mfail(AD_ERR_NOMEM, "device allocation failed");
    }
    double* zero = tmp + 9 * n;
    cudaMemsetAsync(zero, 0, sizeof(double) * n, op->stream);
    pack_weights_f64(op->g, dx, dy, zero, zero, zero, nullptr, nullptr, ax, ay, tmp, op->stream);
    copy_planes_k<<<blocks_for(5 * n), kThreads, 0, op->stream>>>(n, tmp, op->WA);
    cudaStreamSynchronize(op->stream);
    cudaFree(tmp);
  }
  momentum_rows(np, mom->P, mom->dpp, mom->b, mom->loss, op->rows);
  for (int k = 0; k < np; ++k) op->rows[k].beta = mom->beta[k];
  if (cudaMemcpyAsync(op->mc, op->rows.data(), sizeof(MomCoef) * np, cudaMemcpyHostToDevice,
                      op->stream) != cudaSuccess) {
    cudaGetLastError();
    free_mop(op);
    return mfail(AD_ERR_CUDA, "upload of the momentum rows failed");
  }
  // Gershgorin bound (Section 2)
  mom_gershgorin_k<<<op->nblocks, kThreads, 0, op->stream>>>(op->g, np, op->WD,
                                                             op->adv ? op->WA : nullptr, op->mc,
                                                             op->partials);
  reduce_partials(op->partials, op->nblocks, 1, op->dscal, op->stream);
  double a = 0.0;
  if (cudaMemcpyAsync(&a, op->dscal, sizeof(double), cudaMemcpyDeviceToHost, op->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(op->stream) != cudaSuccess) {
    cudaGetLastError();
    free_mop(op);
    return mfail(AD_ERR_CUDA, "operator set-up failed");
  }
  const int r = mop_set_alpha(op, a < 0.0 ? a : -1.0);
  if (r != AD_OK) {
    free_mop(op);
    return r;
  }
  *out = op;
  return AD_OK;
}

int ad_destroy_momentum_operator(ad_momentum_operator* op) {
  if (op) {
    cudaStreamSynchronize(op->stream);
    free_mop(op);
  }
  return AD_OK;
}

int ad_momentum_spectral_bound(const ad_momentum_operator* op, double* alpha) {
  set_error_message("");
  if (!op || !alpha) return mfail(AD_ERR_INVALID, "NULL argument");
  *alpha = op->alpha;
  return AD_OK;
}

int ad_momentum_set_spectral_bound(ad_momentum_operator* op, double alpha) {
  set_error_message("");
  if (!op) return mfail(AD_ERR_INVALID, "op is NULL");
  return mop_set_alpha(op, alpha);
}

int ad_momentum_set_options(ad_momentum_operator* op, double rho_max, int max_iters) {
  set_error_message("");
  if (!op) return mfail(AD_ERR_INVALID, "op is NULL");
  if (max_iters > kMaxIters) return mfail(AD_ERR_INVALID, "max_iters > 500");
  if (rho_max > 0) op->rho_max = rho_max;
  if (max_iters > 0) op->max_iters = max_iters;
  return AD_OK;
}

int ad_momentum_apply(ad_momentum_operator* op, const double* u, double* Au) {
  set_error_message("");
  if (!op || !u || !Au) return mfail(AD_ERR_INVALID, "NULL argument");
  if (!dev_ptr(u) || !dev_ptr(Au)) return mfail(AD_ERR_INVALID, "u and Au must be device pointers");
  if (u == Au) return mfail(AD_ERR_INVALID, "u and Au must not alias");
  mop_apply(op, u, nullptr, Au);
  M_CUDA(cudaGetLastError());
  M_CUDA(cudaStreamSynchronize(op->stream));
  return AD_OK;
}

int ad_momentum_leja_phi1(ad_momentum_operator* op, const double* v, double* out, double dt,
                          double tol, int force_iters, ad_stats* stats) {
  set_error_message("");
  if (!op || !v || !out) return mfail(AD_ERR_INVALID, "NULL argument");
  if (!dev_ptr(v) || !dev_ptr(out)) return mfail(AD_ERR_INVALID, "v and out must be device pointers");
  if (!(dt > 0) || !std::isfinite(dt)) return mfail(AD_ERR_INVALID, "dt must be positive");
  if (force_iters < 0 && !(tol > 0)) return mfail(AD_ERR_INVALID, "tol must be positive");
  if (force_iters > op->max_iters) return mfail(AD_ERR_INVALID, "force_iters > max_iters");
  ad_stats st{};
  st.converged = 1;
  st.alpha = op->alpha;
  const long long l0 = launch_counter();
  const int r = mop_phi1(op, v, out, dt, tol, force_iters < 0 ? -1 : force_iters, &st);
  if (r != AD_OK && r != AD_ERR_NOT_CONVERGED) return r;
  M_CUDA(cudaStreamSynchronize(op->stream));
  st.kernel_launches = (int)(launch_counter() - l0);
  if (stats) *stats = st;
  if (r != AD_OK) return mfail(r, "Leja series reached max_iters");
  return AD_OK;
}

int ad_momentum_step(ad_momentum_operator* op, double* u, double dt, const double* S, double tol,
                     int force_iters, ad_stats* stats) {
  set_error_message("");
  if (!op || !u) return mfail(AD_ERR_INVALID, "NULL argument");
  if (!dev_ptr(u) || (S && !dev_ptr(S)))
    return mfail(AD_ERR_INVALID, "u and S must be device pointers");
  if (!(dt > 0) || !std::isfinite(dt)) return mfail(AD_ERR_INVALID, "dt must be positive");
  if (force_iters < 0 && !(tol > 0)) return mfail(AD_ERR_INVALID, "tol must be positive");
  if (force_iters > op->max_iters) return mfail(AD_ERR_INVALID, "force_iters > max_iters");
  ad_stats st{};
  st.converged = 1;
  st.alpha = op->alpha;
  const long long l0 = launch_counter();
  // v = A u + S in T1, phi_1(dt A) v into T3, u += dt T3
  mop_apply(op, u, S, op->T1);
  st.matvecs += 1;
  const int r = mop_phi1(op, op->T1, op->T3, dt, tol, force_iters < 0 ? -1 : force_iters, &st);
  if (r != AD_OK && r != AD_ERR_NOT_CONVERGED) return r;
  axpby(0, op->N, 1.0, u, dt, op->T3, u, op->stream);
  M_CUDA(cudaGetLastError());
  M_CUDA(cudaStreamSynchronize(op->stream));
  st.kernel_launches = (int)(launch_counter() - l0);
  if (stats) *stats = st;
  if (r != AD_OK) return mfail(r, "Leja series reached max_iters");
  return AD_OK;
}

}  // extern "C"
