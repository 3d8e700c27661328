// FP64 Newton series (Section 2) of a small grid in ONE thread-block cluster.
//
// For grids of a few thousand cells the series is a chain of short
// dependent iterations: at 64^2 a Leja iteration is 4096 cells of a 9-point
// stencil, and the cost of the persistent tile kernel (152 blocks of 27-32
// cells, neighbours synchronised through flags in global memory) is its
// synchronisation latency, about 6 us per iteration.  Here the grid lives in
// the distributed shared memory of one cluster of K <= 16 CTAs (one per SM):
// CTA r owns the row band [r ny / K, (r + 1) ny / K) -- its 9 scaled
// weights, three p buffers and two windows of y with one halo row above and
// below and one halo column on each side.  Per iteration m:
//   phase A: warps 2-9 form z = y_{m+1} and p_{m+1} on the band (the cell
//     arithmetic of the persistent kernels, operation for operation) and
//     their squared-norm terms; meanwhile control warp 1 adds the block's
//     terms of iteration m - 1, and control warp 0 adds the K block sums of
//     iteration m - 2 (published one barrier earlier) and applies the
//     stopping rule to iteration m - 2;
//   one hardware cluster barrier (release / acquire, every thread of the
//     cluster) publishes the new rows, the block sums and the decision;
//   each CTA copies its two halo rows of y_{m+1} from the neighbouring CTAs'
//     shared memory.
// The norms and the decision stay off the critical path: the rule runs two
// iterations late (p after iteration m - 2 survives in the third p buffer)
// and the K sums are added in rank order by every CTA, so every CTA takes the
// same decision and runs the same number of barriers.  Count limits (forced
// counts, max_iters) stop before the iteration they exclude, and a drain
// then tests the two iterations still pending.  Double buffering (y windows
// and block sums by parity) makes one barrier per iteration enough: a buffer
// is overwritten only one barrier after the last remote read of it.  A final
// barrier keeps every CTA's shared memory alive until the others have
// stopped reading it.  The waits are the hardware barrier's own (no spin
// loop, nothing to time out).
//
// The augmented series of two-stage quadrature (Eq. exp_quad) adds the
// couplings e1 w2 + e2 w1 per cell, w1 and w2 held in shared memory beside
// the weights.  With a StepFuse the launch also forms the step's right-hand
// sides w1 = A u + sum a_k g_k and w2 = sum b_k g_k (prologue, the apply
// kernel's arithmetic; y_0 = w1 for the midpoint rule, Eq. exp_midpoint,
// y_0 = 0 for two stages) and the update u += P (epilogue), as the tile
// kernel does: one launch per step.
#include "cluster_f64.h"
#include "stencil9.cuh"

#include <cooperative_groups.h>

#include <cstdlib>
#include <mutex>
#include <vector>

namespace cg = cooperative_groups;

namespace ad {
namespace {

constexpr int kClusterCompute = 256;                  // threads of warps 2-9
constexpr int kClusterThreads = 64 + kClusterCompute;  // + the two control warps
constexpr int kClusterMaxCtas = 16;          // non-portable cluster size (GB300 allows 16)
// Measured per Leja iteration (the 64^2 workload's fields at other sizes,
// this kernel vs the tile kernel): 32^2 1.9 vs 5.1 us, 64^2 2.5 vs 5.4,
// 96^2 3.7 vs 5.5, 112^2 5.2 vs 5.8, 128^2 5.4 vs 5.3, 160^2 7.3 vs 5.7:
// beyond 112^2 the 16 SMs' FP64 pipes, not synchronisation, bound it.
constexpr long long kClusterMaxCells = 112 * 112;

struct ClusterGeom {
  int K;        // CTAs in the cluster
  int rows;     // largest row band (shared-memory plane stride: rows * nx cells)
  int S;        // window row stride, nx + 2
};

template <bool FUSED, bool AUG>
__global__ void __launch_bounds__(kClusterThreads)
    leja_cluster_f64_k(SeriesArgs a, ClusterGeom geo, StepFuse F) {
  extern __shared__ __align__(16) double csm[];
  __shared__ double s_red[2][2][kClusterCompute];  // per-thread norm terms, by parity of m
  __shared__ double s_part[2][2];                  // this CTA's (y, p) sums, by parity of m
  __shared__ int s_fin, s_status;
  __shared__ double s_ty, s_tp;
  cg::cluster_group cl = cg::this_cluster();
  const int K = geo.K, rank = (int)cl.block_rank();
  const int t = threadIdx.x, T = blockDim.x, lane = t & 31, warp = t >> 5;
  const int ct = t - 64;                             // compute thread index (warps 2-9)
  const GridDev g = a.g;
  const int nx = g.nx, ny = g.ny, S = geo.S;
  const long long n = g.n;
  const bool periodic = g.bc == 0;
  const int r0 = (int)((long long)ny * rank / K), r1 = (int)((long long)ny * (rank + 1) / K);
  const int rows = r1 - r0, nc = rows * nx;
  const int cpb = geo.rows * nx;
  const int WB = (geo.rows + 2) * S;
  double* sW = csm;                    // [9][cpb] scaled weights
  double* sP = sW + 9 * cpb;           // [3][cpb]: p after iteration k in buffer (k + 1) % 3
  double* sW1 = sP + 3 * cpb;          // [cpb] w1, [cpb] w2: the augmented couplings (AUG)
  double* sW2 = sW1 + cpb;
  double* win = sP + (AUG ? 5 : 3) * cpb;   // [2][WB]: y_m in buffer m & 1
  const double* __restrict__ Ws = static_cast<const double*>(a.coef);
  Ctrl* ctrl = a.ctrl;
  const int force = FUSED ? F.force : ctrl->force;
  const int max_it = min(FUSED ? F.max_iters : ctrl->max_iters, kMaxIters);
  const double tol = FUSED ? F.tol : ctrl->tol;
  // iterations 0 .. limit - 1 at most (terms <= limit)
  const int limit = max(1, force > 0 ? min(force, kMaxIters) : max_it);
  auto widx = [&](int li, int lj) { return (lj + 1) * S + li + 1; };
  // periodic: the halo columns of a row hold the wrapped values
  auto put = [&](double* wb, int li, int lj, double v) {
    wb[widx(li, lj)] = v;
    if (periodic) {
      if (li == 0) wb[widx(nx, lj)] = v;
      if (li == nx - 1) wb[widx(-1, lj)] = v;
    }
  };
  // the neighbouring bands (periodic wrap; -1: zero Dirichlet, the halo row stays 0)
  const int up_rank = rank > 0 ? rank - 1 : (periodic ? K - 1 : -1);
  const int dn_rank = rank < K - 1 ? rank + 1 : (periodic ? 0 : -1);
  const double* up_win = nullptr;
  const double* dn_win = nullptr;
  int up_row = 0;
  if (up_rank >= 0) {
    up_win = cl.map_shared_rank(win, (unsigned)up_rank);
    const int ur0 = (int)((long long)ny * up_rank / K), ur1 = (int)((long long)ny * (up_rank + 1) / K);
    up_row = ur1 - ur0 - 1;            // its last row
  }
  if (dn_rank >= 0) dn_win = cl.map_shared_rank(win, (unsigned)dn_rank);
  // halo rows of buffer buf from the neighbours' shared memory
  auto fill_halo = [&](int buf) {
    double* wb = win + buf * WB;
    for (int q = t; q < 2 * S; q += T) {
      if (q < S) {
        if (up_win) wb[q] = up_win[buf * WB + (up_row + 1) * S + q];
      } else if (dn_win) {
        wb[(rows + 1) * S + (q - S)] = dn_win[buf * WB + S + (q - S)];
      }
    }
  };
  // control warp 1: the block's sums of the terms of parity par -- lanes
  // 0-15 the y terms, 16-31 the p terms, 16 terms per lane (q = lane mod 16
  // + 16 j) added as a pairwise tree, then a shuffle tree over the half-warp
  // (FP64 adds are slow to issue from one warp, so the dependent chain is
  // kept short)
  auto block_sums = [&](int par) {
    static_assert(kClusterCompute == 256, "16 lanes x 16 terms per norm");
    const double* src = &s_red[par][lane >> 4][lane & 15];
    double v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = src[16 * j];   // lanes on consecutive words
#pragma unroll
    for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
      for (int j = 0; j < w; ++j) v[j] = v[j] + v[j + w];
    double r = v[0];
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (lane == 0) s_part[par][0] = r;
    if (lane == 16) s_part[par][1] = r;
  };
  // control warp: the K block sums of parity par in rank order (identical in
  // every CTA), in every lane
  auto cluster_sums = [&](int par, double& ty, double& tp) {
    const int q = lane & 15;
    double v = 0.0;
    if (q < K) v = cl.map_shared_rank(&s_part[par][0], (unsigned)q)[lane < 16 ? 0 : 1];
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    ty = __shfl_sync(0xffffffffu, v, 0);
    tp = __shfl_sync(0xffffffffu, v, 16);
  };
  // the norm test of series_finish on iteration k (terms = k + 1) with
  // absd = |d_{k+1}|: 0 converged, 3 not finite, -1 go on
  const double tol2 = tol * tol;
  auto norm_test = [&](int k, double absd, double ty, double tp) -> int {
    if (!isfinite(ty) || !isfinite(tp)) return 3;
    if (k + 1 >= 2 && (absd * absd) * ty <= tol2 * tp) return 0;
    return -1;
  };

  for (int q = t; q < 2 * WB; q += T) win[q] = 0.0;   // zero Dirichlet halo
  if (t == 0) s_fin = -1;
  __syncthreads();
  const double* __restrict__ Wu = F.W;
  const double* __restrict__ uu = F.u;
  for (int k = t; k < nc; k += T) {
    const int li = k % nx, lj = k / nx;
    const long long idx = (long long)(r0 + lj) * nx + li;
#pragma unroll
    for (int q = 0; q < 9; ++q) sW[q * cpb + k] = Ws[(long long)q * n + idx];
    if (FUSED) {   // w1 = A u + sum a_k g_k, w2 = sum b_k g_k, as the apply kernel forms them
      const double au = stencil9(Wu, n, uu, li, r0 + lj, nx, ny, g.bc, idx);
      double r = 1.0 * au, r2 = 0.0;
      for (int q = 0; q < F.src.n; ++q) {
        const double gq = static_cast<const double*>(F.src.g[q])[idx];
        r = fma(F.src.a[q], gq, r);
        r2 = fma(F.src.b[q], gq, r2);
      }
      F.w1[idx] = r;
      if (AUG) {                   // two stages: y_0 = 0 (the window stays 0)
        sW1[k] = r;
        sW2[k] = r2;
        sP[k] = F.d0 * 0.0;
      } else {                     // midpoint: y_0 = w1
        put(win, li, lj, r);
        sP[k] = F.d0 * r;
      }
    } else {
      put(win, li, lj, static_cast<const double*>(a.y[0])[idx]);
      sP[k] = static_cast<const double*>(a.p)[idx];
      if (AUG) {
        sW1[k] = static_cast<const double*>(a.w1)[idx];
        sW2[k] = static_cast<const double*>(a.w2)[idx];
      }
    }
  }
  cl.sync();            // every band's y_0 is in place
  fill_halo(0);
  __syncthreads();

  int m = 0;
  // Leja scalars one iteration ahead (their loads stay off the critical path):
  // xi_m, d_{m+1} (and the coupling scalars e1, e2) for the compute warps,
  // |d| of the iteration warp 0 tests next
  double xi_m = a.lc[0].xi, d_m = a.lc[0].d;
  double e1_m = AUG ? a.lc[0].e1 : 0.0, e2_m = AUG ? a.lc[0].e2 : 0.0;
  double absd_next = a.lc[0].absd;
  for (;;) {
    if (m >= limit) break;          // count limit: the drain below decides
    if (warp >= 2) {                // phase A: iteration m
      const double xi = xi_m, dd = d_m, e1 = e1_m, e2 = e2_m;
      if (m + 1 < kMaxIters) {
        xi_m = a.lc[m + 1].xi;
        d_m = a.lc[m + 1].d;
        if (AUG) {
          e1_m = a.lc[m + 1].e1;
          e2_m = a.lc[m + 1].e2;
        }
      }
      const double* wy = win + (m & 1) * WB;
      double* wz = win + ((m + 1) & 1) * WB;
      const double* Pin = sP + (m % 3) * cpb;
      double* Pout = sP + ((m + 1) % 3) * cpb;
      double sy = 0.0, sp = 0.0;
      for (int k = ct; k < nc; k += kClusterCompute) {
        const int li = k % nx, lj = k / nx;
        const double* yc = wy + widx(li, lj);
        // the cell arithmetic of the persistent kernels, in their order
        double z = sW[4 * cpb + k] * yc[0];
        z = fma(sW[0 * cpb + k], yc[-S - 1], z);
        z = fma(sW[1 * cpb + k], yc[-S], z);
        z = fma(sW[2 * cpb + k], yc[-S + 1], z);
        z = fma(sW[3 * cpb + k], yc[-1], z);
        z = fma(sW[5 * cpb + k], yc[1], z);
        z = fma(sW[6 * cpb + k], yc[S - 1], z);
        z = fma(sW[7 * cpb + k], yc[S], z);
        z = fma(sW[8 * cpb + k], yc[S + 1], z);
        z = fma(-xi, yc[0], z);
        if (AUG) {                 // the augmented couplings, as the persistent kernels add them
          if (e1 != 0.0) z = fma(e1, sW2[k], z);
          if (e2 != 0.0) z = fma(e2, sW1[k], z);
        }
        put(wz, li, lj, z);
        const double pn = fma(dd, z, Pin[k]);
        Pout[k] = pn;
        sy = fma(z, z, sy);
        sp = fma(pn, pn, sp);
      }
      s_red[m & 1][0][ct] = sy;
      s_red[m & 1][1][ct] = sp;
    } else if (warp == 1) {         // phase A: the block's sums of iteration m - 1
      if (m >= 1) block_sums((m - 1) & 1);
    } else if (m >= 2) {            // phase A: the rule on iteration m - 2
      const double absd = absd_next;
      absd_next = a.lc[m - 1].absd;
      if (force <= 0) {
        double ty, tp;
        cluster_sums((m - 2) & 1, ty, tp);
        const int r = norm_test(m - 2, absd, ty, tp);
        if (lane == 0 && r >= 0) {
          s_fin = m - 2;
          s_status = r;
          s_ty = ty;
          s_tp = tp;
        }
      }
    }
    // y_{m+1} bands and the block sums of m - 1, cluster-wide; a release /
    // acquire barrier over every thread of the cluster, so it also orders
    // this block's shared memory (the decision s_fin, the terms in s_red)
    cl.sync();
    if (s_fin >= 0) break;          // the same decision in every CTA, after the same barrier
    fill_halo((m + 1) & 1);
    __syncthreads();
    ++m;
  }
  if (s_fin < 0) {   // stopped by a count before iteration m: iterations m - 2, m - 1 pending
    if (warp == 1) block_sums((m - 1) & 1);
    __syncthreads();
    cl.sync();
    if (warp == 0) {
      int fin = m - 1, st = 0;
      double ty = 0.0, tp = 0.0;
      if (force <= 0 && m >= 2) {
        cluster_sums((m - 2) & 1, ty, tp);
        const int r = norm_test(m - 2, a.lc[m - 2].absd, ty, tp);
        if (r >= 0) { fin = m - 2; st = r; }
      }
      if (fin == m - 1) {
        cluster_sums((m - 1) & 1, ty, tp);
        if (force <= 0) st = norm_test(m - 1, a.lc[m - 1].absd, ty, tp) == 0 ? 0 : 3;
      }
      if (lane == 0) {
        s_fin = fin;
        s_status = st;
        s_ty = ty;
        s_tp = tp;
      }
    }
    __syncthreads();
  }
  const int fin = s_fin;
  const double* Pf = sP + ((fin + 1) % 3) * cpb;
  if (FUSED) {   // u = 1 u + b P, as the axpby kernel forms it
    for (int k = t; k < nc; k += T) {
      const long long idx = (long long)(r0 + k / nx) * nx + k % nx;
      F.u[idx] = fma(F.b, Pf[k], 1.0 * F.u[idx]);
    }
  } else {
    double* p = static_cast<double*>(a.p);
    for (int k = t; k < nc; k += T) p[(long long)(r0 + k / nx) * nx + k % nx] = Pf[k];
  }
  cl.sync();            // no CTA leaves while another may still read its shared memory
  if (rank == 0 && t == 0) {
    ctrl->iters = fin + 1;
    ctrl->m = fin + 1;
    ctrl->ynorm2 = s_ty;
    ctrl->pnorm2 = s_tp;
    ctrl->err_est = a.lc[fin].absd;
    ctrl->status = s_status;
    ctrl->stop = 1;
    if (FUSED && F.totals) {   // the asynchronous step's report
      AsyncTotals* tt = F.totals;
      const int it = fin + 1;
      tt->iters += it;
      if (F.timed) tt->timed_iters += it;
      tt->series += 1;
      if (s_status > tt->status) tt->status = s_status;
      const double e = s_tp > 0.0 ? a.lc[fin].absd * sqrt(s_ty / s_tp)
                                  : (s_ty > 0.0 ? INFINITY : 0.0);
      if (e > tt->err_est) tt->err_est = e;
    }
  }
}

// Off with AD_F64_CLUSTER=0, and whenever AD_F64_KERNEL or AD_NO_NSYNC asks
// for one of the persistent kernels by name.
bool cluster_enabled() {
  static const bool on = [] {
    const char* e = getenv("AD_F64_CLUSTER");
    return !(e && e[0] == '0') && !getenv("AD_F64_KERNEL") && !getenv("AD_NO_NSYNC");
  }();
  return on;
}

}  // namespace

int series_run_cluster(const SeriesArgs& a, cudaStream_t s, const StepFuse* fuse) {
  if (!cluster_enabled() || a.prec != 0 || a.g.n > kClusterMaxCells) return 0;
  if (fuse && (fuse->s == 2) != (a.aug != 0)) return 0;
  const int nx = a.g.nx, ny = a.g.ny;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return 0; }
  void* fn = fuse ? (a.aug ? (void*)leja_cluster_f64_k<true, true>
                           : (void*)leja_cluster_f64_k<true, false>)
                  : (a.aug ? (void*)leja_cluster_f64_k<false, true>
                           : (void*)leja_cluster_f64_k<false, false>);
  // once per (device, kernel): all the dynamic shared memory the device
  // offers, and clusters of 16; then per (K, smem): whether one such cluster
  // can be resident (cached: a series is launched on every step)
  struct FnInfo { int dev; const void* fn; size_t max_dyn; bool ok; };
  struct Fit { int dev; const void* fn; int K; size_t smem; bool ok; };
  static std::mutex mu;
  static std::vector<FnInfo> fns;
  static std::vector<Fit> fits;
  std::lock_guard<std::mutex> lock(mu);
  const FnInfo* fi = nullptr;
  for (const FnInfo& f : fns)
    if (f.dev == dev && f.fn == fn) fi = &f;
  if (!fi) {
    FnInfo f{dev, fn, 0, false};
    int optin = 0;
    cudaFuncAttributes fa{};
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
        cudaFuncGetAttributes(&fa, fn) == cudaSuccess && fa.sharedSizeBytes < (size_t)optin) {
      f.max_dyn = (size_t)optin - fa.sharedSizeBytes;
      f.ok = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)f.max_dyn) == cudaSuccess &&
             cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                 cudaSuccess;
    }
    cudaGetLastError();
    fns.push_back(f);
    fi = &fns.back();
  }
  if (!fi->ok) return 0;
  for (int K = std::min(kClusterMaxCtas, ny); K >= 1;
       K = K > 8 ? std::min(8, ny) : (K > 4 ? std::min(4, ny) : 0)) {
    const ClusterGeom geo{K, (ny + K - 1) / K, nx + 2};
    const size_t smem =
        sizeof(double) * ((size_t)(a.aug ? 14 : 12) * geo.rows * nx +
                          2 * (size_t)(geo.rows + 2) * geo.S);
    if (smem > fi->max_dyn) continue;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)K;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)K);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int known = -1;
    for (const Fit& f : fits)
      if (f.dev == dev && f.fn == fn && f.K == K && f.smem == smem) known = f.ok ? 1 : 0;
    if (known < 0) {
      int clusters = 0;
      const bool ok = cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg) == cudaSuccess &&
                      clusters >= 1;
      cudaGetLastError();
      fits.push_back(Fit{dev, fn, K, smem, ok});
      known = ok ? 1 : 0;
    }
    if (!known) continue;
    StepFuse F{};
    if (fuse) F = *fuse;
    SeriesArgs args = a;
    args.nblocks = K;
    ClusterGeom g = geo;
    void* params[] = {&args, &g, &F};
    if (cudaLaunchKernelExC(&cfg, fn, params) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    ++launch_counter();
    return 10;
  }
  return 0;
}

}  // namespace ad
