// Matrix-free 9-point operator A = div(D grad .) + div(a .) of Eq. anidiff and
// the fused Leja iteration of Section 2 (Newton recurrence + polynomial
// update + norm partials in one pass over the grid).
//
// Discretisation (the paper gives none): conservative flux form on the
// cell-centred grid,
//   Fx(i+1/2) = Dxx_e (u_E - u_C)/dx + Dxy_e (u_NE + u_N - u_SE - u_S)/(4 dy) + ax_e (u_C + u_E)/2
//   Fy(j+1/2) = Dyy_n (u_N - u_C)/dy + Dxy_n (u_NE + u_E - u_NW - u_W)/(4 dx) + ay_n (u_C + u_N)/2
//   (A u)_C   = (Fx(i+1/2) - Fx(i-1/2))/dx + (Fy(j+1/2) - Fy(j-1/2))/dy,
// face coefficients = mean of the two adjacent cells; periodic wrap, or zero
// Dirichlet through odd-reflection ghosts (corner ghost: diagonal mirror,
// sign +; ghost coefficients mirror without sign).
//
// FP64 layout: 9 weights per cell, with the Dirichlet ghosts folded into the
// interior slots, so each output costs 9 FMA (GB300 runs FP64 at ~1/58 of
// its FP32 rate, so fewer FP64 operations beat fewer bytes here).
// FP32 layout: 3 (+2 with an advection field) pre-scaled cell fields; the
// face means and fluxes are formed on the fly (fewest bytes).
#include "ad_internal.h"
#include "stencil9.cuh"

#include <algorithm>
#include <cstdlib>

#include "tile_f32.cuh"
#include "series_finish.cuh"
#include "sqsum.cuh"
#include "tile_f32_bulk.cuh"
#include "tile_f32_vec.cuh"
#include "tile_f32_ring.cuh"
#include "tile_f32_pair.cuh"
#include "tile_f32_pair_tma.cuh"

namespace ad {

namespace {

// Deterministic block sum of four values of an NT-thread block; results valid
// in thread 0.  Warp w < 4 adds the w-th value of every thread: eight per lane
// as a pairwise tree, then a butterfly.  The four sums run in parallel, so no
// warp issues more than 12 dependent FP64 additions (one warp issues one FP64
// instruction per 64 cycles on this GPU; two block_sum2 calls on warp 0 took
// 52).
template <int NT>
__device__ __forceinline__ void block_sum4(double& a, double& b, double& c, double& d) {
  static_assert(NT == 256, "eight values per lane of four warps");
  __shared__ double s4[4][NT];
  __shared__ double r4[4];
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  __syncthreads();
  s4[0][t] = a;
  s4[1][t] = b;
  s4[2][t] = c;
  s4[3][t] = d;
  __syncthreads();
  if (w < 4) {
    double x[NT / 32];
#pragma unroll
    for (int j = 0; j < NT / 32; ++j) x[j] = s4[w][lane + 32 * j];
#pragma unroll
    for (int h = NT / 64; h >= 1; h >>= 1)
#pragma unroll
      for (int j = 0; j < h; ++j) x[j] += x[j + h];
    const double v = warp_sum(x[0]);
    if (lane == 0) r4[w] = v;
  }
  __syncthreads();
  if (t == 0) {
    a = r4[0];
    b = r4[1];
    c = r4[2];
    d = r4[3];
  }
}

// Epilogue of a pair launch (two iterations, m and m + 1, m even): publish the
// block's four norm partials; the last block sums them in block order and
// applies the stopping rule after term m + 1, then after term m + 2.  A stop
// after term m + 1 leaves the stored p complete (ctrl->m becomes m + 1, odd);
// otherwise ctrl->m becomes m + 2 and d_{m+2} y_{m+2} is pending (added by the
// next pair launch, or by pair_flush_k after the series).
__device__ void series_finish2(const SeriesArgs& a, double y1, double p1, double y2, double p2) {
  __shared__ unsigned int s_last;
  block_sum4<kPairWarps * 32>(y1, p1, y2, p2);
  Ctrl* ctrl = a.ctrl;
  if (threadIdx.x == 0) {
    double* q = a.partials + 4 * blockIdx.x;
    q[0] = y1;
    q[1] = p1;
    q[2] = y2;
    q[3] = p2;
    __threadfence();
    const unsigned int t = atomicAdd(&ctrl->ticket, 1u);
    s_last = (t == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double t1y = 0.0, t1p = 0.0, t2y = 0.0, t2p = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    t1y += __ldcg(&a.partials[4 * b]);
    t1p += __ldcg(&a.partials[4 * b + 1]);
    t2y += __ldcg(&a.partials[4 * b + 2]);
    t2p += __ldcg(&a.partials[4 * b + 3]);
  }
  block_sum4<kPairWarps * 32>(t1y, t1p, t2y, t2p);
  if (threadIdx.x == 0) {
    const int m = ctrl->m;
    const double tol = ctrl->tol;
    int status = ctrl->status;
    // the rule of series_finish, applied after `terms` terms
    auto stop_after = [&](int terms, double absd, double ty, double tp) -> bool {
      bool stop = false;
      if (ctrl->force > 0) {
        stop = terms >= ctrl->force;
      } else if (!isfinite(ty) || !isfinite(tp)) {
        stop = true;
        status = 3;
      } else if (terms >= 2 && (absd * absd) * ty <= (tol * tol) * tp) {
        stop = true;
      } else if (terms >= ctrl->max_iters) {
        stop = true;
        status = 3;
      }
      return stop || terms >= kMaxIters;
    };
    const LejaCoef& L1 = a.lc[m];
    if (stop_after(m + 1, L1.absd, t1y, t1p)) {
      ctrl->ynorm2 = t1y;
      ctrl->pnorm2 = t1p;
      ctrl->iters = m + 1;
      ctrl->err_est = L1.absd;
      ctrl->m = m + 1;
      ctrl->stop = 1;
    } else {
      const LejaCoef& L2 = a.lc[m + 1];
      const bool stop = stop_after(m + 2, L2.absd, t2y, t2p);
      ctrl->ynorm2 = t2y;
      ctrl->pnorm2 = t2p;
      ctrl->iters = m + 2;
      ctrl->err_est = L2.absd;
      ctrl->m = m + 2;
      ctrl->stop = stop ? 1 : 0;
    }
    ctrl->status = status;
    ctrl->ticket = 0u;
    __threadfence();
    if (a.has_handle)
      cudaGraphSetConditional((cudaGraphConditionalHandle)a.handle, ctrl->stop ? 0u : 1u);
  }
}

// Grid-stride over tiles of one row x 256 columns.
struct RowTiles {
  int tiles_x, ntiles;
  __device__ RowTiles(int nx, int ny) {
    tiles_x = (nx + kThreads - 1) / kThreads;
    ntiles = tiles_x * ny;
  }
};

// Coefficient at a (possibly ghost) cell: mirror (Dirichlet) or wrap, no sign.
__device__ __forceinline__ double coef_at(const double* f, double fc, int i, int j, int nx, int ny,
                                          int bc) {
  if (!f) return fc;
  if (bc == 0) {
    i = (i < 0) ? i + nx : (i >= nx ? i - nx : i);
    j = (j < 0) ? j + ny : (j >= ny ? j - ny : j);
  } else {
    i = (i < 0) ? -1 - i : (i >= nx ? 2 * nx - 1 - i : i);
    j = (j < 0) ? -1 - j : (j >= ny ? 2 * ny - 1 - j : j);
  }
  return f[(long long)j * nx + i];
}

__global__ void pack_weights_f64_k(GridDev g, double dx, double dy, const double* Dxx,
                                   const double* Dxy, const double* Dyy, const double* ax,
                                   const double* ay, double ax_c, double ay_c, double* W) {
  const long long n = g.n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % g.nx), j = (int)(idx / g.nx);
    const int nx = g.nx, ny = g.ny, bc = g.bc;
    auto C = [&](const double* f, double fc, int ii, int jj) { return coef_at(f, fc, ii, jj, nx, ny, bc); };
    const double idx2 = 1.0 / (dx * dx), idy2 = 1.0 / (dy * dy), iq = 1.0 / (4.0 * dx * dy);
    // face coefficients (east/west/north/south faces of cell (i, j))
    const double axx_e = 0.5 * (C(Dxx, 0, i, j) + C(Dxx, 0, i + 1, j)) * idx2;
    const double axx_w = 0.5 * (C(Dxx, 0, i - 1, j) + C(Dxx, 0, i, j)) * idx2;
    const double ayy_n = 0.5 * (C(Dyy, 0, i, j) + C(Dyy, 0, i, j + 1)) * idy2;
    const double ayy_s = 0.5 * (C(Dyy, 0, i, j - 1) + C(Dyy, 0, i, j)) * idy2;
    const double qe = 0.5 * (C(Dxy, 0, i, j) + C(Dxy, 0, i + 1, j)) * iq;
    const double qw = 0.5 * (C(Dxy, 0, i - 1, j) + C(Dxy, 0, i, j)) * iq;
    const double qn = 0.5 * (C(Dxy, 0, i, j) + C(Dxy, 0, i, j + 1)) * iq;
    const double qs = 0.5 * (C(Dxy, 0, i, j - 1) + C(Dxy, 0, i, j)) * iq;
    const double be = 0.25 * (C(ax, ax_c, i, j) + C(ax, ax_c, i + 1, j)) / dx;
    const double bw = 0.25 * (C(ax, ax_c, i - 1, j) + C(ax, ax_c, i, j)) / dx;
    const double bn = 0.25 * (C(ay, ay_c, i, j) + C(ay, ay_c, i, j + 1)) / dy;
    const double bs = 0.25 * (C(ay, ay_c, i, j - 1) + C(ay, ay_c, i, j)) / dy;
    // unfolded weights w[dj+1][di+1] of u(i+di, j+dj)
    double w[3][3];
    w[1][1] = -axx_e + be - axx_w - bw - ayy_n + bn - ayy_s - bs;
    w[1][2] = axx_e + be + qn - qs;
    w[1][0] = axx_w - bw - qn + qs;
    w[2][1] = ayy_n + bn + qe - qw;
    w[0][1] = ayy_s - bs - qe + qw;
    w[2][2] = qe + qn;
    w[2][0] = -qw - qn;
    w[0][2] = -qe - qs;
    w[0][0] = qw + qs;
    double f[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    if (bc == 0) {
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) f[a][b] = w[a][b];
    } else {  // fold odd-reflection ghosts into the interior slots
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
          int ti = i + di, tj = j + dj;
          double sg = 1.0;
          if (ti < 0) { ti = -1 - ti; sg = -sg; } else if (ti >= nx) { ti = 2 * nx - 1 - ti; sg = -sg; }
          if (tj < 0) { tj = -1 - tj; sg = -sg; } else if (tj >= ny) { tj = 2 * ny - 1 - tj; sg = -sg; }
          f[tj - j + 1][ti - i + 1] += sg * w[dj + 1][di + 1];
        }
    }
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) W[(a * 3 + b) * n + idx] = f[a][b];
  }
}

// Ws = (W - c I) / gamma : the Newton basis operator (A - c)/gamma.
__global__ void scale_weights_f64_k(long long n, const double* W, double c, double gamma,
                                    double* Ws) {
  const double ig = 1.0 / gamma;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const double w = W[k * n + idx];
      Ws[k * n + idx] = (k == 4 ? (w - c) : w) * ig;
    }
  }
}

// Gershgorin: per cell a_ii - sum_{j != i} |a_ij| with coincident columns
// merged (periodic wrap on grids narrower than 3 cells).
__global__ void gershgorin_f64_k(GridDev g, const double* W, double* partials) {
  __shared__ double smin[kThreads];
  double mn = 1e308;
  const long long n = g.n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % g.nx), j = (int)(idx / g.nx);
    long long col[9];
    double val[9];
    for (int k = 0; k < 9; ++k) {
      const int di = k % 3 - 1, dj = k / 3 - 1;
      int ti = i + di, tj = j + dj;
      if (g.bc == 0) {
        ti = (ti + g.nx) % g.nx;
        tj = (tj + g.ny) % g.ny;
      }
      col[k] = (ti < 0 || tj < 0 || ti >= g.nx || tj >= g.ny) ? -1 : (long long)tj * g.nx + ti;
      val[k] = W[k * n + idx];
    }
    for (int k = 0; k < 9; ++k)          // merge duplicates into the first slot
      for (int q = k + 1; q < 9; ++q)
        if (col[k] >= 0 && col[q] == col[k]) { val[k] += val[q]; val[q] = 0.0; col[q] = -1; }
    double diag = 0.0, rad = 0.0;
    for (int k = 0; k < 9; ++k) {
      if (col[k] < 0) continue;
      if (col[k] == idx) diag += val[k]; else rad += fabs(val[k]);
    }
    mn = fmin(mn, diag - rad);
  }
  smin[threadIdx.x] = mn;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = smin[0];
}

// out1 = s0 u + s1 A u + sum_k a_k g_k ; out2 = sum_k b_k g_k.
__global__ void apply_f64_k(GridDev g, const double* __restrict__ W, const double* __restrict__ u,
                            double* out1, double* out2, Sources src, double s0, double s1) {
  const RowTiles rt(g.nx, g.ny);
  for (int t = blockIdx.x; t < rt.ntiles; t += gridDim.x) {
    const int j = t / rt.tiles_x, i = (t % rt.tiles_x) * kThreads + threadIdx.x;
    if (i >= g.nx) continue;
    const long long idx = (long long)j * g.nx + i;
    const double au = stencil9(W, g.n, u, i, j, g.nx, g.ny, g.bc, idx);
    double r = s1 * au;
    if (s0 != 0.0) r = fma(s0, u[idx], r);
    double r2 = 0.0;
    for (int k = 0; k < src.n; ++k) {
      const double gk = static_cast<const double*>(src.g[k])[idx];
      r = fma(src.a[k], gk, r);
      r2 = fma(src.b[k], gk, r2);
    }
    out1[idx] = r;
    if (out2) out2[idx] = r2;
  }
}

// Fused Leja iteration m: y_{m+1} = Ws y_m - xi_m y_m [+ e1 w2 + e2 w1],
// p += d_{m+1} y_{m+1}, norm partials; each block owns a contiguous chunk of
// cells (equal FP64 work per block: the kernel is FP64-pipe bound).  SQ: the
// norms' sums of squares on the integer and FP32 pipes (sqsum.cuh), which
// leaves the FP64 pipe 11 instructions per cell instead of 13; otherwise two
// FP64 FMAs per cell.
template <bool AUG, bool SQ>
__global__ void __launch_bounds__(kThreads) leja_iter_f64_k(SeriesArgs a) {
  const volatile Ctrl* vc = a.ctrl;
  if (vc->stop) return;
  const int m = vc->m;
  const LejaCoef lc = a.lc[m];
  const double* __restrict__ yin = static_cast<const double*>(a.y[m & 1]);
  double* __restrict__ yout = static_cast<double*>(a.y[(m + 1) & 1]);
  double* __restrict__ p = static_cast<double*>(a.p);
  const double* __restrict__ Ws = static_cast<const double*>(a.coef);
  const double* __restrict__ w1 = static_cast<const double*>(a.w1);
  const double* __restrict__ w2 = static_cast<const double*>(a.w2);
  const GridDev g = a.g;
  const unsigned int n = (unsigned int)g.n, nx = (unsigned int)g.nx;
  const unsigned int chunk = (n + gridDim.x - 1) / gridDim.x;
  const unsigned int c0 = blockIdx.x * chunk;
  const unsigned int c1 = min(n, c0 + chunk);
  const bool use_w2 = AUG && lc.e1 != 0.0, use_w1 = AUG && lc.e2 != 0.0;
  double sy = 0.0, sp = 0.0;
  SqSum qy, qp;
  // two cells per thread and loop trip, computed side by side (independent
  // FP64 chains and loads in flight)
  for (unsigned int base = c0 + threadIdx.x; base < c1; base += 2 * blockDim.x) {
    unsigned int id[2];
    bool ok[2];
    double z[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const unsigned int idx = base + q * blockDim.x;
      ok[q] = idx < c1;
      id[q] = ok[q] ? idx : base;
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const unsigned int idx = id[q];
      const int j = (int)(idx / nx), i = (int)(idx - (unsigned int)j * nx);
      double zz = stencil9(Ws, g.n, yin, i, j, g.nx, g.ny, g.bc, idx);
      zz = fma(-lc.xi, yin[idx], zz);
      if (use_w2) zz = fma(lc.e1, w2[idx], zz);
      if (use_w1) zz = fma(lc.e2, w1[idx], zz);
      z[q] = zz;
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      if (!ok[q]) continue;
      const unsigned int idx = id[q];
      yout[idx] = z[q];
      const double pn = fma(lc.d, z[q], p[idx]);
      p[idx] = pn;
      if (SQ) {
        qy.add(z[q]);
        qp.add(pn);
      } else {
        sy = fma(z[q], z[q], sy);
        sp = fma(pn, pn, sp);
      }
    }
  }
  if (SQ) {
    sy = qy.value();
    sp = qp.value();
  }
  series_finish(a, sy, sp);
}

// --------------------------------------------------------------------------
// FP32 storage: fields F[5][n] = Dxx/(2dx^2), Dyy/(2dy^2), Dxy/(8dxdy), ax/(4dx), ay/(4dy).
__global__ void pack_fields_f32_k(GridDev g, double dx, double dy, const double* Dxx,
                                  const double* Dxy, const double* Dyy, const double* ax,
                                  const double* ay, double ax_c, double ay_c, float* F) {
  const long long n = g.n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    F[0 * n + idx] = (float)(Dxx[idx] / (2.0 * dx * dx));
    F[1 * n + idx] = (float)(Dyy[idx] / (2.0 * dy * dy));
    F[2 * n + idx] = (float)(Dxy[idx] / (8.0 * dx * dy));
    if (ax || ay) {
      F[3 * n + idx] = (float)((ax ? ax[idx] : ax_c) / (4.0 * dx));
      F[4 * n + idx] = (float)((ay ? ay[idx] : ay_c) / (4.0 * dy));
    }
  }
}


__global__ void gershgorin_f32_k(GridDev g, const float* F, int adv, double abx, double aby,
                                 double* partials) {
  // the 9 weights of the flux form, assembled in double from the float fields
  __shared__ double smin[kThreads];
  double mn = 1e308;
  const long long n = g.n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % g.nx), j = (int)(idx / g.nx);
    auto fld = [&](int k, int ti, int tj) {
      float sg = 1.0f;
      map_idx(ti, tj, sg, g.nx, g.ny, g.bc);
      return (double)F[k * n + (long long)tj * g.nx + ti];
    };
    const double axe = fld(0, i, j) + fld(0, i + 1, j), axw = fld(0, i - 1, j) + fld(0, i, j);
    const double ayn = fld(1, i, j) + fld(1, i, j + 1), ays = fld(1, i, j - 1) + fld(1, i, j);
    const double qe = fld(2, i, j) + fld(2, i + 1, j), qw = fld(2, i - 1, j) + fld(2, i, j);
    const double qn = fld(2, i, j) + fld(2, i, j + 1), qs = fld(2, i, j - 1) + fld(2, i, j);
    double be = abx, bw = abx, bn = aby, bs = aby;
    if (adv == 2) {
      be = fld(3, i, j) + fld(3, i + 1, j); bw = fld(3, i - 1, j) + fld(3, i, j);
      bn = fld(4, i, j) + fld(4, i, j + 1); bs = fld(4, i, j - 1) + fld(4, i, j);
    } else if (adv == 0) {
      be = bw = bn = bs = 0.0;
    }
    double w[3][3];
    w[1][1] = -axe + be - axw - bw - ayn + bn - ays - bs;
    w[1][2] = axe + be + qn - qs;
    w[1][0] = axw - bw - qn + qs;
    w[2][1] = ayn + bn + qe - qw;
    w[0][1] = ays - bs - qe + qw;
    w[2][2] = qe + qn;
    w[2][0] = -qw - qn;
    w[0][2] = -qe - qs;
    w[0][0] = qw + qs;
    long long col[9];
    double val[9];
    for (int k = 0; k < 9; ++k) {
      int ti = i + k % 3 - 1, tj = j + k / 3 - 1;
      float sg = 1.0f;
      map_idx(ti, tj, sg, g.nx, g.ny, g.bc);
      col[k] = (long long)tj * g.nx + ti;
      val[k] = sg * w[k / 3][k % 3];
    }
    for (int k = 0; k < 9; ++k)
      for (int q = k + 1; q < 9; ++q)
        if (col[k] >= 0 && col[q] == col[k]) { val[k] += val[q]; val[q] = 0.0; col[q] = -1; }
    double diag = 0.0, rad = 0.0;
    for (int k = 0; k < 9; ++k) {
      if (col[k] < 0) continue;
      if (col[k] == idx) diag += val[k]; else rad += fabs(val[k]);
    }
    mn = fmin(mn, diag - rad);
  }
  smin[threadIdx.x] = mn;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = smin[0];
}

__global__ void apply_f32_k(GridDev g, const float* __restrict__ F, int adv, float abx, float aby,
                            const float* __restrict__ u, float* out1, float* out2, Sources src,
                            float s0, float s1) {
  const RowTiles rt(g.nx, g.ny);
  for (int t = blockIdx.x; t < rt.ntiles; t += gridDim.x) {
    const int j = t / rt.tiles_x, i = (t % rt.tiles_x) * kThreads + threadIdx.x;
    if (i >= g.nx) continue;
    const long long idx = (long long)j * g.nx + i;
    const bool interior = i > 0 && j > 0 && i + 1 < g.nx && j + 1 < g.ny;
    const float au = flux_apply_f32(F, g.n, u, i, j, g.nx, g.ny, g.bc, interior, adv, abx, aby);
    float r = s1 * au;
    if (s0 != 0.0f) r = fmaf(s0, u[idx], r);
    float r2 = 0.0f;
    for (int k = 0; k < src.n; ++k) {
      const float gk = static_cast<const float*>(src.g[k])[idx];
      r = fmaf((float)src.a[k], gk, r);
      r2 = fmaf((float)src.b[k], gk, r2);
    }
    out1[idx] = r;
    if (out2) out2[idx] = r2;
  }
}

// FP32 fused Leja iteration; Leja scalars arrive in FP64 and are rounded once
// per iteration; per-thread square sums in FP32, block sums in FP64.
// FP32 fused iteration, warp-specialised bulk-copy pipeline (tile_f32_bulk.cuh).
template <bool AUG, int ADV>
__global__ void __launch_bounds__(kBulkThreads) leja_iter_f32_bulk_k(SeriesArgs a) {
  extern __shared__ __align__(16) float ring[];
  __shared__ __align__(8) uint64_t full[kBulkStages], empty[kBulkStages];
  __shared__ float rowsign[kBulkStages];
  const volatile Ctrl* vc = a.ctrl;
  if (vc->stop) return;
  const int m = vc->m;
  const LejaCoef lc = a.lc[m];
  const float* __restrict__ yin = static_cast<const float*>(a.y[m & 1]);
  float* __restrict__ yout = static_cast<float*>(a.y[(m + 1) & 1]);
  float* __restrict__ p = static_cast<float*>(a.p);
  const float ig = (float)(1.0 / a.gamma);
  const float sh = (float)(a.c / a.gamma + lc.xi);
  const float d = (float)lc.d, e1 = (float)lc.e1, e2 = (float)lc.e2;
  if (threadIdx.x == 0) {
    for (int k = 0; k < kBulkStages; ++k) {
      mbar_init(&full[k], 2u);               // producer's expect_tx arrive + cp.async arrive
      mbar_init(&empty[k], kThreads / 32);   // one arrive per consumer warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  BulkItems it;
  it.tiles_x = (a.g.nx + kTileCols - 1) / kTileCols;
  it.ntiles = it.tiles_x * ((a.g.ny + kBulkTY - 1) / kBulkTY);
  it.tile0 = blockIdx.x;
  it.stride = gridDim.x;
  double accy = 0.0, accp = 0.0;
  int failed = 0;
  if (threadIdx.x >= kThreads)
    bulk_producer<AUG, ADV>(a, yin, it, ring, full, empty, rowsign, failed);
  else
    bulk_consumer<AUG, ADV>(a, lc, yout, p, it, ring, full, empty, rowsign, ig, sh, d, e1, e2,
                            accy, accp, failed);
  if (failed) a.ctrl->status = 4;            // AD_ERR_TIMEOUT; the series stops
  series_finish(a, accy, accp);
}

// FP32 fused iteration by register marching (tile_f32_vec.cuh).
template <bool AUG, int ADV>
__global__ void __launch_bounds__(kVecThreads, 2) leja_iter_f32_vec_k(SeriesArgs a) {
  const volatile Ctrl* vc = a.ctrl;
  if (vc->stop) return;
  const int m = vc->m;
  const LejaCoef lc = a.lc[m];
  const float* __restrict__ yin = static_cast<const float*>(a.y[m & 1]);
  float* __restrict__ yout = static_cast<float*>(a.y[(m + 1) & 1]);
  float* __restrict__ p = static_cast<float*>(a.p);
  const float ig = (float)(1.0 / a.gamma);
  const float sh = (float)(a.c / a.gamma + lc.xi);
  const float d = (float)lc.d, e1 = (float)lc.e1, e2 = (float)lc.e2;
  VGeo G;
  G.nx = a.g.nx;
  G.ny = a.g.ny;
  G.bc = a.g.bc;
  G.n = a.g.n;
  G.lane = threadIdx.x & 31;
  const long long strips = (G.nx + kVecCols - 1) / kVecCols;
  const long long units = strips * G.ny;
  const long long warps = (long long)gridDim.x * (kVecThreads / 32);
  const long long w = (long long)blockIdx.x * (kVecThreads / 32) + (threadIdx.x >> 5);
  long long u0, u1;
  vec_range(units, warps, w, u0, u1);
  float ly = 0.f, lp = 0.f;
  for (long long u = u0; u < u1;) {
    const int strip = (int)(u / G.ny);
    const int r0 = (int)(u - (long long)strip * G.ny);
    const long long rr = r0 + (u1 - u);
    const int r1 = (int)(rr < G.ny ? rr : G.ny);
    G.x = strip * kVecCols + 4 * G.lane;
    G.active = G.x < G.nx;
    vec_run<AUG, ADV>(a, G, r0, r1, yin, yout, p, ig, sh, d, e1, e2, ly, lp);
    u += r1 - r0;
  }
  series_finish(a, (double)ly, (double)lp);
}

// FP32 fused iteration by register marching from per-warp cp.async rings
// (tile_f32_ring.cuh); one block of 8 warps per SM.
template <bool AUG, int ADV>
__global__ void __launch_bounds__(kRingThreads, 1) leja_iter_f32_ring_k(SeriesArgs a) {
  extern __shared__ __align__(16) float ring_smem[];
  const volatile Ctrl* vc = a.ctrl;
  if (vc->stop) return;
  const int m = vc->m;
  const LejaCoef lc = a.lc[m];
  const float* __restrict__ yin = static_cast<const float*>(a.y[m & 1]);
  float* __restrict__ yout = static_cast<float*>(a.y[(m + 1) & 1]);
  float* __restrict__ p = static_cast<float*>(a.p);
  const float ig = (float)(1.0 / a.gamma);
  const float sh = (float)(a.c / a.gamma + lc.xi);
  const float d = (float)lc.d, e1 = (float)lc.e1, e2 = (float)lc.e2;
  using L = RingLayout<AUG, ADV>;
  float* ring = ring_smem + (size_t)(threadIdx.x >> 5) * L::STAGES * L::SIZE;
  VGeo G;
  G.nx = a.g.nx;
  G.ny = a.g.ny;
  G.bc = a.g.bc;
  G.n = a.g.n;
  G.lane = threadIdx.x & 31;
  const long long strips = (G.nx + kVecCols - 1) / kVecCols;
  const long long units = strips * G.ny;
  const long long warps = (long long)gridDim.x * kRingWarps;
  const long long w = (long long)blockIdx.x * kRingWarps + (threadIdx.x >> 5);
  long long u0, u1;
  vec_range(units, warps, w, u0, u1);
  float ly = 0.f, lp = 0.f;
  for (long long u = u0; u < u1;) {
    const int strip = (int)(u / G.ny);
    const int r0 = (int)(u - (long long)strip * G.ny);
    const long long rr = r0 + (u1 - u);
    const int r1 = (int)(rr < G.ny ? rr : G.ny);
    G.x = strip * kVecCols + 4 * G.lane;
    G.active = G.x < G.nx;
    ring_run<AUG, ADV>(a, G, ring, r0, r1, yin, yout, p, ig, sh, d, e1, e2, ly, lp);
    u += r1 - r0;
  }
  series_finish(a, (double)ly, (double)lp);
}

// Two fused FP32 iterations per launch by register marching over overlapped
// 120-column strips fed by per-warp cp.async rings (tile_f32_pair.cuh); one
// block of 8 warps per SM.
template <int ADV, int MODE>
__global__ void __launch_bounds__(kPairWarps * 32, 1) leja_iter2_f32_ring_k(SeriesArgs a) {
  extern __shared__ __align__(16) float pair_smem[];
  const volatile Ctrl* vc = a.ctrl;
  if (vc->stop) return;
  const int m = vc->m;                                 // even in pair mode
  const LejaCoef lc1 = a.lc[m], lc2 = a.lc[m + 1];
  PairCtx X;
  X.F = static_cast<const float*>(a.coef);
  X.yin = static_cast<const float*>(a.y[(m >> 1) & 1]);
  X.yout = static_cast<float*>(a.y[((m >> 1) + 1) & 1]);
  X.p = static_cast<float*>(a.p);
  X.ring = pair_smem + (size_t)(threadIdx.x >> 5) * PairLayout::STAGES * PairLayout::SIZE;
  X.stages = PairLayout::STAGES;
  X.G.nx = a.g.nx;
  X.G.ny = a.g.ny;
  X.G.bc = a.g.bc;
  X.G.n = a.g.n;
  X.G.lane = threadIdx.x & 31;
  X.ig = (float)(1.0 / a.gamma);
  X.sh1 = (float)(a.c / a.gamma + lc1.xi);
  X.sh2 = (float)(a.c / a.gamma + lc2.xi);
  X.d0 = m > 0 ? (float)a.lc[m - 1].d : 0.0f;          // pending d_m y_m
  X.d1 = (float)lc1.d;
  X.d2 = (float)lc2.d;
  X.abx = a.abx;
  X.aby = a.aby;
  // bands of rows, one per warp of each strip (at least 8 rows each)
  const int strips = (X.G.nx + kPairOwn - 1) / kPairOwn;
  const long long warps = (long long)gridDim.x * kPairWarps;
  long long bands = warps / strips;
  if (bands > X.G.ny / 8) bands = X.G.ny / 8;
  if (bands < 1) bands = 1;
  const long long units = bands * strips;
  const long long w = (long long)blockIdx.x * kPairWarps + (threadIdx.x >> 5);
  long long u0, u1;
  vec_range(units, warps, w, u0, u1);
  float ly1 = 0.f, lp1 = 0.f, ly2 = 0.f, lp2 = 0.f;
  for (long long u = u0; u < u1; ++u) {
    const long long b = u / strips;
    const int X0 = (int)(u - b * strips) * kPairOwn;
    X.y0 = (int)(X.G.ny * b / bands);
    X.y1 = (int)(X.G.ny * (b + 1) / bands);
    X.L = pair_lane(X0, X.G.lane, X.G.nx, X.G.bc);
    X.gx = X0 - 4 + 4 * X.G.lane;
    X.fix = X.G.bc != 0 && (X0 == 0 || X0 + kPairOwn >= X.G.nx);
    CpAsyncLoader ldr;
    if (MODE == 2) pair_run_pf<ADV, true>(X, ldr, ly1, lp1, ly2, lp2);
    else if (MODE == 1) pair_run_pf<ADV>(X, ldr, ly1, lp1, ly2, lp2);
    else pair_run<ADV>(X, ldr, ly1, lp1, ly2, lp2);
  }
  series_finish2(a, (double)ly1, (double)lp1, (double)ly2, (double)lp2);
}

size_t pair_smem_bytes() {
  return sizeof(float) * (size_t)kPairWarps * PairLayout::STAGES * PairLayout::SIZE;
}

// The same two iterations with the row records brought in by TMA
// (tile_f32_pair_tma.cuh): zero-Dirichlet grids.  Dynamic shared memory: the
// rings (aligned to 128 bytes for the copies), then each warp's STAGES
// mbarriers.
template <int ADV>
__global__ void __launch_bounds__(kPairWarps * 32, 1)
    leja_iter2_f32_tma_k(SeriesArgs a, const __grid_constant__ PairTmaMaps maps) {
  extern __shared__ __align__(16) unsigned char pair_tma_smem[];
  const volatile Ctrl* vc = a.ctrl;
  if (vc->stop) return;
  const int m = vc->m;                                 // even in pair mode
  const LejaCoef lc1 = a.lc[m], lc2 = a.lc[m + 1];
  float* rings = reinterpret_cast<float*>(
      (reinterpret_cast<uintptr_t>(pair_tma_smem) + 127) & ~uintptr_t(127));
  const int warp = threadIdx.x >> 5;
  constexpr int stages = PairLayout::STAGES;   // a constant: the slot index is a cheap modulo
  uint64_t* bars = reinterpret_cast<uint64_t*>(
                       rings + (size_t)kPairWarps * stages * PairLayout::SIZE) +
                   warp * stages;
  PairCtx X;
  X.F = static_cast<const float*>(a.coef);
  X.stages = stages;
  X.yin = static_cast<const float*>(a.y[(m >> 1) & 1]);
  X.yout = static_cast<float*>(a.y[((m >> 1) + 1) & 1]);
  X.p = static_cast<float*>(a.p);
  X.ring = rings + (size_t)warp * stages * PairLayout::SIZE;
  X.G.nx = a.g.nx;
  X.G.ny = a.g.ny;
  X.G.bc = a.g.bc;
  X.G.n = a.g.n;
  X.G.lane = threadIdx.x & 31;
  X.ig = (float)(1.0 / a.gamma);
  X.sh1 = (float)(a.c / a.gamma + lc1.xi);
  X.sh2 = (float)(a.c / a.gamma + lc2.xi);
  X.d0 = m > 0 ? (float)a.lc[m - 1].d : 0.0f;          // pending d_m y_m
  X.d1 = (float)lc1.d;
  X.d2 = (float)lc2.d;
  X.abx = a.abx;
  X.aby = a.aby;
  if (X.G.lane == 0) {
    for (int s = 0; s < stages; ++s) mbar_init(bars + s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  TmaLoader ldr{&maps, &maps.y[(m >> 1) & 1], bars, a.ctrl, 0u, 0u, false};
  // bands of rows, one per warp of each strip (at least 8 rows each)
  const int strips = (X.G.nx + kPairOwn - 1) / kPairOwn;
  const long long warps = (long long)gridDim.x * kPairWarps;
  long long bands = warps / strips;
  if (bands > X.G.ny / 8) bands = X.G.ny / 8;
  if (bands < 1) bands = 1;
  const long long units = bands * strips;
  const long long w = (long long)blockIdx.x * kPairWarps + warp;
  long long u0, u1;
  vec_range(units, warps, w, u0, u1);
  float ly1 = 0.f, lp1 = 0.f, ly2 = 0.f, lp2 = 0.f;
  for (long long u = u0; u < u1; ++u) {
    const long long b = u / strips;
    const int X0 = (int)(u - b * strips) * kPairOwn;
    X.y0 = (int)(X.G.ny * b / bands);
    X.y1 = (int)(X.G.ny * (b + 1) / bands);
    X.L = pair_lane(X0, X.G.lane, X.G.nx, X.G.bc);
    X.gx = X0 - 4 + 4 * X.G.lane;
    X.fix = X.G.bc != 0 && (X0 == 0 || X0 + kPairOwn >= X.G.nx);
    pair_run<ADV>(X, ldr, ly1, lp1, ly2, lp2);
  }
  series_finish2(a, (double)ly1, (double)lp1, (double)ly2, (double)lp2);
}

size_t pair_tma_smem_bytes() {
  return pair_smem_bytes() + 128 + sizeof(uint64_t) * kPairWarps * PairLayout::STAGES;
}

// The TMA row loader is measured slower than the cp.async rings on this
// kernel (116 vs 95 us per 4096^2 launch: the marching is bound by issue
// latency, and lane 0's copy issue sits on the warp's critical path), so it
// runs only when asked for: AD_F32_TMA=1.
bool pair_tma_enabled() {
  static const bool on = [] {
    const char* e = getenv("AD_F32_TMA");
    return e && e[0] == '1';
  }();
  return on;
}

// After a pair-mode series: add the pending d_m y_m when it stopped after an
// even count m (y_m in buffer (m / 2) & 1).
__global__ void pair_flush_k(SeriesArgs a) {
  const int m = a.ctrl->m;
  if (m == 0 || (m & 1)) return;
  const float d = (float)a.lc[m - 1].d;
  const float* y = static_cast<const float*>(a.y[(m >> 1) & 1]);
  float* p = static_cast<float*>(a.p);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.g.n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = fmaf(d, y[i], p[i]);
}

template <bool AUG, int ADV>
size_t ring_smem_bytes() {
  return sizeof(float) * (size_t)kRingWarps * RingLayout<AUG, ADV>::STAGES *
         RingLayout<AUG, ADV>::SIZE;
}

// The start of an FP32 phi_1 series whose vector is w1 = A u + sum_k c_k g_k
// (the midpoint step's right-hand side), in one marching pass of the ring
// kernel: the pass reads u with scale 1 and shift 0, the source fields as the
// couplings of the augmented form (g0 through w2, g1 through w1; SRC: any
// source at all), and p as 0, and writes y_0 = w1 and p_0 = d0 y_0.  Block 0
// resets the control block as series_init does.  Replaces the apply kernel,
// which forms each cell from 21 cached loads, and the series start.
template <bool SRC, int ADV>
__global__ void __launch_bounds__(kRingThreads, 1)
    series_start_f32_ring_k(SeriesArgs a, const float* __restrict__ u, float c0, float c1,
                            float d0, int force, int max_iters, double tol) {
  extern __shared__ __align__(16) float ring_smem[];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Ctrl* c = a.ctrl;
    c->m = 0;
    c->stop = 0;
    c->iters = 0;
    c->status = 0;
    c->force = force;
    c->max_iters = max_iters;
    c->ticket = 0u;
    c->tol = tol;
    c->err_est = 0.0;
    c->ynorm2 = 0.0;
    c->pnorm2 = 0.0;
  }
  float* __restrict__ y0 = static_cast<float*>(a.y[0]);
  float* __restrict__ p = static_cast<float*>(a.p);
  using L = RingLayout<SRC, ADV>;
  float* ring = ring_smem + (size_t)(threadIdx.x >> 5) * L::STAGES * L::SIZE;
  VGeo G;
  G.nx = a.g.nx;
  G.ny = a.g.ny;
  G.bc = a.g.bc;
  G.n = a.g.n;
  G.lane = threadIdx.x & 31;
  const long long strips = (G.nx + kVecCols - 1) / kVecCols;
  const long long units = strips * G.ny;
  const long long warps = (long long)gridDim.x * kRingWarps;
  const long long w = (long long)blockIdx.x * kRingWarps + (threadIdx.x >> 5);
  long long u0, u1;
  vec_range(units, warps, w, u0, u1);
  float ly = 0.f, lp = 0.f;
  for (long long q = u0; q < u1;) {
    const int strip = (int)(q / G.ny);
    const int r0 = (int)(q - (long long)strip * G.ny);
    const long long rr = r0 + (u1 - q);
    const int r1 = (int)(rr < G.ny ? rr : G.ny);
    G.x = strip * kVecCols + 4 * G.lane;
    G.active = G.x < G.nx;
    ring_run<SRC, ADV>(a, G, ring, r0, r1, u, y0, p, 1.0f, 0.0f, d0, c0, c1, ly, lp, true);
    q += r1 - r0;
  }
}

template <bool AUG, int ADV>
__global__ void __launch_bounds__(kThreads) leja_iter_f32_k(SeriesArgs a) {
  __shared__ float sy[3][kTileCols + 2];
  __shared__ float sxy[2][kTileCols + 2];
  __shared__ float sxx[kTileCols + 2];
  __shared__ float sax[kTileCols + 2];
  const volatile Ctrl* vc = a.ctrl;
  if (vc->stop) return;
  const int m = vc->m;
  const LejaCoef lc = a.lc[m];
  const float* __restrict__ yin = static_cast<const float*>(a.y[m & 1]);
  float* __restrict__ yout = static_cast<float*>(a.y[(m + 1) & 1]);
  float* __restrict__ p = static_cast<float*>(a.p);
  const float ig = (float)(1.0 / a.gamma);
  const float sh = (float)(a.c / a.gamma + lc.xi);
  const float d = (float)lc.d, e1 = (float)lc.e1, e2 = (float)lc.e2;
  const int tiles_x = (a.g.nx + kTileCols - 1) / kTileCols;
  const int tiles_y = (a.g.ny + kTileRows - 1) / kTileRows;
  double accy = 0.0, accp = 0.0;
  for (int tile = blockIdx.x; tile < tiles_x * tiles_y; tile += gridDim.x)
    tile_f32<AUG, ADV>(a, lc, tile % tiles_x, tile / tiles_x, yin, yout, p, ig, sh, d, e1, e2,
                       sy, sxx, sxy, sax, accy, accp);
  series_finish(a, accy, accp);
}

}  // namespace

// Marching of the two-iteration kernels: 1 pair_run_pf (one row of
// lookahead in registers, the default of single series), 0 pair_run, 2
// pair_run_pf with the stencil levels in packed FP32 pairs (AD_F32_MARCH
// selects; batches tune 1 against 2 on their persistent kernel).  Measured
// at 4096^2 without advection: 0: 94.6, 1: 90.7, 2: 93.5 us per launch; on the
// 128-slice batch (constant advection) a full pass of the persistent kernel
// takes 0.859 ms with 1 and 0.814 ms with 2.  A marching with level 2 one row
// further behind level 1 (two independent chains per step) took 98.9 us and
// was dropped.
int pair_march_env() {
  static const int mode = [] {
    const char* e = getenv("AD_F32_MARCH");
    return e && e[0] >= '0' && e[0] <= '2' && e[1] == 0 ? e[0] - '0' : -1;
  }();
  return mode;
}

int pair_march() {
  const int m = pair_march_env();
  return m < 0 ? 1 : m;
}

namespace {
// The two-iteration kernels by marching (pair_march) and advection (none,
// constant): the launch picks from this table, and the shared-memory opt-in
// runs over all of it.
void* const kPairKernels[3][2] = {
    {(void*)leja_iter2_f32_ring_k<0, 0>, (void*)leja_iter2_f32_ring_k<1, 0>},
    {(void*)leja_iter2_f32_ring_k<0, 1>, (void*)leja_iter2_f32_ring_k<1, 1>},
    {(void*)leja_iter2_f32_ring_k<0, 2>, (void*)leja_iter2_f32_ring_k<1, 2>}};
}  // namespace

// Failure-detection check of the bounded waits: one block waits on an
// mbarrier whose phase never completes (two arrivals expected, one made) and
// must give up after timeout_ns, recording 4 (timeout) in *status.
__global__ void wait_timeout_probe_k(unsigned long long timeout_ns, int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 2u);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_arrive(&bar);
    const unsigned long long t0 = global_ns_();
    int st = 0;
    while (!mbar_try_wait(&bar, 0u)) {
      if (global_ns_() - t0 > timeout_ns) { st = 4; break; }
    }
    *status = st;
    mbar_arrive(&bar);   // complete the phase so the barrier is left consistent
  }
}

int wait_timeout_probe(unsigned long long timeout_ns, int* status_dev, cudaStream_t s) {
  ++launch_counter();
  wait_timeout_probe_k<<<1, 32, 0, s>>>(timeout_ns, status_dev);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

// FP64 FMA rate probe: every thread runs four independent chains
// a <- a * b + c (b just below 1, so the chains stay finite); the result is
// stored only under a condition that never holds, which keeps the chains
// live without a memory stream.
__global__ void __launch_bounds__(kThreads) dfma_rate_k(int iters, double* sink) {
  double a0 = 1.0 + 1e-3 * threadIdx.x, a1 = a0 + 0.25, a2 = a0 + 0.5, a3 = a0 + 0.75;
  const double b = 0.99999999, c = 1e-9;
#pragma unroll 4
  for (int k = 0; k < iters; ++k) {
    a0 = fma(a0, b, c);
    a1 = fma(a1, b, c);
    a2 = fma(a2, b, c);
    a3 = fma(a3, b, c);
  }
  if (a0 + a1 + a2 + a3 < -1.0) sink[blockIdx.x] = a0;
}

int fp64_fma_rate(int blocks, int iters, cudaStream_t s, double* tflops) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return 2;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return 2; }
  launch_counter() += 2;
  dfma_rate_k<<<blocks, kThreads, 0, s>>>(iters, nullptr);      // warm-up (clocks up)
  cudaEventRecord(e0, s);
  dfma_rate_k<<<blocks, kThreads, 0, s>>>(iters, nullptr);
  cudaEventRecord(e1, s);
  float ms = 0.f;
  const bool ok = cudaEventSynchronize(e1) == cudaSuccess &&
                  cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) return 2;
  *tflops = 2.0 * 4.0 * iters * (double)kThreads * blocks / (ms * 1e-3) / 1e12;
  return 0;
}

int series_blocks(int prec, long long n) {
  // FP64: 4 blocks per SM (two cells per thread per trip keep the FP64 pipe
  // fed; fewer blocks keep the block reductions cheap); FP32: 8 blocks per SM
  // for memory parallelism.
  if (prec == 0) {
    const long long want = (n + kThreads - 1) / kThreads;
    const long long cap = 152LL * 4;
    return (int)(want < cap ? (want < 1 ? 1 : want) : cap);
  }
  return -1;  // FP32: depends on the tile count, see series_blocks_grid
}

int series_f32_kernel(int prec, int nx) {
  if (prec != 1) return 0;
  static const int pick = [] {
    const char* e = getenv("AD_F32_KERNEL");     // tuning override: ring | vec | bulk | tile
    if (!e) return 3;
    if (e[0] == 'b') return 1;
    if (e[0] == 't') return 0;
    if (e[0] == 'v') return 2;
    return 3;
  }();
  return nx % 4 == 0 ? pick : 0;
}

int series_blocks_grid(int prec, int nx, int ny) {
  if (prec == 0) return series_blocks(0, (long long)nx * ny);
  const int kind = series_f32_kernel(prec, nx);
  if (kind == 3) {
    static bool attr = false;
    if (!attr) {   // the rings need more than the default 48 KB of dynamic shared memory
#define AD_RING_ATTR(AUGV, ADVV)                                                         \
      cudaFuncSetAttribute((void*)leja_iter_f32_ring_k<AUGV, ADVV>,                      \
                           cudaFuncAttributeMaxDynamicSharedMemorySize,                  \
                           (int)ring_smem_bytes<AUGV, ADVV>())
      AD_RING_ATTR(false, 0); AD_RING_ATTR(false, 1); AD_RING_ATTR(false, 2);
      AD_RING_ATTR(true, 0); AD_RING_ATTR(true, 1); AD_RING_ATTR(true, 2);
#undef AD_RING_ATTR
      for (const auto& row : kPairKernels)      // every marching the launches can pick
        for (void* fn : row)
          cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)pair_smem_bytes());
      cudaFuncSetAttribute((void*)leja_iter2_f32_tma_k<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)pair_tma_smem_bytes());
      cudaFuncSetAttribute((void*)leja_iter2_f32_tma_k<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)pair_tma_smem_bytes());
      attr = true;
    }
    // one block of 8 warps per SM; fewer for small grids (>= 16 rows per warp)
    const long long units = (long long)((nx + kVecCols - 1) / kVecCols) * ny;
    const long long want = (units + kRingWarps * 16 - 1) / (kRingWarps * 16);
    const long long cap = 152LL;
    return (int)(want < cap ? (want < 1 ? 1 : want) : cap);
  }
  if (kind == 2) {
    // one warp per contiguous range of >= 16 (strip, row) pairs; 2 blocks of
    // 256 threads per SM at up to 128 registers
    const long long units = (long long)((nx + kVecCols - 1) / kVecCols) * ny;
    const long long want = (units + 8 * 16 - 1) / (8 * 16);
    const long long cap = 152LL * 2;
    return (int)(want < cap ? (want < 1 ? 1 : want) : cap);
  }
  if (kind == 1) {
    static bool attr = false;
    if (!attr) {   // the ring needs more than the default 48 KB of dynamic shared memory
      const int smem = kBulkStages * kStageFloats * (int)sizeof(float);
      for (void* f : {(void*)leja_iter_f32_bulk_k<false, 0>, (void*)leja_iter_f32_bulk_k<false, 1>,
                      (void*)leja_iter_f32_bulk_k<false, 2>, (void*)leja_iter_f32_bulk_k<true, 0>,
                      (void*)leja_iter_f32_bulk_k<true, 1>, (void*)leja_iter_f32_bulk_k<true, 2>})
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      attr = true;
    }
    const long long tiles = (long long)((nx + kTileCols - 1) / kTileCols) *
                            ((ny + kBulkTY - 1) / kBulkTY);
    const long long cap = 152LL * 3;   // 3 blocks of 288 threads and 66.5 KB per SM
    return (int)(tiles < cap ? tiles : cap);
  }
  const long long tiles = (long long)((nx + kTileCols - 1) / kTileCols) *
                          ((ny + kTileRows - 1) / kTileRows);
  const long long cap = 152LL * 4;   // resident blocks of 256 threads at 64-80 registers
  return (int)(tiles < cap ? tiles : cap);
}

int stream_blocks(long long n) {
  // 152 SMs x 8 resident blocks of 256 threads, or fewer for small grids
  const long long want = (n + kThreads - 1) / kThreads;
  const long long cap = 152LL * 8;
  return (int)(want < cap ? (want < 1 ? 1 : want) : cap);
}

void pack_weights_f64(const GridDev& g, double dx, double dy, const double* Dxx, const double* Dxy,
                      const double* Dyy, const double* ax, const double* ay, double ax_c,
                      double ay_c, double* W, cudaStream_t s) {
  ++launch_counter();
  pack_weights_f64_k<<<stream_blocks(g.n), kThreads, 0, s>>>(g, dx, dy, Dxx, Dxy, Dyy, ax, ay,
                                                              ax_c, ay_c, W);
}

void scale_weights_f64(const GridDev& g, const double* W, double c, double gamma, double* Ws,
                       cudaStream_t s) {
  ++launch_counter();
  scale_weights_f64_k<<<stream_blocks(g.n), kThreads, 0, s>>>(g.n, W, c, gamma, Ws);
}

void gershgorin_partials_f64(const GridDev& g, const double* W, double* partials, int nblocks,
                             cudaStream_t s) {
  ++launch_counter();
  gershgorin_f64_k<<<nblocks, kThreads, 0, s>>>(g, W, partials);
}

void apply_f64(const GridDev& g, const double* W, const double* u, double* out1, double* out2,
               const Sources& src, cudaStream_t s) {
  ++launch_counter();
  apply_f64_k<<<stream_blocks(g.n), kThreads, 0, s>>>(g, W, u, out1, out2, src, 0.0, 1.0);
}

void pack_fields_f32(const GridDev& g, double dx, double dy, const double* Dxx, const double* Dxy,
                     const double* Dyy, const double* ax, const double* ay, double ax_c,
                     double ay_c, float* F, cudaStream_t s) {
  ++launch_counter();
  pack_fields_f32_k<<<stream_blocks(g.n), kThreads, 0, s>>>(g, dx, dy, Dxx, Dxy, Dyy, ax, ay,
                                                             ax_c, ay_c, F);
}

void gershgorin_partials_f32(const GridDev& g, const float* F, int adv, float abx, float aby,
                             double* partials, int nblocks, cudaStream_t s) {
  ++launch_counter();
  gershgorin_f32_k<<<nblocks, kThreads, 0, s>>>(g, F, adv, abx, aby, partials);
}

void apply_f32(const GridDev& g, const float* F, int adv, float abx, float aby, const float* u,
               float* out1, float* out2, const Sources& src, cudaStream_t s) {
  ++launch_counter();
  apply_f32_k<<<stream_blocks(g.n), kThreads, 0, s>>>(g, F, adv, abx, aby, u, out1, out2, src,
                                                       0.0f, 1.0f);
}

// The large-grid FP64 iteration forms its norms' sums of squares off the FP64
// pipe (SqSum) unless AD_F64_NORMS=fp64 asks for FP64 FMAs.  Measured on the
// 4096^2 workload: 0.397 against 0.428 ms per iteration (the FP64 pipe is fed
// 11 instructions per cell instead of 13, at 89 % of a plain DFMA loop's rate
// against 96 %); with one cell per thread and 6 blocks per SM 0.394 ms, with
// four cells per thread 0.399 ms.
static bool f64_int_squares() {
  static const bool on = [] {
    const char* e = getenv("AD_F64_NORMS");
    return !(e && e[0] == 'f');
  }();
  return on;
}

void series_iteration(const SeriesArgs& a, cudaStream_t s) {
  if (a.prec == 0) {
    ++launch_counter();
    if (f64_int_squares()) {
      if (a.aug) leja_iter_f64_k<true, true><<<a.nblocks, kThreads, 0, s>>>(a);
      else leja_iter_f64_k<false, true><<<a.nblocks, kThreads, 0, s>>>(a);
    } else {
      if (a.aug) leja_iter_f64_k<true, false><<<a.nblocks, kThreads, 0, s>>>(a);
      else leja_iter_f64_k<false, false><<<a.nblocks, kThreads, 0, s>>>(a);
    }
  } else if (series_pair(a)) {
    ++launch_counter();
    if (series_pair_tma(a)) {
      const size_t smem = pair_tma_smem_bytes();
      if (a.adv == 0)
        leja_iter2_f32_tma_k<0><<<a.nblocks, kPairWarps * 32, smem, s>>>(a, *a.tma);
      else
        leja_iter2_f32_tma_k<1><<<a.nblocks, kPairWarps * 32, smem, s>>>(a, *a.tma);
    } else {
      void* args[] = {const_cast<SeriesArgs*>(&a)};
      cudaLaunchKernel(kPairKernels[pair_march()][a.adv == 0 ? 0 : 1], dim3(a.nblocks),
                       dim3(kPairWarps * 32), args, pair_smem_bytes(), s);
    }
  } else if (a.f32k == 3) {
    ++launch_counter();
#define AD_F32R_LAUNCH(AUGV, ADVV)                                                  \
    leja_iter_f32_ring_k<AUGV, ADVV><<<a.nblocks, kRingThreads,                      \
                                       ring_smem_bytes<AUGV, ADVV>(), s>>>(a)
    if (a.aug) {
      if (a.adv == 0) AD_F32R_LAUNCH(true, 0);
      else if (a.adv == 1) AD_F32R_LAUNCH(true, 1);
      else AD_F32R_LAUNCH(true, 2);
    } else {
      if (a.adv == 0) AD_F32R_LAUNCH(false, 0);
      else if (a.adv == 1) AD_F32R_LAUNCH(false, 1);
      else AD_F32R_LAUNCH(false, 2);
    }
#undef AD_F32R_LAUNCH
  } else if (a.f32k == 2) {
    ++launch_counter();
#define AD_F32V_LAUNCH(AUGV, ADVV) \
    leja_iter_f32_vec_k<AUGV, ADVV><<<a.nblocks, kVecThreads, 0, s>>>(a)
    if (a.aug) {
      if (a.adv == 0) AD_F32V_LAUNCH(true, 0);
      else if (a.adv == 1) AD_F32V_LAUNCH(true, 1);
      else AD_F32V_LAUNCH(true, 2);
    } else {
      if (a.adv == 0) AD_F32V_LAUNCH(false, 0);
      else if (a.adv == 1) AD_F32V_LAUNCH(false, 1);
      else AD_F32V_LAUNCH(false, 2);
    }
#undef AD_F32V_LAUNCH
  } else if (a.f32k == 1) {
    // bulk-copy pipeline
    ++launch_counter();
    const size_t smem = (size_t)kBulkStages * kStageFloats * sizeof(float);
#define AD_F32B_LAUNCH(AUGV, ADVV) \
    leja_iter_f32_bulk_k<AUGV, ADVV><<<a.nblocks, kBulkThreads, smem, s>>>(a)
    if (a.aug) {
      if (a.adv == 0) AD_F32B_LAUNCH(true, 0);
      else if (a.adv == 1) AD_F32B_LAUNCH(true, 1);
      else AD_F32B_LAUNCH(true, 2);
    } else {
      if (a.adv == 0) AD_F32B_LAUNCH(false, 0);
      else if (a.adv == 1) AD_F32B_LAUNCH(false, 1);
      else AD_F32B_LAUNCH(false, 2);
    }
#undef AD_F32B_LAUNCH
  } else {
    ++launch_counter();
#define AD_F32_LAUNCH(AUGV, ADVV) leja_iter_f32_k<AUGV, ADVV><<<a.nblocks, kThreads, 0, s>>>(a)
    if (a.aug) {
      if (a.adv == 0) AD_F32_LAUNCH(true, 0);
      else if (a.adv == 1) AD_F32_LAUNCH(true, 1);
      else AD_F32_LAUNCH(true, 2);
    } else {
      if (a.adv == 0) AD_F32_LAUNCH(false, 0);
      else if (a.adv == 1) AD_F32_LAUNCH(false, 1);
      else AD_F32_LAUNCH(false, 2);
    }
#undef AD_F32_LAUNCH
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

bool encode_pair_tma(const GridDev& g, const void* y0, const void* y1, const void* p,
                     const float* F, PairTmaMaps* out) {
  static const EncodeTiledFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (EncodeTiledFn) nullptr;
    }
    return (EncodeTiledFn)f;
  }();
  if (!fn || g.nx % 4 != 0) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny};
  const cuuint64_t strides[1] = {(cuuint64_t)g.nx * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)PairLayout::XY, 1};    // 128 columns, one row
  const cuuint32_t step[2] = {1, 1};
  auto enc = [&](CUtensorMap* m, const void* base) {
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box,
              step, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;   // out of range: zeros
  };
  const long long n = g.n;
  return enc(&out->y[0], y0) && enc(&out->y[1], y1) && enc(&out->p, p) && enc(&out->xx, F) &&
         enc(&out->yy, F + n) && enc(&out->xy, F + 2 * n);
}

bool series_pair(const SeriesArgs& a) {
  static const bool off = [] {
    const char* e = getenv("AD_F32_PAIR");        // tuning override: 0 = one iteration per launch
    return e && e[0] == '0';
  }();
  return !off && a.prec == 1 && a.f32k == 3 && !a.aug && a.adv != 2 && a.g.ny >= 2;
}

bool series_pair_tma(const SeriesArgs& a) {
  return series_pair(a) && a.tma && a.g.bc != 0 && pair_tma_enabled();
}

void series_flush_pair(const SeriesArgs& a, cudaStream_t s) {
  ++launch_counter();
  pair_flush_k<<<stream_blocks(a.g.n), kThreads, 0, s>>>(a);
}

// u = 1 u + b (p + the pending d_m y_m of an even count) in one pass: the
// flush and the axpby that follows it, with their arithmetic (p is completed
// in registers, not written back).
__global__ void pair_finish_update_k(SeriesArgs a, float* u, float b) {
  const int m = a.ctrl->m;
  const bool pending = m > 0 && !(m & 1);
  const float d = pending ? (float)a.lc[m - 1].d : 0.0f;
  const float* y = static_cast<const float*>(a.y[(m >> 1) & 1]);
  const float* p = static_cast<const float*>(a.p);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.g.n;
       i += (long long)gridDim.x * blockDim.x) {
    const float pv = pending ? fmaf(d, y[i], p[i]) : p[i];
    u[i] = fmaf(b, pv, 1.0f * u[i]);
  }
}

void series_finish_pair_update(const SeriesArgs& a, void* u, double b, cudaStream_t s) {
  ++launch_counter();
  pair_finish_update_k<<<stream_blocks(a.g.n), kThreads, 0, s>>>(a, static_cast<float*>(u),
                                                                  (float)b);
}

bool series_start_f32(const SeriesArgs& a, const void* u, const Sources& S, double d0, int force,
                      int max_iters, double tol, cudaStream_t s) {
  if (a.prec != 1 || a.aug || a.f32k != 3 || S.n > 2) return false;
  // the ring pass reads u and the source fields with 16-byte copies: a caller
  // vector on a weaker alignment takes the apply path instead
  uintptr_t bits = reinterpret_cast<uintptr_t>(u);
  for (int k = 0; k < S.n; ++k) bits |= reinterpret_cast<uintptr_t>(S.g[k]);
  if (bits & 15u) return false;
  SeriesArgs b = a;
  b.w2 = S.n > 0 ? S.g[0] : nullptr;
  b.w1 = S.n > 1 ? S.g[1] : nullptr;
  const float c0 = S.n > 0 ? (float)S.a[0] : 0.0f, c1 = S.n > 1 ? (float)S.a[1] : 0.0f;
  const float* uf = static_cast<const float*>(u);
  const float fd0 = (float)d0;
  const bool src = S.n > 0;
  void* fn = nullptr;
  size_t smem = 0;
#define AD_START(SRCV, ADVV)                                                  \
  fn = (void*)series_start_f32_ring_k<SRCV, ADVV>;                            \
  smem = ring_smem_bytes<SRCV, ADVV>();
  if (src) {
    if (a.adv == 0) { AD_START(true, 0) } else if (a.adv == 1) { AD_START(true, 1) } else { AD_START(true, 2) }
  } else {
    if (a.adv == 0) { AD_START(false, 0) } else if (a.adv == 1) { AD_START(false, 1) } else { AD_START(false, 2) }
  }
#undef AD_START
  static bool attr[2][3] = {};
  if (!attr[src][a.adv]) {   // the rings need more than the default 48 KB of shared memory
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    attr[src][a.adv] = true;
  }
  void* args[] = {&b, &uf, (void*)&c0, (void*)&c1, (void*)&fd0, &force, &max_iters, &tol};
  ++launch_counter();
  return cudaLaunchKernel(fn, dim3(a.nblocks), dim3(kRingThreads), args, smem, s) == cudaSuccess;
}

// shifted operator for GMRES: out = s0 u + s1 A u (+ sources)
void apply_shifted_f64(const GridDev& g, const double* W, const double* u, double* out, double s0,
                       double s1, cudaStream_t s) {
  Sources none{};
  ++launch_counter();
  apply_f64_k<<<stream_blocks(g.n), kThreads, 0, s>>>(g, W, u, out, nullptr, none, s0, s1);
}

}  // namespace ad
