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

namespace ad {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum of two values; result valid in thread 0.  Lanes of
// warp 0 add eight values each, then one butterfly: far fewer FP64 additions
// than a butterfly in every warp (FP64 is the scarce pipe on this GPU).
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[kThreads], sb[kThreads];
  const int t = threadIdx.x;
  __syncthreads();
  sa[t] = a;
  sb[t] = b;
  __syncthreads();
  if (t < 32) {
    double x = 0.0, y = 0.0;
    for (int k = t; k < (int)blockDim.x; k += 32) {
      x += sa[k];
      y += sb[k];
    }
    a = warp_sum(x);
    b = warp_sum(y);
  }
}

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
    } else if (!(ty == ty) || !(tp == tp)) {       // NaN: give up
      stop = 1;
      ctrl->status = 3;
    } else if (terms >= 2 && (absd * absd) * ty <= (tol * tol) * tp) {   // squared test
      stop = 1;
    } else if (terms >= ctrl->max_iters) {
      stop = 1;
      ctrl->status = 3;
    }
    if (terms >= kMaxIters) stop = 1;               // hard cap, independent of the settings
    ctrl->ticket = 0u;
    ctrl->stop = stop;
    ctrl->m = m + 1;
    __threadfence();
    if (a.has_handle)
      cudaGraphSetConditional((cudaGraphConditionalHandle)a.handle, stop ? 0u : 1u);
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

// --------------------------------------------------------------------------
// FP64: folded 9-weight stencil, branch-free.  Periodic: neighbour indices
// wrap.  Dirichlet: the ghosts are folded into the interior slots, so every
// out-of-domain slot has weight exactly 0; its index is clamped into the
// domain (any finite value times 0 adds nothing), which keeps all nine loads
// unconditional and independent.
__device__ __forceinline__ double stencil9(const double* __restrict__ W, long long n,
                                           const double* __restrict__ u, int i, int j, int nx,
                                           int ny, int bc, long long idx) {
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
  const double* rm = u + (long long)jm * nx;
  const double* r0 = u + (long long)j * nx;
  const double* rp = u + (long long)jp * nx;
  double acc = W[4 * n + idx] * r0[i];
  acc = fma(W[0 * n + idx], rm[im], acc);
  acc = fma(W[1 * n + idx], rm[i], acc);
  acc = fma(W[2 * n + idx], rm[ip], acc);
  acc = fma(W[3 * n + idx], r0[im], acc);
  acc = fma(W[5 * n + idx], r0[ip], acc);
  acc = fma(W[6 * n + idx], rp[im], acc);
  acc = fma(W[7 * n + idx], rp[i], acc);
  acc = fma(W[8 * n + idx], rp[ip], acc);
  return acc;
}

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
// cells (equal FP64 work per block: the kernel is FP64-pipe bound).
template <bool AUG>
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
      sy = fma(z[q], z[q], sy);
      sp = fma(pn, pn, sp);
    }
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

// Neighbourhood of cell (i, j) with ghost values (sign) and ghost coefficients (mirror).
struct Nbr32 {
  float u[3][3];      // u[dj+1][di+1]
  float fxx[3], fyy[3], fxy[5], fax[3], fay[3];  // centre, -, + along the axis; fxy: C,W,E,S,N
};

__device__ __forceinline__ void map_idx(int& ti, int& tj, float& sg, int nx, int ny, int bc) {
  if (bc == 0) {
    ti = (ti < 0) ? ti + nx : (ti >= nx ? ti - nx : ti);
    tj = (tj < 0) ? tj + ny : (tj >= ny ? tj - ny : tj);
  } else {
    if (ti < 0) { ti = -1 - ti; sg = -sg; } else if (ti >= nx) { ti = 2 * nx - 1 - ti; sg = -sg; }
    if (tj < 0) { tj = -1 - tj; sg = -sg; } else if (tj >= ny) { tj = 2 * ny - 1 - tj; sg = -sg; }
  }
}

// A u at one cell from the flux form (FP32 arithmetic).
// adv: 0 none, 1 constant (be = bw = abx, bn = bs = aby), 2 fields F[3], F[4].
__device__ __forceinline__ float flux_apply_f32(const float* __restrict__ F, long long n,
                                                const float* __restrict__ u, int i, int j, int nx,
                                                int ny, int bc, bool interior, int adv, float abx,
                                                float aby) {
  float U[3][3];
  float cxx[3], cyy[3], cxyx[3], cxyy[3], cax[3], cay[3];
  if (interior) {
    const long long idx = (long long)j * nx + i;
#pragma unroll
    for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
      for (int di = -1; di <= 1; ++di) U[dj + 1][di + 1] = u[idx + (long long)dj * nx + di];
#pragma unroll
    for (int d = -1; d <= 1; ++d) {
      cxx[d + 1] = F[0 * n + idx + d];
      cxyx[d + 1] = F[2 * n + idx + d];
      cyy[d + 1] = F[1 * n + idx + (long long)d * nx];
      cxyy[d + 1] = F[2 * n + idx + (long long)d * nx];
      if (adv == 2) {
        cax[d + 1] = F[3 * n + idx + d];
        cay[d + 1] = F[4 * n + idx + (long long)d * nx];
      }
    }
  } else {
#pragma unroll
    for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
      for (int di = -1; di <= 1; ++di) {
        int ti = i + di, tj = j + dj;
        float sg = 1.0f;
        map_idx(ti, tj, sg, nx, ny, bc);
        U[dj + 1][di + 1] = sg * u[(long long)tj * nx + ti];
      }
#pragma unroll
    for (int d = -1; d <= 1; ++d) {
      int ti = i + d, tj = j;
      float sg = 1.0f;
      map_idx(ti, tj, sg, nx, ny, bc);
      long long q = (long long)tj * nx + ti;
      cxx[d + 1] = F[0 * n + q];
      cxyx[d + 1] = F[2 * n + q];
      if (adv == 2) cax[d + 1] = F[3 * n + q];
      ti = i; tj = j + d; sg = 1.0f;
      map_idx(ti, tj, sg, nx, ny, bc);
      q = (long long)tj * nx + ti;
      cyy[d + 1] = F[1 * n + q];
      cxyy[d + 1] = F[2 * n + q];
      if (adv == 2) cay[d + 1] = F[4 * n + q];
    }
  }
  // face coefficients (factors 1/2 and the grid scalings are folded into F)
  const float axe = cxx[1] + cxx[2], axw = cxx[0] + cxx[1];
  const float ayn = cyy[1] + cyy[2], ays = cyy[0] + cyy[1];
  const float qe = cxyx[1] + cxyx[2], qw = cxyx[0] + cxyx[1];
  const float qn = cxyy[1] + cxyy[2], qs = cxyy[0] + cxyy[1];
  float be = abx, bw = abx, bn = aby, bs = aby;
  if (adv == 2) {
    be = cax[1] + cax[2]; bw = cax[0] + cax[1];
    bn = cay[1] + cay[2]; bs = cay[0] + cay[1];
  }
  const float uC = U[1][1], uE = U[1][2], uW = U[1][0], uN = U[2][1], uS = U[0][1];
  const float uNE = U[2][2], uNW = U[2][0], uSE = U[0][2], uSW = U[0][0];
  float fe = axe * (uE - uC) + qe * ((uNE + uN) - (uSE + uS));
  float fw = axw * (uC - uW) + qw * ((uN + uNW) - (uS + uSW));
  float fn = ayn * (uN - uC) + qn * ((uNE + uE) - (uNW + uW));
  float fs = ays * (uC - uS) + qs * ((uE + uSE) - (uW + uSW));
  if (adv != 0) {
    fe = fmaf(be, uC + uE, fe);
    fw = fmaf(bw, uW + uC, fw);
    fn = fmaf(bn, uC + uN, fn);
    fs = fmaf(bs, uS + uC, fs);
  }
  return (fe - fw) + (fn - fs);
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
// ---- FP32 fused iteration: tiles of 256 columns x kTileRows rows, marching in y.
// Each thread owns one column of the tile; rows j-1, j, j+1 of y and the rows
// of Dxx/Dxy that need x-neighbours live in shared-memory rings, the next row
// is prefetched into registers while the current row is computed.  Steady
// state global traffic per cell: y, Dxx, Dxy, Dyy, p read, y', p written
// (28 B), + w2 (augmented) + ax, ay (advection fields).
constexpr int kTileRows = 32;
constexpr int kTileCols = kThreads;

struct RowMap {
  long long off;   // mapped row offset j' * nx
  float sg;        // ghost sign for values (Dirichlet odd reflection)
};

__device__ __forceinline__ RowMap map_row(int j, int nx, int ny, int bc) {
  RowMap r;
  float sg = 1.0f;
  if (bc == 0) j = (j < 0) ? j + ny : (j >= ny ? j - ny : j);
  else if (j < 0) { j = -1 - j; sg = -1.0f; }
  else if (j >= ny) { j = 2 * ny - 1 - j; sg = -1.0f; }
  r.off = (long long)j * nx;
  r.sg = sg;
  return r;
}

__device__ __forceinline__ int map_col(int i, int nx, int bc, float& sg) {
  sg = 1.0f;
  if (bc == 0) return (i < 0) ? i + nx : (i >= nx ? i - nx : i);
  if (i < 0) { sg = -1.0f; return -1 - i; }
  if (i >= nx) { sg = -1.0f; return 2 * nx - 1 - i; }
  return i;
}

// Values needed from row r (for y, Dxy, Dxx rows with x-halo): this thread's
// column and, for thread 0, the two halo columns.
struct RowVals {
  float c, l, r;
};

__device__ __forceinline__ RowVals load_row(const float* __restrict__ f, const RowMap& rm,
                                            bool values, int ci, float csg, bool cvalid,
                                            int li, float lsg, int ri, float rsg, bool halo) {
  RowVals v;
  const float s = values ? rm.sg : 1.0f;
  v.c = cvalid ? f[rm.off + ci] * (values ? s * csg : 1.0f) : 0.0f;
  v.l = v.r = 0.0f;
  if (halo) {
    v.l = f[rm.off + li] * (values ? s * lsg : 1.0f);
    v.r = f[rm.off + ri] * (values ? s * rsg : 1.0f);
  }
  return v;
}

template <bool AUG, int ADV>
__device__ __forceinline__ void tile_f32(const SeriesArgs& a, const LejaCoef& lc, int tx, int ty,
                                         const float* __restrict__ yin, float* __restrict__ yout,
                                         float* __restrict__ p, float ig, float sh, float d,
                                         float e1, float e2, float (*sy)[kTileCols + 2],
                                         float* sxx, float (*sxy)[kTileCols + 2], float* sax,
                                         double& accy, double& accp) {
  const GridDev g = a.g;
  const int nx = g.nx, ny = g.ny, bc = g.bc;
  const long long n = g.n;
  const float* __restrict__ F = static_cast<const float*>(a.coef);
  const float* Fxx = F;
  const float* Fyy = F + n;
  const float* Fxy = F + 2 * n;
  const float* Fax = F + 3 * n;
  const float* Fay = F + 4 * n;
  const float* __restrict__ w1 = static_cast<const float*>(a.w1);
  const float* __restrict__ w2 = static_cast<const float*>(a.w2);
  const int t = threadIdx.x;
  const int x0 = tx * kTileCols, y0 = ty * kTileRows;
  const int y1 = min(ny, y0 + kTileRows);
  const int i = x0 + t;
  const bool compute = i < nx;
  const bool cvalid = i <= nx;            // column nx is the right ghost
  float csg, lsg, rsg;
  const int ci = cvalid ? map_col(i, nx, bc, csg) : 0;
  const int li = map_col(x0 - 1, nx, bc, lsg);
  const int ri = map_col(min(x0 + kTileCols, nx), nx, bc, rsg);
  const bool halo = (t == 0);
  const int rslot = min(kTileCols, nx - x0) + 1;  // smem index of the right halo
  __syncthreads();   // the previous tile's last row may still be read
  // prologue: rows y0-1 and y0 of y, row y0 of Dxy (with halos), Dyy/Dxy/ay columns
  {
    const RowMap rm = map_row(y0 - 1, nx, ny, bc), r0 = map_row(y0, nx, ny, bc);
    RowVals v = load_row(yin, rm, true, ci, csg, cvalid, li, lsg, ri, rsg, halo);
    sy[(y0 + 2) % 3][t + 1] = v.c;
    if (halo) { sy[(y0 + 2) % 3][0] = v.l; sy[(y0 + 2) % 3][rslot] = v.r; }
    v = load_row(yin, r0, true, ci, csg, cvalid, li, lsg, ri, rsg, halo);
    sy[y0 % 3][t + 1] = v.c;
    if (halo) { sy[y0 % 3][0] = v.l; sy[y0 % 3][rslot] = v.r; }
    v = load_row(Fxy, r0, false, ci, csg, cvalid, li, lsg, ri, rsg, halo);
    sxy[y0 & 1][t + 1] = v.c;
    if (halo) { sxy[y0 & 1][0] = v.l; sxy[y0 & 1][rslot] = v.r; }
  }
  float dyy_s = 0.f, dyy_c = 0.f, dxy_s = 0.f, ay_s = 0.f, ay_c = 0.f;
  {
    const RowMap rm = map_row(y0 - 1, nx, ny, bc), r0 = map_row(y0, nx, ny, bc);
    if (cvalid) {
      dyy_s = Fyy[rm.off + ci];
      dyy_c = Fyy[r0.off + ci];
      dxy_s = Fxy[rm.off + ci];
      if (ADV == 2) { ay_s = Fay[rm.off + ci]; ay_c = Fay[r0.off + ci]; }
    }
  }
  // prefetch for the first row
  RowVals ynext, xynext, xxcur, axcur;
  float dyy_n = 0.f, ay_n = 0.f, pc = 0.f, w2c = 0.f, w1c = 0.f;
  auto prefetch = [&](int j) {
    const RowMap rn = map_row(j + 1, nx, ny, bc), rc = map_row(j, nx, ny, bc);
    ynext = load_row(yin, rn, true, ci, csg, cvalid, li, lsg, ri, rsg, halo);
    xynext = load_row(Fxy, rn, false, ci, csg, cvalid, li, lsg, ri, rsg, halo);
    xxcur = load_row(Fxx, rc, false, ci, csg, cvalid, li, lsg, ri, rsg, halo);
    if (ADV == 2) axcur = load_row(Fax, rc, false, ci, csg, cvalid, li, lsg, ri, rsg, halo);
    if (cvalid) {
      dyy_n = Fyy[rn.off + ci];
      if (ADV == 2) ay_n = Fay[rn.off + ci];
    }
    if (compute) {
      const long long idx = (long long)j * nx + i;
      pc = p[idx];
      if (AUG) {
        if (e1 != 0.0f) w2c = w2[idx];
        if (e2 != 0.0f) w1c = w1[idx];
      }
    }
  };
  prefetch(y0);
  float ly = 0.f, lp = 0.f;
  for (int j = y0; j < y1; ++j) {
    __syncthreads();                       // previous row's readers are done
    const int sn = (j + 1) % 3, sc = j % 3, ss = (j + 2) % 3;
    sy[sn][t + 1] = ynext.c;
    sxy[(j + 1) & 1][t + 1] = xynext.c;
    sxx[t + 1] = xxcur.c;
    if (ADV == 2) sax[t + 1] = axcur.c;
    if (halo) {
      sy[sn][0] = ynext.l; sy[sn][rslot] = ynext.r;
      sxy[(j + 1) & 1][0] = xynext.l; sxy[(j + 1) & 1][rslot] = xynext.r;
      sxx[0] = xxcur.l; sxx[rslot] = xxcur.r;
      if (ADV == 2) { sax[0] = axcur.l; sax[rslot] = axcur.r; }
    }
    const float dyyn = dyy_n, ayn = ay_n, pcur = pc, w2cur = w2c, w1cur = w1c;
    __syncthreads();
    if (j + 1 < y1) prefetch(j + 1);       // overlap the next row's loads with this row
    if (compute) {
      const float uC = sy[sc][t + 1], uE = sy[sc][t + 2], uW = sy[sc][t];
      const float uN = sy[sn][t + 1], uNE = sy[sn][t + 2], uNW = sy[sn][t];
      const float uS = sy[ss][t + 1], uSE = sy[ss][t + 2], uSW = sy[ss][t];
      const float dxy_c = sxy[j & 1][t + 1];
      const float axe = sxx[t + 1] + sxx[t + 2], axw = sxx[t] + sxx[t + 1];
      const float qe = dxy_c + sxy[j & 1][t + 2], qw = sxy[j & 1][t] + dxy_c;
      const float qn = dxy_c + sxy[(j + 1) & 1][t + 1], qs = dxy_s + dxy_c;
      const float ayn_ = dyy_c + dyyn, ays = dyy_s + dyy_c;
      float fe = axe * (uE - uC) + qe * ((uNE + uN) - (uSE + uS));
      float fw = axw * (uC - uW) + qw * ((uN + uNW) - (uS + uSW));
      float fn = ayn_ * (uN - uC) + qn * ((uNE + uE) - (uNW + uW));
      float fs = ays * (uC - uS) + qs * ((uE + uSE) - (uW + uSW));
      if (ADV == 1) {
        fe = fmaf(a.abx, uC + uE, fe);
        fw = fmaf(a.abx, uW + uC, fw);
        fn = fmaf(a.aby, uC + uN, fn);
        fs = fmaf(a.aby, uS + uC, fs);
      } else if (ADV == 2) {
        fe = fmaf(sax[t + 1] + sax[t + 2], uC + uE, fe);
        fw = fmaf(sax[t] + sax[t + 1], uW + uC, fw);
        fn = fmaf(ay_c + ayn, uC + uN, fn);
        fs = fmaf(ay_s + ay_c, uS + uC, fs);
      }
      const float au = (fe - fw) + (fn - fs);
      float z = fmaf(au, ig, -sh * uC);
      if (AUG) {
        if (e1 != 0.0f) z = fmaf(e1, w2cur, z);
        if (e2 != 0.0f) z = fmaf(e2, w1cur, z);
      }
      const long long idx = (long long)j * nx + i;
      yout[idx] = z;
      const float pn = fmaf(d, z, pcur);
      p[idx] = pn;
      ly = fmaf(z, z, ly);
      lp = fmaf(pn, pn, lp);
    }
    // roll the column registers
    dxy_s = sxy[j & 1][t + 1];
    dyy_s = dyy_c;
    dyy_c = dyyn;
    if (ADV == 2) { ay_s = ay_c; ay_c = ayn; }
  }
  accy += (double)ly;
  accp += (double)lp;
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

int series_blocks_grid(int prec, int nx, int ny) {
  if (prec == 0) return series_blocks(0, (long long)nx * ny);
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

void series_iteration(const SeriesArgs& a, cudaStream_t s) {
  if (a.prec == 0) {
    if (a.aug) {
      ++launch_counter();
      leja_iter_f64_k<true><<<a.nblocks, kThreads, 0, s>>>(a);
    }
    else {
      ++launch_counter();
      leja_iter_f64_k<false><<<a.nblocks, kThreads, 0, s>>>(a);
    }
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

// shifted operator for GMRES: out = s0 u + s1 A u (+ sources)
void apply_shifted_f64(const GridDev& g, const double* W, const double* u, double* out, double s0,
                       double s1, cudaStream_t s) {
  Sources none{};
  ++launch_counter();
  apply_f64_k<<<stream_blocks(g.n), kThreads, 0, s>>>(g, W, u, out, nullptr, none, s0, s1);
}

}  // namespace ad
