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

// Deterministic block sum of two values; result valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[32], sb[32];
  a = warp_sum(a);
  b = warp_sum(b);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sa[wid] = a; sb[wid] = b; }
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    a = lane < nw ? sa[lane] : 0.0;
    b = lane < nw ? sb[lane] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
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
// FP64: folded 9-weight stencil.
__device__ __forceinline__ double stencil9(const double* __restrict__ W, long long n,
                                           const double* __restrict__ u, int i, int j, int nx,
                                           int ny, int bc, long long idx) {
  const double* r0 = u + (long long)j * nx;
  double acc = W[4 * n + idx] * r0[i];
  if (bc == 0) {  // periodic: wrap
    const int im = i ? i - 1 : nx - 1, ip = (i + 1 < nx) ? i + 1 : 0;
    const int jm = j ? j - 1 : ny - 1, jp = (j + 1 < ny) ? j + 1 : 0;
    const double* rm = u + (long long)jm * nx;
    const double* rp = u + (long long)jp * nx;
    acc = fma(W[0 * n + idx], rm[im], acc);
    acc = fma(W[1 * n + idx], rm[i], acc);
    acc = fma(W[2 * n + idx], rm[ip], acc);
    acc = fma(W[3 * n + idx], r0[im], acc);
    acc = fma(W[5 * n + idx], r0[ip], acc);
    acc = fma(W[6 * n + idx], rp[im], acc);
    acc = fma(W[7 * n + idx], rp[i], acc);
    acc = fma(W[8 * n + idx], rp[ip], acc);
  } else {        // Dirichlet: ghosts are folded, out-of-domain slots are 0
    const bool hm = i > 0, hp = i + 1 < nx;
    if (j > 0) {
      const double* rm = r0 - nx;
      if (hm) acc = fma(W[0 * n + idx], rm[i - 1], acc);
      acc = fma(W[1 * n + idx], rm[i], acc);
      if (hp) acc = fma(W[2 * n + idx], rm[i + 1], acc);
    }
    if (hm) acc = fma(W[3 * n + idx], r0[i - 1], acc);
    if (hp) acc = fma(W[5 * n + idx], r0[i + 1], acc);
    if (j + 1 < ny) {
      const double* rp = r0 + nx;
      if (hm) acc = fma(W[6 * n + idx], rp[i - 1], acc);
      acc = fma(W[7 * n + idx], rp[i], acc);
      if (hp) acc = fma(W[8 * n + idx], rp[i + 1], acc);
    }
  }
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
// p += d_{m+1} y_{m+1}, block partials of ||y_{m+1}||^2, ||p||^2.
template <bool AUG>
__global__ void __launch_bounds__(kThreads) leja_iter_f64_k(SeriesArgs a) {
  const Ctrl* ctrl = a.ctrl;
  if (ctrl->stop) return;
  const int m = ctrl->m;
  const LejaCoef lc = a.lc[m];
  const double* __restrict__ yin = static_cast<const double*>(a.y[m & 1]);
  double* __restrict__ yout = static_cast<double*>(a.y[(m + 1) & 1]);
  double* __restrict__ p = static_cast<double*>(a.p);
  const double* __restrict__ Ws = static_cast<const double*>(a.coef);
  const double* __restrict__ w1 = static_cast<const double*>(a.w1);
  const double* __restrict__ w2 = static_cast<const double*>(a.w2);
  const GridDev g = a.g;
  const RowTiles rt(g.nx, g.ny);
  double sy = 0.0, sp = 0.0;
  for (int t = blockIdx.x; t < rt.ntiles; t += gridDim.x) {
    const int j = t / rt.tiles_x, i = (t % rt.tiles_x) * kThreads + threadIdx.x;
    if (i >= g.nx) continue;
    const long long idx = (long long)j * g.nx + i;
    double z = stencil9(Ws, g.n, yin, i, j, g.nx, g.ny, g.bc, idx);
    z = fma(-lc.xi, yin[idx], z);
    if (AUG) {
      if (lc.e1 != 0.0) z = fma(lc.e1, w2[idx], z);
      if (lc.e2 != 0.0) z = fma(lc.e2, w1[idx], z);
    }
    yout[idx] = z;
    const double pn = fma(lc.d, z, p[idx]);
    p[idx] = pn;
    sy = fma(z, z, sy);
    sp = fma(pn, pn, sp);
  }
  block_sum2(sy, sp);
  if (threadIdx.x == 0) {
    a.partials[2 * blockIdx.x] = sy;
    a.partials[2 * blockIdx.x + 1] = sp;
  }
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
template <bool AUG>
__global__ void __launch_bounds__(kThreads) leja_iter_f32_k(SeriesArgs a) {
  const Ctrl* ctrl = a.ctrl;
  if (ctrl->stop) return;
  const int m = ctrl->m;
  const LejaCoef lc = a.lc[m];
  const float* __restrict__ yin = static_cast<const float*>(a.y[m & 1]);
  float* __restrict__ yout = static_cast<float*>(a.y[(m + 1) & 1]);
  float* __restrict__ p = static_cast<float*>(a.p);
  const float* __restrict__ F = static_cast<const float*>(a.coef);
  const float* __restrict__ w1 = static_cast<const float*>(a.w1);
  const float* __restrict__ w2 = static_cast<const float*>(a.w2);
  const GridDev g = a.g;
  const float ig = (float)(1.0 / a.gamma);
  const float sh = (float)(a.c / a.gamma + lc.xi);
  const float d = (float)lc.d, e1 = (float)lc.e1, e2 = (float)lc.e2;
  const RowTiles rt(g.nx, g.ny);
  double sy = 0.0, sp = 0.0;
  for (int t = blockIdx.x; t < rt.ntiles; t += gridDim.x) {
    const int j = t / rt.tiles_x, i = (t % rt.tiles_x) * kThreads + threadIdx.x;
    if (i >= g.nx) continue;
    const long long idx = (long long)j * g.nx + i;
    const bool interior = i > 0 && j > 0 && i + 1 < g.nx && j + 1 < g.ny;
    const float au =
        flux_apply_f32(F, g.n, yin, i, j, g.nx, g.ny, g.bc, interior, a.adv, a.abx, a.aby);
    float z = fmaf(au, ig, -sh * yin[idx]);
    if (AUG) {
      if (e1 != 0.0f) z = fmaf(e1, w2[idx], z);
      if (e2 != 0.0f) z = fmaf(e2, w1[idx], z);
    }
    yout[idx] = z;
    const float pn = fmaf(d, z, p[idx]);
    p[idx] = pn;
    sy += (double)(z * z);
    sp += (double)(pn * pn);
  }
  block_sum2(sy, sp);
  if (threadIdx.x == 0) {
    a.partials[2 * blockIdx.x] = sy;
    a.partials[2 * blockIdx.x + 1] = sp;
  }
}

}  // namespace

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
    if (a.aug) {
      ++launch_counter();
      leja_iter_f32_k<true><<<a.nblocks, kThreads, 0, s>>>(a);
    }
    else {
      ++launch_counter();
      leja_iter_f32_k<false><<<a.nblocks, kThreads, 0, s>>>(a);
    }
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
