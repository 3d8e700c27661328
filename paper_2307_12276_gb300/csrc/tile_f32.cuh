// FP32 tile machinery shared by the single-operator and batched Leja kernels:
// ghost mapping, the flux-form operator at one cell, and one tile of the fused
// Leja iteration marching in y with shared-memory row rings.  Included by
// stencil_kernels.cu and batched.cu; everything has internal linkage.
#pragma once
#include "ad_internal.h"

namespace ad {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One face flux of the flux form, a du + q dd, with its rounding fixed: every
// FP32 kernel forms it the same way, so kernels that evaluate the stencil in
// different code (one and two iterations per pass) agree bit for bit.
__device__ __forceinline__ float face_flux(float a, float du, float q, float dd) {
  return fmaf(a, du, q * dd);
}

// Deterministic block sum of two values; result valid in thread 0.  Lanes of
// warp 0 add eight values each, then one butterfly: far fewer FP64 additions
// than a butterfly in every warp (FP64 is the scarce pipe on this GPU).
template <int CAP = kThreads + 32>   // CAP: the most threads a calling block has
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[CAP], sb[CAP];
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

// Neighbourhood of cell (i, j) with ghost values (sign) and ghost coefficients (mirror).
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
  float fe = face_flux(axe, uE - uC, qe, (uNE + uN) - (uSE + uS));
  float fw = face_flux(axw, uC - uW, qw, (uN + uNW) - (uS + uSW));
  float fn = face_flux(ayn, uN - uC, qn, (uNE + uE) - (uNW + uW));
  float fs = face_flux(ays, uC - uS, qs, (uE + uSE) - (uW + uSW));
  if (adv != 0) {
    fe = fmaf(be, uC + uE, fe);
    fw = fmaf(bw, uW + uC, fw);
    fn = fmaf(bn, uC + uN, fn);
    fs = fmaf(bs, uS + uC, fs);
  }
  return (fe - fw) + (fn - fs);
}

// ---- FP32 fused iteration: tiles of 256 columns x TY rows, marching in y.
// Each thread owns one column of the tile; rows j-1, j, j+1 of y and the rows
// of Dxx/Dxy that need x-neighbours live in shared-memory rings, the next row
// is prefetched into registers while the current row is computed.  Steady
// state global traffic per cell: y, Dxx, Dxy, Dyy, p read, y', p written
// (28 B), + w2 (augmented) + ax, ay (advection fields).
constexpr int kTileRows = 32;      // default tile height of the single-operator kernel
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

template <bool AUG, int ADV, int TY = kTileRows>
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
  const int x0 = tx * kTileCols, y0 = ty * TY;
  const int y1 = min(ny, y0 + TY);
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
      float fe = face_flux(axe, uE - uC, qe, (uNE + uN) - (uSE + uS));
      float fw = face_flux(axw, uC - uW, qw, (uN + uNW) - (uS + uSW));
      float fn = face_flux(ayn_, uN - uC, qn, (uNE + uE) - (uNW + uW));
      float fs = face_flux(ays, uC - uS, qs, (uE + uSE) - (uW + uSW));
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

}  // namespace
}  // namespace ad
