// FP32 fused Leja iteration by register marching (rows of float4).
//
// A warp owns a strip of 128 columns; lane l holds columns x .. x+3 with
// x = x0 + 4 l, so every row of every field arrives as one coalesced 512-byte
// float4 load per warp.  The warp walks down a contiguous range of rows of its
// strip keeping three rows of y (j-1, j, j+1) and two rows of Dxy/Dyy in
// registers; the x-neighbours at x-1 and x+4 come from the neighbouring lanes
// (shuffles), lanes at the strip or domain edges load or mirror them.  Each
// face flux is formed once: the x-faces of row j as five fluxes per lane (the
// east face of a cell is the west face of the next), the north faces of row j
// are kept as the south faces of row j+1.  The same expressions as the
// per-cell form (flux_apply_f32), term for term.
//
// Work split: the (strip, row) pairs of the grid, strip-major, are divided
// into equal contiguous ranges, one per warp of the grid; a range crossing a
// strip boundary is two marching runs.  Each run re-reads two halo rows of y,
// Dxy and Dyy.  Rows of the next step are prefetched into registers while the
// current row is computed.
//
// Requirement (checked by the launcher): nx % 4 == 0, so rows start on
// 16-byte boundaries.
#pragma once
#include "tile_f32.cuh"

namespace ad {
namespace {

constexpr int kVecCols = 128;       // columns per warp strip
constexpr int kVecThreads = 256;    // 8 warps per block

struct VGeo {
  int nx, ny, bc;
  long long n;
  int x;        // first column of this lane
  int lane;
  bool active;  // x < nx
};

// One row (ghost-mapped) around the lane's four columns.
template <int ADV>
struct VRow {
  float y[6];    // columns x-1 .. x+4, row sign applied (Dirichlet ghost rows)
  float xy[6];
  float yy[4];
  float ay[ADV == 2 ? 4 : 1];
};

template <int ADV, bool AUG>
struct VCen {    // data of the row being computed
  float xx[6];
  float ax[ADV == 2 ? 6 : 1];
  float4 p;
  float4 w2;
};

__device__ __forceinline__ float4 ldg4(const float* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}

// Fill v[0] (column x-1) and v[5] (column x+4) of a row of field f.  values:
// a field of unknowns (Dirichlet mirrors carry a minus sign) rather than a
// coefficient (mirrors without sign).  rowp points at the mapped row start;
// s is the row sign already applied to v[1..4].
__device__ __forceinline__ void vhalo(float* v, const float* __restrict__ rowp, float s,
                                      bool values, const VGeo& G) {
  const float left = __shfl_up_sync(0xffffffffu, v[4], 1);
  const float right = __shfl_down_sync(0xffffffffu, v[1], 1);
  v[0] = left;
  v[5] = right;
  if (!G.active) return;
  const bool dir = G.bc != 0;
  if (G.x == 0) {
    if (dir) v[0] = values ? -v[1] : v[1];                 // mirror of column 0
    else v[0] = s * __ldg(rowp + G.nx - 1);                 // wrap
  } else if (G.lane == 0) {
    v[0] = s * __ldg(rowp + G.x - 1);
  }
  if (G.x + 4 == G.nx) {
    if (dir) v[5] = values ? -v[4] : v[4];                 // mirror of column nx-1
    else v[5] = s * __ldg(rowp);                            // wrap
  } else if (G.lane == 31) {
    v[5] = s * __ldg(rowp + G.x + 4);
  }
}

template <int ADV>
__device__ __forceinline__ void vload_row(VRow<ADV>& R, const float* __restrict__ yin,
                                          const float* __restrict__ Fxy,
                                          const float* __restrict__ Fyy,
                                          const float* __restrict__ Fay, int r, const VGeo& G) {
  const RowMap rm = map_row(r, G.nx, G.ny, G.bc);
  float4 y4 = make_float4(0.f, 0.f, 0.f, 0.f), q4 = y4, b4 = y4, a4 = y4;
  if (G.active) {
    y4 = ldg4(yin + rm.off + G.x);
    q4 = ldg4(Fxy + rm.off + G.x);
    b4 = ldg4(Fyy + rm.off + G.x);
    if (ADV == 2) a4 = ldg4(Fay + rm.off + G.x);
  }
  R.y[1] = rm.sg * y4.x; R.y[2] = rm.sg * y4.y; R.y[3] = rm.sg * y4.z; R.y[4] = rm.sg * y4.w;
  R.xy[1] = q4.x; R.xy[2] = q4.y; R.xy[3] = q4.z; R.xy[4] = q4.w;
  R.yy[0] = b4.x; R.yy[1] = b4.y; R.yy[2] = b4.z; R.yy[3] = b4.w;
  if (ADV == 2) { R.ay[0] = a4.x; R.ay[1] = a4.y; R.ay[2] = a4.z; R.ay[3] = a4.w; }
  vhalo(R.y, yin + rm.off, rm.sg, true, G);
  vhalo(R.xy, Fxy + rm.off, 1.0f, false, G);
}

template <int ADV, bool AUG>
__device__ __forceinline__ void vload_cen(VCen<ADV, AUG>& C, const float* __restrict__ Fxx,
                                          const float* __restrict__ Fax,
                                          const float* __restrict__ p,
                                          const float* __restrict__ w2, int r, const VGeo& G) {
  const long long off = (long long)r * G.nx;       // a computed row is never a ghost
  float4 x4 = make_float4(0.f, 0.f, 0.f, 0.f), a4 = x4;
  C.p = x4;
  C.w2 = x4;
  if (G.active) {
    x4 = ldg4(Fxx + off + G.x);
    if (ADV == 2) a4 = ldg4(Fax + off + G.x);
    C.p = ldg4(p + off + G.x);
    if (AUG) C.w2 = ldg4(w2 + off + G.x);
  }
  C.xx[1] = x4.x; C.xx[2] = x4.y; C.xx[3] = x4.z; C.xx[4] = x4.w;
  vhalo(C.xx, Fxx + off, 1.0f, false, G);
  if (ADV == 2) {
    C.ax[1] = a4.x; C.ax[2] = a4.y; C.ax[3] = a4.z; C.ax[4] = a4.w;
    vhalo(C.ax, Fax + off, 1.0f, false, G);
  }
}

// North-face fluxes of row B (towards row N), one per lane column.
template <int ADV>
__device__ __forceinline__ void vnorth(float* fn, const VRow<ADV>& B, const VRow<ADV>& N,
                                       float aby) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int c = k + 1;
    const float ayn = B.yy[k] + N.yy[k];
    const float qn = B.xy[c] + N.xy[c];
    float f = face_flux(ayn, N.y[c] - B.y[c], qn, (N.y[c + 1] + B.y[c + 1]) - (N.y[c - 1] + B.y[c - 1]));
    if (ADV == 1) f = fmaf(aby, B.y[c] + N.y[c], f);
    if (ADV == 2) f = fmaf(B.ay[k] + N.ay[k], B.y[c] + N.y[c], f);
    fn[k] = f;
  }
}

// One marching run: rows [y0, y1) of the strip at this lane's columns.
template <bool AUG, int ADV>
__device__ __forceinline__ void vec_run(const SeriesArgs& a, const VGeo& G, int y0, int y1,
                                        const float* __restrict__ yin, float* __restrict__ yout,
                                        float* __restrict__ p, float ig, float sh, float d,
                                        float e1, float e2, float& ly, float& lp) {
  const long long n = G.n;
  const float* __restrict__ F = static_cast<const float*>(a.coef);
  const float* Fxx = F;
  const float* Fyy = F + n;
  const float* Fxy = F + 2 * n;
  const float* Fax = F + 3 * n;
  const float* Fay = F + 4 * n;
  const float* __restrict__ w1 = static_cast<const float*>(a.w1);
  const float* __restrict__ w2 = static_cast<const float*>(a.w2);
  VRow<ADV> A, B, N, Rn;
  VCen<ADV, AUG> C, Cn;
  vload_row<ADV>(A, yin, Fxy, Fyy, Fay, y0 - 1, G);
  vload_row<ADV>(B, yin, Fxy, Fyy, Fay, y0, G);
  vload_row<ADV>(N, yin, Fxy, Fyy, Fay, y0 + 1, G);
  vload_cen<ADV, AUG>(C, Fxx, Fax, p, w2, y0, G);
  float fs[4];
  vnorth<ADV>(fs, A, B, a.aby);
  for (int j = y0; j < y1; ++j) {
    // prefetch the next step's rows
    if (j + 2 <= y1) vload_row<ADV>(Rn, yin, Fxy, Fyy, Fay, j + 2, G);
    if (j + 1 < y1) vload_cen<ADV, AUG>(Cn, Fxx, Fax, p, w2, j + 1, G);
    float fn[4];
    vnorth<ADV>(fn, B, N, a.aby);
    float fx[5];
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      const int L = f, R = f + 1;
      const float axf = C.xx[L] + C.xx[R];
      const float qf = B.xy[L] + B.xy[R];
      float v = face_flux(axf, B.y[R] - B.y[L], qf, (N.y[R] + N.y[L]) - (A.y[R] + A.y[L]));
      if (ADV == 1) v = fmaf(a.abx, B.y[L] + B.y[R], v);
      if (ADV == 2) v = fmaf(C.ax[L] + C.ax[R], B.y[L] + B.y[R], v);
      fx[f] = v;
    }
    if (G.active) {
      const long long idx = (long long)j * G.nx + G.x;
      float4 w1v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (AUG && e2 != 0.0f) w1v = ldg4(w1 + idx);
      const float pin[4] = {C.p.x, C.p.y, C.p.z, C.p.w};
      const float w2v[4] = {C.w2.x, C.w2.y, C.w2.z, C.w2.w};
      const float w1a[4] = {w1v.x, w1v.y, w1v.z, w1v.w};
      float z[4], pn[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float au = (fx[k + 1] - fx[k]) + (fn[k] - fs[k]);
        float zz = fmaf(au, ig, -sh * B.y[k + 1]);
        if (AUG) {
          if (e1 != 0.0f) zz = fmaf(e1, w2v[k], zz);
          if (e2 != 0.0f) zz = fmaf(e2, w1a[k], zz);
        }
        z[k] = zz;
        pn[k] = fmaf(d, zz, pin[k]);
        ly = fmaf(zz, zz, ly);
        lp = fmaf(pn[k], pn[k], lp);
      }
      *reinterpret_cast<float4*>(yout + idx) = make_float4(z[0], z[1], z[2], z[3]);
      *reinterpret_cast<float4*>(p + idx) = make_float4(pn[0], pn[1], pn[2], pn[3]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) fs[k] = fn[k];
    A = B;
    B = N;
    N = Rn;
    C = Cn;
  }
}

// The rows of this warp: units u = strip * ny + row in [u0, u1).
__device__ __forceinline__ void vec_range(long long units, long long warps, long long w,
                                          long long& u0, long long& u1) {
  u0 = units * w / warps;
  u1 = units * (w + 1) / warps;
}

}  // namespace
}  // namespace ad
