// FP32 fused Leja iteration: register marching fed by a per-warp ring of
// asynchronous copies (cp.async) in shared memory.
//
// Same warp geometry, flux expressions and work split as tile_f32_vec.cuh
// (a warp owns a 128-column strip, lane l columns x0 + 4l .. x0 + 4l + 3, and
// marches down a contiguous range of rows).  The difference is where the rows
// wait: every row of every field is copied global -> shared by the warp's own
// lanes with 16-byte cp.async (4 bytes for the two halo columns) into a ring
// of S records, so each warp keeps S - 3 rows of loads in flight without
// holding them in registers.  Before step j the ring holds rows j - 1 ..
// j + S - 2, one commit group per row; the warp waits until at most S - 3
// groups are pending (rows <= j + 1 complete); after step j the slot of row
// j - 1 is refilled with row j + S - 1.  Waits are the hardware's own
// (cp.async.wait_group): nothing spins.
//
// A row record holds, at float offsets, y and Dxy and Dxx with one halo
// column on each side (index 4 + c for column x0 + c, c = -1 .. 128), Dyy,
// p, w2 and the advection fields.  Ghost columns are copied from their mapped
// source (wrap or mirror); the Dirichlet sign of ghost values is applied when
// the row is read.  Halo rows of a run (y0 - 1 and y1) skip Dxx, p and w2.
#pragma once
#include "tile_f32_vec.cuh"

namespace ad {
namespace {

constexpr int kRingWarps = 8;
constexpr int kRingThreads = kRingWarps * 32;
constexpr int kRingHalo = 136;     // floats per haloed row segment

template <bool AUG, int ADV>
struct RingLayout {
  static constexpr int Y = 0, XY = kRingHalo, XX = 2 * kRingHalo;
  static constexpr int AX = 3 * kRingHalo;                         // ADV == 2
  static constexpr int YY = AX + (ADV == 2 ? kRingHalo : 0);
  static constexpr int P = YY + 128;
  static constexpr int W2 = P + 128;                                // AUG
  static constexpr int AY = W2 + (AUG ? 128 : 0);                   // ADV == 2
  static constexpr int SIZE = AY + (ADV == 2 ? 128 : 0);            // floats, multiple of 4
  // stages per warp: as many as fit 8 warps in ~220 KB, at most 8
  static constexpr int STAGES_FIT = (220 * 1024) / (kRingWarps * SIZE * 4);
  static constexpr int STAGES = STAGES_FIT > 8 ? 8 : STAGES_FIT;
};

__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async4f(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Issue the copies of row r (centre: also Dxx, p, w2, ax) into record S.
// pzero: p is taken as 0 and not read.
template <bool AUG, int ADV>
__device__ __forceinline__ void ring_issue(float* S, const SeriesArgs& a, const VGeo& G,
                                           const float* __restrict__ yin, int r, bool centre,
                                           int x0, int wcols, bool pzero = false) {
  using L = RingLayout<AUG, ADV>;
  const long long n = G.n;
  const float* F = static_cast<const float*>(a.coef);
  const float* Fxx = F;
  const float* Fyy = F + n;
  const float* Fxy = F + 2 * n;
  const float* Fax = F + 3 * n;
  const float* Fay = F + 4 * n;
  const RowMap rm = map_row(r, G.nx, G.ny, G.bc);
  const long long off = rm.off;
  const int c = 4 * G.lane;
  if (G.active) {
    cp_async16(S + L::Y + 4 + c, yin + off + G.x);
    cp_async16(S + L::XY + 4 + c, Fxy + off + G.x);
    cp_async16(S + L::YY + c, Fyy + off + G.x);
    if (ADV == 2) cp_async16(S + L::AY + c, Fay + off + G.x);
    if (centre) {
      cp_async16(S + L::XX + 4 + c, Fxx + off + G.x);
      if (!pzero) cp_async16(S + L::P + c, static_cast<const float*>(a.p) + off + G.x);
      if (AUG) cp_async16(S + L::W2 + c, static_cast<const float*>(a.w2) + off + G.x);
      if (ADV == 2) cp_async16(S + L::AX + 4 + c, Fax + off + G.x);
    }
  }
  // halo columns: lane 0 the left one (column x0 - 1), lane 1 the right one
  if (G.lane < 2) {
    const bool left = G.lane == 0;
    const int col = left ? x0 - 1 : x0 + wcols;
    float sg;
    const int mc = map_col(col, G.nx, G.bc, sg);
    const int pos = left ? 3 : 4 + wcols;
    cp_async4f(S + L::Y + pos, yin + off + mc);
    cp_async4f(S + L::XY + pos, Fxy + off + mc);
    if (centre) {
      cp_async4f(S + L::XX + pos, Fxx + off + mc);
      if (ADV == 2) cp_async4f(S + L::AX + pos, Fax + off + mc);
    }
  }
}

// v[0..5] = columns x-1 .. x+4 of a haloed segment (own four as one float4).
__device__ __forceinline__ void ring_read6(float* v, const float* seg, const VGeo& G, int wcols,
                                           float edge_sign) {
  const int c = 4 * G.lane;
  float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
  if (G.active) q = *reinterpret_cast<const float4*>(seg + 4 + c);
  v[1] = q.x; v[2] = q.y; v[3] = q.z; v[4] = q.w;
  v[0] = __shfl_up_sync(0xffffffffu, q.w, 1);
  v[5] = __shfl_down_sync(0xffffffffu, q.x, 1);
  if (!G.active) return;
  if (G.lane == 0) v[0] = seg[3] * (G.x == 0 ? edge_sign : 1.0f);
  if (c + 4 == wcols) v[5] = seg[4 + wcols] * (G.x + 4 == G.nx ? edge_sign : 1.0f);
}

template <bool AUG, int ADV>
__device__ __forceinline__ void ring_read_row(VRow<ADV>& R, const float* S, const VGeo& G,
                                              int r, int wcols) {
  using L = RingLayout<AUG, ADV>;
  const float sg = (G.bc != 0 && (r < 0 || r >= G.ny)) ? -1.0f : 1.0f;
  const float esg = G.bc != 0 ? -1.0f : 1.0f;     // Dirichlet ghost column of a value
  ring_read6(R.y, S + L::Y, G, wcols, esg);
#pragma unroll
  for (int k = 0; k < 6; ++k) R.y[k] *= sg;
  ring_read6(R.xy, S + L::XY, G, wcols, 1.0f);
  const int c = 4 * G.lane;
  float4 b = make_float4(0.f, 0.f, 0.f, 0.f), ay = b;
  if (G.active) {
    b = *reinterpret_cast<const float4*>(S + L::YY + c);
    if (ADV == 2) ay = *reinterpret_cast<const float4*>(S + L::AY + c);
  }
  R.yy[0] = b.x; R.yy[1] = b.y; R.yy[2] = b.z; R.yy[3] = b.w;
  if (ADV == 2) { R.ay[0] = ay.x; R.ay[1] = ay.y; R.ay[2] = ay.z; R.ay[3] = ay.w; }
}

template <bool AUG, int ADV>
__device__ __forceinline__ void ring_read_cen(VCen<ADV, AUG>& C, const float* S, const VGeo& G,
                                              int wcols, bool pzero = false) {
  using L = RingLayout<AUG, ADV>;
  ring_read6(C.xx, S + L::XX, G, wcols, 1.0f);
  if (ADV == 2) ring_read6(C.ax, S + L::AX, G, wcols, 1.0f);
  const int c = 4 * G.lane;
  C.p = make_float4(0.f, 0.f, 0.f, 0.f);
  C.w2 = C.p;
  if (G.active) {
    if (!pzero) C.p = *reinterpret_cast<const float4*>(S + L::P + c);
    if (AUG) C.w2 = *reinterpret_cast<const float4*>(S + L::W2 + c);
  }
}

// One marching run of rows [y0, y1) through this warp's ring.  pzero: p
// starts from 0 (not read), which with ig = 1, sh = 0 and the couplings
// holding source fields makes the run a series start: y_0 = A u + sources,
// p_0 = d y_0.
template <bool AUG, int ADV>
__device__ __forceinline__ void ring_run(const SeriesArgs& a, const VGeo& G, float* ring, int y0,
                                         int y1, const float* __restrict__ yin,
                                         float* __restrict__ yout, float* __restrict__ p, float ig,
                                         float sh, float d, float e1, float e2, float& ly,
                                         float& lp, bool pzero = false) {
  using L = RingLayout<AUG, ADV>;
  constexpr int S = L::STAGES;
  const int x0 = G.x - 4 * G.lane;
  const int wcols = min(kVecCols, G.nx - x0);
  const float* __restrict__ w1 = static_cast<const float*>(a.w1);
  auto slot = [&](int r) { return ring + (size_t)((r - (y0 - 1)) % S) * L::SIZE; };
  // rows y0 - 1 .. y0 + S - 2 in flight (one group each; empty past y1)
  __syncwarp();
#pragma unroll 1
  for (int q = 0; q < S; ++q) {
    const int r = y0 - 1 + q;
    if (r <= y1) ring_issue<AUG, ADV>(slot(r), a, G, yin, r, r >= y0 && r < y1, x0, wcols, pzero);
    cp_async_commit();
  }
  cp_async_wait_group<S - 3>();      // rows y0 - 1, y0 and y0 + 1 complete
  __syncwarp();
  VRow<ADV> A, B, N;
  VCen<ADV, AUG> C;
  ring_read_row<AUG, ADV>(A, slot(y0 - 1), G, y0 - 1, wcols);
  ring_read_row<AUG, ADV>(B, slot(y0), G, y0, wcols);
  float fs[4];
  vnorth<ADV>(fs, A, B, a.aby);
#pragma unroll 1
  for (int j = y0; j < y1; ++j) {
    if (j > y0) {
      cp_async_wait_group<S - 3>();  // row j + 1 complete
      __syncwarp();
    }
    ring_read_row<AUG, ADV>(N, slot(j + 1), G, j + 1, wcols);
    ring_read_cen<AUG, ADV>(C, slot(j), G, wcols, pzero);
    float fn[4];
    vnorth<ADV>(fn, B, N, a.aby);
    float fx[5];
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      const int Lc = f, Rc = f + 1;
      const float axf = C.xx[Lc] + C.xx[Rc];
      const float qf = B.xy[Lc] + B.xy[Rc];
      float v = face_flux(axf, B.y[Rc] - B.y[Lc], qf, (N.y[Rc] + N.y[Lc]) - (A.y[Rc] + A.y[Lc]));
      if (ADV == 1) v = fmaf(a.abx, B.y[Lc] + B.y[Rc], v);
      if (ADV == 2) v = fmaf(C.ax[Lc] + C.ax[Rc], B.y[Lc] + B.y[Rc], v);
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
    // row j - 1 is no longer read: refill its slot with row j + S - 1
    __syncwarp();
    const int r = j + S - 1;
    if (r <= y1) ring_issue<AUG, ADV>(slot(r), a, G, yin, r, r < y1, x0, wcols, pzero);
    cp_async_commit();
#pragma unroll
    for (int k = 0; k < 4; ++k) fs[k] = fn[k];
    A = B;
    B = N;
  }
  cp_async_wait_group<0>();          // nothing may land in the ring after the run
  __syncwarp();
}

}  // namespace
}  // namespace ad
