// FP32 fused Leja iterations two at a time (temporal blocking): one pass over
// HBM computes y_{m+1} and y_{m+2} of the Newton recurrence (Section 2).
//
// Overlapped strips.  A warp produces 120 columns [X0, X0 + 120) and computes
// the first iteration (level 1) on the 128 columns [X0 - 4, X0 + 124): lane l
// holds the group of four columns gx = X0 - 4 + 4 l .. gx + 3.  Lanes 1 .. 30
// own their groups; lanes 0 and 31 compute level 1 only, so that their
// columns X0 - 1 and X0 + 120 supply the x-neighbours of level 2 at the strip
// edges.  Their other columns see a neighbour value the lane does not have (a
// shuffle returns its own) and are never used.  So neither level needs halo
// loads or edge-lane extra cells: each row of each field is one 16-byte copy
// per lane, and both levels run the register marching of tile_f32_vec.cuh
// with its flux expressions term for term.
//
// Marching down rows, the warp computes at step j level 1 on row j + 1 (from
// rows j .. j + 2 of y_m) and level 2 on row j (from rows j - 1 .. j + 1 of
// y_{m+1}, held in registers).  Rows come through a per-warp ring of
// cp.async records: a record is refilled with the row S ahead as soon as it
// has been read into registers, so S - 1 rows stay in flight.
//
// Ghost values.  A group outside [0, nx) is copied from its wrapped source
// (periodic) or from its mirror group (zero Dirichlet: read back reversed,
// values negated).  y_{m+1} must obey the boundary condition of every vector
// the operator acts on, so with zero Dirichlet its ghost column and ghost
// rows are set to the odd reflection of the computed values; with the
// periodic wrap they are computed like any other cell.
//
// Traffic per cell and pass: y_m, p, Dxx, Dxy, Dyy read, y_{m+2} and p
// written (28 bytes for two iterations), plus 8 of every 128 columns of the
// four read fields read again by the edge lanes.  The pass stores p_{m+1} and
// leaves d_{m+2} y_{m+2} pending: the next pass adds it (it reads y_{m+2}
// anyway), and a flush kernel adds it when the series stops after an even
// count.  In pair mode y_m lives in y buffer (m / 2) & 1.
//
// Eligible: the phi_1 form (no augmented couplings), no advection or constant
// advection, nx % 4 == 0, ny >= 2.
#pragma once
#include "tile_f32_ring.cuh"

namespace ad {
namespace {

constexpr int kPairOwn = 120;        // columns a warp strip produces

struct PairLayout {                  // one row record, floats (lane l at 4 l)
  static constexpr int Y = 0, XY = 128, YY = 256, XX = 384, P = 512;
  static constexpr int SIZE = 640;
  static constexpr int STAGES = 10;
};

struct PairLane {
  int src;       // first column of the copied source group
  bool load;     // the group is needed: -4 <= gx <= nx
  bool rev;      // zero-Dirichlet ghost group: the mirror group, reversed on read
  float csg;     // sign of values in the group (-1 for a zero-Dirichlet ghost group)
  bool own;      // lanes 1 .. 30 inside the domain: produce y_{m+2} and p
};

__device__ __forceinline__ PairLane pair_lane(int X0, int lane, int nx, int bc) {
  PairLane L;
  const int gx = X0 - 4 + 4 * lane;
  L.load = gx >= -4 && gx <= nx;
  L.rev = false;
  L.csg = 1.0f;
  L.src = gx;
  if (gx < 0) {
    if (bc == 0) L.src = gx + nx;
    else { L.src = 0; L.rev = true; L.csg = -1.0f; }
  } else if (gx >= nx) {
    if (bc == 0) L.src = gx - nx;
    else { L.src = nx - 4; L.rev = true; L.csg = -1.0f; }
  }
  L.own = lane >= 1 && lane <= 30 && gx < nx;
  return L;
}

struct PRow {          // one row of y_m and its Dxy, Dyy around the lane's group
  float y[6];          // columns gx - 1 .. gx + 4, signs applied
  float xy[6];
  float yy[4];
};

struct PCen {          // the row level 1 computes: Dxx (with x-neighbours) and p
  float xx[6];
  float4 p;
};

__device__ __forceinline__ float4 pair_ld4(const float* s, const PairLane& L) {
  float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
  if (L.load) q = *reinterpret_cast<const float4*>(s);
  if (L.rev) q = make_float4(q.w, q.z, q.y, q.x);
  return q;
}

__device__ __forceinline__ void pair_spread(float* v, float4 q, float s) {
  v[1] = s * q.x; v[2] = s * q.y; v[3] = s * q.z; v[4] = s * q.w;
  v[0] = __shfl_up_sync(0xffffffffu, v[4], 1);
  v[5] = __shfl_down_sync(0xffffffffu, v[1], 1);
}

// Copies of row r into record S: y, Dxy, Dyy always; Dxx for the rows level 1
// computes; p for own rows on own lanes.
__device__ __forceinline__ void pair_issue(float* S, const SeriesArgs& a, const VGeo& G,
                                           const PairLane& L, const float* __restrict__ yin,
                                           int r, bool want_xx, bool want_p) {
  using PL = PairLayout;
  if (!L.load) return;
  const long long n = G.n;
  const float* F = static_cast<const float*>(a.coef);
  const long long off = map_row(r, G.nx, G.ny, G.bc).off + L.src;
  const int c = 4 * G.lane;
  cp_async16(S + PL::Y + c, yin + off);
  cp_async16(S + PL::XY + c, F + 2 * n + off);
  cp_async16(S + PL::YY + c, F + n + off);
  if (want_xx) cp_async16(S + PL::XX + c, F + off);
  if (want_p && L.own) cp_async16(S + PL::P + c, static_cast<const float*>(a.p) + off);
}

__device__ __forceinline__ void pair_read(PRow& R, PCen* C, const float* S, const VGeo& G,
                                          const PairLane& L, int r) {
  using PL = PairLayout;
  const int c = 4 * G.lane;
  const float rsg = (G.bc != 0 && (r < 0 || r >= G.ny)) ? -1.0f : 1.0f;
  pair_spread(R.y, pair_ld4(S + PL::Y + c, L), rsg * L.csg);
  pair_spread(R.xy, pair_ld4(S + PL::XY + c, L), 1.0f);
  const float4 b = pair_ld4(S + PL::YY + c, L);
  R.yy[0] = b.x; R.yy[1] = b.y; R.yy[2] = b.z; R.yy[3] = b.w;
  if (C) {
    pair_spread(C->xx, pair_ld4(S + PL::XX + c, L), 1.0f);
    C->p = make_float4(0.f, 0.f, 0.f, 0.f);
    if (L.own) C->p = *reinterpret_cast<const float4*>(S + PL::P + c);
  }
}

// North-face fluxes of row B towards row N (the expressions of vnorth).
template <int ADV>
__device__ __forceinline__ void pair_north(const float* uB, const float* uN, const float* xyB,
                                           const float* xyN, const float* yyB, const float* yyN,
                                           float aby, float* fn) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int c = k + 1;
    const float ayn = yyB[k] + yyN[k];
    const float qn = xyB[c] + xyN[c];
    float f = face_flux(ayn, uN[c] - uB[c], qn, (uN[c + 1] + uB[c + 1]) - (uN[c - 1] + uB[c - 1]));
    if (ADV == 1) f = fmaf(aby, uB[c] + uN[c], f);
    fn[k] = f;
  }
}

// The fused stencil on row B of one level (rows A, B, N of its input vector
// u): the north fluxes fn of row B, and z = (A u - c u) / gamma - xi u on the
// lane's four columns, with the south fluxes fs carried from the row above.
// The x-face and north-face fluxes of ring_run, term for term.
template <int ADV>
__device__ __forceinline__ void pair_level(const float* uA, const float* uB, const float* uN,
                                           const float* xx, const float* xyB, const float* xyN,
                                           const float* yyB, const float* yyN, float abx,
                                           float aby, const float* fs, float* fn, float ig,
                                           float sh, float* z) {
  pair_north<ADV>(uB, uN, xyB, xyN, yyB, yyN, aby, fn);
  float fx[5];
#pragma unroll
  for (int f = 0; f < 5; ++f) {
    const int Lc = f, Rc = f + 1;
    const float axf = xx[Lc] + xx[Rc];
    const float qf = xyB[Lc] + xyB[Rc];
    float v = face_flux(axf, uB[Rc] - uB[Lc], qf, (uN[Rc] + uN[Lc]) - (uA[Rc] + uA[Lc]));
    if (ADV == 1) v = fmaf(abx, uB[Lc] + uB[Rc], v);
    fx[f] = v;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float au = (fx[k + 1] - fx[k]) + (fn[k] - fs[k]);
    z[k] = fmaf(au, ig, -sh * uB[k + 1]);
  }
}

// A row of y_{m+1} from the level-1 values z of the lane's group: with zero
// Dirichlet, column -1 (in a left ghost group) and column nx (in a right
// one) become the odd reflection of their mirror; then the x-neighbours.
__device__ __forceinline__ void pair_y1(float* u, const float* z, bool fix, int gx, int nx) {
  u[1] = z[0]; u[2] = z[1]; u[3] = z[2]; u[4] = z[3];
  if (fix) {                                   // warp-uniform: the strip has a ghost group
    const float right_of = __shfl_down_sync(0xffffffffu, z[0], 1);
    const float left_of = __shfl_up_sync(0xffffffffu, z[3], 1);
    if (gx < 0) u[4] = -right_of;              // column -1 = -(column 0)
    if (gx == nx) u[1] = -left_of;             // column nx = -(column nx - 1)
  }
  u[0] = __shfl_up_sync(0xffffffffu, u[4], 1);
  u[5] = __shfl_down_sync(0xffffffffu, u[1], 1);
}

// One marching run of rows [y0, y1) of the strip that starts at column X0.
template <int ADV>
__device__ __forceinline__ void pair_run(const SeriesArgs& a, const VGeo& G, float* ring, int X0,
                                         int y0, int y1, const float* __restrict__ yin,
                                         float* __restrict__ yout, float* __restrict__ p,
                                         float ig, float sh1, float sh2, float d1, float d2,
                                         float d0, float& ly1, float& lp1, float& ly2,
                                         float& lp2) {
  using PL = PairLayout;
  constexpr int S = PL::STAGES;
  const PairLane L = pair_lane(X0, G.lane, G.nx, G.bc);
  const int gx = X0 - 4 + 4 * G.lane;
  const bool dir = G.bc != 0;
  const bool fix = dir && (X0 == 0 || X0 + kPairOwn >= G.nx);
  const float abx = a.abx, aby = a.aby;
  auto slot = [&](int r) { return ring + (size_t)((r - (y0 - 2)) % S) * PL::SIZE; };
  auto issue = [&](int r) {            // rows y0 - 2 .. y1 + 1; one commit group each
    if (r <= y1 + 1)
      pair_issue(slot(r), a, G, L, yin, r, r >= y0 - 1 && r <= y1, r >= y0 && r < y1);
    cp_async_commit();
  };
  // Read row r into registers, then refill its record with row r + S.  Row r
  // is the oldest pending group: the S - 1 younger ones stay in flight.
  auto consume = [&](int r, PRow& R, PCen* C) {
    cp_async_wait_group<S - 1>();
    __syncwarp();
    pair_read(R, C, slot(r), G, L, r);
    __syncwarp();
    issue(r + S);
  };
  __syncwarp();
#pragma unroll 1
  for (int q = 0; q < S; ++q) issue(y0 - 2 + q);

  PRow A, B, N;
  PCen C, Cn;
  float fs1[4], fn1[4], fs2[4], fn2[4], z[4];
  float U1a[6], U1b[6], U1n[6];       // y_{m+1} on the level-2 rows j - 1, j, j + 1
  float xx2[6];                       // Dxx of the level-2 row
  float p1[4] = {0.f, 0.f, 0.f, 0.f}; // p_{m+1} of the last own level-1 row

  // level 1 on the row of B (A, B, N: rows r - 1 .. r + 1; C: row r); own
  // rows also store p_{m+1} and add to the level-1 norms
  auto level1 = [&](int r, float* u1) {
    pair_level<ADV>(A.y, B.y, N.y, C.xx, B.xy, N.xy, B.yy, N.yy, abx, aby, fs1, fn1, ig, sh1, z);
    pair_y1(u1, z, fix, gx, G.nx);
    if (L.own && r >= y0 && r < y1) {
      const float pin[4] = {C.p.x, C.p.y, C.p.z, C.p.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float pm = fmaf(d0, B.y[k + 1], pin[k]);   // the pending d_m y_m
        p1[k] = fmaf(d1, z[k], pm);
        ly1 = fmaf(z[k], z[k], ly1);
        lp1 = fmaf(p1[k], p1[k], lp1);
      }
      const long long idx = (long long)r * G.nx + gx;
      *reinterpret_cast<float4*>(p + idx) = make_float4(p1[0], p1[1], p1[2], p1[3]);
    }
  };

  consume(y0 - 2, A, nullptr);
  consume(y0 - 1, B, &C);
  pair_north<ADV>(A.y, B.y, A.xy, B.xy, A.yy, B.yy, aby, fs1);   // south faces of row y0 - 1
  // prologue: level 1 on rows y0 - 1 and y0
  consume(y0, N, &Cn);
  level1(y0 - 1, U1b);
#pragma unroll
  for (int k = 0; k < 4; ++k) fs1[k] = fn1[k];
  A = B; B = N; C = Cn;
  consume(y0 + 1, N, &Cn);
  level1(y0, U1n);
  if (dir && y0 == 0) {               // y_{m+1} row -1 = -(row 0)
#pragma unroll
    for (int k = 0; k < 6; ++k) U1b[k] = -U1n[k];
  }
  // south faces of level 2 on row y0: y_{m+1} rows y0 - 1, y0 with the
  // coefficient rows y0 - 1 (A) and y0 (B)
  pair_north<ADV>(U1b, U1n, A.xy, B.xy, A.yy, B.yy, aby, fs2);
#pragma unroll
  for (int k = 0; k < 6; ++k) { U1a[k] = U1b[k]; U1b[k] = U1n[k]; xx2[k] = C.xx[k]; }
#pragma unroll
  for (int k = 0; k < 4; ++k) fs1[k] = fn1[k];
  A = B; B = N; C = Cn;

#pragma unroll 1
  for (int j = y0; j < y1; ++j) {
    // here A, B, C hold rows j, j + 1, j + 1; U1a, U1b rows j - 1, j
    const float p1j[4] = {p1[0], p1[1], p1[2], p1[3]};        // p_{m+1} of row j
    consume(j + 2, N, &Cn);
    level1(j + 1, U1n);
    if (dir && j + 1 == G.ny) {       // y_{m+1} row ny = -(row ny - 1)
#pragma unroll
      for (int k = 0; k < 6; ++k) U1n[k] = -U1b[k];
    }
    // level 2 on row j: coefficient rows j (A) and j + 1 (B), Dxx of row j
    pair_level<ADV>(U1a, U1b, U1n, xx2, A.xy, B.xy, A.yy, B.yy, abx, aby, fs2, fn2, ig, sh2, z);
    if (L.own) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float p2 = fmaf(d2, z[k], p1j[k]);
        ly2 = fmaf(z[k], z[k], ly2);
        lp2 = fmaf(p2, p2, lp2);
      }
      const long long idx = (long long)j * G.nx + gx;
      *reinterpret_cast<float4*>(yout + idx) = make_float4(z[0], z[1], z[2], z[3]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) { fs2[k] = fn2[k]; fs1[k] = fn1[k]; }
#pragma unroll
    for (int k = 0; k < 6; ++k) { U1a[k] = U1b[k]; U1b[k] = U1n[k]; xx2[k] = C.xx[k]; }
    A = B; B = N; C = Cn;
  }
  cp_async_wait_group<0>();          // nothing may land in the ring after the run
  __syncwarp();
}

}  // namespace
}  // namespace ad
