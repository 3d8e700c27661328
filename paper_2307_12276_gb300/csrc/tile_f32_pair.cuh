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
// y_{m+1}, held in registers; three row slots rotate, with no copies).  Rows
// come through a per-warp ring of cp.async records: a record is refilled with
// the row S ahead as soon as it has been read into registers, so S - 1 rows
// stay in flight.
//
// Ghost values.  With the periodic wrap a group outside [0, nx) is copied
// from its wrapped source and computed like any other.  With zero Dirichlet
// it is not read: the lanes at columns 0 and nx - 1 mirror their own values
// into the missing x-neighbour (negated for y), and y_{m+1}, which must obey
// the boundary condition of every vector the operator acts on, gets its
// ghost column and ghost rows as the odd reflection of the computed values.
//
// Work split: the rows are cut into bands, one per warp of each strip, and a
// warp takes a band of one strip (band-major order), so the warps of
// neighbouring strips march the same rows at the same time and the sectors
// both read at a strip edge come from L2 the second time.  Each band re-reads
// four halo rows (two above, two below).
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
#include <type_traits>

#include "tile_f32_ring.cuh"

namespace ad {
namespace {

constexpr int kPairOwn = 120;        // columns a warp strip produces
constexpr int kPairWarps = 8;        // warps per block (one block per SM)

struct PairLayout {                  // one row record, floats (lane l at 4 l)
  static constexpr int Y = 0, XY = 128, YY = 256, XX = 384, P = 512;
  static constexpr int SIZE = 640;
  // Ring depth.  Measured on GB300 (4096^2 pair launch / 128-slice batch step):
  // 10 stages 98.3 us / 13.21 ms, 5-8 stages 96.0-96.7 us / 12.62-12.70 ms
  // (less shared memory leaves more of the unified L1).
  static constexpr int STAGES = 6;
};

struct PairLane {
  int src;       // first column of the copied source group
  bool load;     // the lane copies its group (periodic: the wrapped one)
  bool own;      // lanes 1 .. 30 inside the domain: produce y_{m+2} and p
  bool west;     // zero Dirichlet: the group starts at column 0
  bool east;     // zero Dirichlet: the group ends at column nx - 1
};

__device__ __forceinline__ PairLane pair_lane(int X0, int lane, int nx, int bc) {
  PairLane L;
  const int gx = X0 - 4 + 4 * lane;
  if (bc == 0) {
    L.load = gx >= -4 && gx <= nx;
    L.src = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
  } else {                     // ghost groups are not read: their values are mirrored
    L.load = gx >= 0 && gx < nx;
    L.src = gx;
  }
  L.own = lane >= 1 && lane <= 30 && gx < nx;
  L.west = bc != 0 && gx == 0;
  L.east = bc != 0 && gx + 4 == nx;
  return L;
}

struct PRow {          // one row around the lane's group, columns gx - 1 .. gx + 4
  float y[6];          // y_m (Dirichlet ghost signs applied)
  float xy[6];
  float xx[6];         // rows level 1 computes
  float yy[4];
  float p[4];          // p_m; after level 1 on an own row, p_{m+1}
};

struct PairCtx {       // per-run constants (registers: no per-row loads through a struct in memory)
  const float* F;      // the coefficient fields [3][n]
  int stages;          // ring depth (records per warp)
  const float* yin;
  float* yout;
  float* p;
  float* ring;
  VGeo G;
  PairLane L;
  int gx, y0, y1;
  bool fix;            // zero Dirichlet and the strip reaches column 0 or nx - 1
  float ig, sh1, sh2, d0, d1, d2, abx, aby;
};

// x-neighbours from the adjacent lanes; zero Dirichlet mirrors at the domain
// edge (sgn -1 for values, +1 for coefficients).
__device__ __forceinline__ void pair_spread(float* v, float4 q, const PairCtx& X, float sgn) {
  v[1] = q.x; v[2] = q.y; v[3] = q.z; v[4] = q.w;
  v[0] = __shfl_up_sync(0xffffffffu, v[4], 1);
  v[5] = __shfl_down_sync(0xffffffffu, v[1], 1);
  if (X.fix) {
    if (X.L.west) v[0] = sgn * v[1];
    if (X.L.east) v[5] = sgn * v[4];
  }
}

__device__ __forceinline__ float* pair_slot(const PairCtx& X, int r) {
  return X.ring + (size_t)((r - (X.y0 - 2)) % X.stages) * PairLayout::SIZE;
}

// Copies of row r into record S (rows y0 - 2 .. y1 + 1; one commit group per
// row, empty past the end): y, Dxy, Dyy always; Dxx for the rows level 1
// computes; p for own rows on own lanes.
__device__ __forceinline__ void pair_issue(const PairCtx& X, int r, float* S) {
  using PL = PairLayout;
  if (r <= X.y1 + 1 && X.L.load) {
    const long long n = X.G.n;
    const float* F = X.F;
    const long long off = map_row(r, X.G.nx, X.G.ny, X.G.bc).off + X.L.src;
    const int c = 4 * X.G.lane;
    cp_async16(S + PL::Y + c, X.yin + off);
    cp_async16(S + PL::XY + c, F + 2 * n + off);
    cp_async16(S + PL::YY + c, F + n + off);
    if (r >= X.y0 - 1 && r <= X.y1) cp_async16(S + PL::XX + c, F + off);
    if (r >= X.y0 && r < X.y1 && X.L.own)
      cp_async16(S + PL::P + c, X.p + off);
  }
  cp_async_commit();
}

// The row copies of a warp's ring: 16-byte cp.async per lane, one commit
// group per row.  A lane that copies nothing for its group leaves zeros.
// Every lane reads back only the 16 bytes per field that it copied itself
// (neighbouring columns come by shuffles), so neither the wait nor the refill
// of a record needs a warp barrier: cp.async.wait_group makes a thread's own
// copies visible to it, and the refill of a record is issued after the
// thread's reads of it.  The records are used in row order, so the slot is
// a rolling counter: the initial fill writes records 0 .. S - 1, and each
// refill writes the record just read.
struct CpAsyncLoader {
  static constexpr bool kReadAll = false;   // records hold data only where a lane copied
  int slot = 0;                             // record of the next row read (and refilled)
  __device__ __forceinline__ float* rec(const PairCtx& X) const {
    return X.ring + slot * PairLayout::SIZE;
  }
  __device__ __forceinline__ void issue(const PairCtx& X, int r) {
    pair_issue(X, r, rec(X));
    slot = slot + 1 == PairLayout::STAGES ? 0 : slot + 1;
  }
  // row r (the oldest pending group: the S - 1 younger ones stay in flight)
  __device__ __forceinline__ const float* wait(const PairCtx& X, int) {
    cp_async_wait_group<PairLayout::STAGES - 1>();
    return rec(X);
  }
  __device__ __forceinline__ void drain(const PairCtx&) {
    cp_async_wait_group<0>();          // nothing may land in the ring after the run
    __syncwarp();
  }
};

// Read row r into registers, then refill its record with row r + S.
template <class Ld>
__device__ __forceinline__ void pair_consume(const PairCtx& X, Ld& ldr, int r, PRow& R) {
  using PL = PairLayout;
  const float* S = ldr.wait(X, r);
  const int c = 4 * X.G.lane;
  const bool ld = Ld::kReadAll || X.L.load;
  float4 y4 = make_float4(0.f, 0.f, 0.f, 0.f), q4 = y4, b4 = y4, x4 = y4, p4 = y4;
  if (ld) {
    y4 = *reinterpret_cast<const float4*>(S + PL::Y + c);
    q4 = *reinterpret_cast<const float4*>(S + PL::XY + c);
    b4 = *reinterpret_cast<const float4*>(S + PL::YY + c);
    x4 = *reinterpret_cast<const float4*>(S + PL::XX + c);
    p4 = *reinterpret_cast<const float4*>(S + PL::P + c);
  }
  if (X.G.bc != 0 && (r < 0 || r >= X.G.ny)) {       // zero Dirichlet ghost row
    y4.x = -y4.x; y4.y = -y4.y; y4.z = -y4.z; y4.w = -y4.w;
  }
  pair_spread(R.y, y4, X, -1.0f);
  pair_spread(R.xy, q4, X, 1.0f);
  pair_spread(R.xx, x4, X, 1.0f);
  R.yy[0] = b4.x; R.yy[1] = b4.y; R.yy[2] = b4.z; R.yy[3] = b4.w;
  R.p[0] = p4.x; R.p[1] = p4.y; R.p[2] = p4.z; R.p[3] = p4.w;
  ldr.issue(X, r + X.stages);
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
// u): z = (A u - c u) / gamma - xi u on the lane's four columns, with the
// south fluxes fs of row B; on return fs holds the north fluxes of row B
// (the south fluxes of the next row).  The x-face and north-face fluxes of
// ring_run, term for term.
template <int ADV>
__device__ __forceinline__ void pair_level(const float* uA, const float* uB, const float* uN,
                                           const float* xx, const float* xyB, const float* xyN,
                                           const float* yyB, const float* yyN, float abx,
                                           float aby, float* fs, float ig, float sh, float* z) {
  float fn[4];
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
    fs[k] = fn[k];
  }
}

// Packed FP32 pairs (the f32x2 arithmetic of sm_100 and later): each half is
// rounded exactly as the scalar operation, so a packed expression gives the
// scalar expression's results bit for bit with half the instructions.  Pairs
// are formed only where both halves sit in one aligned register pair or come
// straight from scalar results; sums across neighbouring columns of another
// alignment stay scalar.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
      "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
      "sub.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}

// pair_north with packed pairs: columns (1, 2) and (3, 4) of the lane's six.
template <int ADV>
__device__ __forceinline__ void pair_north_x2(const float* uB, const float* uN, const float* xyB,
                                              const float* xyN, const float* yyB, const float* yyN,
                                              float aby, float* fn) {
  float s[6];                           // uN + uB, the sums of both dd terms
  s[0] = uN[0] + uB[0];
  s[5] = uN[5] + uB[5];
#pragma unroll
  for (int h = 1; h < 5; h += 2) {
    const float2 t = add2(f2(uN[h], uN[h + 1]), f2(uB[h], uB[h + 1]));
    s[h] = t.x;
    s[h + 1] = t.y;
  }
#pragma unroll
  for (int h = 1; h < 5; h += 2) {      // columns h, h + 1
    const int k = h - 1;
    const float2 ayn = add2(f2(yyB[k], yyB[k + 1]), f2(yyN[k], yyN[k + 1]));
    const float2 qn = add2(f2(xyB[h], xyB[h + 1]), f2(xyN[h], xyN[h + 1]));
    const float2 du = sub2(f2(uN[h], uN[h + 1]), f2(uB[h], uB[h + 1]));
    const float2 dd = f2(s[h + 1] - s[h - 1], s[h + 2] - s[h]);
    float2 f = fma2(ayn, du, mul2(qn, dd));
    if (ADV == 1) f = fma2(f2(aby, aby), f2(s[h], s[h + 1]), f);
    fn[k] = f.x;
    fn[k + 1] = f.y;
  }
}

// pair_level with packed pairs: faces (0, 1) and (2, 3) and columns (1, 2),
// (3, 4); face 4 scalar.
template <int ADV>
__device__ __forceinline__ void pair_level_x2(const float* uA, const float* uB, const float* uN,
                                              const float* xx, const float* xyB, const float* xyN,
                                              const float* yyB, const float* yyN, float abx,
                                              float aby, float* fs, float ig, float sh, float* z) {
  float fn[4];
  pair_north_x2<ADV>(uB, uN, xyB, xyN, yyB, yyN, aby, fn);
  float fx[5];
#pragma unroll
  for (int f = 0; f < 4; f += 2) {      // faces f, f + 1
    const float2 axf = f2(xx[f] + xx[f + 1], xx[f + 1] + xx[f + 2]);
    const float2 qf = f2(xyB[f] + xyB[f + 1], xyB[f + 1] + xyB[f + 2]);
    const float2 du = f2(uB[f + 1] - uB[f], uB[f + 2] - uB[f + 1]);
    const float2 sn = f2(uN[f + 1] + uN[f], uN[f + 2] + uN[f + 1]);
    const float2 sa = f2(uA[f + 1] + uA[f], uA[f + 2] + uA[f + 1]);
    float2 v = fma2(axf, du, mul2(qf, sub2(sn, sa)));
    if (ADV == 1) v = fma2(f2(abx, abx), f2(uB[f] + uB[f + 1], uB[f + 1] + uB[f + 2]), v);
    fx[f] = v.x;
    fx[f + 1] = v.y;
  }
  {
    const float axf = xx[4] + xx[5];
    const float qf = xyB[4] + xyB[5];
    float v = face_flux(axf, uB[5] - uB[4], qf, (uN[5] + uN[4]) - (uA[5] + uA[4]));
    if (ADV == 1) v = fmaf(abx, uB[4] + uB[5], v);
    fx[4] = v;
  }
#pragma unroll
  for (int k = 0; k < 4; k += 2) {      // columns k + 1, k + 2
    const float2 au = add2(f2(fx[k + 1] - fx[k], fx[k + 2] - fx[k + 1]),
                           sub2(f2(fn[k], fn[k + 1]), f2(fs[k], fs[k + 1])));
    const float2 zz = fma2(au, f2(ig, ig), mul2(f2(-sh, -sh), f2(uB[k + 1], uB[k + 2])));
    z[k] = zz.x;
    z[k + 1] = zz.y;
    fs[k] = fn[k];
    fs[k + 1] = fn[k + 1];
  }
}

// Norm-sum accumulators: one float (scalar marching) or a packed pair.
__device__ __forceinline__ void acc_sq4(float& a, const float* v) {
#pragma unroll
  for (int k = 0; k < 4; ++k) a = fmaf(v[k], v[k], a);
}
__device__ __forceinline__ void acc_sq4(float2& a, const float* v) {
  const float2 lo = f2(v[0], v[1]), hi = f2(v[2], v[3]);
  a = fma2(lo, lo, a);
  a = fma2(hi, hi, a);
}
__device__ __forceinline__ float acc_total(float a) { return a; }
__device__ __forceinline__ float acc_total(float2 a) { return a.x + a.y; }

template <int ADV, bool X2>
__device__ __forceinline__ void pair_north_any(const float* uB, const float* uN, const float* xyB,
                                               const float* xyN, const float* yyB,
                                               const float* yyN, float aby, float* fn) {
  if constexpr (X2) pair_north_x2<ADV>(uB, uN, xyB, xyN, yyB, yyN, aby, fn);
  else pair_north<ADV>(uB, uN, xyB, xyN, yyB, yyN, aby, fn);
}

// A row of y_{m+1} from the level-1 values z of the lane's group: with zero
// Dirichlet, column -1 (in the group left of column 0) and column nx (in the
// group right of nx - 1) become the odd reflection of their mirror; then the
// x-neighbours.
__device__ __forceinline__ void pair_y1(float* u, const float* z, const PairCtx& X) {
  u[1] = z[0]; u[2] = z[1]; u[3] = z[2]; u[4] = z[3];
  if (X.fix) {
    const float right_of = __shfl_down_sync(0xffffffffu, z[0], 1);
    const float left_of = __shfl_up_sync(0xffffffffu, z[3], 1);
    if (X.gx == -4) u[4] = -right_of;          // column -1 = -(column 0)
    if (X.gx == X.G.nx) u[1] = -left_of;       // column nx = -(column nx - 1)
  }
  u[0] = __shfl_up_sync(0xffffffffu, u[4], 1);
  u[5] = __shfl_down_sync(0xffffffffu, u[1], 1);
}

// Level 1 on row r (A, B, N: rows r - 1 .. r + 1 of y_m) into u1; on a row of
// the run also p_{m+1} = p_m + d_m y_m + d_{m+1} y_{m+1} (stored by own lanes,
// and kept in B.p for level 2) and the level-1 norm terms.  Every lane forms
// the terms (no divergent branch); the run's sums of lanes that own no group
// are dropped when the run ends (pair_run_sums).
template <int ADV, bool X2 = false, class Acc>
__device__ __forceinline__ void pair_level1(const PairCtx& X, int r, const PRow& A, PRow& B,
                                            const PRow& N, float* fs1, float* u1, Acc& ly1,
                                            Acc& lp1) {
  float z[4];
  if constexpr (X2)
    pair_level_x2<ADV>(A.y, B.y, N.y, B.xx, B.xy, N.xy, B.yy, N.yy, X.abx, X.aby, fs1, X.ig,
                       X.sh1, z);
  else
    pair_level<ADV>(A.y, B.y, N.y, B.xx, B.xy, N.xy, B.yy, N.yy, X.abx, X.aby, fs1, X.ig, X.sh1, z);
  pair_y1(u1, z, X);
  if (r >= X.y0 && r < X.y1) {               // uniform over the warp
    if constexpr (X2) {
#pragma unroll
      for (int k = 0; k < 4; k += 2) {
        const float2 pm = fma2(f2(X.d0, X.d0), f2(B.y[k + 1], B.y[k + 2]), f2(B.p[k], B.p[k + 1]));
        const float2 pn = fma2(f2(X.d1, X.d1), f2(z[k], z[k + 1]), pm);
        B.p[k] = pn.x;
        B.p[k + 1] = pn.y;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float pm = fmaf(X.d0, B.y[k + 1], B.p[k]);   // the pending d_m y_m
        B.p[k] = fmaf(X.d1, z[k], pm);
      }
    }
    acc_sq4(ly1, z);
    acc_sq4(lp1, B.p);
    const long long idx = (long long)r * X.G.nx + X.gx;
    if (X.L.own)
      *reinterpret_cast<float4*>(X.p + idx) = make_float4(B.p[0], B.p[1], B.p[2], B.p[3]);
  }
}

// The norm sums of one run added to the thread's totals: only lanes that own
// their group contribute (the others' terms may come from records they never
// filled).
template <class Acc>
__device__ __forceinline__ void pair_run_sums(const PairCtx& X, const Acc* r, float& ly1,
                                              float& lp1, float& ly2, float& lp2) {
  if (X.L.own) {
    ly1 += acc_total(r[0]);
    lp1 += acc_total(r[1]);
    ly2 += acc_total(r[2]);
    lp2 += acc_total(r[3]);
  }
}

// Step j: level 1 on row j + 1 and level 2 on row j.  On entry A, B hold rows
// j, j + 1 (B.p: p_m of row j + 1; A.p: p_{m+1} of row j) and Ua, Ub the
// y_{m+1} rows j - 1, j; N and Un are free.  The next step's roles are
// (B, N, A) and (Ub, Un, Ua).
template <int ADV, class Ld>
__device__ __forceinline__ void pair_step(const PairCtx& X, Ld& ldr, int j, PRow& A, PRow& B,
                                          PRow& N, const float* Ua, const float* Ub, float* Un,
                                          float* fs1, float* fs2, float& ly1, float& lp1,
                                          float& ly2, float& lp2) {
  pair_consume(X, ldr, j + 2, N);
  pair_level1<ADV>(X, j + 1, A, B, N, fs1, Un, ly1, lp1);
  if (X.G.bc != 0 && j + 1 == X.G.ny) {     // y_{m+1} row ny = -(row ny - 1)
#pragma unroll
    for (int k = 0; k < 6; ++k) Un[k] = -Ub[k];
  }
  // level 2 on row j: coefficient rows j (A) and j + 1 (B)
  float z[4];
  pair_level<ADV>(Ua, Ub, Un, A.xx, A.xy, B.xy, A.yy, B.yy, X.abx, X.aby, fs2, X.ig, X.sh2, z);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float p2 = fmaf(X.d2, z[k], A.p[k]);
    ly2 = fmaf(z[k], z[k], ly2);
    lp2 = fmaf(p2, p2, lp2);
  }
  const long long idx = (long long)j * X.G.nx + X.gx;
  if (X.L.own) *reinterpret_cast<float4*>(X.yout + idx) = make_float4(z[0], z[1], z[2], z[3]);
}

// One marching run of rows [y0, y1) (X.y0, X.y1) of the strip of X, its rows
// brought into the warp's ring by the loader ldr.
template <int ADV, class Ld>
__device__ __forceinline__ void pair_run(const PairCtx& X, Ld& ldr, float& ly1, float& lp1,
                                         float& ly2, float& lp2) {
  float rs[4] = {0.f, 0.f, 0.f, 0.f};   // this run's norm sums
  const int y0 = X.y0, y1 = X.y1;
  __syncwarp();
#pragma unroll 1
  for (int q = 0; q < X.stages; ++q) ldr.issue(X, y0 - 2 + q);
  PRow r0, r1, r2;
  float u0[6], u1[6], u2[6], fs1[4], fs2[4];
  pair_consume(X, ldr, y0 - 2, r0);
  pair_consume(X, ldr, y0 - 1, r1);
  pair_north<ADV>(r0.y, r1.y, r0.xy, r1.xy, r0.yy, r1.yy, X.aby, fs1);   // south faces, row y0 - 1
  pair_consume(X, ldr, y0, r2);
  pair_level1<ADV>(X, y0 - 1, r0, r1, r2, fs1, u1, rs[0], rs[1]);
  pair_consume(X, ldr, y0 + 1, r0);
  pair_level1<ADV>(X, y0, r1, r2, r0, fs1, u2, rs[0], rs[1]);
  if (X.G.bc != 0 && y0 == 0) {               // y_{m+1} row -1 = -(row 0)
#pragma unroll
    for (int k = 0; k < 6; ++k) u1[k] = -u2[k];
  }
  // south faces of level 2 on row y0: coefficient rows y0 - 1 (r1) and y0 (r2)
  pair_north<ADV>(u1, u2, r1.xy, r2.xy, r1.yy, r2.yy, X.aby, fs2);
  // rows: r2 = y0, r0 = y0 + 1, r1 free; y_{m+1}: u1 = y0 - 1, u2 = y0, u0 free
  int j = y0;
#pragma unroll 1
  for (; j + 3 <= y1; j += 3) {
    pair_step<ADV>(X, ldr, j, r2, r0, r1, u1, u2, u0, fs1, fs2, rs[0], rs[1], rs[2], rs[3]);
    pair_step<ADV>(X, ldr, j + 1, r0, r1, r2, u2, u0, u1, fs1, fs2, rs[0], rs[1], rs[2], rs[3]);
    pair_step<ADV>(X, ldr, j + 2, r1, r2, r0, u0, u1, u2, fs1, fs2, rs[0], rs[1], rs[2], rs[3]);
  }
  if (j < y1) pair_step<ADV>(X, ldr, j, r2, r0, r1, u1, u2, u0, fs1, fs2, rs[0], rs[1], rs[2], rs[3]);
  if (j + 1 < y1)
    pair_step<ADV>(X, ldr, j + 1, r0, r1, r2, u2, u0, u1, fs1, fs2, rs[0], rs[1], rs[2], rs[3]);
  ldr.drain(X);
  pair_run_sums(X, rs, ly1, lp1, ly2, lp2);
}

// Step j with the next row prefetched: on entry A, B, N hold rows j, j + 1,
// j + 2 (N was read by the previous step) and Q is free; Q receives row
// j + 3 first, so its shared-memory loads and shuffles overlap this step's
// arithmetic instead of heading its dependency chain.  Otherwise pair_step.
// The next step's roles are (B, N, Q, A) and (Ub, Un, Ua's successor).  X2:
// the levels in packed pairs (same results).
template <int ADV, bool X2, class Ld, class Acc>
__device__ __forceinline__ void pair_step_pf(const PairCtx& X, Ld& ldr, int j, PRow& A, PRow& B,
                                             PRow& N, PRow& Q, const float* Ua, const float* Ub,
                                             float* Un, float* fs1, float* fs2, Acc& ly1,
                                             Acc& lp1, Acc& ly2, Acc& lp2) {
  if (j + 3 <= X.y1 + 1) pair_consume(X, ldr, j + 3, Q);   // rows are issued up to y1 + 1
  pair_level1<ADV, X2>(X, j + 1, A, B, N, fs1, Un, ly1, lp1);
  if (X.G.bc != 0 && j + 1 == X.G.ny) {     // y_{m+1} row ny = -(row ny - 1)
#pragma unroll
    for (int k = 0; k < 6; ++k) Un[k] = -Ub[k];
  }
  float z[4], p2[4];
  if constexpr (X2) {
    pair_level_x2<ADV>(Ua, Ub, Un, A.xx, A.xy, B.xy, A.yy, B.yy, X.abx, X.aby, fs2, X.ig, X.sh2,
                       z);
#pragma unroll
    for (int k = 0; k < 4; k += 2) {
      const float2 t = fma2(f2(X.d2, X.d2), f2(z[k], z[k + 1]), f2(A.p[k], A.p[k + 1]));
      p2[k] = t.x;
      p2[k + 1] = t.y;
    }
  } else {
    pair_level<ADV>(Ua, Ub, Un, A.xx, A.xy, B.xy, A.yy, B.yy, X.abx, X.aby, fs2, X.ig, X.sh2, z);
#pragma unroll
    for (int k = 0; k < 4; ++k) p2[k] = fmaf(X.d2, z[k], A.p[k]);
  }
  acc_sq4(ly2, z);
  acc_sq4(lp2, p2);
  const long long idx = (long long)j * X.G.nx + X.gx;
  if (X.L.own) *reinterpret_cast<float4*>(X.yout + idx) = make_float4(z[0], z[1], z[2], z[3]);
}

// pair_run with one row of lookahead in registers: four row records and four
// y_{m+1} rows rotate with period 4 (the loop is unrolled four times, so no
// row is copied).  The same operations in the same order as pair_run; with
// X2 the levels run in packed pairs and each norm sum is kept as two
// interleaved partial sums.
template <int ADV, bool X2 = false, class Ld>
__device__ __forceinline__ void pair_run_pf(const PairCtx& X, Ld& ldr, float& ly1, float& lp1,
                                            float& ly2, float& lp2) {
  using Acc = std::conditional_t<X2, float2, float>;
  Acc rs[4] = {};                       // this run's norm sums
  const int y0 = X.y0, y1 = X.y1;
  __syncwarp();
#pragma unroll 1
  for (int q = 0; q < X.stages; ++q) ldr.issue(X, y0 - 2 + q);
  PRow R0, R1, R2, R3;
  float U0[6], U1[6], U2[6], U3[6], fs1[4], fs2[4];
  pair_consume(X, ldr, y0 - 2, R0);
  pair_consume(X, ldr, y0 - 1, R1);
  pair_north_any<ADV, X2>(R0.y, R1.y, R0.xy, R1.xy, R0.yy, R1.yy, X.aby, fs1);   // south faces, row y0 - 1
  pair_consume(X, ldr, y0, R2);
  pair_level1<ADV, X2>(X, y0 - 1, R0, R1, R2, fs1, U1, rs[0], rs[1]);
  pair_consume(X, ldr, y0 + 1, R3);
  pair_level1<ADV, X2>(X, y0, R1, R2, R3, fs1, U2, rs[0], rs[1]);
  if (X.G.bc != 0 && y0 == 0) {               // y_{m+1} row -1 = -(row 0)
#pragma unroll
    for (int k = 0; k < 6; ++k) U1[k] = -U2[k];
  }
  // south faces of level 2 on row y0: coefficient rows y0 - 1 (R1) and y0 (R2)
  pair_north_any<ADV, X2>(U1, U2, R1.xy, R2.xy, R1.yy, R2.yy, X.aby, fs2);
  pair_consume(X, ldr, y0 + 2, R0);           // y0 + 2 <= y1 + 1: always issued
  // rows: R2 = y0, R3 = y0 + 1, R0 = y0 + 2, R1 free; y_{m+1}: U1 = y0 - 1, U2 = y0
  int j = y0;
#pragma unroll 1
  for (; j + 4 <= y1; j += 4) {
    pair_step_pf<ADV, X2>(X, ldr, j, R2, R3, R0, R1, U1, U2, U3, fs1, fs2, rs[0], rs[1], rs[2], rs[3]);
    pair_step_pf<ADV, X2>(X, ldr, j + 1, R3, R0, R1, R2, U2, U3, U0, fs1, fs2, rs[0], rs[1], rs[2], rs[3]);
    pair_step_pf<ADV, X2>(X, ldr, j + 2, R0, R1, R2, R3, U3, U0, U1, fs1, fs2, rs[0], rs[1], rs[2], rs[3]);
    pair_step_pf<ADV, X2>(X, ldr, j + 3, R1, R2, R3, R0, U0, U1, U2, fs1, fs2, rs[0], rs[1], rs[2], rs[3]);
  }
  if (j < y1)
    pair_step_pf<ADV, X2>(X, ldr, j, R2, R3, R0, R1, U1, U2, U3, fs1, fs2, rs[0], rs[1], rs[2], rs[3]);
  if (j + 1 < y1)
    pair_step_pf<ADV, X2>(X, ldr, j + 1, R3, R0, R1, R2, U2, U3, U0, fs1, fs2, rs[0], rs[1], rs[2], rs[3]);
  if (j + 2 < y1)
    pair_step_pf<ADV, X2>(X, ldr, j + 2, R0, R1, R2, R3, U3, U0, U1, fs1, fs2, rs[0], rs[1], rs[2], rs[3]);
  ldr.drain(X);
  pair_run_sums(X, rs, ly1, lp1, ly2, lp2);
}

}  // namespace
}  // namespace ad
