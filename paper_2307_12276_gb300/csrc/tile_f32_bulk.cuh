// FP32 fused Leja iteration with a warp-specialised bulk-copy pipeline.
//
// A tile is 256 columns x TY rows.  The block has 8 consumer warps (thread t
// owns column x0 + t) and 1 producer warp.  Each row r of a tile is an "item":
// the producer's lane 0 streams the row's segments of y, Dxy, Dxx, Dyy, p (and
// w2 / advection fields) from global memory into one stage of a D-deep
// shared-memory ring with cp.async.bulk (completion counted in bytes on the
// stage's "full" mbarrier); the two halo columns come with 4-byte cp.async
// whose completion arrives on the same mbarrier.  Consumers wait for the
// stage, compute the row from shared memory only, and release the stage on
// its "empty" mbarrier once the row is no longer needed (a row is read by
// three consecutive steps).  Ghost rows/columns are copied from their mapped
// (mirrored or wrapped) source and the Dirichlet sign is applied on read.
//
// Requirements (checked by the launcher): nx % 4 == 0, so every row segment
// starts and ends on a 16-byte boundary.  Every wait is bounded by
// kBulkTimeoutNs of global time; on a timeout the block records status 4 in
// the control block, the producer waits (again bounded) for the copies it
// has in flight, and the block leaves.
#pragma once
#include <cstdint>

#include "tile_f32.cuh"

namespace ad {
namespace {

constexpr int kBulkStages = 8;
constexpr int kBulkTY = 32;
constexpr int kBulkThreads = kThreads + 32;        // 8 consumer warps + 1 producer warp
constexpr unsigned long long kBulkTimeoutNs = 2000000000ULL;

// stage layout (floats); halo arrays keep the interior 16-byte aligned at +4
constexpr int kHalo = 264;                          // [3] left halo, [4..259] interior, [4+W] right
constexpr int kOffY = 0, kOffXY = kHalo, kOffXX = 2 * kHalo, kOffYY = 3 * kHalo;
constexpr int kOffP = kOffYY + kTileCols, kOffW2 = kOffP + kTileCols;
constexpr int kOffAX = kOffW2 + kTileCols, kOffAY = kOffAX + kHalo;
constexpr int kStageFloats = kOffAY + kTileCols;     // 2080 floats = 8320 B

__device__ __forceinline__ unsigned long long global_ns_() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns_();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns_() - t0 > kBulkTimeoutNs) return false;
  }
  return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

struct BulkItems {
  // the block's items: tiles tile0, tile0 + stride, ... ; rows y0 - 1 .. y1 of each
  int tiles_x, ntiles, tile0, stride;
};

// Producer: stream every item of this block's tiles through the ring.
template <bool AUG, int ADV>
__device__ void bulk_producer(const SeriesArgs& a, const float* yin, const BulkItems& it,
                              float* ring, uint64_t* full, uint64_t* empty, float* rowsign,
                              int& failed) {
  const GridDev g = a.g;
  const int nx = g.nx, ny = g.ny, bc = g.bc;
  const long long n = g.n;
  const float* F = static_cast<const float*>(a.coef);
  const float* Fxx = F;
  const float* Fyy = F + n;
  const float* Fxy = F + 2 * n;
  const float* Fax = F + 3 * n;
  const float* Fay = F + 4 * n;
  const float* p = static_cast<const float*>(a.p);
  const float* w2 = static_cast<const float*>(a.w2);
  const int lane = threadIdx.x & 31;
  long long q = 0;      // item counter of this block
  for (int tile = it.tile0; tile < it.ntiles; tile += it.stride) {
    const int x0 = (tile % it.tiles_x) * kTileCols, y0 = (tile / it.tiles_x) * kBulkTY;
    const int y1 = min(ny, y0 + kBulkTY);
    const int W = min(kTileCols, nx - x0);
    float sl, sr;
    const int li = map_col(x0 - 1, nx, bc, sl);
    const int ri = map_col(x0 + W, nx, bc, sr);
    for (int r = y0 - 1; r <= y1; ++r, ++q) {
      const int slot = (int)(q % kBulkStages);
      const unsigned use = (unsigned)(q / kBulkStages);
      if (lane == 0) {
        if (use > 0 && !mbar_wait(&empty[slot], (use - 1) & 1u)) { failed = 1; }
      }
      failed = __shfl_sync(0xffffffffu, failed, 0);
      if (failed) break;
      if (lane == 0) {
        float* S = ring + (size_t)slot * kStageFloats;
        const RowMap rm = map_row(r, nx, ny, bc);
        const bool inner = (r >= y0 && r < y1);
        rowsign[slot] = rm.sg;
        // halo columns (4-byte async copies, mapped source columns)
        cp_async4(S + kOffY + 3, yin + rm.off + li);
        cp_async4(S + kOffY + 4 + W, yin + rm.off + ri);
        cp_async4(S + kOffXY + 3, Fxy + rm.off + li);
        cp_async4(S + kOffXY + 4 + W, Fxy + rm.off + ri);
        if (inner) {
          cp_async4(S + kOffXX + 3, Fxx + rm.off + li);
          cp_async4(S + kOffXX + 4 + W, Fxx + rm.off + ri);
          if (ADV == 2) {
            cp_async4(S + kOffAX + 3, Fax + rm.off + li);
            cp_async4(S + kOffAX + 4 + W, Fax + rm.off + ri);
          }
        }
        cp_async_arrive_noinc(&full[slot]);
        const unsigned seg = (unsigned)W * 4u;
        unsigned bytes = 3u * seg;                       // y, Dxy, Dyy
        if (ADV == 2) bytes += seg;                      // ay
        if (inner) bytes += 2u * seg + (AUG ? seg : 0u) + (ADV == 2 ? seg : 0u);  // Dxx, p, w2, ax
        mbar_arrive_expect_tx(&full[slot], bytes);
        const long long base = rm.off + x0;
        bulk_g2s(S + kOffY + 4, yin + base, seg, &full[slot]);
        bulk_g2s(S + kOffXY + 4, Fxy + base, seg, &full[slot]);
        bulk_g2s(S + kOffYY, Fyy + base, seg, &full[slot]);
        if (ADV == 2) bulk_g2s(S + kOffAY, Fay + base, seg, &full[slot]);
        if (inner) {
          const long long cb = (long long)r * nx + x0;   // inner rows are never ghosts
          bulk_g2s(S + kOffXX + 4, Fxx + base, seg, &full[slot]);
          bulk_g2s(S + kOffP, p + cb, seg, &full[slot]);
          if (AUG) bulk_g2s(S + kOffW2, w2 + cb, seg, &full[slot]);
          if (ADV == 2) bulk_g2s(S + kOffAX + 4, Fax + base, seg, &full[slot]);
        }
      }
    }
    if (failed) break;
  }
  // drain: every issued stage must complete before the block may leave
  if (lane == 0) {
    const long long nitems = q;
    for (long long k = (nitems > kBulkStages ? nitems - kBulkStages : 0); k < nitems; ++k) {
      const int slot = (int)(k % kBulkStages);
      if (!mbar_wait(&full[slot], (unsigned)((k / kBulkStages) & 1))) { failed = 1; break; }
    }
  }
}

// Consumer thread t: compute every row of this block's tiles from the ring.
template <bool AUG, int ADV>
__device__ void bulk_consumer(const SeriesArgs& a, const LejaCoef& lc, float* yout, float* p,
                              const BulkItems& it, float* ring, uint64_t* full, uint64_t* empty,
                              const float* rowsign, float ig, float sh, float d, float e1,
                              float e2, double& accy, double& accp, int& failed) {
  const GridDev g = a.g;
  const int nx = g.nx, ny = g.ny, bc = g.bc;
  const int t = threadIdx.x, lane = t & 31;
  long long q = 0;
  for (int tile = it.tile0; tile < it.ntiles; tile += it.stride) {
    const int x0 = (tile % it.tiles_x) * kTileCols, y0 = (tile / it.tiles_x) * kBulkTY;
    const int y1 = min(ny, y0 + kBulkTY);
    const int i = x0 + t;
    const bool compute = i < nx;
    // Dirichlet ghost columns change the sign of values
    const float cl = (bc == 1 && i == 0) ? -1.f : 1.f;
    const float cr = (bc == 1 && i == nx - 1) ? -1.f : 1.f;
    const long long q0 = q;                       // item of row y0 - 1
    const int nrows = y1 - y0;
    // lane 0 waits, the warp follows (uniform control flow within the warp)
    auto wait_item = [&](long long qq) {
      int ok = 1;
      if (lane == 0) ok = mbar_wait(&full[qq % kBulkStages], (unsigned)((qq / kBulkStages) & 1));
      ok = __shfl_sync(0xffffffffu, ok, 0);
      __syncwarp();
      if (!ok) failed = 1;
    };
    wait_item(q0);          // row y0 - 1
    if (!failed) wait_item(q0 + 1);   // row y0
    float ly = 0.f, lp = 0.f;
    for (int s = 0; s < nrows && !failed; ++s) {
      const long long qm = q0 + s, qc = qm + 1, qp = qm + 2;
      wait_item(qp);
      if (failed) break;
      const float* Sm = ring + (size_t)(qm % kBulkStages) * kStageFloats;
      const float* S0 = ring + (size_t)(qc % kBulkStages) * kStageFloats;
      const float* Sp = ring + (size_t)(qp % kBulkStages) * kStageFloats;
      if (compute) {
        const float sgm = rowsign[qm % kBulkStages], sgp = rowsign[qp % kBulkStages];
        const int c = 4 + t;
        const float uC = S0[kOffY + c], uW = cl * S0[kOffY + c - 1], uE = cr * S0[kOffY + c + 1];
        const float uN = sgp * Sp[kOffY + c], uNW = sgp * cl * Sp[kOffY + c - 1];
        const float uNE = sgp * cr * Sp[kOffY + c + 1];
        const float uS = sgm * Sm[kOffY + c], uSW = sgm * cl * Sm[kOffY + c - 1];
        const float uSE = sgm * cr * Sm[kOffY + c + 1];
        const float xyC = S0[kOffXY + c];
        const float axe = S0[kOffXX + c] + S0[kOffXX + c + 1], axw = S0[kOffXX + c - 1] + S0[kOffXX + c];
        const float qe = xyC + S0[kOffXY + c + 1], qw = S0[kOffXY + c - 1] + xyC;
        const float qn = xyC + Sp[kOffXY + c], qs = Sm[kOffXY + c] + xyC;
        const float yyC = S0[kOffYY + t];
        const float ayn = yyC + Sp[kOffYY + t], ays = Sm[kOffYY + t] + yyC;
        float fe = face_flux(axe, uE - uC, qe, (uNE + uN) - (uSE + uS));
        float fw = face_flux(axw, uC - uW, qw, (uN + uNW) - (uS + uSW));
        float fn = face_flux(ayn, uN - uC, qn, (uNE + uE) - (uNW + uW));
        float fs = face_flux(ays, uC - uS, qs, (uE + uSE) - (uW + uSW));
        if (ADV == 1) {
          fe = fmaf(a.abx, uC + uE, fe);
          fw = fmaf(a.abx, uW + uC, fw);
          fn = fmaf(a.aby, uC + uN, fn);
          fs = fmaf(a.aby, uS + uC, fs);
        } else if (ADV == 2) {
          const float axC = S0[kOffAX + c], ayC = S0[kOffAY + t];
          fe = fmaf(axC + S0[kOffAX + c + 1], uC + uE, fe);
          fw = fmaf(S0[kOffAX + c - 1] + axC, uW + uC, fw);
          fn = fmaf(ayC + Sp[kOffAY + t], uC + uN, fn);
          fs = fmaf(Sm[kOffAY + t] + ayC, uS + uC, fs);
        }
        const float au = (fe - fw) + (fn - fs);
        float z = fmaf(au, ig, -sh * uC);
        if (AUG) {
          if (e1 != 0.0f) z = fmaf(e1, S0[kOffW2 + t], z);
          if (e2 != 0.0f) z = fmaf(e2, static_cast<const float*>(a.w1)[(long long)(y0 + s) * nx + i], z);
        }
        const long long idx = (long long)(y0 + s) * nx + i;
        yout[idx] = z;
        const float pn = fmaf(d, z, S0[kOffP + t]);
        p[idx] = pn;
        ly = fmaf(z, z, ly);
        lp = fmaf(pn, pn, lp);
      }
      // row y0 + s - 1 (item qm) is no longer needed by this warp
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[qm % kBulkStages]);
    }
    if (!failed) {
      __syncwarp();
      if (lane == 0) {                     // the tile's last two rows
        mbar_arrive(&empty[(q0 + nrows) % kBulkStages]);
        mbar_arrive(&empty[(q0 + nrows + 1) % kBulkStages]);
      }
    }
    q = q0 + nrows + 2;
    accy += (double)ly;
    accp += (double)lp;
    if (failed) break;
  }
}

}  // namespace
}  // namespace ad
