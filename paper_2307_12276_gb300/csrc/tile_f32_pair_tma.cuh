// Row records of the FP32 two-iteration kernel brought in by the Tensor
// Memory Accelerator instead of per-lane cp.async.
//
// Each field (y_m, p, Dxx, Dyy, Dxy) has a 2-D tensor map over the [ny][nx]
// grid with a box of 128 columns x 1 row: exactly one row record field of
// PairLayout (lane l's group at 4 l).  For row r of a run, lane 0 of the warp
// announces the record's byte count on the slot's mbarrier
// (arrive.expect_tx) and issues one cp.async.bulk.tensor.2d per field at
// (X0 - 4, mapped row); the copies complete the barrier's phase.  The other
// lanes issue nothing: the 32 x 5 per-lane copies, their address arithmetic
// and the commit groups of the cp.async ring are gone.  Columns outside
// [0, nx) are filled with zeros by the copy engine, which is what the
// cp.async ring leaves for the zero-Dirichlet ghost groups it does not read;
// so every record holds the same values and the kernel's results are bit for
// bit those of the cp.async kernel.  Periodic grids keep the cp.async ring
// (their ghost groups are wrapped copies, which a tile box cannot express).
//
// Measured on GB300 (4096^2, one launch = two iterations): 116 us with this
// loader against 95 us with the cp.async ring, at every ring depth from 6 to
// 11 records.  The marching is bound by the issue latency of its dependent
// stencil levels, not by the copies, and lane 0's issue of the copies sits on
// the warp's critical path where the per-lane cp.async it replaces did not.
// So the cp.async ring stays the default and this loader is opt-in
// (AD_F32_TMA=1); the GPU tests hold the two bit for bit.
//
// Ordering: a slot is refilled by the warp that just read it; after
// __syncwarp (in issue), lane 0 fences the generic-proxy reads against the copy
// engine's writes (fence.proxy.async) before it issues the next copies.
// Every wait is bounded (kBulkTimeoutNs of global time): on a timeout the
// warp records status 4 in the control block, stops issuing and waiting, and
// before it leaves waits (bounded again) for the copies it still has in
// flight.
#pragma once
#include <cuda.h>

#include "tile_f32_bulk.cuh"
#include "tile_f32_pair.cuh"

namespace ad {
namespace {

__device__ __forceinline__ void tma_row(float* dst, const CUtensorMap* map, int x, int y,
                                        uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

struct TmaLoader {
  static constexpr bool kReadAll = true;   // out-of-range columns arrive as zeros
  const PairTmaMaps* maps;
  const CUtensorMap* yin;
  uint64_t* bar;                           // the warp's STAGES barriers
  Ctrl* ctrl;
  unsigned ph;                             // per slot: parity of its next completion
  unsigned pend;                           // per slot: copies issued, not yet consumed
  bool failed;

  __device__ __forceinline__ int slot_of(const PairCtx& X, int r) const {
    return (r - (X.y0 - 2)) % X.stages;
  }

  // (called by the whole warp: the barrier orders every lane's reads of the
  // record before lane 0 hands it to the copy engine)
  __device__ __forceinline__ void issue(const PairCtx& X, int r) {
    __syncwarp();
    if (failed || r > X.y1 + 1) return;
    using PL = PairLayout;
    const int s = slot_of(X, r);
    pend |= 1u << s;
    if (X.G.lane == 0) {
      const int ny = X.G.ny;
      const int jr = r < 0 ? -1 - r : (r >= ny ? 2 * ny - 1 - r : r);   // zero-Dirichlet mirror
      const bool xx = r >= X.y0 - 1 && r <= X.y1, p = r >= X.y0 && r < X.y1;
      float* S = pair_slot(X, r);
      uint64_t* b = bar + s;
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(b, 512u * (3u + (xx ? 1u : 0u) + (p ? 1u : 0u)));
      tma_row(S + PL::Y, yin, X.gx, jr, b);
      tma_row(S + PL::XY, &maps->xy, X.gx, jr, b);
      tma_row(S + PL::YY, &maps->yy, X.gx, jr, b);
      if (xx) tma_row(S + PL::XX, &maps->xx, X.gx, jr, b);
      if (p) tma_row(S + PL::P, &maps->p, X.gx, jr, b);
    }
  }

  __device__ __forceinline__ const float* wait(const PairCtx& X, int r) {
    const int s = slot_of(X, r);
    if (!failed) {
      const bool ok = __all_sync(0xffffffffu, mbar_wait(bar + s, (ph >> s) & 1u));
      if (ok) {
        ph ^= 1u << s;
        pend &= ~(1u << s);
      } else {
        failed = true;                     // the slot keeps its pending copy
        if (X.G.lane == 0) *(volatile int*)&ctrl->status = 4;
      }
    }
    return pair_slot(X, r);
  }

  __device__ __forceinline__ void drain(const PairCtx& X) {
    if (failed)                            // copies still in flight land before the warp leaves
      for (int s = 0; s < X.stages; ++s)
        if (pend & (1u << s)) (void)mbar_wait(bar + s, (ph >> s) & 1u);
    __syncwarp();
  }
};

}  // namespace
}  // namespace ad
