// Batched exponential-midpoint step over many independent problems of uneven
// size (the momentum slices of a cosmic-ray transport grid: the momentum
// terms of the full transport equation are dropped, so each momentum p only
// sets its own diffusion coefficients).  Every slice is an FP32-storage
// operator; one step of Eq. exp_midpoint,
//     u_s += dt phi_1(dt A_s)(A_s u_s + S_s(t + dt/2)),
// runs for all slices as ONE CUDA graph launch:
//   apply (v_s = A_s u_s + S_s)  ->  init (y_0 = v_s, p = d_0 v_s)
//   -> WHILE { 4 x fused Leja iteration over every active slice's tiles }
//   -> update (u_s += dt p_s).
// The iteration kernel is persistent: its blocks stride over one flat list of
// 256 x TY tiles of all slices.  Each slice keeps its own Leja scalars,
// control block and stopping decision: the last tile of a slice to finish
// reduces that slice's tile partials (fixed order) and applies the stopping
// rule; slices that stopped are skipped; the last block of a launch keeps the
// loop running while any slice is active.  The tile height TY and the number
// of resident blocks are chosen per batch by a small autotuner whose choice is
// cached in a JSON file.
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "ad_internal.h"
#include "anidiff.h"
#include "leja_host.h"
#include "tile_f32.cuh"
#include "tile_f32_ring.cuh"
#include "tile_f32_pair.cuh"

namespace ad {
namespace {

constexpr int kBatchSources = 4;
constexpr int kBatchUnroll = 4;
constexpr unsigned long long kPersistTimeoutNs = 2000000000ULL;   // bound of every wait

// Device words of a batched step (the kernels take a pointer to `ticket`).
struct BatchSync {
  unsigned int ticket;        // launches of the graph loop: warps of the launch done
  int active;                 // persistent iteration: slices still iterating
  int abort;                  // persistent iteration: a bounded wait gave up
  int pad;
  unsigned long long next;    // persistent iteration: next (pass, tile) item
};

__device__ __forceinline__ unsigned long long batch_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct BatchSlice {
  SeriesArgs a;                     // operator buffers, batch-owned lc/ctrl
  float* u;                         // the slice's state (caller memory)
  const float* src_g[kBatchSources];
  float src_c[kBatchSources];       // h_k(t + dt/2)
  int nsrc;
  float dt;
  double d0;
  int tile_off, ntiles, tiles_x;     // 256 x TY tiles (streaming kernels, tile iteration)
  int rt_off, rt_n, rt_x;            // 128-column x R-row warp tiles (ring iteration)
};

// Stopping rule of the Newton series (same reading as the single-operator
// kernels): squared form of |d_{m+1}| ||y|| <= tol ||p|| for m+1 >= 2.
__device__ int decide(Ctrl* ctrl, const LejaCoef& lc, int m, double ty, double tp) {
  const int terms = m + 1;
  ctrl->ynorm2 = ty;
  ctrl->pnorm2 = tp;
  ctrl->iters = terms;
  ctrl->err_est = lc.absd;
  const double tol = ctrl->tol;
  int stop = 0;
  if (ctrl->force > 0) {
    stop = terms >= ctrl->force;
  } else if (!isfinite(ty) || !isfinite(tp)) {
    stop = 1;
    ctrl->status = 3;
  } else if (terms >= 2 && (lc.absd * lc.absd) * ty <= (tol * tol) * tp) {
    stop = 1;
  } else if (terms >= ctrl->max_iters) {
    stop = 1;
    ctrl->status = 3;
  }
  if (terms >= kMaxIters) stop = 1;
  return stop;
}

// ---------------------------------------------------------------- kernels
template <int ADV>
__global__ void __launch_bounds__(kThreads) batch_apply_k(const BatchSlice* slices,
                                                         const int* tile_slice, int ntiles, int TY) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const BatchSlice& S = slices[tile_slice[t]];
    const GridDev g = S.a.g;
    const int local = t - S.tile_off;
    const int x0 = (local % S.tiles_x) * kTileCols, y0 = (local / S.tiles_x) * TY;
    const int i = x0 + threadIdx.x;
    if (i >= g.nx) continue;
    const float* F = static_cast<const float*>(S.a.coef);
    float* v = static_cast<float*>(const_cast<void*>(S.a.w1));
    for (int j = y0; j < min(g.ny, y0 + TY); ++j) {
      const long long idx = (long long)j * g.nx + i;
      const bool interior = i > 0 && j > 0 && i + 1 < g.nx && j + 1 < g.ny;
      float r = flux_apply_f32(F, g.n, S.u, i, j, g.nx, g.ny, g.bc, interior, ADV, S.a.abx, S.a.aby);
      for (int k = 0; k < S.nsrc; ++k) r = fmaf(S.src_c[k], S.src_g[k][idx], r);
      v[idx] = r;
    }
  }
}

__global__ void __launch_bounds__(kThreads) batch_init_k(const BatchSlice* slices,
                                                        const int* tile_slice, int ntiles, int TY,
                                                        int nslices, int force, int max_iters,
                                                        double tol, unsigned int* bticket) {
  if (blockIdx.x == 0) {
    for (int s = threadIdx.x; s < nslices; s += blockDim.x) {
      Ctrl* c = slices[s].a.ctrl;
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
      c->gen = 0u;                // passes completed (persistent iteration)
    }
    if (threadIdx.x == 0) {
      BatchSync* bs = reinterpret_cast<BatchSync*>(bticket);
      bs->ticket = 0u;
      bs->active = nslices;
      bs->abort = 0;
      bs->next = 0ull;
    }
  }
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const BatchSlice& S = slices[tile_slice[t]];
    const GridDev g = S.a.g;
    const int local = t - S.tile_off;
    const int x0 = (local % S.tiles_x) * kTileCols, y0 = (local / S.tiles_x) * TY;
    const int i = x0 + threadIdx.x;
    if (i >= g.nx) continue;
    const float* v = static_cast<const float*>(S.a.w1);
    float* y = static_cast<float*>(S.a.y[0]);
    float* p = static_cast<float*>(S.a.p);
    const float d0 = (float)S.d0;
    for (int j = y0; j < min(g.ny, y0 + TY); ++j) {
      const long long idx = (long long)j * g.nx + i;
      const float x = v[idx];
      y[idx] = x;
      p[idx] = d0 * x;
    }
  }
}

template <int ADV, int TY>
__global__ void __launch_bounds__(kThreads) batch_iter_k(const BatchSlice* slices,
                                                        const int* tile_slice, int ntiles,
                                                        int nslices, double* tile_partials,
                                                        unsigned int* bticket,
                                                        unsigned long long handle, int has_handle) {
  __shared__ float sy[3][kTileCols + 2];
  __shared__ float sxy[2][kTileCols + 2];
  __shared__ float sxx[kTileCols + 2];
  __shared__ float sax[kTileCols + 2];
  __shared__ int s_last;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int s = tile_slice[t];
    const BatchSlice& S = slices[s];
    const volatile Ctrl* vc = S.a.ctrl;
    if (vc->stop) continue;                    // uniform over the block
    const int m = vc->m;
    const LejaCoef lc = S.a.lc[m];
    const float* yin = static_cast<const float*>(S.a.y[m & 1]);
    float* yout = static_cast<float*>(S.a.y[(m + 1) & 1]);
    float* p = static_cast<float*>(S.a.p);
    const float ig = (float)(1.0 / S.a.gamma);
    const float sh = (float)(S.a.c / S.a.gamma + lc.xi);
    const int local = t - S.tile_off;
    double ty = 0.0, tp = 0.0;
    tile_f32<false, ADV, TY>(S.a, lc, local % S.tiles_x, local / S.tiles_x, yin, yout, p, ig, sh,
                             (float)lc.d, 0.0f, 0.0f, sy, sxx, sxy, sax, ty, tp);
    block_sum2(ty, tp);
    if (threadIdx.x == 0) {
      tile_partials[2 * t] = ty;
      tile_partials[2 * t + 1] = tp;
      __threadfence();
      const unsigned int k = atomicAdd(&S.a.ctrl->ticket, 1u);
      s_last = (k == (unsigned int)S.ntiles - 1u) ? 1 : 0;
    }
    __syncthreads();
    if (s_last) {                              // this slice's last tile: decide for it
      __threadfence();
      double ay = 0.0, ap = 0.0;
      // unrolled: the loads of several tiles in flight, the sums still in tile order
#pragma unroll 8
      for (int q = threadIdx.x; q < S.ntiles; q += blockDim.x) {
        const double2 v = __ldcg(reinterpret_cast<const double2*>(tile_partials) + S.tile_off + q);
        ay += v.x;
        ap += v.y;
      }
      block_sum2(ay, ap);
      if (threadIdx.x == 0) {
        Ctrl* ctrl = S.a.ctrl;
        const int stop = decide(ctrl, lc, m, ay, ap);
        ctrl->ticket = 0u;
        ctrl->stop = stop;
        ctrl->m = m + 1;
        __threadfence();
      }
    }
  }
  // the launch's last block keeps the loop running while any slice is active
  __syncthreads();                             // every warp has read s_last
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int k = atomicAdd(bticket, 1u);
    s_last = (k == gridDim.x - 1u) ? 1 : 0;
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    int active = 0;
    for (int s = 0; s < nslices; ++s) active |= !*(volatile int*)&slices[s].a.ctrl->stop;
    *bticket = 0u;
    __threadfence();
    if (has_handle) cudaGraphSetConditional((cudaGraphConditionalHandle)handle, active ? 1u : 0u);
  }
}

// Fused Leja iteration over the flat list of warp tiles (128 columns x R
// rows of one slice) with the register-marching kernel of the single-operator
// FP32 path (tile_f32_ring.cuh): each warp takes tiles gw, gw + GW, ..., skips
// tiles of slices that have stopped, marches its tile through its cp.async
// ring and publishes the tile's two norm partials.  The warp that completes
// a slice's last tile of the launch (ticket) sums that slice's partials in
// tile order and applies the stopping rule; the launch's last warp keeps the
// graph loop running while any slice is active.  Requires nx % 4 == 0 for
// every slice (rows on 16-byte boundaries).
template <int ADV>
__global__ void __launch_bounds__(kRingThreads, 1)
    batch_ring_k(const BatchSlice* slices, const int* rtile_slice, int nrtiles, int nslices,
                 int R, double* tile_partials, unsigned int* bticket, unsigned long long handle,
                 int has_handle) {
  extern __shared__ __align__(16) float ring_smem[];
  using L = RingLayout<false, ADV>;
  float* ring = ring_smem + (size_t)(threadIdx.x >> 5) * L::STAGES * L::SIZE;
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kRingWarps + (threadIdx.x >> 5);
  const int GW = gridDim.x * kRingWarps;
  for (int tile = gw; tile < nrtiles; tile += GW) {
    const int s = rtile_slice[tile];
    const BatchSlice& S = slices[s];
    const volatile Ctrl* vc = S.a.ctrl;
    if (vc->stop) continue;                    // uniform over the warp
    const int m = vc->m;
    const LejaCoef lc = S.a.lc[m];
    const float* yin = static_cast<const float*>(S.a.y[m & 1]);
    float* yout = static_cast<float*>(S.a.y[(m + 1) & 1]);
    float* p = static_cast<float*>(S.a.p);
    const float ig = (float)(1.0 / S.a.gamma);
    const float sh = (float)(S.a.c / S.a.gamma + lc.xi);
    const int local = tile - S.rt_off;
    const int x0 = (local % S.rt_x) * kVecCols, y0 = (local / S.rt_x) * R;
    const int y1 = min(S.a.g.ny, y0 + R);
    VGeo G;
    G.nx = S.a.g.nx;
    G.ny = S.a.g.ny;
    G.bc = S.a.g.bc;
    G.n = S.a.g.n;
    G.lane = lane;
    G.x = x0 + 4 * lane;
    G.active = G.x < G.nx;
    float ly = 0.f, lp = 0.f;
    ring_run<false, ADV>(S.a, G, ring, y0, y1, yin, yout, p, ig, sh, (float)lc.d, 0.f, 0.f, ly,
                         lp);
    double ty = ly, tp = lp;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ty += __shfl_down_sync(0xffffffffu, ty, o);
      tp += __shfl_down_sync(0xffffffffu, tp, o);
    }
    int last = 0;
    if (lane == 0) {
      tile_partials[2 * tile] = ty;
      tile_partials[2 * tile + 1] = tp;
      __threadfence();
      const unsigned int k = atomicAdd(&S.a.ctrl->ticket, 1u);
      last = (k == (unsigned int)S.rt_n - 1u) ? 1 : 0;
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) {                                // this slice's last tile: decide for it
      __threadfence();
      double ay = 0.0, ap = 0.0;
      // unrolled: the loads of several tiles in flight, the sums still in tile order
#pragma unroll 8
      for (int q = lane; q < S.rt_n; q += 32) {
        const double2 v = __ldcg(reinterpret_cast<const double2*>(tile_partials) + S.rt_off + q);
        ay += v.x;
        ap += v.y;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ay += __shfl_down_sync(0xffffffffu, ay, o);
        ap += __shfl_down_sync(0xffffffffu, ap, o);
      }
      if (lane == 0) {
        Ctrl* ctrl = S.a.ctrl;
        const int stop = decide(ctrl, lc, m, ay, ap);
        ctrl->ticket = 0u;
        ctrl->stop = stop;
        ctrl->m = m + 1;
        __threadfence();
      }
    }
  }
  // the launch's last warp keeps the loop running while any slice is active
  if (lane == 0) {
    __threadfence();
    const unsigned int k = atomicAdd(bticket, 1u);
    if (k == (unsigned int)GW - 1u) {
      __threadfence();
      int active = 0;
      for (int s = 0; s < nslices; ++s) active |= !*(volatile int*)&slices[s].a.ctrl->stop;
      *bticket = 0u;
      __threadfence();
      if (has_handle)
        cudaGraphSetConditional((cudaGraphConditionalHandle)handle, active ? 1u : 0u);
    }
  }
}

// Two fused Leja iterations per launch (temporal blocking, tile_f32_pair.cuh)
// over the flat list of warp tiles (120 produced columns x R rows of one
// slice).  In pair mode a slice's y_m lives in y buffer (m / 2) & 1, p holds
// p_{m-1} + pending d_m y_m (added by the next launch or by batch_finish_k).
// The warp completing a slice's last tile sums the tile partials of both
// iterations in tile order and applies the stopping rule after iteration m
// and, if it does not fire, after iteration m + 1.  Eligible batches: every
// slice with nx % 4 == 0 and ny >= 2, constant or no advection.
template <int ADV, int MODE>
__global__ void __launch_bounds__(kRingThreads, 1)
    batch_pair_k(const BatchSlice* slices, const int* rtile_slice, int nrtiles, int nslices,
                 int R, double* tile_partials, unsigned int* bticket, unsigned long long handle,
                 int has_handle) {
  extern __shared__ __align__(16) float pair_smem[];
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kRingWarps + (threadIdx.x >> 5);
  const int GW = gridDim.x * kRingWarps;
  float* ring = pair_smem + (size_t)(threadIdx.x >> 5) * PairLayout::STAGES * PairLayout::SIZE;
  for (int tile = gw; tile < nrtiles; tile += GW) {
    const int s = rtile_slice[tile];
    const BatchSlice& S = slices[s];
    const volatile Ctrl* vc = S.a.ctrl;
    if (vc->stop) continue;                    // uniform over the warp
    const int m = vc->m;                       // even
    const LejaCoef lc1 = S.a.lc[m], lc2 = S.a.lc[m + 1];
    PairCtx X;
    X.F = static_cast<const float*>(S.a.coef);
    X.yin = static_cast<const float*>(S.a.y[(m >> 1) & 1]);
    X.yout = static_cast<float*>(S.a.y[((m >> 1) + 1) & 1]);
    X.p = static_cast<float*>(S.a.p);
    X.ring = ring;
    X.stages = PairLayout::STAGES;
    X.G.nx = S.a.g.nx;
    X.G.ny = S.a.g.ny;
    X.G.bc = S.a.g.bc;
    X.G.n = S.a.g.n;
    X.G.lane = lane;
    X.ig = (float)(1.0 / S.a.gamma);
    X.sh1 = (float)(S.a.c / S.a.gamma + lc1.xi);
    X.sh2 = (float)(S.a.c / S.a.gamma + lc2.xi);
    X.d0 = m > 0 ? (float)S.a.lc[m - 1].d : 0.0f;
    X.d1 = (float)lc1.d;
    X.d2 = (float)lc2.d;
    X.abx = S.a.abx;
    X.aby = S.a.aby;
    const int local = tile - S.rt_off;
    const int X0 = (local % S.rt_x) * kPairOwn;
    X.y0 = (local / S.rt_x) * R;
    X.y1 = min(S.a.g.ny, X.y0 + R);
    X.L = pair_lane(X0, lane, X.G.nx, X.G.bc);
    X.gx = X0 - 4 + 4 * lane;
    X.fix = X.G.bc != 0 && (X0 == 0 || X0 + kPairOwn >= X.G.nx);
    float ly1 = 0.f, lp1 = 0.f, ly2 = 0.f, lp2 = 0.f;
    CpAsyncLoader ldr;
    if (MODE == 2) pair_run_pf<ADV, true>(X, ldr, ly1, lp1, ly2, lp2);
    else if (MODE == 1) pair_run_pf<ADV>(X, ldr, ly1, lp1, ly2, lp2);
    else pair_run<ADV>(X, ldr, ly1, lp1, ly2, lp2);
    double q[4] = {ly1, lp1, ly2, lp2};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int k = 0; k < 4; ++k) q[k] += __shfl_down_sync(0xffffffffu, q[k], o);
    int last = 0;
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < 4; ++k) tile_partials[4 * tile + k] = q[k];
      __threadfence();
      const unsigned int k = atomicAdd(&S.a.ctrl->ticket, 1u);
      last = (k == (unsigned int)S.rt_n - 1u) ? 1 : 0;
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) {                                // this slice's last tile: decide for it
      __threadfence();
      double t4[4] = {0.0, 0.0, 0.0, 0.0};
      // unrolled: the loads of several tiles in flight, the sums still in tile order
#pragma unroll 8
      for (int r = lane; r < S.rt_n; r += 32) {
        const double2* tp = reinterpret_cast<const double2*>(tile_partials) + 2 * (S.rt_off + r);
        const double2 v0 = __ldcg(tp), v1 = __ldcg(tp + 1);
        t4[0] += v0.x;
        t4[1] += v0.y;
        t4[2] += v1.x;
        t4[3] += v1.y;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 4; ++k) t4[k] += __shfl_down_sync(0xffffffffu, t4[k], o);
      if (lane == 0) {
        Ctrl* ctrl = S.a.ctrl;
        int stop = decide(ctrl, lc1, m, t4[0], t4[1]);
        if (stop) {
          ctrl->m = m + 1;                     // p is complete (no pending term)
        } else {
          stop = decide(ctrl, lc2, m + 1, t4[2], t4[3]);
          ctrl->m = m + 2;
        }
        ctrl->ticket = 0u;
        ctrl->stop = stop;
        __threadfence();
      }
    }
  }
  if (lane == 0) {
    __threadfence();
    const unsigned int k = atomicAdd(bticket, 1u);
    if (k == (unsigned int)GW - 1u) {
      __threadfence();
      int active = 0;
      for (int s = 0; s < nslices; ++s) active |= !*(volatile int*)&slices[s].a.ctrl->stop;
      *bticket = 0u;
      __threadfence();
      if (has_handle)
        cudaGraphSetConditional((cudaGraphConditionalHandle)handle, active ? 1u : 0u);
    }
  }
}

// The whole Newton series of every slice in ONE persistent (cooperative)
// launch: warps take (pass, tile) items in order from a global counter, an
// item being one two-iteration pass (pair_run, as batch_pair_k) of one warp
// tile.  A tile of pass k waits only for pass k - 1 of its own slice (the
// slice's completed-pass counter, set by the warp that applies the slice's
// stopping rule), so slices at different passes overlap and no launch
// boundary separates the passes.  Items are taken in pass order, so every
// item of pass k - 1 is taken, and running on a resident warp, before any
// warp waits on it; each wait is bounded (kPersistTimeoutNs of global time:
// on expiry the kernel records status 4 and every warp leaves).  Items of a
// slice that has stopped are skipped; the warps leave once no slice is
// iterating.
template <int ADV, int MODE>
__global__ void __launch_bounds__(kRingThreads, 1)
    batch_persist_k(const BatchSlice* slices, const int* rtile_slice, int nrtiles, int nslices,
                    int R, double* tile_partials, unsigned int* bticket) {
  extern __shared__ __align__(16) float pair_smem[];
  BatchSync* bs = reinterpret_cast<BatchSync*>(bticket);
  const int lane = threadIdx.x & 31;
  float* ring = pair_smem + (size_t)(threadIdx.x >> 5) * PairLayout::STAGES * PairLayout::SIZE;
  const unsigned long long limit = (unsigned long long)(kMaxIters / 2 + 1) * nrtiles;
  for (;;) {
    unsigned long long it = 0ull;
    if (lane == 0) it = atomicAdd(&bs->next, 1ull);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= limit) break;                    // no series runs past kMaxIters
    const int k = (int)(it / (unsigned long long)nrtiles);
    const int tile = (int)(it - (unsigned long long)k * nrtiles);
    const BatchSlice& S = slices[rtile_slice[tile]];
    Ctrl* ctrl = S.a.ctrl;
    int state = 0;                             // 0 run, 1 slice stopped, 2 leave
    if (lane == 0) {
      const unsigned long long t0 = batch_ns();
      for (;;) {
        if (*(volatile int*)&bs->abort) { state = 2; break; }
        if (*(volatile int*)&ctrl->stop) { state = 1; break; }
        if (*(volatile unsigned int*)&ctrl->gen >= (unsigned int)k) {
          // the slice's flags are written stop first, then (after a fence) the
          // pass count: a stop that came with this count must be seen here
          __threadfence();
          if (*(volatile int*)&ctrl->stop) state = 1;
          break;
        }
        if (batch_ns() - t0 > kPersistTimeoutNs) {
          *(volatile int*)&ctrl->status = 4;
          *(volatile int*)&bs->abort = 1;
          state = 2;
          break;
        }
        __nanosleep(256);                      // back off: the polls share L2 with the work
      }
      if (state == 1 && *(volatile int*)&bs->active == 0) state = 2;   // nothing iterates
      __threadfence();
    }
    state = __shfl_sync(0xffffffffu, state, 0);
    if (state == 2) break;
    if (state == 1) continue;
    const int m = *(volatile int*)&ctrl->m;    // 2 k
    const LejaCoef lc1 = S.a.lc[m], lc2 = S.a.lc[m + 1];
    PairCtx X;
    X.F = static_cast<const float*>(S.a.coef);
    X.yin = static_cast<const float*>(S.a.y[(m >> 1) & 1]);
    X.yout = static_cast<float*>(S.a.y[((m >> 1) + 1) & 1]);
    X.p = static_cast<float*>(S.a.p);
    X.ring = ring;
    X.stages = PairLayout::STAGES;
    X.G.nx = S.a.g.nx;
    X.G.ny = S.a.g.ny;
    X.G.bc = S.a.g.bc;
    X.G.n = S.a.g.n;
    X.G.lane = lane;
    X.ig = (float)(1.0 / S.a.gamma);
    X.sh1 = (float)(S.a.c / S.a.gamma + lc1.xi);
    X.sh2 = (float)(S.a.c / S.a.gamma + lc2.xi);
    X.d0 = m > 0 ? (float)S.a.lc[m - 1].d : 0.0f;
    X.d1 = (float)lc1.d;
    X.d2 = (float)lc2.d;
    X.abx = S.a.abx;
    X.aby = S.a.aby;
    const int local = tile - S.rt_off;
    const int X0 = (local % S.rt_x) * kPairOwn;
    X.y0 = (local / S.rt_x) * R;
    X.y1 = min(S.a.g.ny, X.y0 + R);
    X.L = pair_lane(X0, lane, X.G.nx, X.G.bc);
    X.gx = X0 - 4 + 4 * lane;
    X.fix = X.G.bc != 0 && (X0 == 0 || X0 + kPairOwn >= X.G.nx);
    float ly1 = 0.f, lp1 = 0.f, ly2 = 0.f, lp2 = 0.f;
    CpAsyncLoader ldr;
    if (MODE == 2) pair_run_pf<ADV, true>(X, ldr, ly1, lp1, ly2, lp2);
    else if (MODE == 1) pair_run_pf<ADV>(X, ldr, ly1, lp1, ly2, lp2);
    else pair_run<ADV>(X, ldr, ly1, lp1, ly2, lp2);
    double q[4] = {ly1, lp1, ly2, lp2};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) q[kk] += __shfl_down_sync(0xffffffffu, q[kk], o);
    int last = 0;
    if (lane == 0) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) tile_partials[4 * tile + kk] = q[kk];
      __threadfence();
      const unsigned int t = atomicAdd(&ctrl->ticket, 1u);
      last = (t == (unsigned int)S.rt_n - 1u) ? 1 : 0;
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (last) {                                // the slice's last tile of pass k: decide
      __threadfence();
      double t4[4] = {0.0, 0.0, 0.0, 0.0};
      // unrolled: the loads of several tiles in flight, the sums still in tile order
#pragma unroll 8
      for (int r = lane; r < S.rt_n; r += 32) {
        const double2* tp = reinterpret_cast<const double2*>(tile_partials) + 2 * (S.rt_off + r);
        const double2 v0 = __ldcg(tp), v1 = __ldcg(tp + 1);
        t4[0] += v0.x;
        t4[1] += v0.y;
        t4[2] += v1.x;
        t4[3] += v1.y;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) t4[kk] += __shfl_down_sync(0xffffffffu, t4[kk], o);
      if (lane == 0) {
        int stop = decide(ctrl, lc1, m, t4[0], t4[1]);
        if (stop) {
          ctrl->m = m + 1;                     // p is complete (no pending term)
        } else {
          stop = decide(ctrl, lc2, m + 1, t4[2], t4[3]);
          ctrl->m = m + 2;
        }
        if (*(volatile int*)&bs->abort) stop = 1;
        ctrl->ticket = 0u;
        __threadfence();                       // the pass's data and scalars before its flags
        if (stop) {
          *(volatile int*)&ctrl->stop = 1;
          atomicSub(&bs->active, 1);
          __threadfence();                     // stop before the pass count that reveals it
        }
        *(volatile unsigned int*)&ctrl->gen = (unsigned int)(k + 1);
        __threadfence();
      }
    }
  }
}

// Series start of every slice in one marching pass (the ring kernels'
// run with scale 1, shift 0 and p taken as 0): y_0 = A u + c0 g0 + c1 g1,
// p_0 = d0 y_0, over 128-column x TY-row units (the two halves of each
// streaming tile); block 0 resets every slice's control block as
// batch_init_k does.  SRC: some slice has sources (at most two per slice; a
// slice without points the coupling fields at its own u with coefficient 0,
// which the run skips).  Replaces batch_apply_k + batch_init_k in the ring
// and pair modes.
template <bool SRC, int ADV>
__global__ void __launch_bounds__(kRingThreads, 1)
    batch_start_k(const BatchSlice* slices, const int* tile_slice, int ntiles, int TY,
                  int nslices, int force, int max_iters, double tol, unsigned int* bticket) {
  extern __shared__ __align__(16) float ring_smem[];
  if (blockIdx.x == 0) {
    for (int s = threadIdx.x; s < nslices; s += blockDim.x) {
      Ctrl* c = slices[s].a.ctrl;
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
      c->gen = 0u;                // passes completed (persistent iteration)
    }
    if (threadIdx.x == 0) {
      BatchSync* bs = reinterpret_cast<BatchSync*>(bticket);
      bs->ticket = 0u;
      bs->active = nslices;
      bs->abort = 0;
      bs->next = 0ull;
    }
  }
  using L = RingLayout<SRC, ADV>;
  float* ring = ring_smem + (size_t)(threadIdx.x >> 5) * L::STAGES * L::SIZE;
  const int lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kRingWarps + (threadIdx.x >> 5);
  const int GW = gridDim.x * kRingWarps;
  for (int unit = gw; unit < 2 * ntiles; unit += GW) {
    const int t = unit >> 1;
    const BatchSlice& S = slices[tile_slice[t]];
    const int local = t - S.tile_off;
    const int x0 = (local % S.tiles_x) * kTileCols + (unit & 1) * kVecCols;
    if (x0 >= S.a.g.nx) continue;              // uniform over the warp
    const int y0 = (local / S.tiles_x) * TY, y1 = min(S.a.g.ny, y0 + TY);
    SeriesArgs b = S.a;
    b.w2 = S.nsrc > 0 ? S.src_g[0] : S.u;
    b.w1 = S.nsrc > 1 ? S.src_g[1] : S.u;
    const float c0 = S.nsrc > 0 ? S.src_c[0] : 0.0f, c1 = S.nsrc > 1 ? S.src_c[1] : 0.0f;
    VGeo G;
    G.nx = S.a.g.nx;
    G.ny = S.a.g.ny;
    G.bc = S.a.g.bc;
    G.n = S.a.g.n;
    G.lane = lane;
    G.x = x0 + 4 * lane;
    G.active = G.x < G.nx;
    float ly = 0.f, lp = 0.f;
    ring_run<SRC, ADV>(b, G, ring, y0, y1, S.u, static_cast<float*>(S.a.y[0]),
                       static_cast<float*>(S.a.p), 1.0f, 0.0f, (float)S.d0, c0, c1, ly, lp, true);
  }
}

template <bool SRC, int ADV>
size_t batch_start_smem() {
  return sizeof(float) * (size_t)kRingWarps * RingLayout<SRC, ADV>::STAGES *
         RingLayout<SRC, ADV>::SIZE;
}

void* pick_start(bool src, int adv) {
  if (src) return adv == 0 ? (void*)batch_start_k<true, 0>
                           : (adv == 1 ? (void*)batch_start_k<true, 1> : (void*)batch_start_k<true, 2>);
  return adv == 0 ? (void*)batch_start_k<false, 0>
                  : (adv == 1 ? (void*)batch_start_k<false, 1> : (void*)batch_start_k<false, 2>);
}

size_t start_smem_for(bool src, int adv) {
  if (src) return adv == 0 ? batch_start_smem<true, 0>()
                           : (adv == 1 ? batch_start_smem<true, 1>() : batch_start_smem<true, 2>());
  return adv == 0 ? batch_start_smem<false, 0>()
                  : (adv == 1 ? batch_start_smem<false, 1>() : batch_start_smem<false, 2>());
}

// The end of the step in one pass: a converged slice gets u += dt (p + the
// pending d_m y_m of an even pair-mode count: p is completed in registers,
// not written back); a slice that did not converge keeps its input state.
__global__ void __launch_bounds__(kThreads) batch_finish_k(const BatchSlice* slices,
                                                          const int* tile_slice, int ntiles,
                                                          int TY, int pair) {
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const BatchSlice& S = slices[tile_slice[t]];
    if (S.a.ctrl->status != 0) continue;      // not converged: keep the input state
    const GridDev g = S.a.g;
    const int local = t - S.tile_off;
    const int x0 = (local % S.tiles_x) * kTileCols, y0 = (local / S.tiles_x) * TY;
    const int i = x0 + threadIdx.x;
    if (i >= g.nx) continue;
    const int m = S.a.ctrl->m;
    const bool pending = pair && m > 0 && !(m & 1);
    const float d = pending ? (float)S.a.lc[m - 1].d : 0.0f;
    const float* y = static_cast<const float*>(S.a.y[(m >> 1) & 1]);
    const float* p = static_cast<const float*>(S.a.p);
    for (int j = y0; j < min(g.ny, y0 + TY); ++j) {
      const long long idx = (long long)j * g.nx + i;
      const float pv = pending ? fmaf(d, y[idx], p[idx]) : p[idx];
      S.u[idx] = fmaf(S.dt, pv, S.u[idx]);
    }
  }
}

// batch_finish_k with 16-byte accesses, for batches whose rows and vectors
// are 16-byte aligned (every nx % 4 == 0; the ring and pair modes with the
// one-pass start): a thread updates four columns of every fourth row of its
// tile, four rows in flight.  The same operations per element.
__global__ void __launch_bounds__(kThreads) batch_finish_vec_k(const BatchSlice* slices,
                                                              const int* tile_slice, int ntiles,
                                                              int TY, int pair) {
  const int cg = threadIdx.x & 63, rg = threadIdx.x >> 6;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const BatchSlice& S = slices[tile_slice[t]];
    if (S.a.ctrl->status != 0) continue;      // not converged: keep the input state
    const GridDev g = S.a.g;
    const int local = t - S.tile_off;
    const int x0 = (local % S.tiles_x) * kTileCols, y0 = (local / S.tiles_x) * TY;
    const int i = x0 + 4 * cg;
    if (i >= g.nx) continue;                  // nx % 4 == 0: the group is all inside
    const int m = S.a.ctrl->m;
    const bool pending = pair && m > 0 && !(m & 1);
    const float d = pending ? (float)S.a.lc[m - 1].d : 0.0f;
    const float* y = static_cast<const float*>(S.a.y[(m >> 1) & 1]);
    const float* p = static_cast<const float*>(S.a.p);
    const int y1 = min(g.ny, y0 + TY);
    const float dt = S.dt;
#pragma unroll 4
    for (int j = y0 + rg; j < y1; j += 4) {
      const long long idx = (long long)j * g.nx + i;
      float4 pv = *reinterpret_cast<const float4*>(p + idx);
      float4 uv = *reinterpret_cast<const float4*>(S.u + idx);
      if (pending) {
        const float4 yv = *reinterpret_cast<const float4*>(y + idx);
        pv.x = fmaf(d, yv.x, pv.x);
        pv.y = fmaf(d, yv.y, pv.y);
        pv.z = fmaf(d, yv.z, pv.z);
        pv.w = fmaf(d, yv.w, pv.w);
      }
      uv.x = fmaf(dt, pv.x, uv.x);
      uv.y = fmaf(dt, pv.y, uv.y);
      uv.z = fmaf(dt, pv.z, uv.z);
      uv.w = fmaf(dt, pv.w, uv.w);
      *reinterpret_cast<float4*>(S.u + idx) = uv;
    }
  }
}

size_t batch_pair_smem() {
  return sizeof(float) * (size_t)kRingWarps * PairLayout::STAGES * PairLayout::SIZE;
}

void* pick_pair(int adv, int march) {
  static void* const fn[3][2] = {{(void*)batch_pair_k<0, 0>, (void*)batch_pair_k<1, 0>},
                                 {(void*)batch_pair_k<0, 1>, (void*)batch_pair_k<1, 1>},
                                 {(void*)batch_pair_k<0, 2>, (void*)batch_pair_k<1, 2>}};
  return fn[march][adv == 0 ? 0 : 1];
}

template <int ADV>
size_t batch_ring_smem() {
  return sizeof(float) * (size_t)kRingWarps * RingLayout<false, ADV>::STAGES *
         RingLayout<false, ADV>::SIZE;
}

void* pick_ring(int adv) {
  return adv == 0 ? (void*)batch_ring_k<0> : (adv == 1 ? (void*)batch_ring_k<1> : (void*)batch_ring_k<2>);
}

size_t ring_smem_for(int adv) {
  return adv == 0 ? batch_ring_smem<0>() : (adv == 1 ? batch_ring_smem<1>() : batch_ring_smem<2>());
}

using IterFn = void (*)(const BatchSlice*, const int*, int, int, double*, unsigned int*,
                        unsigned long long, int);

template <int ADV>
IterFn iter_fn(int TY) {
  switch (TY) {
    case 8: return batch_iter_k<ADV, 8>;
    case 16: return batch_iter_k<ADV, 16>;
    case 32: return batch_iter_k<ADV, 32>;
    default: return batch_iter_k<ADV, 64>;
  }
}

IterFn pick_iter(int adv, int TY) {
  return adv == 0 ? iter_fn<0>(TY) : (adv == 1 ? iter_fn<1>(TY) : iter_fn<2>(TY));
}

void* pick_apply(int adv) {
  return adv == 0 ? (void*)batch_apply_k<0> : (adv == 1 ? (void*)batch_apply_k<1> : (void*)batch_apply_k<2>);
}

}  // namespace
}  // namespace ad

using namespace ad;

struct ad_batch {
  std::vector<ad_operator*> ops;
  int S = 0;
  int adv = 0;
  cudaStream_t stream = nullptr;
  int TY = 32;
  int nblocks = 608;
  double tuned_ms = 0.0;
  bool ring = false;                  // warp-tile ring iteration (every nx % 4 == 0)
  bool pair = false;                  // ... two iterations per launch (see batch_pair_k)
  int R = 64;                         // rows per warp tile
  int* d_rtile_slice = nullptr;
  int nrtiles = 0;
  double* d_rpartials = nullptr;
  std::vector<BatchSlice> hs;
  BatchSlice* d_slices = nullptr;
  int* d_tile_slice = nullptr;
  int ntiles = 0;
  double* d_partials = nullptr;
  LejaCoef* d_lc = nullptr;
  Ctrl* d_ctrl = nullptr;
  unsigned int* d_bticket = nullptr;
  std::vector<LejaCoef> h_lc;
  std::vector<double> lc_dt, lc_alpha;
  std::vector<Ctrl> h_ctrl;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  int graph_force = -2;
  double graph_tol = -1.0;
  int graph_start = -1;               // start_mode the graph was built with
  bool persist = false;               // the graph runs the persistent iteration kernel
  bool persist_off = false;           // the persistent kernel could not be built here
  int march = 1;                      // marching of the two-iteration kernels (pair_march)
  // vectors and sources bound by ad_batch_bind (caller memory), for ad_batch_step
  std::vector<void*> bound_u;
  std::vector<ad_source> bound_src;
  std::vector<std::vector<const void*>> bound_g;
  bool bound_has_src = false;
  // Queue order of the slices' warp tiles (empty: slice order): slices expected
  // to iterate longest first, from ad_batch_iteration_hint and then from the
  // counts of each step; order_dirty asks the next step to rebuild the list.
  std::vector<int> order;
  bool order_dirty = false;
};

namespace {

int bfail(int code, const std::string& m) {
  set_error_message(m.c_str());
  return code;
}

#define B_CUDA(expr)                                                                     \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      cudaGetLastError();                                                                \
      return bfail(AD_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));     \
    }                                                                                    \
  } while (0)

// Tile table for tile height TY: slice s owns tiles [off_s, off_s + n_s).
void build_tiles(ad_batch* b, int TY, std::vector<int>& tile_slice) {
  tile_slice.clear();
  for (int s = 0; s < b->S; ++s) {
    BatchSlice& hs = b->hs[s];
    const int tx = (hs.a.g.nx + kTileCols - 1) / kTileCols;
    const int ty = (hs.a.g.ny + TY - 1) / TY;
    hs.tiles_x = tx;
    hs.ntiles = tx * ty;
    hs.tile_off = (int)tile_slice.size();
    for (int k = 0; k < hs.ntiles; ++k) tile_slice.push_back(s);
  }
}

int upload_tiles(ad_batch* b, int TY) {
  std::vector<int> ts;
  build_tiles(b, TY, ts);
  if ((int)ts.size() > b->ntiles) {
    if (b->d_tile_slice) cudaFree(b->d_tile_slice);
    if (b->d_partials) cudaFree(b->d_partials);
    b->d_tile_slice = nullptr;
    b->d_partials = nullptr;
    B_CUDA(cudaMalloc(&b->d_tile_slice, sizeof(int) * ts.size()));
    B_CUDA(cudaMalloc(&b->d_partials, sizeof(double) * 2 * ts.size()));
  }
  b->ntiles = (int)ts.size();
  b->TY = TY;
  B_CUDA(cudaMemcpyAsync(b->d_tile_slice, ts.data(), sizeof(int) * ts.size(),
                         cudaMemcpyHostToDevice, b->stream));
  B_CUDA(cudaMemcpyAsync(b->d_slices, b->hs.data(), sizeof(BatchSlice) * b->S,
                         cudaMemcpyHostToDevice, b->stream));
  B_CUDA(cudaStreamSynchronize(b->stream));
  return AD_OK;
}

// Warp-tile table for rows per tile R: slice s owns ring tiles [rt_off, rt_off + rt_n).
int upload_ring_tiles(ad_batch* b, int R, bool sync = true) {
  std::vector<int> ts;
  for (int q = 0; q < b->S; ++q) {
    const int s = b->order.empty() ? q : b->order[q];
    BatchSlice& hs = b->hs[s];
    const int cols = b->pair ? kPairOwn : kVecCols;
    hs.rt_x = (hs.a.g.nx + cols - 1) / cols;
    hs.rt_n = hs.rt_x * ((hs.a.g.ny + R - 1) / R);
    hs.rt_off = (int)ts.size();
    for (int k = 0; k < hs.rt_n; ++k) ts.push_back(s);
  }
  if ((int)ts.size() > b->nrtiles || !b->d_rtile_slice) {
    if (b->d_rtile_slice) cudaFree(b->d_rtile_slice);
    if (b->d_rpartials) cudaFree(b->d_rpartials);
    b->d_rtile_slice = nullptr;
    b->d_rpartials = nullptr;
    B_CUDA(cudaMalloc(&b->d_rtile_slice, sizeof(int) * ts.size()));
    B_CUDA(cudaMalloc(&b->d_rpartials, sizeof(double) * 4 * ts.size()));
  }
  b->nrtiles = (int)ts.size();
  b->R = R;
  B_CUDA(cudaMemcpyAsync(b->d_rtile_slice, ts.data(), sizeof(int) * ts.size(),
                         cudaMemcpyHostToDevice, b->stream));
  B_CUDA(cudaMemcpyAsync(b->d_slices, b->hs.data(), sizeof(BatchSlice) * b->S,
                         cudaMemcpyHostToDevice, b->stream));
  if (sync) B_CUDA(cudaStreamSynchronize(b->stream));
  return AD_OK;
}

// Queue the slices' warp tiles by decreasing expected iteration count (ties in
// slice order).  In every pass the series that run longest are then handed
// out first, so their next pass is not held behind the tiles of slices that
// stop earlier; the tile sums of each slice keep their order, so results do
// not depend on the queue order.
void order_by_iterations(ad_batch* b, const double* iters) {
  std::vector<int> o(b->S);
  for (int s = 0; s < b->S; ++s) o[s] = s;
  if (iters)
    std::stable_sort(o.begin(), o.end(), [&](int x, int y) { return iters[x] > iters[y]; });
  if (o != b->order) {
    b->order = o;
    b->order_dirty = true;
  }
}

bool order_auto() {
  static const bool on = [] {
    const char* e = getenv("AD_BATCH_ORDER");         // tuning override: 0 keeps slice order
    return !(e && e[0] == '0');
  }();
  return on;
}

int ring_grid(const ad_batch* b) { return std::max(1, std::min(152, (b->nrtiles + 7) / 8)); }

void* pick_persist(int adv, int march) {
  static void* const fn[3][2] = {{(void*)batch_persist_k<0, 0>, (void*)batch_persist_k<1, 0>},
                                 {(void*)batch_persist_k<0, 1>, (void*)batch_persist_k<1, 1>},
                                 {(void*)batch_persist_k<0, 2>, (void*)batch_persist_k<1, 2>}};
  return fn[march][adv == 0 ? 0 : 1];
}

// Blocks of the persistent iteration kernel: one per SM when a block fits on
// every SM at once (co-residency of all blocks is what its waits rely on);
// 0 to keep the graph loop (also with AD_BATCH_PERSIST=0).
int persist_grid(const ad_batch* b) {
  static const bool off = [] {
    const char* e = getenv("AD_BATCH_PERSIST");
    return e && e[0] == '0';
  }();
  if (off || !b->pair || b->persist_off) return 0;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  for (int march = 0; march <= 2; ++march) {    // every marching a batch may run
    void* fn = pick_persist(b->adv, march);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)batch_pair_smem()) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kRingThreads,
                                                      batch_pair_smem()) != cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      return 0;
    }
  }
  return sms;
}

void destroy_batch_graph(ad_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// start_mode: 0 apply + init kernels, 1 batch_start_k without sources, 2 with.
int build_batch_graph(ad_batch* b, int force, double tol, int start_mode) {
  destroy_batch_graph(b);
  cudaGraph_t g;
  B_CUDA(cudaGraphCreate(&g, 0));
  b->graph = g;
  // the two-iteration passes as ONE persistent cooperative launch (one block
  // per SM, every block resident) instead of the graph loop
  const int pgrid = persist_grid(b);
  b->persist = b->pair && start_mode > 0 && pgrid > 0;
  cudaGraphConditionalHandle h{};
  if (!b->persist) B_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  int TY = b->TY, nt = b->ntiles, S = b->S, maxit = kMaxIters;
  const BatchSlice* sl = b->d_slices;
  const int* ts = b->d_tile_slice;
  unsigned int* bt = b->d_bticket;
  double* parts = b->d_partials;
  unsigned long long hv = (unsigned long long)h;
  int one = 1;
  const int grid = std::min(nt, b->nblocks);
  cudaKernelNodeParams kp = {};
  kp.blockDim = dim3(kThreads);
  kp.gridDim = dim3(grid);
  cudaGraphNode_t n_apply, n_init, n_cond, n_upd;
  if (start_mode > 0) {   // the series start in one ring pass (batch_start_k)
    void* args[] = {&sl, &ts, &nt, &TY, &S, &force, &maxit, &tol, &bt};
    cudaKernelNodeParams sp = kp;
    sp.func = pick_start(start_mode == 2, b->adv);
    sp.kernelParams = args;
    sp.blockDim = dim3(kRingThreads);
    sp.gridDim = dim3(std::max(1, std::min(152, (2 * nt + kRingWarps - 1) / kRingWarps)));
    sp.sharedMemBytes = (unsigned)start_smem_for(start_mode == 2, b->adv);
    B_CUDA(cudaGraphAddKernelNode(&n_init, g, nullptr, 0, &sp));
  } else {
    {
      void* args[] = {&sl, &ts, &nt, &TY};
      kp.func = pick_apply(b->adv);
      kp.kernelParams = args;
      B_CUDA(cudaGraphAddKernelNode(&n_apply, g, nullptr, 0, &kp));
    }
    {
      void* args[] = {&sl, &ts, &nt, &TY, &S, &force, &maxit, &tol, &bt};
      kp.func = (void*)batch_init_k;
      kp.kernelParams = args;
      B_CUDA(cudaGraphAddKernelNode(&n_init, g, &n_apply, 1, &kp));
    }
  }
  const int* rts = b->d_rtile_slice;
  int nrt = b->nrtiles, R = b->R;
  double* rparts = b->d_rpartials;
  if (b->persist) {
    void* pargs[] = {&sl, &rts, &nrt, &S, &R, &rparts, &bt};
    cudaKernelNodeParams pp = kp;
    pp.func = pick_persist(b->adv, b->march);
    pp.kernelParams = pargs;
    pp.blockDim = dim3(kRingThreads);
    pp.gridDim = dim3(pgrid);
    pp.sharedMemBytes = (unsigned)batch_pair_smem();
    B_CUDA(cudaGraphAddKernelNode(&n_cond, g, &n_init, 1, &pp));
    cudaKernelNodeAttrValue coop{};
    coop.cooperative = 1;
    if (cudaGraphKernelNodeSetAttribute(n_cond, cudaKernelNodeAttributeCooperative, &coop) !=
        cudaSuccess) {             // no cooperative graph nodes here: build the graph loop
      cudaGetLastError();
      b->persist_off = true;
      return build_batch_graph(b, force, tol, start_mode);
    }
  } else {
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  B_CUDA(cudaGraphAddNode(&n_cond, g, &n_init, nullptr, 1, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  {
    void* args[] = {&sl, &ts, &nt, &S, &parts, &bt, &hv, &one};
    void* rargs[] = {&sl, &rts, &nrt, &S, &R, &rparts, &bt, &hv, &one};
    cudaKernelNodeParams ip = kp;
    if (b->ring) {
      ip.func = b->pair ? pick_pair(b->adv, b->march) : pick_ring(b->adv);
      ip.kernelParams = rargs;
      ip.blockDim = dim3(kRingThreads);
      ip.gridDim = dim3(ring_grid(b));
      ip.sharedMemBytes = (unsigned)(b->pair ? batch_pair_smem() : ring_smem_for(b->adv));
    } else {
      ip.func = (void*)pick_iter(b->adv, TY);
      ip.kernelParams = args;
    }
    cudaGraphNode_t prev = nullptr;
    for (int u = 0; u < kBatchUnroll; ++u) {
      cudaGraphNode_t nn;
      B_CUDA(cudaGraphAddKernelNode(&nn, body, prev ? &prev : nullptr, prev ? 1 : 0, &ip));
      prev = nn;
    }
  }
  }
  {   // u += dt (p + the pending term of even pair-mode counts)
    int pr = b->pair ? 1 : 0;
    void* args[] = {&sl, &ts, &nt, &TY, &pr};
    // the one-pass start certifies 16-byte aligned rows and vectors
    kp.func = start_mode > 0 ? (void*)batch_finish_vec_k : (void*)batch_finish_k;
    kp.kernelParams = args;
    B_CUDA(cudaGraphAddKernelNode(&n_upd, g, &n_cond, 1, &kp));
  }
  if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
    cudaGetLastError();
    if (!b->persist) return bfail(AD_ERR_CUDA, "cudaGraphInstantiate failed");
    b->persist_off = true;         // the cooperative node was refused: build the graph loop
    return build_batch_graph(b, force, tol, start_mode);
  }
  b->graph_force = force;
  b->graph_tol = tol;
  b->graph_start = start_mode;
  return AD_OK;
}

// --------------------------------------------------------------- autotune cache
std::string cache_path() {
  if (const char* e = getenv("AD_AUTOTUNE_CACHE")) return e;
  Dl_info info;
  if (dladdr((void*)&cache_path, &info) && info.dli_fname) {
    std::string f = info.dli_fname;
    const size_t k = f.rfind('/');
    return (k == std::string::npos ? std::string(".") : f.substr(0, k)) + "/autotune_cache.json";
  }
  return "autotune_cache.json";
}

struct TuneEntry {
  int ty, bps;
  double ms;
  int march;       // marching of the two-iteration kernels (1 where not tuned)
};

// The cache is a JSON object with one entry per line:
//   "key": {"ty": 16, "bps": 4, "ms": 0.1234, "march": 1},
std::map<std::string, TuneEntry> read_cache() {
  std::map<std::string, TuneEntry> m;
  FILE* f = fopen(cache_path().c_str(), "r");
  if (!f) return m;
  char line[1024];
  while (fgets(line, sizeof line, f)) {
    char key[512];
    TuneEntry e{};
    e.march = 1;
    const int got = sscanf(line, " \"%511[^\"]\": {\"ty\": %d, \"bps\": %d, \"ms\": %lf, \"march\": %d",
                           key, &e.ty, &e.bps, &e.ms, &e.march);
    if (got >= 4 && e.march >= 0 && e.march <= 2) m[key] = e;
  }
  fclose(f);
  return m;
}

void write_cache(const std::map<std::string, TuneEntry>& m) {
  const std::string path = cache_path();
  const std::string tmp = path + ".tmp";
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return;
  fprintf(f, "{\n");
  size_t k = 0;
  for (const auto& kv : m) {
    fprintf(f, "  \"%s\": {\"ty\": %d, \"bps\": %d, \"ms\": %.6f, \"march\": %d}%s\n",
            kv.first.c_str(), kv.second.ty, kv.second.bps, kv.second.ms, kv.second.march,
            (++k < m.size()) ? "," : "");
  }
  fprintf(f, "}\n");
  fclose(f);
  rename(tmp.c_str(), path.c_str());
}

std::string tune_key(const ad_batch* b) {
  std::map<std::pair<int, int>, int> sizes;
  for (const auto& s : b->hs) sizes[{s.a.g.nx, s.a.g.ny}]++;
  // the pair mode is tuned on the persistent kernel where that runs
  std::string k = std::string(b->pair ? (persist_grid(b) > 0 ? "persist" : "pair")
                                      : (b->ring ? "ring" : "tile")) + "-f32-adv" +
                  std::to_string(b->adv) +
                  "-S" + std::to_string(b->S);
  if (b->pair && pair_march_env() >= 0)       // a marching fixed by AD_F32_MARCH is not tuned
    k += "-march" + std::to_string(pair_march_env());
  for (const auto& kv : sizes)
    k += "-" + std::to_string(kv.first.first) + "x" + std::to_string(kv.first.second) + "*" +
         std::to_string(kv.second);
  return k;
}

// Time `reps` forced iterations of the ring kernel for R rows per warp tile.
int time_ring(ad_batch* b, int R, int reps, double* ms_out) {
  {
    const int r = upload_ring_tiles(b, R);
    if (r != AD_OK) return r;
  }
  int force = b->pair ? 2 * reps : reps, maxit = kMaxIters;
  double tol = 0.0;
  const int sgrid = std::min(b->ntiles, b->nblocks);
  batch_init_k<<<sgrid, kThreads, 0, b->stream>>>(b->d_slices, b->d_tile_slice, b->ntiles, b->TY,
                                                  b->S, force, maxit, tol, b->d_bticket);
  void* fn = b->pair ? pick_pair(b->adv, b->march) : pick_ring(b->adv);
  const size_t smem = b->pair ? batch_pair_smem() : ring_smem_for(b->adv);
  const int grid = ring_grid(b);
  cudaEvent_t e0, e1;
  B_CUDA(cudaEventCreate(&e0));
  B_CUDA(cudaEventCreate(&e1));
  B_CUDA(cudaEventRecord(e0, b->stream));
  const BatchSlice* sl = b->d_slices;
  const int* rts = b->d_rtile_slice;
  int nrt = b->nrtiles, S = b->S, zero = 0;
  double* rparts = b->d_rpartials;
  unsigned int* bt = b->d_bticket;
  unsigned long long hv = 0ULL;
  void* args[] = {&sl, &rts, &nrt, &S, &R, &rparts, &bt, &hv, &zero};
  for (int r = 0; r < reps; ++r)
    B_CUDA(cudaLaunchKernel(fn, dim3(grid), dim3(kRingThreads), args, smem, b->stream));
  B_CUDA(cudaEventRecord(e1, b->stream));
  B_CUDA(cudaStreamSynchronize(b->stream));
  float ms = 0.f;
  B_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_out = ms / reps;
  return AD_OK;
}

// Time `reps` forced two-iteration passes of the persistent series kernel
// (one cooperative launch, every slice active in every pass) for R rows per
// warp tile.
int time_persist(ad_batch* b, int R, int reps, int grid, double* ms_out) {
  {
    const int r = upload_ring_tiles(b, R);
    if (r != AD_OK) return r;
  }
  int force = 2 * reps, maxit = kMaxIters;
  double tol = 0.0;
  const int sgrid = std::min(b->ntiles, b->nblocks);
  batch_init_k<<<sgrid, kThreads, 0, b->stream>>>(b->d_slices, b->d_tile_slice, b->ntiles, b->TY,
                                                  b->S, force, maxit, tol, b->d_bticket);
  cudaEvent_t e0, e1;
  B_CUDA(cudaEventCreate(&e0));
  B_CUDA(cudaEventCreate(&e1));
  const BatchSlice* sl = b->d_slices;
  const int* rts = b->d_rtile_slice;
  int nrt = b->nrtiles, S = b->S;
  double* rparts = b->d_rpartials;
  unsigned int* bt = b->d_bticket;
  void* args[] = {&sl, &rts, &nrt, &S, &R, &rparts, &bt};
  B_CUDA(cudaEventRecord(e0, b->stream));
  const cudaError_t le = cudaLaunchCooperativeKernel(pick_persist(b->adv, b->march), dim3(grid),
                                                     dim3(kRingThreads), args,
                                                     batch_pair_smem(), b->stream);
  B_CUDA(cudaEventRecord(e1, b->stream));
  const cudaError_t se = cudaStreamSynchronize(b->stream);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (le != cudaSuccess || se != cudaSuccess) {
    cudaGetLastError();
    return bfail(AD_ERR_CUDA, "persistent series kernel failed in the autotuner");
  }
  *ms_out = ms / reps;
  return AD_OK;
}

// Time `reps` forced iterations of the batched kernel for one (TY, blocks).
int time_config(ad_batch* b, int TY, int nblocks, int reps, double* ms_out) {
  {
    const int r = upload_tiles(b, TY);
    if (r != AD_OK) return r;
  }
  const int grid = std::min(b->ntiles, nblocks);
  int force = reps, maxit = kMaxIters;
  double tol = 0.0;
  batch_init_k<<<grid, kThreads, 0, b->stream>>>(b->d_slices, b->d_tile_slice, b->ntiles, TY, b->S,
                                                 force, maxit, tol, b->d_bticket);
  IterFn fn = pick_iter(b->adv, TY);
  cudaEvent_t e0, e1;
  B_CUDA(cudaEventCreate(&e0));
  B_CUDA(cudaEventCreate(&e1));
  B_CUDA(cudaEventRecord(e0, b->stream));
  for (int r = 0; r < reps; ++r)
    fn<<<grid, kThreads, 0, b->stream>>>(b->d_slices, b->d_tile_slice, b->ntiles, b->S,
                                         b->d_partials, b->d_bticket, 0ULL, 0);
  B_CUDA(cudaEventRecord(e1, b->stream));
  B_CUDA(cudaStreamSynchronize(b->stream));
  float ms = 0.f;
  B_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_out = ms / reps;
  return AD_OK;
}

}  // namespace

extern "C" {

int ad_create_batch(ad_operator* const* ops, int nslices, int autotune, ad_batch** out) {
  set_error_message("");
  if (!out || !ops || nslices < 1) return bfail(AD_ERR_INVALID, "ops/out NULL or nslices < 1");
  *out = nullptr;
  ad_batch* b = new ad_batch();
  b->S = nslices;
  b->hs.resize(nslices);
  for (int s = 0; s < nslices; ++s) {
    OperatorView v;
    if (!ops[s] || !operator_view(ops[s], &v)) {
      delete b;
      return bfail(AD_ERR_INVALID, "NULL operator in the batch");
    }
    if (v.prec != 1) {
      delete b;
      return bfail(AD_ERR_INVALID, "batched steps need AD_FP32_STORAGE operators");
    }
    if (s == 0) {
      b->adv = v.adv;
      b->stream = v.stream;
    } else if (v.adv != b->adv || v.stream != b->stream) {
      delete b;
      return bfail(AD_ERR_INVALID, "batch slices must share the advection mode and the stream");
    }
    b->ops.push_back(ops[s]);
    BatchSlice& hs = b->hs[s];
    hs = BatchSlice{};
    hs.a.g = v.g;
    hs.a.prec = 1;
    hs.a.coef = v.coef;
    hs.a.y[0] = v.y0;
    hs.a.y[1] = v.y1;
    hs.a.p = v.p;
    hs.a.w1 = v.w1;
    hs.a.adv = v.adv;
    hs.a.abx = v.abx;
    hs.a.aby = v.aby;
    hs.a.c = v.c;
    hs.a.gamma = v.gamma;
    // the autotuner iterates on whatever the workspace holds: start from zeros
    cudaMemsetAsync(v.w1, 0, sizeof(float) * (size_t)v.g.n, v.stream);
  }
  bool ok = cudaMalloc(&b->d_slices, sizeof(BatchSlice) * nslices) == cudaSuccess &&
            cudaMalloc(&b->d_lc, sizeof(LejaCoef) * kMaxIters * nslices) == cudaSuccess &&
            cudaMalloc(&b->d_ctrl, sizeof(Ctrl) * nslices) == cudaSuccess &&
            cudaMalloc(&b->d_bticket, sizeof(BatchSync)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    ad_destroy_batch(b);
    return bfail(AD_ERR_NOMEM, "batch allocation failed");
  }
  cudaMemsetAsync(b->d_ctrl, 0, sizeof(Ctrl) * nslices, b->stream);
  cudaMemsetAsync(b->d_bticket, 0, sizeof(BatchSync), b->stream);
  for (int s = 0; s < nslices; ++s) {
    b->hs[s].a.lc = b->d_lc + (size_t)s * kMaxIters;
    b->hs[s].a.ctrl = b->d_ctrl + s;
  }
  b->h_lc.resize((size_t)kMaxIters * nslices);
  b->lc_dt.assign(nslices, -1.0);
  b->lc_alpha.assign(nslices, 0.0);
  b->h_ctrl.resize(nslices);
  // iteration kernel: warp-tile rings when every slice's rows are 16-byte aligned
  {
    static const bool tile_only = [] {
      const char* e = getenv("AD_BATCH_KERNEL");         // tuning override: ring | tile
      return e && e[0] == 't';
    }();
    bool aligned = true;
    for (const auto& hs : b->hs) aligned = aligned && hs.a.g.nx % 4 == 0;
    b->ring = aligned && !tile_only;
    static const bool no_pair = [] {
      const char* e = getenv("AD_F32_PAIR");             // tuning override: 0 = one iteration
      return e && e[0] == '0';
    }();
    bool rows2 = true;
    for (const auto& hs : b->hs) rows2 = rows2 && hs.a.g.ny >= 2;
    b->pair = b->ring && b->adv <= 1 && rows2 && !no_pair;
    if (b->ring) {
      static bool attr = false;
      if (!attr) {
        for (int adv = 0; adv < 3; ++adv)
          cudaFuncSetAttribute(pick_ring(adv), cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)ring_smem_for(adv));
        for (int adv = 0; adv < 2; ++adv)
          for (int march = 0; march <= 2; ++march)
            cudaFuncSetAttribute(pick_pair(adv, march),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)batch_pair_smem());
        for (int src = 0; src < 2; ++src)
          for (int adv = 0; adv < 3; ++adv)
            cudaFuncSetAttribute(pick_start(src != 0, adv),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)start_smem_for(src != 0, adv));
        attr = true;
      }
    }
  }
  // tile shape: cached autotune result, a fresh autotune, or the default
  int TY = 32, bps = 4, march = pair_march();
  double tuned = 0.0;
  const std::string key = tune_key(b);
  auto cache = read_cache();
  auto it = cache.find(key);
  static const int rows_override = [] {
    const char* e = getenv("AD_BATCH_ROWS");          // tuning override: rows per warp tile
    const int v = e ? atoi(e) : 0;
    return (v == 16 || v == 32 || v == 64 || v == 128) ? v : 0;
  }();
  if (rows_override && b->ring) {
    TY = rows_override;
    bps = 1;
  } else if (it != cache.end()) {
    TY = it->second.ty;
    bps = it->second.bps;
    tuned = it->second.ms;
    if (pair_march_env() < 0) march = it->second.march;
  } else if (autotune && b->ring) {
    // streaming kernels keep 256 x 32 tiles; tune the rows per warp tile
    {
      const int r = upload_tiles(b, 32);
      if (r != AD_OK) {
        std::string msg = ad_last_error();
        ad_destroy_batch(b);
        return bfail(r, msg);
      }
    }
    double best = 1e30;
    // The persistent series kernel (pair mode) is tuned on itself, over the
    // rows per warp tile and the marching of its two stencil levels (scalar
    // or packed FP32 pairs, unless AD_F32_MARCH fixes it).  Its adaptive
    // steps end with passes over few slices, where small tiles spread the
    // work over more warps: it takes the smallest R whose full pass is within
    // 10 % of the fastest (on the 128-slice workload R = 64: 7.96 ms per step
    // against 8.39 ms with the fastest full pass, R = 128).
    const int pgrid = b->pair ? persist_grid(b) : 0;
    const bool tune_march = pgrid > 0 && pair_march_env() < 0;
    double tr[4] = {0.0, 0.0, 0.0, 0.0};
    int tm[4] = {march, march, march, march};
    const int rows[4] = {16, 32, 64, 128};
    for (int q = 0; q < 4; ++q) {
      tr[q] = 1e30;
      for (int m = tune_march ? 1 : march; m <= (tune_march ? 2 : march); ++m) {
        b->march = m;
        double ms = 0.0;
        const int r = pgrid > 0 ? time_persist(b, rows[q], 6, pgrid, &ms)
                                : time_ring(b, rows[q], 6, &ms);
        if (r != AD_OK) {
          std::string msg = ad_last_error();
          ad_destroy_batch(b);
          return bfail(r, msg);
        }
        if (ms < tr[q]) { tr[q] = ms; tm[q] = m; }
      }
      if (tr[q] < best) { best = tr[q]; TY = rows[q]; march = tm[q]; }
    }
    if (pgrid > 0)
      for (int q = 0; q < 4; ++q)
        if (tr[q] <= 1.1 * best) { TY = rows[q]; best = tr[q]; march = tm[q]; break; }
    bps = 1;
    tuned = best;
    cache[key] = TuneEntry{TY, bps, best, march};
    write_cache(cache);
  } else if (autotune) {
    double best = 1e30;
    for (int ty : {8, 16, 32, 64})
      for (int bp : {2, 3, 4}) {
        double ms = 0.0;
        const int r = time_config(b, ty, 152 * bp, 6, &ms);
        if (r != AD_OK) {
          std::string msg = ad_last_error();
          ad_destroy_batch(b);
          return bfail(r, msg);
        }
        if (ms < best) { best = ms; TY = ty; bps = bp; }
      }
    tuned = best;
    cache[key] = TuneEntry{TY, bps, best, march};
    write_cache(cache);
  }
  b->tuned_ms = tuned;
  b->march = march;
  int r;
  if (b->ring) {
    b->nblocks = 152 * 4;                 // streaming kernels: 4 blocks of 256 per SM
    r = upload_tiles(b, 32);
    if (r == AD_OK) r = upload_ring_tiles(b, TY);
  } else {
    b->nblocks = 152 * bps;
    r = upload_tiles(b, TY);
  }
  if (r != AD_OK) {
    std::string msg = ad_last_error();
    ad_destroy_batch(b);
    return bfail(r, msg);
  }
  *out = b;
  return AD_OK;
}

int ad_destroy_batch(ad_batch* b) {
  if (!b) return AD_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  destroy_batch_graph(b);
  for (void* p : {(void*)b->d_slices, (void*)b->d_tile_slice, (void*)b->d_partials, (void*)b->d_lc,
                  (void*)b->d_ctrl, (void*)b->d_bticket, (void*)b->d_rtile_slice,
                  (void*)b->d_rpartials})
    if (p) cudaFree(p);
  delete b;
  return AD_OK;
}

int ad_batch_info(const ad_batch* b, int* tile_rows, int* blocks, int* ntiles, double* tuned_ms,
                  int* marching) {
  if (!b) return bfail(AD_ERR_INVALID, "NULL batch");
  if (tile_rows) *tile_rows = b->ring ? b->R : b->TY;
  if (blocks) *blocks = b->ring ? ring_grid(b) : std::min(b->ntiles, b->nblocks);
  if (ntiles) *ntiles = b->ring ? b->nrtiles : b->ntiles;
  if (tuned_ms) *tuned_ms = b->tuned_ms;
  if (marching) *marching = b->march;
  return AD_OK;
}

int ad_batch_iteration_hint(ad_batch* b, const double* iters) {
  set_error_message("");
  if (!b) return bfail(AD_ERR_INVALID, "NULL batch");
  if (iters)
    for (int s = 0; s < b->S; ++s)
      if (!std::isfinite(iters[s])) return bfail(AD_ERR_INVALID, "iteration hints must be finite");
  order_by_iterations(b, iters);
  return AD_OK;
}

int ad_batch_order(const ad_batch* b, int* order) {
  set_error_message("");
  if (!b || !order) return bfail(AD_ERR_INVALID, "NULL argument");
  for (int q = 0; q < b->S; ++q) order[q] = b->order.empty() ? q : b->order[q];
  return AD_OK;
}

int ad_batch_midpoint_step(ad_batch* b, void* const* u, double t, double dt,
                           const ad_source* src, double tol, int force_iters,
                           ad_stats* per_slice) {
  set_error_message("");
  if (!b || !u) return bfail(AD_ERR_INVALID, "NULL argument");
  if (!(dt > 0) || !std::isfinite(dt) || !std::isfinite(t)) return bfail(AD_ERR_INVALID, "bad t or dt");
  if (force_iters < 0 && !(tol > 0)) return bfail(AD_ERR_INVALID, "tol must be positive");
  if (force_iters > kMaxIters) return bfail(AD_ERR_INVALID, "force_iters > 500");
  const std::vector<double>& xi = leja_points();
  const long long l0 = launch_counter();
  bool lc_dirty = false;
  for (int s = 0; s < b->S; ++s) {
    OperatorView v;
    operator_view(b->ops[s], &v);
    BatchSlice& hs = b->hs[s];
    if (!u[s]) return bfail(AD_ERR_INVALID, "u[s] is NULL");
    hs.u = static_cast<float*>(u[s]);
    hs.a.c = v.c;
    hs.a.gamma = v.gamma;
    hs.dt = (float)dt;
    if (v.gamma * dt > v.rho_max)
      return bfail(AD_ERR_INVALID, "batched steps need gamma*dt <= rho_max for every slice "
                                   "(one substep); reduce dt or raise rho_max");
    hs.nsrc = 0;
    if (src) {
      const ad_source& q = src[s];
      if (q.nterms < 0 || q.nterms > kBatchSources)
        return bfail(AD_ERR_INVALID, "batched sources: at most 4 terms per slice");
      hs.nsrc = q.nterms;
      for (int k = 0; k < q.nterms; ++k) {
        hs.src_g[k] = static_cast<const float*>(q.g[k]);
        hs.src_c[k] = (float)(q.h ? q.h(k, t + 0.5 * dt, q.ctx) : 1.0);
      }
    }
    if (b->lc_dt[s] != dt || b->lc_alpha[s] != v.alpha) {
      double f[kMaxIters + 1], d[kMaxIters + 1];
      for (int m = 0; m <= kMaxIters; ++m) f[m] = phi1((v.c + v.gamma * xi[m]) * dt);
      divided_differences(xi.data(), f, kMaxIters + 1, d);
      for (int m = 0; m < kMaxIters; ++m)
        b->h_lc[(size_t)s * kMaxIters + m] =
            LejaCoef{xi[m], d[m + 1], std::fabs(d[m + 1]), 0.0, 0.0, {0.0, 0.0, 0.0}};
      hs.d0 = d[0];
      b->lc_dt[s] = dt;
      b->lc_alpha[s] = v.alpha;
      lc_dirty = true;
    }
  }
  if (b->ring && b->order_dirty) {         // a new queue order of the warp tiles
    const int r = upload_ring_tiles(b, b->R, false);
    if (r != AD_OK) return r;
    b->order_dirty = false;
  }
  if (lc_dirty)
    B_CUDA(cudaMemcpyAsync(b->d_lc, b->h_lc.data(), sizeof(LejaCoef) * b->h_lc.size(),
                           cudaMemcpyHostToDevice, b->stream));
  B_CUDA(cudaMemcpyAsync(b->d_slices, b->hs.data(), sizeof(BatchSlice) * b->S,
                         cudaMemcpyHostToDevice, b->stream));
  const int force = force_iters < 0 ? -1 : force_iters;
  // the one-pass series start serves the ring and pair modes with at most two
  // source terms per slice
  int max_src = 0;
  uintptr_t bits = 0;       // the ring pass reads u and the sources with 16-byte copies
  for (const BatchSlice& hs : b->hs) {
    max_src = std::max(max_src, hs.nsrc);
    bits |= reinterpret_cast<uintptr_t>(hs.u);
    for (int k = 0; k < hs.nsrc; ++k) bits |= reinterpret_cast<uintptr_t>(hs.src_g[k]);
  }
  const bool aligned16 = (bits & 15u) == 0;
  const int start_mode = (b->ring && max_src <= 2 && aligned16) ? (max_src > 0 ? 2 : 1) : 0;
  if (!b->exec || b->graph_force != force || b->graph_tol != tol ||
      b->graph_start != start_mode) {
    const int r = build_batch_graph(b, force, tol, start_mode);
    if (r != AD_OK) return r;
  }
  if (force == 0) return bfail(AD_ERR_INVALID, "force_iters == 0 is not supported in batches");
  B_CUDA(cudaGraphLaunch(b->exec, b->stream));
  B_CUDA(cudaMemcpyAsync(b->h_ctrl.data(), b->d_ctrl, sizeof(Ctrl) * b->S, cudaMemcpyDeviceToHost,
                         b->stream));
  B_CUDA(cudaStreamSynchronize(b->stream));
  int status = AD_OK;
  int total_iters = 0;
  for (int s = 0; s < b->S; ++s) {
    const Ctrl& c = b->h_ctrl[s];
    total_iters += c.iters;
    if (c.status == 4) status = AD_ERR_TIMEOUT;
    else if (c.status != 0 && status != AD_ERR_TIMEOUT) status = AD_ERR_NOT_CONVERGED;
    if (per_slice) {
      ad_stats& st = per_slice[s];
      st = ad_stats{};
      st.iters = c.iters;
      st.matvecs = c.iters + 1;
      st.substeps = 1;
      st.converged = c.status == 0;
      st.err_est = c.pnorm2 > 0.0 ? c.err_est * std::sqrt(c.ynorm2 / c.pnorm2) : 0.0;
      st.alpha = b->lc_alpha[s];
    }
  }
  if (b->ring && order_auto()) {           // the next step queues the longest series first
    std::vector<double> it(b->S);
    for (int s = 0; s < b->S; ++s) it[s] = b->h_ctrl[s].iters;
    order_by_iterations(b, it.data());
  }
  if (per_slice) {
    // kernels of the whole batched step: apply, init, update and every kernel of
    // every loop-body run (kBatchUnroll per run, enough runs for the slowest slice)
    int max_it = 0;
    for (int s = 0; s < b->S; ++s) max_it = std::max(max_it, b->h_ctrl[s].iters);
    const int per_run = kBatchUnroll * (b->pair ? 2 : 1);     // iterations per body run
    const int launches =
        b->persist ? (int)(launch_counter() - l0) + 3          // start, persistent, finish
                   : (int)(launch_counter() - l0) + 3 + (b->pair ? 1 : 0) +
                         kBatchUnroll * ((max_it + per_run - 1) / per_run);
    for (int s = 0; s < b->S; ++s) per_slice[s].kernel_launches = launches;
  }
  if (status == AD_ERR_TIMEOUT) return bfail(status, "a bounded wait of the batched series gave up");
  if (status != AD_OK) return bfail(status, "a slice's Leja series reached max_iters");
  return AD_OK;
}

int ad_batch_bind(ad_batch* b, void* const* u, const ad_source* src) {
  set_error_message("");
  if (!b || !u) return bfail(AD_ERR_INVALID, "NULL argument");
  for (int s = 0; s < b->S; ++s) {
    if (!u[s]) return bfail(AD_ERR_INVALID, "u[s] is NULL");
    if (src && (src[s].nterms < 0 || src[s].nterms > kBatchSources))
      return bfail(AD_ERR_INVALID, "batched sources: at most 4 terms per slice");
    if (src && src[s].nterms > 0 && !src[s].g) return bfail(AD_ERR_INVALID, "source: g is NULL");
  }
  b->bound_u.assign(u, u + b->S);
  b->bound_has_src = src != nullptr;
  b->bound_src.assign(b->S, ad_source{});
  b->bound_g.assign(b->S, {});
  if (src)
    for (int s = 0; s < b->S; ++s) {       // the term pointers are copied; the fields are not
      b->bound_g[s].assign(src[s].g, src[s].g + src[s].nterms);
      b->bound_src[s] = src[s];
      b->bound_src[s].g = b->bound_g[s].data();
    }
  return AD_OK;
}

int ad_batch_step(ad_batch* b, double t, double dt, double tol, int force_iters,
                  ad_stats* per_slice) {
  set_error_message("");
  if (!b) return bfail(AD_ERR_INVALID, "NULL batch");
  if ((int)b->bound_u.size() != b->S) return bfail(AD_ERR_INVALID, "no vectors bound (ad_batch_bind)");
  return ad_batch_midpoint_step(b, b->bound_u.data(), t, dt,
                                b->bound_has_src ? b->bound_src.data() : nullptr, tol, force_iters,
                                per_slice);
}

}  // extern "C"
