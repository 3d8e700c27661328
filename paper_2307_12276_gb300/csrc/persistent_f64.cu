// Persistent FP64 Newton series (Section 2): one cooperative launch runs
// every Leja iteration of a series for grids up to kPersistMaxCells.  Each
// block's 9 scaled weights, p and w2 stay in shared memory for the whole
// series (loaded once).
//
// Three kernels:
//  * leja_tile_f64_k (default wherever its tiles fit): block b owns a 2-D
//    tile, synchronises with its up to 8 neighbours only, and the stopping
//    rule runs two iterations behind; for a step of one substep it also runs
//    the step's right-hand side and update (StepFuse), so a step is one launch;
//  * leja_nsync_f64_k: the same protocol on contiguous row ranges;
//  * leja_persistent_f64_k: one grid barrier per iteration, used when neither
//    window fits in shared memory.
#include "ad_internal.h"
#include "stencil9.cuh"

#include <algorithm>
#include <cstdlib>
#include <mutex>
#include <vector>

namespace ad {
namespace {

// ---------------------------------------------------------------- shared pieces
// Every wait of both kernels is bounded by kBarrierTimeoutNs of global time,
// after which the block records a timeout status and leaves, so neither
// kernel can hang.
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ULL;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Tree sum of two values over the block (FP64; result in every thread):
// contiguous halving, then a shuffle tree in warp 0.  Measured on GB300: a
// __syncthreads costs ~0.5k cycles in a 1024-thread block and ~0.1k with 64
// threads, so the persistent kernels use small blocks.
__device__ __forceinline__ void block_tree_sum2(double& a, double& b, double* sa, double* sb) {
  const int t = threadIdx.x, nt = blockDim.x;  // nt is a power of two
  __syncthreads();
  sa[t] = a;
  sb[t] = b;
  __syncthreads();
  for (int s = nt >> 1; s >= 32; s >>= 1) {
    if (t < s) {
      sa[t] += sa[t + s];
      sb[t] += sb[t + s];
    }
    __syncthreads();
  }
  if (t < 32) {
    double x = sa[t], y = sb[t];
    if (nt < 32) {                 // tiny blocks: lanes beyond the block hold nothing
      x = t < nt ? x : 0.0;
      y = t < nt ? y : 0.0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_down_sync(0xffffffffu, x, o);
      y += __shfl_down_sync(0xffffffffu, y, o);
    }
    if (t == 0) {
      sa[0] = x;
      sb[0] = y;
    }
  }
  __syncthreads();
  a = sa[0];
  b = sb[0];
}

// One cell of the fused iteration (Section 2 recurrence),
//   z = ((A - c)/gamma) y - xi_m y  [+ e1 w2 + e2 w1 in the augmented form],
// as one FMA chain: 12 FP64 instructions (+ 3 for p and the norms).  On
// GB300 a warp issues at most one FP64 instruction per 64 cycles and four
// warps per SM saturate the FP64 pipe, so the instruction count is what
// matters, not the chain length.  Both persistent kernels use this order.
struct Nb9 {
  double sw, s, se, w, c, e, nw, n, ne;
};

// w1 is read with a plain (coherent) load: the fused step of the tile kernel
// writes it in the same launch.
template <bool AUG>
__device__ __forceinline__ double f64_cell(const double* __restrict__ sW, int cpb, int k,
                                           const Nb9& y, const LejaCoef& lc, double w2v,
                                           const double* w1, int idx) {
  double z = sW[4 * cpb + k] * y.c;
  z = fma(sW[0 * cpb + k], y.sw, z);
  z = fma(sW[1 * cpb + k], y.s, z);
  z = fma(sW[2 * cpb + k], y.se, z);
  z = fma(sW[3 * cpb + k], y.w, z);
  z = fma(sW[5 * cpb + k], y.e, z);
  z = fma(sW[6 * cpb + k], y.nw, z);
  z = fma(sW[7 * cpb + k], y.n, z);
  z = fma(sW[8 * cpb + k], y.ne, z);
  z = fma(-lc.xi, y.c, z);
  if (AUG) {
    if (lc.e1 != 0.0) z = fma(lc.e1, w2v, z);
    if (lc.e2 != 0.0) z = fma(lc.e2, w1[idx], z);
  }
  return z;
}

// Neighbour offsets of cell (i, j): periodic wrap, or Dirichlet clamping (the
// folded ghost weights are exactly 0, any in-domain value serves).
// cyclic: offsets into a window indexed modulo n (the row wrap is implicit).
__device__ __forceinline__ void f64_offsets(bool periodic, bool cyclic, int i, int j, int nx,
                                            int ny, int& dxm, int& dxp, int& dym, int& dyp) {
  if (periodic) {
    dxm = i ? -1 : nx - 1;
    dxp = (i + 1 < nx) ? 1 : 1 - nx;
    dym = (j || cyclic) ? -nx : (ny - 1) * nx;
    dyp = (j + 1 < ny || cyclic) ? nx : -(ny - 1) * nx;
  } else {
    dxm = i ? -1 : 0;
    dxp = (i + 1 < nx) ? 1 : 0;
    dym = j ? -nx : 0;
    dyp = (j + 1 < ny) ? nx : 0;
  }
}

__device__ __forceinline__ Nb9 gather9(const double* yc, int dxm, int dxp, int dym, int dyp) {
  Nb9 y;
  y.c = yc[0];
  y.w = yc[dxm];
  y.e = yc[dxp];
  y.s = yc[dym];
  y.sw = yc[dym + dxm];
  y.se = yc[dym + dxp];
  y.n = yc[dyp];
  y.nw = yc[dyp + dxm];
  y.ne = yc[dyp + dxp];
  return y;
}

// Asynchronous 8-byte global -> shared copy (completion: cp_async_wait_all).
__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Warp-wide sums of (ty, tp) over G blocks' partials base[2 b], base[2 b + 1]
// in a fixed order (lane-strided, then a shuffle tree), result in lane 0.
__device__ __forceinline__ void warp_sum_partials(const double* base, int G, double& ty,
                                                  double& tp) {
  const int lane = threadIdx.x & 31;
  double y = 0.0, p = 0.0;
  for (int b = lane; b < G; b += 32) {
    y += __ldcg(base + 2 * b);
    p += __ldcg(base + 2 * b + 1);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    y += __shfl_down_sync(0xffffffffu, y, o);
    p += __shfl_down_sync(0xffffffffu, p, o);
  }
  ty = y;
  tp = p;
}

// Threads per persistent block owning cpb cells: the smallest power of two
// >= cpb, at most 256.  Four warps per SM already saturate GB300's FP64 pipe
// (one FP64 instruction per 64 cycles per sub-partition); more warps only
// make every block barrier dearer.
int persist_threads(int cpb) {
  int T = 32;
  while (T < cpb && T < 256) T <<= 1;
  return T;
}

// ---------------------------------------------------------------- grid-barrier kernel
// y ping-pongs through global memory.  One grid barrier per iteration: the
// last block to arrive reduces the norm partials in block order, applies the
// stopping rule and publishes it; the others wait for the barrier generation
// to change.
template <bool AUG>
__global__ void __launch_bounds__(256) leja_persistent_f64_k(SeriesArgs a, unsigned int cpb_u,
                                                             unsigned int* gen) {
  extern __shared__ double smem[];
  __shared__ double ra[256], rb[256];
  __shared__ int s_flag;
  const GridDev g = a.g;
  const int n = (int)g.n, nx = g.nx, ny = g.ny, cpb = (int)cpb_u;
  const bool periodic = g.bc == 0;
  const int T = blockDim.x, t = threadIdx.x;
  const int c0 = blockIdx.x * cpb;
  const int c1 = min(n, c0 + cpb);
  const int nc = c1 > c0 ? c1 - c0 : 0;
  double* sW = smem;                 // [9][cpb]
  double* sP = smem + 9 * cpb;       // [cpb]
  double* sW2 = sP + cpb;            // [cpb] (augmented)
  const double* __restrict__ Ws = static_cast<const double*>(a.coef);
  double* __restrict__ p = static_cast<double*>(a.p);
  const double* __restrict__ w1 = static_cast<const double*>(a.w1);
  const double* __restrict__ w2 = static_cast<const double*>(a.w2);
  Ctrl* ctrl = a.ctrl;
  for (int k = t; k < nc; k += T) {
#pragma unroll
    for (int q = 0; q < 9; ++q) sW[q * cpb + k] = Ws[(long long)q * n + c0 + k];
    sP[k] = p[c0 + k];
    if (AUG) sW2[k] = w2[c0 + k];
  }
  unsigned int my_gen = 0;
  if (t == 0) my_gen = *(volatile unsigned int*)gen;
  int m = 0;
  for (;;) {
    const LejaCoef lc = a.lc[m];
    const double* yin = static_cast<const double*>(a.y[m & 1]);
    double* yout = static_cast<double*>(a.y[(m + 1) & 1]);
    __syncthreads();                 // shared weights/p ready; previous iteration done
    double sy = 0.0, sp = 0.0;
    for (int k = t; k < nc; k += T) {
      const int idx = c0 + k;
      const int j = idx / nx, i = idx - j * nx;
      int dxm, dxp, dym, dyp;
      f64_offsets(periodic, false, i, j, nx, ny, dxm, dxp, dym, dyp);
      // plain loads: L1 hits for the neighbours; the fence that follows every
      // grid barrier orders them after the other blocks' writes
      const Nb9 y = gather9(yin + idx, dxm, dxp, dym, dyp);
      const double z = f64_cell<AUG>(sW, cpb, k, y, lc, AUG ? sW2[k] : 0.0, w1, idx);
      __stcg(yout + idx, z);
      const double pn = fma(lc.d, z, sP[k]);
      sP[k] = pn;
      sy = fma(z, z, sy);
      sp = fma(pn, pn, sp);
    }
    block_tree_sum2(sy, sp, ra, rb);
    // grid barrier; the last arriver decides
    if (t == 0) {
      a.partials[2 * blockIdx.x] = sy;
      a.partials[2 * blockIdx.x + 1] = sp;
      __threadfence();
      const unsigned int tk = atomicAdd(&ctrl->ticket, 1u);
      s_flag = (tk == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (s_flag) {
      double ty = 0.0, tp = 0.0;
      if (t < 32) {
        __threadfence();
        warp_sum_partials(a.partials, (int)gridDim.x, ty, tp);
      }
      if (t == 0) {
        const int terms = m + 1;
        const double absd = lc.absd, tol = ctrl->tol;
        ctrl->ynorm2 = ty;
        ctrl->pnorm2 = tp;
        ctrl->iters = terms;
        ctrl->err_est = absd;
        int stop = 0;
        if (ctrl->force > 0) {
          stop = terms >= ctrl->force;
        } else if (!isfinite(ty) || !isfinite(tp)) {
          stop = 1;
          ctrl->status = 3;
        } else if (terms >= 2 && (absd * absd) * ty <= (tol * tol) * tp) {
          stop = 1;
        } else if (terms >= ctrl->max_iters) {
          stop = 1;
          ctrl->status = 3;
        }
        if (terms >= kMaxIters) stop = 1;
        ctrl->stop = stop;
        ctrl->m = m + 1;
        ctrl->ticket = 0u;
        __threadfence();
        atomicAdd(gen, 1u);           // release the waiting blocks
        my_gen += 1u;
        s_flag = stop ? 2 : 0;
      }
    } else if (t == 0) {
      const unsigned long long t0 = global_ns();
      int state = 0;
      while (*(volatile unsigned int*)gen == my_gen) {
        if (global_ns() - t0 > kBarrierTimeoutNs) { state = 3; break; }
        __nanosleep(64);
      }
      if (state == 3) {
        ctrl->status = 4;              // a wait gave up: AD_ERR_TIMEOUT
        s_flag = 3;
      } else {
        __threadfence();
        my_gen += 1u;
        s_flag = (*(volatile int*)&ctrl->stop) ? 2 : 0;
      }
    }
    __syncthreads();
    if (s_flag != 0) break;
    ++m;
  }
  __syncthreads();
  for (int k = t; k < nc; k += T) p[c0 + k] = sP[k];
}

// ---------------------------------------------------------------- neighbour-synchronised kernel
// Iteration m of block b needs y_m only on its own cells and on the cells
// within H of them (H = nx + 1 with clamped Dirichlet indices, 2 nx with the
// periodic wrap), a "window" of cpb + 2H values kept in shared memory (two
// buffers: y_m is read while y_{m+1} is written).  Own cells farther than H
// from both ends of the block's range ("interior") need no other block's
// data; the others ("boundary") need the two halo strips.  Per iteration:
//
//   A  warp 0 applies the lagged stopping rule (below); warp 1 waits for the
//      blocks owning the halo cells (flags >= m) and copies the halo strips
//      of y_m from global memory into the window; warps 2.. compute z on the
//      interior cells (into the window only: no other block reads them).
//   C  all warps compute z on the boundary cells, into the window and into
//      global y_{m+1}; then thread 0 publishes flags[b] = m + 1.
//   D  all threads update p and accumulate the two squared norms; the block
//      sums are written to the write-once slot (m, b).
//
// The wait of phase A is hidden behind the interior cells.  flags[b] >= m + 1
// also tells the neighbours that block b has finished reading the global
// buffer they overwrite next.
//
// Stopping rule with a lag of two: at the start of iteration m every block
// reads the slots of iteration m - 2 of all blocks (normally long written),
// sums them in block order and applies the test of Section 2, so every block
// reaches the same decision.  If the series should have stopped after
// iteration m - 2, iteration m - 1 was computed for nothing and its p (kept
// in a second buffer) is dropped; phase A of iteration m writes nothing that
// survives the decision.  Count-based stops (forced iteration counts,
// max_iters) need no norms and end without a lag.
//
// Slots hold a signalling NaN until written (arithmetic never produces one),
// reset by their owner at the start of each launch, followed by one grid
// barrier.  Every wait is bounded by kBarrierTimeoutNs; a block that gives up
// records status 4 and leaves, and the blocks waiting on it do the same.
constexpr unsigned long long kSlotEmpty = 0x7FF0DEAD0000BEEFULL;
constexpr int kNsyncMaxNeighbours = 32;
constexpr int kNsyncMaxBlocks = 160;     // slots per iteration (>= 152 SMs)

struct NsyncGeom {
  int cpb;   // cells per block (the last block may own fewer)
  int H;     // window half-width
  int W;     // window length, cpb + 2 H
};

__device__ __forceinline__ unsigned long long ld_volatile_u64(const double* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}

// Warp-wide: norm sums of iteration k over all G blocks, in block order
// (lane-strided partial sums, then a shuffle tree), identical in every block.
// Returns false if a slot stayed empty for kBarrierTimeoutNs.
__device__ bool nsync_read_norms(const double* slots, int k, int G, double& ty, double& tp) {
  const int lane = threadIdx.x & 31;
  constexpr int R = (kNsyncMaxBlocks + 31) / 32;
  double vy[R], vp[R];
  bool have[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    have[r] = lane + 32 * r >= G;
    vy[r] = 0.0;
    vp[r] = 0.0;
  }
  const double* base = slots + 2LL * k * kNsyncMaxBlocks;
  const unsigned long long t0 = global_ns();
  bool ok = true;
  for (;;) {
    bool all = true;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!have[r]) {
        const int bb = lane + 32 * r;
        const unsigned long long y = ld_volatile_u64(base + 2 * bb);
        const unsigned long long p = ld_volatile_u64(base + 2 * bb + 1);
        if (y != kSlotEmpty && p != kSlotEmpty) {
          vy[r] = __longlong_as_double((long long)y);
          vp[r] = __longlong_as_double((long long)p);
          have[r] = true;
        } else {
          all = false;
        }
      }
    }
    if (__all_sync(0xffffffffu, all)) break;
    if (__any_sync(0xffffffffu, global_ns() - t0 > kBarrierTimeoutNs)) { ok = false; break; }
  }
  double y = 0.0, p = 0.0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    y += vy[r];
    p += vp[r];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    y += __shfl_down_sync(0xffffffffu, y, o);
    p += __shfl_down_sync(0xffffffffu, p, o);
  }
  ty = __shfl_sync(0xffffffffu, y, 0);
  tp = __shfl_sync(0xffffffffu, p, 0);
  return ok;
}

// Stopping test of Section 2 on the norms of iteration k (terms = k + 1):
// 0 converged, 3 not finite, -1 keep going.
__device__ __forceinline__ int nsync_test(const LejaCoef& lc, int terms, double tol, double ty,
                                          double tp) {
  if (!isfinite(ty) || !isfinite(tp)) return 3;
  if (terms >= 2 && (lc.absd * lc.absd) * ty <= (tol * tol) * tp) return 0;
  return -1;
}

template <bool AUG>
__global__ void __launch_bounds__(256) leja_nsync_f64_k(SeriesArgs a, NsyncGeom geo,
                                                        double* slots, unsigned int* flags,
                                                        unsigned int* gen) {
  extern __shared__ double smem[];
  __shared__ double ra[256], rb[256];
  __shared__ int s_nb[kNsyncMaxNeighbours];
  __shared__ int s_nnb, s_final, s_status, s_fail;
  __shared__ double s_ty, s_tp;
  const GridDev g = a.g;
  const int n = (int)g.n, nx = g.nx, ny = g.ny;
  const bool periodic = g.bc == 0;
  const int G = gridDim.x, b = blockIdx.x, T = blockDim.x, t = threadIdx.x;
  const int warp = t >> 5, lane = t & 31, nwarps = T >> 5;
  const int cpb = geo.cpb, H = geo.H, W = geo.W;
  const int c0 = b * cpb;
  const int c1 = min(n, c0 + cpb);
  const int nc = max(0, c1 - c0);
  // interior own cells [H, nc - H); boundary: the rest
  const int nA = nc > 2 * H ? nc - 2 * H : 0;
  const int nB = nc - nA;
  // roles: warp 0 decides, warp 1 (or 0) polls and copies the halo,
  // warps 2.. (or all) compute the interior
  const int poll_warp = nwarps >= 2 ? 1 : 0;
  const int wA = nwarps >= 3 ? warp - 2 : warp, nwA = nwarps >= 3 ? nwarps - 2 : nwarps;
  double* sW = smem;                        // [9][cpb] scaled weights
  double* sP = sW + 9 * cpb;                // [2][cpb]: P_k lives in buffer (k + 1) & 1
  double* sW2 = sP + 2 * cpb;               // [cpb] (augmented)
  double* win = sW2 + (AUG ? cpb : 0);      // [2][W]: y_m lives in buffer m & 1
  const double* __restrict__ Ws = static_cast<const double*>(a.coef);
  const double* __restrict__ w1 = static_cast<const double*>(a.w1);
  const double* __restrict__ w2 = static_cast<const double*>(a.w2);
  Ctrl* ctrl = a.ctrl;
  const int force = ctrl->force;
  const int max_it = min(ctrl->max_iters, kMaxIters);
  const double tol = ctrl->tol;

  // ---- reset this block's slots and flag, load the resident data
  for (int k = t; k < kMaxIters; k += T) {
    double* s2 = slots + 2LL * ((long long)k * kNsyncMaxBlocks + b);
    reinterpret_cast<unsigned long long*>(s2)[0] = kSlotEmpty;
    reinterpret_cast<unsigned long long*>(s2)[1] = kSlotEmpty;
  }
  if (t == 0) {
    flags[b] = 0u;
    s_fail = 0;
    // blocks owning the halo cells [c0 - H, c0) and [c1, c1 + H)
    int cnt = 0;
    for (int side = 0; side < 2 && cnt >= 0; ++side) {
      long long c = side == 0 ? (long long)c0 - H : (long long)c1;
      const long long hi = side == 0 ? (long long)c0 - 1 : (long long)c1 + H - 1;
      while (c <= hi) {
        long long cm = c;
        if (periodic) {
          cm = ((c % n) + n) % n;
        } else if (c < 0) {
          c = 0;
          continue;
        } else if (c >= n) {
          break;
        }
        const int owner = (int)(cm / cpb);
        bool seen = owner == b;
        for (int q = 0; q < cnt; ++q) seen = seen || s_nb[q] == owner;
        if (!seen) {
          if (cnt == kNsyncMaxNeighbours) { cnt = -1; break; }
          s_nb[cnt++] = owner;
        }
        const long long end = (long long)(owner + 1) * cpb;
        c += (end < n ? end : n) - cm;                   // to the owner's last cell
      }
    }
    s_nnb = cnt;
    if (cnt < 0) s_fail = 1;                 // the launcher bounds the neighbour count
  }
  for (int k = t; k < nc; k += T) {
#pragma unroll
    for (int q = 0; q < 9; ++q) sW[q * cpb + k] = Ws[(long long)q * n + c0 + k];
    sP[k] = static_cast<const double*>(a.p)[c0 + k];
    if (AUG) sW2[k] = w2[c0 + k];
  }
  {  // the whole window of y_0
    const double* y0 = static_cast<const double*>(a.y[0]);
    for (int q = t; q < 2 * H + nc; q += T) {
      long long c = (long long)c0 - H + q;
      if (periodic) c = ((c % n) + n) % n;
      else if (c < 0 || c >= n) continue;
      win[q] = y0[c];
    }
  }
  // ---- one grid barrier: no block reads a slot or flag before its owner reset it
  __threadfence();
  __syncthreads();
  if (t == 0) {
    const unsigned int my_gen = *(volatile unsigned int*)gen;
    __threadfence();
    const unsigned int tk = atomicAdd(&ctrl->ticket, 1u);
    if (tk == (unsigned int)G - 1) {
      ctrl->ticket = 0u;
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*(volatile unsigned int*)gen == my_gen) {
        if (global_ns() - t0 > kBarrierTimeoutNs) { s_fail = 1; break; }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();

  int m = 0;
  int fin = -1;
  if (!s_fail) {
    for (;;) {
      const LejaCoef lc = a.lc[m];
      const double* wy = win + (m & 1) * W;
      double* wz = win + ((m + 1) & 1) * W;
      // ---- phase A
      if (warp == 0) {                              // the lagged decisions
        int f = -1, st = 0;
        double ty = 0.0, tp = 0.0;
        bool ok = true;
        if (force <= 0 && m >= 2) {                 // norm test on iteration m - 2
          ok = nsync_read_norms(slots, m - 2, G, ty, tp);
          const int r = nsync_test(a.lc[m - 2], m - 1, tol, ty, tp);
          if (ok && r >= 0) { f = m - 2; st = r; }
        }
        if (ok && f < 0 && m >= 1) {                // count-based stop after iteration m - 1
          const bool cnt = (force > 0 ? m >= force : m >= max_it) || m >= kMaxIters;
          if (cnt) {
            f = m - 1;
            if (b == 0) {                           // norms for the report (block 0 only)
              ok = nsync_read_norms(slots, m - 1, G, ty, tp);
              if (force <= 0) {
                const int r = nsync_test(a.lc[m - 1], m, tol, ty, tp);
                st = r == 0 ? 0 : 3;
              }
            }
          }
        }
        if (lane == 0) {
          s_final = f;
          s_status = st;
          s_ty = ty;
          s_tp = tp;
          if (!ok) s_fail = 1;
        }
      }
      if (warp == poll_warp && m >= 1) {            // neighbours, then the halo strips of y_m
        if (lane < s_nnb) {
          const unsigned int* fl = flags + s_nb[lane];
          if (*(const volatile unsigned int*)fl < (unsigned int)m) {
            const unsigned long long t0 = global_ns();
            while (*(const volatile unsigned int*)fl < (unsigned int)m) {
              if (global_ns() - t0 > kBarrierTimeoutNs) { s_fail = 1; break; }
            }
          }
          __threadfence();
        }
        __syncwarp();
        // asynchronous copies: every lane has all its copies in flight at once
        const double* yg = static_cast<const double*>(a.y[m & 1]);
        double* wh = win + (m & 1) * W;
        for (int q = lane; q < 2 * H; q += 32) {
          const int w = q < H ? q : q + nc;
          long long c = (long long)c0 - H + w;
          if (periodic) c = ((c % n) + n) % n;
          else if (c < 0 || c >= n) continue;
          cp_async8(wh + w, yg + c);
        }
        cp_async_wait_all();
      }
      if (warp >= 2 || nwarps < 3) {                // interior cells (own data only)
        for (int q = wA * 32 + lane; q < nA; q += nwA * 32) {
          const int k = H + q;
          const int idx = c0 + k;
          const int j = idx / nx, i = idx - j * nx;
          int dxm, dxp, dym, dyp;
          f64_offsets(periodic, true, i, j, nx, ny, dxm, dxp, dym, dyp);
          const Nb9 y = gather9(wy + H + k, dxm, dxp, dym, dyp);
          wz[H + k] = f64_cell<AUG>(sW, cpb, k, y, lc, AUG ? sW2[k] : 0.0, w1, idx);
        }
      }
      __syncthreads();
      if (s_fail || s_final >= 0) break;
      // ---- phase C: boundary cells
      double* yout = static_cast<double*>(a.y[(m + 1) & 1]);
      for (int q = t; q < nB; q += T) {
        const int k = (nA > 0 && q >= H) ? q + nA : q;
        const int idx = c0 + k;
        const int j = idx / nx, i = idx - j * nx;
        int dxm, dxp, dym, dyp;
        f64_offsets(periodic, true, i, j, nx, ny, dxm, dxp, dym, dyp);
        const Nb9 y = gather9(wy + H + k, dxm, dxp, dym, dyp);
        const double z = f64_cell<AUG>(sW, cpb, k, y, lc, AUG ? sW2[k] : 0.0, w1, idx);
        wz[H + k] = z;
        __stcg(yout + idx, z);
      }
      __syncthreads();
      if (t == 0) {
        __threadfence();
        *(volatile unsigned int*)(flags + b) = (unsigned int)(m + 1);
      }
      // ---- phase D: p and the norms
      const double* Pin = sP + (m & 1) * cpb;
      double* Pout = sP + ((m + 1) & 1) * cpb;
      double sy = 0.0, sp = 0.0;
      for (int k = t; k < nc; k += T) {
        const double z = wz[H + k];
        const double pn = fma(lc.d, z, Pin[k]);
        Pout[k] = pn;
        sy = fma(z, z, sy);
        sp = fma(pn, pn, sp);
      }
      block_tree_sum2(sy, sp, ra, rb);
      if (t == 0) {                                 // the slot value itself is the signal
        double* s2 = slots + 2LL * ((long long)m * kNsyncMaxBlocks + b);
        s2[0] = sy;
        s2[1] = sp;
      }
      ++m;
    }
    fin = s_final;
  }
  // ---- result: P_fin, and the report of block 0
  if (s_fail) {
    if (t == 0) {
      atomicMax(&ctrl->status, 4);           // AD_ERR_TIMEOUT
      ctrl->stop = 1;
    }
    return;
  }
  const double* Pf = sP + ((fin + 1) & 1) * cpb;
  double* p = static_cast<double*>(a.p);
  for (int k = t; k < nc; k += T) p[c0 + k] = Pf[k];
  if (b == 0 && t == 0) {
    ctrl->iters = fin + 1;
    ctrl->m = fin + 1;
    ctrl->ynorm2 = s_ty;
    ctrl->pnorm2 = s_tp;
    ctrl->err_est = a.lc[fin].absd;
    atomicMax(&ctrl->status, s_status);
    ctrl->stop = 1;
  }
}

// ---------------------------------------------------------------- 2-D tile kernel
// leja_tile_f64_k: the protocol of leja_nsync_f64_k (neighbour flags,
// write-once norm slots, the decision two iterations late, bounded waits) on
// a 2-D decomposition.  Block b owns a tile of tw x th cells (TX x TY tiles
// cover the grid; the last column and row of tiles may be smaller).  Its
// window holds y on the tile plus a one-cell halo ring, (tw + 2) x (th + 2)
// values per buffer, so every stencil offset is constant (the halo carries the
// wrapped values, or zeros outside a zero-Dirichlet domain where the folded
// weights are 0).  Only the tile's outer ring ("ring cells") depends on other
// blocks; the interior -- most of the tile, unlike the row kernel whose
// cells within one grid row of either end all wait for the halo -- is
// computed while warp 1 waits for the up to 8 neighbours and copies the halo.
// Ring cells are also stored to global y_{m+1}, where the neighbours read them.
// p and the two squared norms are formed with z, cell by cell, in both compute
// phases (no separate pass): three p buffers keep the result that the lagged
// decision may still return (P after iteration m - 2) out of the way.  After
// the ring cells thread 0 publishes flags[b] = m + 1; the per-thread norm
// partials of iteration m are added by warp 0 at the start of iteration m + 1
// (one packed shuffle tree instead of one per warp: GB300's FP64 pipe is
// shared by the SM's four sub-partitions, so every FP64 instruction of the
// block counts) and written to the slot (m, b) before warp 0 waits for
// anything.
struct TileGeom {
  int TX, TY;   // tiles per grid row / column (G = TX * TY)
  int tw, th;   // tile width / height (full tiles)
  int S;        // window row stride, tw + 2
};

// tile-local (li, lj) of ring cell q of a tw x th tile
__device__ __forceinline__ void ring_cell(int q, int tw, int th, int& li, int& lj) {
  if (q < tw) { li = q; lj = 0; return; }
  if (th > 1 && q < 2 * tw) { li = q - tw; lj = th - 1; return; }
  const int r = q - (th > 1 ? 2 * tw : tw);
  if (r < th - 2) { li = 0; lj = 1 + r; } else { li = tw - 1; lj = 1 + r - (th - 2); }
}

// halo position q of a tw x th tile: (hx, hy) in the ring around it
__device__ __forceinline__ void halo_cell(int q, int tw, int th, int& hx, int& hy) {
  if (q < tw + 2) { hx = q - 1; hy = -1; return; }
  if (q < 2 * (tw + 2)) { hx = q - (tw + 2) - 1; hy = th; return; }
  const int r = q - 2 * (tw + 2);
  if (r < th) { hx = -1; hy = r; } else { hx = tw; hy = r - th; }
}

template <bool AUG>
__global__ void __launch_bounds__(256) leja_tile_f64_k(SeriesArgs a, TileGeom geo, double* slots,
                                                       unsigned int* flags, unsigned int* gen,
                                                       StepFuse F) {
  extern __shared__ double smem[];
  __shared__ double s_py[2][256], s_pp[2][256];   // per-thread norm partials, double-buffered
  __shared__ int s_nb[8];
  __shared__ int s_nnb, s_final, s_status, s_fail;
  __shared__ double s_ty, s_tp;
  const GridDev g = a.g;
  const int n = (int)g.n, nx = g.nx, ny = g.ny;
  const bool periodic = g.bc == 0;
  const int G = gridDim.x, b = blockIdx.x, T = blockDim.x, t = threadIdx.x;
  const int warp = t >> 5, lane = t & 31, nwarps = T >> 5;
  const int bx = b % geo.TX, by = b / geo.TX;
  const int x0 = bx * geo.tw, y0 = by * geo.th;
  const int tw = min(geo.tw, nx - x0), th = min(geo.th, ny - y0);
  const int nc = tw * th;
  const int cpb = geo.tw * geo.th;                 // plane stride of the resident data
  const int S = geo.S;
  const int WB = S * (geo.th + 2);                 // one window buffer
  const int nI = (tw > 2 && th > 2) ? (tw - 2) * (th - 2) : 0;
  const int nR = nc - nI;
  const int nH = 2 * (tw + 2) + 2 * th;
  const int poll_warp = nwarps >= 2 ? 1 : 0;
  const int wA = nwarps >= 3 ? warp - 2 : warp, nwA = nwarps >= 3 ? nwarps - 2 : nwarps;
  double* sW = smem;                        // [9][cpb] scaled weights
  double* sP = sW + 9 * cpb;                // [3][cpb]: P after iteration k in buffer (k + 1) % 3
  double* sW2 = sP + 3 * cpb;               // [cpb] (augmented)
  double* win = sW2 + (AUG ? cpb : 0);      // [2][WB]: y_m lives in buffer m & 1
  const double* __restrict__ Ws = static_cast<const double*>(a.coef);
  const double* w1 = static_cast<const double*>(a.w1);
  const double* __restrict__ w2 = static_cast<const double*>(a.w2);
  Ctrl* ctrl = a.ctrl;
  const bool fused = F.s != 0;                     // a whole step (see StepFuse)
  const int force = fused ? F.force : ctrl->force;
  const int max_it = min(fused ? F.max_iters : ctrl->max_iters, kMaxIters);
  const double tol = fused ? F.tol : ctrl->tol;
  auto gidx = [&](int li, int lj) { return (y0 + lj) * nx + x0 + li; };
  auto widx = [&](int li, int lj) { return (lj + 1) * S + li + 1; };

  // ---- reset this block's slots and flag, load the resident data
  for (int k = t; k < kMaxIters; k += T) {
    double* s2 = slots + 2LL * ((long long)k * kNsyncMaxBlocks + b);
    reinterpret_cast<unsigned long long*>(s2)[0] = kSlotEmpty;
    reinterpret_cast<unsigned long long*>(s2)[1] = kSlotEmpty;
  }
  if (t == 0) {
    flags[b] = 0u;
    s_fail = 0;
    int cnt = 0;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (dx == 0 && dy == 0) continue;
        int tx = bx + dx, ty = by + dy;
        if (periodic) {
          tx = (tx + geo.TX) % geo.TX;
          ty = (ty + geo.TY) % geo.TY;
        } else if (tx < 0 || ty < 0 || tx >= geo.TX || ty >= geo.TY) {
          continue;
        }
        const int nb = ty * geo.TX + tx;
        bool seen = nb == b;
        for (int q = 0; q < cnt; ++q) seen = seen || s_nb[q] == nb;
        if (!seen) s_nb[cnt++] = nb;
      }
    s_nnb = cnt;
  }
  for (int q = t; q < 2 * WB; q += T) win[q] = 0.0;   // the Dirichlet halo stays 0
  if (fused && t == 0 && b == 0) {                 // what series_init resets
    ctrl->m = 0;
    ctrl->stop = 0;
    ctrl->iters = 0;
    ctrl->status = 0;
    ctrl->force = F.force;
    ctrl->max_iters = F.max_iters;
    ctrl->tol = F.tol;
    ctrl->err_est = 0.0;
    ctrl->ynorm2 = 0.0;
    ctrl->pnorm2 = 0.0;
  }
  __syncthreads();
  // The prologue only reads u, the weights and the sources and only writes
  // w1 (all distinct buffers): restrict-qualified pointers and two cells per
  // round let the loads of one cell overlap the work of the other.
  const double* __restrict__ Wu = F.W;
  const double* __restrict__ uu = F.u;
  double* __restrict__ w1o = F.w1;
#pragma unroll 2
  for (int k = t; k < nc; k += T) {
    const int li = k % tw, lj = k / tw;
    const int idx = gidx(li, lj);
#pragma unroll
    for (int q = 0; q < 9; ++q) sW[q * cpb + k] = Ws[(long long)q * n + idx];
    if (!fused) {
      sP[k] = static_cast<const double*>(a.p)[idx];
      if (AUG) sW2[k] = w2[idx];
      continue;
    }
    // the step's right-hand sides, as the apply kernel forms them
    const double au = stencil9(Wu, n, uu, x0 + li, y0 + lj, nx, ny, g.bc, idx);
    double r = 1.0 * au, r2 = 0.0;
    for (int q = 0; q < F.src.n; ++q) {
      const double gq = static_cast<const double*>(F.src.g[q])[idx];
      r = fma(F.src.a[q], gq, r);
      r2 = fma(F.src.b[q], gq, r2);
    }
    w1o[idx] = r;
    if (F.s == 2) {                                // y_0 = 0: the window stays 0
      if (AUG) sW2[k] = r2;
      sP[k] = F.d0 * 0.0;
    } else {                                       // y_0 = w1
      win[widx(li, lj)] = r;
      sP[k] = F.d0 * r;
    }
  }
  if (!fused) {  // y_0 on tile + halo (a fused phi_1 step loads its halo after the barrier)
    const double* y0g = static_cast<const double*>(a.y[0]);
    for (int k = t; k < nc; k += T) win[widx(k % tw, k / tw)] = y0g[gidx(k % tw, k / tw)];
    for (int q = t; q < nH; q += T) {
      int hx, hy;
      halo_cell(q, tw, th, hx, hy);
      int gx = x0 + hx, gy = y0 + hy;
      if (periodic) {
        gx = (gx + nx) % nx;
        gy = (gy + ny) % ny;
      } else if (gx < 0 || gy < 0 || gx >= nx || gy >= ny) {
        continue;
      }
      win[(hy + 1) * S + hx + 1] = y0g[gy * nx + gx];
    }
  }
  // ---- one grid barrier: no block reads a slot or flag before its owner reset it
  __threadfence();
  __syncthreads();
  if (t == 0) {
    const unsigned int my_gen = *(volatile unsigned int*)gen;
    __threadfence();
    const unsigned int tk = atomicAdd(&ctrl->ticket, 1u);
    if (tk == (unsigned int)G - 1) {
      ctrl->ticket = 0u;
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*(volatile unsigned int*)gen == my_gen) {
        if (global_ns() - t0 > kBarrierTimeoutNs) { s_fail = 1; break; }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  if (fused && F.s == 1) {   // the halo of y_0 = w1, which the neighbours wrote before the barrier
    for (int q = t; q < nH; q += T) {
      int hx, hy;
      halo_cell(q, tw, th, hx, hy);
      int gx = x0 + hx, gy = y0 + hy;
      if (periodic) {
        gx = (gx + nx) % nx;
        gy = (gy + ny) % ny;
      } else if (gx < 0 || gy < 0 || gx >= nx || gy >= ny) {
        continue;
      }
      win[(hy + 1) * S + hx + 1] = __ldcg(F.w1 + gy * nx + gx);
    }
    __syncthreads();
  }

  int m = 0;
  int fin = -1;
  if (!s_fail) {
    for (;;) {
      const LejaCoef lc = a.lc[m];
      const double* wy = win + (m & 1) * WB;
      double* wz = win + ((m + 1) & 1) * WB;
      // p of iteration m is formed with z, cell by cell: P after iteration
      // m - 1 in buffer m % 3, after iteration m into (m + 1) % 3.  The lagged
      // decision of this iteration may still return P after iteration m - 2,
      // in the third buffer, which nothing here overwrites.
      const double* Pin = sP + (m % 3) * cpb;
      double* Pout = sP + ((m + 1) % 3) * cpb;
      double sy = 0.0, sp = 0.0;
      // ---- phase A
      if (warp == 0) {
        // the block's norm sums of iteration m - 1 into slot (m - 1, b): the
        // per-thread partials (double-buffered) in thread order per lane, then
        // one shuffle tree that carries both sums (lanes 0-15 the y sum, lanes
        // 16-31 the p sum)
        if (m >= 1) {
          const double* py = s_py[(m - 1) & 1];
          const double* pp = s_pp[(m - 1) & 1];
          double ty = 0.0, tp = 0.0;
          for (int q = lane; q < T; q += 32) {
            ty += py[q];
            tp += pp[q];
          }
          const bool lo = lane < 16;
          double v = (lo ? ty : tp) + __shfl_xor_sync(0xffffffffu, lo ? tp : ty, 16);
#pragma unroll
          for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          const double vp = __shfl_sync(0xffffffffu, v, 16);
          if (lane == 0) {                          // the slot value itself is the signal
            double* s2 = slots + 2LL * ((long long)(m - 1) * kNsyncMaxBlocks + b);
            s2[0] = v;
            s2[1] = vp;
          }
          __syncwarp();
        }
        // the lagged decisions
        int f = -1, st = 0;
        double ty = 0.0, tp = 0.0;
        bool ok = true;
        if (force <= 0 && m >= 2) {                 // norm test on iteration m - 2
          ok = nsync_read_norms(slots, m - 2, G, ty, tp);
          const int r = nsync_test(a.lc[m - 2], m - 1, tol, ty, tp);
          if (ok && r >= 0) { f = m - 2; st = r; }
        }
        if (ok && f < 0 && m >= 1) {                // count-based stop after iteration m - 1
          const bool cnt = (force > 0 ? m >= force : m >= max_it) || m >= kMaxIters;
          if (cnt) {
            f = m - 1;
            if (b == 0) {                           // norms for the report (block 0 only)
              ok = nsync_read_norms(slots, m - 1, G, ty, tp);
              if (force <= 0) {
                const int r = nsync_test(a.lc[m - 1], m, tol, ty, tp);
                st = r == 0 ? 0 : 3;
              }
            }
          }
        }
        if (lane == 0) {
          s_final = f;
          s_status = st;
          s_ty = ty;
          s_tp = tp;
          if (!ok) s_fail = 1;
        }
      }
      if (warp == poll_warp && m >= 1) {            // neighbours, then the halo of y_m
        if (lane < s_nnb) {
          const unsigned int* fl = flags + s_nb[lane];
          if (*(const volatile unsigned int*)fl < (unsigned int)m) {
            const unsigned long long t0 = global_ns();
            while (*(const volatile unsigned int*)fl < (unsigned int)m) {
              if (global_ns() - t0 > kBarrierTimeoutNs) { s_fail = 1; break; }
            }
          }
          __threadfence();
        }
        __syncwarp();
        const double* yg = static_cast<const double*>(a.y[m & 1]);
        double* wh = win + (m & 1) * WB;
        for (int q = lane; q < nH; q += 32) {
          int hx, hy;
          halo_cell(q, tw, th, hx, hy);
          int gx = x0 + hx, gy = y0 + hy;
          if (periodic) {
            gx = (gx + nx) % nx;
            gy = (gy + ny) % ny;
          } else if (gx < 0 || gy < 0 || gx >= nx || gy >= ny) {
            continue;
          }
          cp_async8(wh + (hy + 1) * S + hx + 1, yg + gy * nx + gx);
        }
        cp_async_wait_all();
      }
      if (warp >= 2 || nwarps < 3) {                // interior cells (own data only)
        for (int q = wA * 32 + lane; q < nI; q += nwA * 32) {
          const int li = 1 + q % (tw - 2), lj = 1 + q / (tw - 2);
          const int k = lj * tw + li;
          const int w = widx(li, lj);
          const int idx = gidx(li, lj);
          const Nb9 y = gather9(wy + w, -1, 1, -S, S);
          const double z = f64_cell<AUG>(sW, cpb, k, y, lc, AUG ? sW2[k] : 0.0, w1, idx);
          wz[w] = z;
          const double pn = fma(lc.d, z, Pin[k]);
          Pout[k] = pn;
          sy = fma(z, z, sy);
          sp = fma(pn, pn, sp);
        }
      }
      __syncthreads();
      if (s_fail || s_final >= 0) break;
      // ---- phase C: ring cells, into the window and global y_{m+1}
      double* yout = static_cast<double*>(a.y[(m + 1) & 1]);
      for (int q = t; q < nR; q += T) {
        int li, lj;
        ring_cell(q, tw, th, li, lj);
        const int k = lj * tw + li;
        const int w = widx(li, lj);
        const int idx = gidx(li, lj);
        const Nb9 y = gather9(wy + w, -1, 1, -S, S);
        const double z = f64_cell<AUG>(sW, cpb, k, y, lc, AUG ? sW2[k] : 0.0, w1, idx);
        wz[w] = z;
        __stcg(yout + idx, z);
        const double pn = fma(lc.d, z, Pin[k]);
        Pout[k] = pn;
        sy = fma(z, z, sy);
        sp = fma(pn, pn, sp);
      }
      // the norm partials go to warp 0 (reduced there during the next
      // iteration); the flag publishes the ring cells of y_{m+1}
      s_py[m & 1][t] = sy;
      s_pp[m & 1][t] = sp;
      __syncthreads();
      if (t == 0) {
        __threadfence();
        *(volatile unsigned int*)(flags + b) = (unsigned int)(m + 1);
      }
      ++m;
    }
    fin = s_final;
  }
  if (s_fail) {
    if (t == 0) {
      atomicMax(&ctrl->status, 4);           // AD_ERR_TIMEOUT
      ctrl->stop = 1;
      if (fused && F.totals) atomicMax(&F.totals->status, 4);
    }
    return;
  }
  const double* Pf = sP + ((fin + 1) % 3) * cpb;
  if (fused) {   // u = 1 u + b P, as the axpby kernel forms it
    for (int k = t; k < nc; k += T) {
      const int idx = gidx(k % tw, k / tw);
      F.u[idx] = fma(F.b, Pf[k], 1.0 * F.u[idx]);
    }
  } else {
    double* p = static_cast<double*>(a.p);
    for (int k = t; k < nc; k += T) p[gidx(k % tw, k / tw)] = Pf[k];
  }
  if (b == 0 && t == 0) {
    ctrl->iters = fin + 1;
    ctrl->m = fin + 1;
    ctrl->ynorm2 = s_ty;
    ctrl->pnorm2 = s_tp;
    ctrl->err_est = a.lc[fin].absd;
    atomicMax(&ctrl->status, s_status);
    ctrl->stop = 1;
    if (fused && F.totals) {   // the asynchronous step's report
      AsyncTotals* tt = F.totals;
      const int it = fin + 1;
      tt->iters += it;
      if (F.timed) tt->timed_iters += it;
      tt->series += 1;
      if (s_status > tt->status) tt->status = s_status;
      const double e = s_tp > 0.0 ? a.lc[fin].absd * sqrt(s_ty / s_tp)
                                  : (s_ty > 0.0 ? INFINITY : 0.0);
      if (e > tt->err_est) tt->err_est = e;
    }
  }
}

}  // namespace

namespace {

// Cooperative launch of fn on G blocks of T threads with smem bytes of dynamic
// shared memory, if they fit (shared memory, co-residency); false, with no
// error left pending, if not.  The checks are cached per (device, kernel,
// smem, T): a series is launched on every step, and the attribute and
// occupancy queries would otherwise keep the device waiting for the host.
bool coop_launch(const void* fn, int G, int T, size_t smem, void** params, cudaStream_t s) {
  struct DevInfo {
    int dev, sms, optin;
  };
  struct FnInfo {
    int dev;
    const void* fn;
    size_t static_smem;
    bool ok;
  };
  struct Fit {
    int dev;
    const void* fn;
    size_t smem;
    int T, per_sm;
  };
  static std::mutex mu;
  static std::vector<DevInfo> devs;
  static std::vector<FnInfo> fns;
  static std::vector<Fit> fits;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int per_sm = -1, sms = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    const DevInfo* di = nullptr;
    for (const DevInfo& d : devs)
      if (d.dev == dev) di = &d;
    if (!di) {
      DevInfo d{dev, 0, 0};
      cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
      cudaDeviceGetAttribute(&d.optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      devs.push_back(d);
      di = &devs.back();
    }
    sms = di->sms;
    const FnInfo* fi = nullptr;
    for (const FnInfo& f : fns)
      if (f.dev == dev && f.fn == fn) fi = &f;
    if (!fi) {   // once per kernel: allow all the dynamic shared memory the device has
      cudaFuncAttributes fa{};
      FnInfo f{dev, fn, 0, false};
      if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess && fa.sharedSizeBytes <= (size_t)di->optin) {
        f.static_smem = fa.sharedSizeBytes;
        f.ok = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    di->optin - (int)fa.sharedSizeBytes) == cudaSuccess;
      }
      cudaGetLastError();
      fns.push_back(f);
      fi = &fns.back();
    }
    if (!fi->ok || smem + fi->static_smem > (size_t)di->optin) return false;
    for (const Fit& f : fits)
      if (f.dev == dev && f.fn == fn && f.smem == smem && f.T == T) per_sm = f.per_sm;
    if (per_sm < 0) {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, T, smem) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 0;
      }
      fits.push_back(Fit{dev, fn, smem, T, per_sm});
    }
  }
  if ((long long)per_sm * sms < G) return false;
  if (cudaLaunchCooperativeKernel(fn, dim3(G), dim3(T), params, smem, s) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  ++launch_counter();
  return true;
}

}  // namespace

// Cooperative persistent series (FP64).  Returns 7 (2-D tile kernel), 2 (row
// kernel with neighbour synchronisation) or 1 (grid-barrier kernel) when
// launched, 0 when the grid is too large or the launch is refused (the caller
// then uses the per-iteration path).  The tile kernel runs whenever its tiles
// fit in shared memory, else the row kernel; AD_F64_KERNEL=row forces the row
// kernel, AD_NO_NSYNC the grid-barrier kernel (A/B overrides).
int series_run_persistent(const SeriesArgs& a, unsigned int* gen, const NsyncScratch* ns,
                          cudaStream_t s, const StepFuse* fuse) {
  if (a.prec != 0 || a.g.n > kPersistMaxCells) return 0;
  if (fuse && (fuse->s == 2) != (a.aug != 0)) return 0;
  const long long n = a.g.n;
  const int G = (int)std::min<long long>(152, (n + 31) / 32);
  const unsigned int cpb = (unsigned int)((n + G - 1) / G);
  const int T = persist_threads((int)cpb);
  static const int optin = [] {   // the geometry search below needs the device's limit
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
  }();
  static const bool no_nsync = getenv("AD_NO_NSYNC") != nullptr;
  SeriesArgs args = a;
  args.nblocks = G;
  auto try_launch = [&](void* fn, size_t smem, void** params) -> bool {
    return coop_launch(fn, G, T, smem, params, s);
  };
  // 0 tiles where they fit, 1 rows (AD_F64_KERNEL=row|tile: A/B overrides)
  static const int f64_kernel = [] {
    const char* e = getenv("AD_F64_KERNEL");
    return !e ? 0 : (e[0] == 'r' ? 1 : (e[0] == 't' ? 2 : 0));
  }();
  if (ns && ns->slots && ns->flags && !no_nsync && f64_kernel != 1) {
    // tiles: the fewest cells per block (most blocks), then the shortest perimeter
    const int nx = a.g.nx, ny = a.g.ny;
    TileGeom best{};
    long long best_cells = -1;
    int best_G = 0;
    for (int TX = 1; TX <= std::min(nx, 152); ++TX) {
      const int tw = (nx + TX - 1) / TX;
      const int TXa = (nx + tw - 1) / tw;
      const int TY = std::min(ny, 152 / TX);
      if (TY < 1) break;
      const int th = (ny + TY - 1) / TY;
      const int TYa = (ny + th - 1) / th;
      const int Ga = TXa * TYa;
      if (Ga > kNsyncMaxBlocks) continue;
      const long long cells = (long long)tw * th;
      const size_t smem_t =
          sizeof(double) * ((size_t)cells * (a.aug ? 13 : 12) + 2 * (size_t)(tw + 2) * (th + 2));
      if (smem_t + 12 * 1024 > (size_t)optin) continue;   // + the static shared arrays
      const bool better = best_cells < 0 || cells < best_cells ||
                          (cells == best_cells && tw + th < best.tw + best.th);
      if (better) {
        best = TileGeom{TXa, TYa, tw, th, tw + 2};
        best_cells = cells;
        best_G = Ga;
      }
    }
    // Measured on GB300 (two-stage workloads, us per iteration, tile / row):
    // 64^2 5.9 / 6.5, 128^2 5.4 / 5.2, 192^2 5.6 / 5.7, 256^2 6.3 / 6.7,
    // 384^2 6.9 / 8.8, 512^2 9.0 / 10.9: the tiles win or tie at every size.
    if (best_cells > 0) {
      const size_t smem = sizeof(double) * ((size_t)best_cells * (a.aug ? 13 : 12) +
                                            2 * (size_t)best.S * (best.th + 2));
      void* fn = a.aug ? (void*)leja_tile_f64_k<true> : (void*)leja_tile_f64_k<false>;
      SeriesArgs targs = a;
      targs.nblocks = best_G;
      double* slots = ns->slots;
      unsigned int* flags = ns->flags;
      StepFuse F{};
      if (fuse) F = *fuse;
      void* params[] = {&targs, &best, &slots, &flags, &gen, &F};
      if (coop_launch(fn, best_G, 256, smem, params, s)) return 7;
    }
  }
  if (fuse) return 0;   // only the tile kernel runs whole steps
  if (ns && ns->slots && ns->flags && !no_nsync && G <= kNsyncMaxBlocks) {
    NsyncGeom geo;
    geo.cpb = (int)cpb;
    geo.H = a.g.bc == 0 ? 2 * a.g.nx : a.g.nx + 1;
    geo.W = geo.cpb + 2 * geo.H;
    const long long per_side = (geo.H + (long long)cpb - 1) / cpb + 1;
    const size_t smem = sizeof(double) * ((size_t)cpb * (a.aug ? 12 : 11) + 2 * (size_t)geo.W);
    void* fn = a.aug ? (void*)leja_nsync_f64_k<true> : (void*)leja_nsync_f64_k<false>;
    double* slots = ns->slots;
    unsigned int* flags = ns->flags;
    void* params[] = {&args, &geo, &slots, &flags, &gen};
    if (2 * per_side <= kNsyncMaxNeighbours && try_launch(fn, smem, params)) return 2;
  }
  const size_t smem = (size_t)cpb * (a.aug ? 11 : 10) * sizeof(double);
  void* fn = a.aug ? (void*)leja_persistent_f64_k<true> : (void*)leja_persistent_f64_k<false>;
  unsigned int cpb_arg = cpb;
  void* params[] = {&args, &cpb_arg, &gen};
  return try_launch(fn, smem, params) ? 1 : 0;
}


size_t nsync_slots_bytes() { return sizeof(double) * 2 * (size_t)kMaxIters * kNsyncMaxBlocks; }
int nsync_max_blocks() { return kNsyncMaxBlocks; }

}  // namespace ad
