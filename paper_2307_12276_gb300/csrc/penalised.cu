// Kernels of the penalised IMEX step (the alternative method Section 4 names):
// conjugate gradients on M = I - c L, with L the operator of Eq. anidiff for
// the unit isotropic tensor (the 5-point Laplacian of the flux form, same
// boundary rule: periodic wrap, or zero Dirichlet through odd-reflection
// ghosts, u_ghost = -u_C).  M is symmetric positive definite for c >= 0.
//
// The CG scalars stay on the device: scal[1] = <p, Mp>, scal[2] = <r, r> of
// the current iteration, scal[3] = <r, r> after the update.  One iteration is
// matvec (+ dot partials) -> reduce -> update (+ dot partials) -> reduce ->
// direction; the host reads scal[3] only every few iterations to test
// convergence.  A zero denominator gives a zero step (a converged residual
// stays converged instead of turning into NaN).
#include <cstring>
#include <mutex>

#include "ad_internal.h"

namespace ad {
namespace {

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sm[kThreads];
  sm[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  return sm[0];
}

// (L u) at cell (i, j): (u_W - 2 u_C + u_E) / dx^2 + (u_S - 2 u_C + u_N) / dy^2
__device__ __forceinline__ double lap5(const double* __restrict__ u, long long idx, int i, int j,
                                       const GridDev& g, double idx2, double idy2) {
  const double c = u[idx];
  double w, e, s, n;
  if (g.bc == 0) {
    w = u[idx - i + (i ? i - 1 : g.nx - 1)];
    e = u[idx - i + (i + 1 < g.nx ? i + 1 : 0)];
    s = u[(long long)(j ? j - 1 : g.ny - 1) * g.nx + i];
    n = u[(long long)(j + 1 < g.ny ? j + 1 : 0) * g.nx + i];
  } else {
    w = i ? u[idx - 1] : -c;
    e = i + 1 < g.nx ? u[idx + 1] : -c;
    s = j ? u[idx - g.nx] : -c;
    n = j + 1 < g.ny ? u[idx + g.nx] : -c;
  }
  return ((w - 2.0 * c) + e) * idx2 + ((s - 2.0 * c) + n) * idy2;
}

// Mp = p - c L p; partials of <p, Mp>.  Block 0 first moves scal[3] (the
// residual norm of the last update) into scal[2].
__global__ void pen_matvec_k(GridDev g, double idx2, double idy2, double c,
                             const double* __restrict__ p, double* __restrict__ Mp,
                             double* __restrict__ partials, double* scal) {
  if (blockIdx.x == 0 && threadIdx.x == 0) scal[2] = scal[3];
  double acc = 0.0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < g.n;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % g.nx), j = (int)(idx / g.nx);
    const double v = p[idx] - c * lap5(p, idx, i, j, g, idx2, idy2);
    Mp[idx] = v;
    acc = fma(p[idx], v, acc);
  }
  const double b = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = b;
}

// alpha = <r,r> / <p,Mp>; x += alpha p; r -= alpha Mp; partials of <r, r>.
__global__ void pen_update_k(long long n, const double* scal, double* __restrict__ x,
                             double* __restrict__ r, const double* __restrict__ p,
                             const double* __restrict__ Mp, double* __restrict__ partials) {
  const double rr = scal[2], pMp = scal[1];
  const double alpha = pMp != 0.0 ? rr / pMp : 0.0;
  double acc = 0.0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    x[idx] = fma(alpha, p[idx], x[idx]);
    const double rv = fma(-alpha, Mp[idx], r[idx]);
    r[idx] = rv;
    acc = fma(rv, rv, acc);
  }
  const double b = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = b;
}

// p = r + (<r,r>_new / <r,r>_old) p
__global__ void pen_direction_k(long long n, const double* scal, const double* __restrict__ r,
                                double* __restrict__ p) {
  const double old = scal[2], nw = scal[3];
  const double beta = old != 0.0 ? nw / old : 0.0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x)
    p[idx] = fma(beta, p[idx], r[idx]);
}

// -lambda_max(D) per cell, block minimum (the caller reduces with min)
// Order-preserving map of doubles onto unsigned 64-bit integers (IEEE 754
// bit patterns: flip all bits of negatives, the sign bit of the rest), so
// that an integer atomicMax gives the largest double.
__device__ __forceinline__ unsigned long long order_key(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// max over cells of lambda_max(D) = (Dxx + Dyy)/2 + sqrt(((Dxx - Dyy)/2)^2 + Dxy^2),
// folded into one device word by atomicMax on its order key (no scratch).
__device__ unsigned long long g_lambda_max_key;

__global__ void lambda_max_k(long long n, const double* __restrict__ Dxx,
                             const double* __restrict__ Dxy, const double* __restrict__ Dyy) {
  __shared__ double sm[kThreads];
  double mx = -1e308;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const double a = Dxx[idx], b = Dxy[idx], d = Dyy[idx];
    const double h = 0.5 * (a - d);
    mx = fmax(mx, 0.5 * (a + d) + sqrt(h * h + b * b));
  }
  sm[threadIdx.x] = mx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(&g_lambda_max_key, order_key(sm[0]));
}

}  // namespace

int lambda_max_reduce(long long n, const double* Dxx, const double* Dxy, const double* Dyy,
                      int nblocks, cudaStream_t s, double* out) {
  // one word of device state shared by every call: host threads are serialised
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  const unsigned long long lowest = 0ull;           // below the key of every double
  if (cudaMemcpyToSymbolAsync(g_lambda_max_key, &lowest, sizeof(lowest), 0,
                              cudaMemcpyHostToDevice, s) != cudaSuccess)
    return 1;
  ++launch_counter();
  lambda_max_k<<<nblocks, kThreads, 0, s>>>(n, Dxx, Dxy, Dyy);
  unsigned long long key = 0ull;
  if (cudaMemcpyFromSymbolAsync(&key, g_lambda_max_key, sizeof(key), 0, cudaMemcpyDeviceToHost,
                                s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return 1;
  const unsigned long long b = (key >> 63) ? (key & 0x7fffffffffffffffull) : ~key;
  std::memcpy(out, &b, sizeof(double));
  return 0;
}

void penalty_cg_iteration(const GridDev& g, double dx, double dy, double c, double* x, double* r,
                          double* p, double* Mp, double* partials, int nblocks, double* scal,
                          cudaStream_t s) {
  launch_counter() += 3;      // the two reductions count themselves
  pen_matvec_k<<<nblocks, kThreads, 0, s>>>(g, 1.0 / (dx * dx), 1.0 / (dy * dy), c, p, Mp,
                                            partials, scal);
  reduce_partials(partials, nblocks, 0, scal + 1, s);
  pen_update_k<<<nblocks, kThreads, 0, s>>>(g.n, scal, x, r, p, Mp, partials);
  reduce_partials(partials, nblocks, 0, scal + 3, s);
  pen_direction_k<<<nblocks, kThreads, 0, s>>>(g.n, scal, r, p);
}

}  // namespace ad
