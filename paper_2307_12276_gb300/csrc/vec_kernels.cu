// Streaming vector kernels and the device-side control of the Leja series:
// series start (y_0, p_0 = d_0 y_0), the per-iteration control kernel
// (deterministic norm reduction + stopping rule of the Newton series,
// Section 2), axpby, norms, the SplitMix64 start vector of the power
// iteration, and the Gram-Schmidt kernels of the GMRES comparison solver.
#include "ad_internal.h"

namespace ad {

namespace {

template <typename T> struct Vec;
template <> struct Vec<double> { using type = double; };
template <> struct Vec<float> { using type = float; };

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// deterministic block sum, result in thread 0
__device__ __forceinline__ double block_sum(double a) {
  __shared__ double sa[32];
  a = warp_sum(a);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sa[wid] = a;
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    a = lane < nw ? sa[lane] : 0.0;
    a = warp_sum(a);
  }
  return a;
}

template <typename T>
__global__ void series_init_k(SeriesArgs a, const T* src, double d0, int force, int max_iters,
                              double tol) {
  T* y = static_cast<T*>(a.y[0]);
  T* p = static_cast<T*>(a.p);
  const long long n = a.g.n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const T v = src ? src[i] : T(0);
    y[i] = v;
    p[i] = (T)d0 * v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Ctrl* c = a.ctrl;
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
  }
}

// z = a x + b y in the storage type's own arithmetic (no FP64 for float data:
// FP64 is the scarce pipe on this GPU).
template <typename T>
__global__ void axpby_k(long long n, T a, const T* x, T b, const T* y, T* z) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    T r = T(0);
    if (x) r = a * x[i];
    if (y) r = fma(b, y[i], r);
    z[i] = r;
  }
}

template <typename T>
__global__ void norm2_k(long long n, const T* x, double* partials) {
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = (double)x[i];
    s = fma(v, v, s);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void reduce_k(const double* partials, int nb, int op, double* out) {
  __shared__ double sm[kThreads];
  double acc = (op == 1) ? 1e308 : 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
    acc = (op == 1) ? fmin(acc, partials[b]) : acc + partials[b];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      sm[threadIdx.x] = (op == 1) ? fmin(sm[threadIdx.x], sm[threadIdx.x + s])
                                  : sm[threadIdx.x] + sm[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = (op == 2) ? sqrt(sm[0]) : sm[0];
}

template <typename T>
__global__ void scale_by_inv_k(long long n, const T* y, const double* sc, T* x) {
  const double s = sc[0];
  const double inv = s != 0.0 ? 1.0 / s : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] = (T)((double)y[i] * inv);
}

// SplitMix64 (Steele, Lea & Flood 2014), counter form: output k mixes
// seed + (k+1) * 0x9E3779B97F4A7C15; mapped to [-0.5, 0.5) by (z >> 11) 2^-53 - 1/2.
template <typename T>
__global__ void splitmix_k(long long n, unsigned long long seed, T* x) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = seed + (unsigned long long)(k + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z = z ^ (z >> 31);
    x[k] = (T)((double)(z >> 11) * 0x1.0p-53 - 0.5);
  }
}

// ---------------------------------------------------------------- GMRES helpers
// partials[i * nb + block] = sum over the block's cells of V_i * w, i < k.
__global__ void multi_dot_k(long long n, const double* __restrict__ V, long long ldv, int k,
                            const double* __restrict__ w, double* partials) {
  extern __shared__ double sh[];  // [k][32] warp sums
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i0 = 0; i0 < k; i0 += 8) {
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int cnt = (k - i0) < 8 ? (k - i0) : 8;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
      const double wc = w[c];
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (q < cnt) acc[q] = fma(V[(long long)(i0 + q) * ldv + c], wc, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (q >= cnt) break;
      const double v = warp_sum(acc[q]);
      if (lane == 0) sh[q * 32 + wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
      double s = 0.0;
      for (int u = 0; u < nw; ++u) s += sh[threadIdx.x * 32 + u];
      partials[(long long)(i0 + threadIdx.x) * gridDim.x + blockIdx.x] = s;
    }
    __syncthreads();
  }
}

__global__ void multi_dot_finalize_k(const double* partials, int nb, int k, double* h) {
  // one block per row i; fixed-order reduction
  const int i = blockIdx.x;
  if (i >= k) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += partials[(long long)i * nb + b];
  s = block_sum(s);
  if (threadIdx.x == 0) h[i] = s;
}

__global__ void multi_axpy_norm_k(long long n, const double* __restrict__ V, long long ldv, int k,
                                  const double* __restrict__ h, double* w, double* partials) {
  double s2 = 0.0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    double r = w[c];
    for (int i = 0; i < k; ++i) r = fma(-h[i], V[(long long)i * ldv + c], r);
    w[c] = r;
    s2 = fma(r, r, s2);
  }
  s2 = block_sum(s2);
  if (threadIdx.x == 0) partials[blockIdx.x] = s2;
}

__global__ void multi_axpy_add_k(long long n, const double* __restrict__ V, long long ldv, int k,
                                 const double* __restrict__ y, double* x) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    double r = x[c];
    for (int i = 0; i < k; ++i) r = fma(y[i], V[(long long)i * ldv + c], r);
    x[c] = r;
  }
}

}  // namespace

long long& launch_counter() {
  static thread_local long long count = 0;
  return count;
}

void series_init(const SeriesArgs& a, const void* src, double d0, int force, int max_iters,
                 double tol, cudaStream_t s) {
  const int nb = stream_blocks(a.g.n);
  ++launch_counter();
  if (a.prec == 0)
    series_init_k<double><<<nb, kThreads, 0, s>>>(a, static_cast<const double*>(src), d0, force,
                                                  max_iters, tol);
  else
    series_init_k<float><<<nb, kThreads, 0, s>>>(a, static_cast<const float*>(src), d0, force,
                                                 max_iters, tol);
}

void axpby(int prec, long long n, double a, const void* x, double b, const void* y, void* z,
           cudaStream_t s) {
  const int nb = stream_blocks(n);
  ++launch_counter();
  if (prec == 0)
    axpby_k<double><<<nb, kThreads, 0, s>>>(n, a, static_cast<const double*>(x), b,
                                            static_cast<const double*>(y), static_cast<double*>(z));
  else
    axpby_k<float><<<nb, kThreads, 0, s>>>(n, (float)a, static_cast<const float*>(x), (float)b,
                                           static_cast<const float*>(y), static_cast<float*>(z));
}

void norm2_partials(int prec, long long n, const void* x, double* partials, int nblocks,
                    cudaStream_t s) {
  ++launch_counter();
  if (prec == 0)
    norm2_k<double><<<nblocks, kThreads, 0, s>>>(n, static_cast<const double*>(x), partials);
  else
    norm2_k<float><<<nblocks, kThreads, 0, s>>>(n, static_cast<const float*>(x), partials);
}

void reduce_partials(const double* partials, int nblocks, int op, double* out, cudaStream_t s) {
  ++launch_counter();
  reduce_k<<<1, kThreads, 0, s>>>(partials, nblocks, op, out);
}

void scale_by_inv(int prec, long long n, const void* y, const double* dev_scalar, void* x,
                  cudaStream_t s) {
  const int nb = stream_blocks(n);
  ++launch_counter();
  if (prec == 0)
    scale_by_inv_k<double><<<nb, kThreads, 0, s>>>(n, static_cast<const double*>(y), dev_scalar,
                                                   static_cast<double*>(x));
  else
    scale_by_inv_k<float><<<nb, kThreads, 0, s>>>(n, static_cast<const float*>(y), dev_scalar,
                                                  static_cast<float*>(x));
}

void splitmix_fill(int prec, long long n, unsigned long long seed, void* x, cudaStream_t s) {
  const int nb = stream_blocks(n);
  if (prec == 0) {
    ++launch_counter();
    splitmix_k<double><<<nb, kThreads, 0, s>>>(n, seed, static_cast<double*>(x));
  }
  else {
    ++launch_counter();
    splitmix_k<float><<<nb, kThreads, 0, s>>>(n, seed, static_cast<float*>(x));
  }
}

void multi_dot_partials(long long n, const double* V, long long ldv, int k, const double* w,
                        double* partials, int nblocks, cudaStream_t s) {
  ++launch_counter();
  multi_dot_k<<<nblocks, kThreads, 8 * 32 * sizeof(double), s>>>(n, V, ldv, k, w, partials);
}

void multi_dot_finalize(const double* partials, int nblocks, int k, double* h, cudaStream_t s) {
  ++launch_counter();
  multi_dot_finalize_k<<<k, kThreads, 0, s>>>(partials, nblocks, k, h);
}

void multi_axpy_norm(long long n, const double* V, long long ldv, int k, const double* h,
                     double* w, double* partials, int nblocks, cudaStream_t s) {
  ++launch_counter();
  multi_axpy_norm_k<<<nblocks, kThreads, 0, s>>>(n, V, ldv, k, h, w, partials);
}

void multi_axpy_add(long long n, const double* V, long long ldv, int k, const double* y, double* x,
                    cudaStream_t s) {
  ++launch_counter();
  multi_axpy_add_k<<<stream_blocks(n), kThreads, 0, s>>>(n, V, ldv, k, y, x);
}

}  // namespace ad
