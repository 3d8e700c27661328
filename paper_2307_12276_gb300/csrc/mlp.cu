// Learned spectral bound: a small multilayer perceptron that predicts, from
// per-field features, the quantities the Leja method otherwise estimates
// with a spectral-bound pass (Section 2 uses Gershgorin discs; power iteration
// is the tighter alternative) and the number of Leja iterations.
//
//   h1 = tanh(x W1 + b1), h2 = tanh(h1 W2 + b2), y = h2 W3 + b3
//
// Inputs are standardised and outputs de-standardised with statistics the
// training call computes on the GPU.  Training runs in FP32 with these
// kernels (forward, backward of the mean squared error, Adam); inference
// runs in BF16 storage with FP32 accumulation.  The network is tiny (about
// 6k parameters) and its batches are at most ~10^4 rows, so plain CUDA-core
// kernels are used: no step is large enough for tensor cores to matter.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "ad_internal.h"
#include "anidiff.h"

namespace {

using namespace ad;

constexpr int kT = 256;

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Y[b, j] = act(sum_i X[b, i] W[i, j] + bias[j]); act 1 = tanh, 0 = identity.
__global__ void dense_fwd_k(const float* X, int B, int nin, const float* W, const float* bias,
                            int nout, int act, float* Y) {
  const long long tot = (long long)B * nout;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < tot;
       q += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(q / nout), j = (int)(q % nout);
    float acc = bias[j];
    const float* x = X + (long long)b * nin;
    for (int i = 0; i < nin; ++i) acc = fmaf(x[i], W[i * nout + j], acc);
    Y[q] = act ? tanhf(acc) : acc;
  }
}

// BF16 inference layer: BF16 inputs and weights, FP32 accumulation.
__global__ void dense_fwd_bf16_k(const __nv_bfloat16* X, int B, int nin, const __nv_bfloat16* W,
                                 const __nv_bfloat16* bias, int nout, int act,
                                 __nv_bfloat16* Yb, float* Yf) {
  const long long tot = (long long)B * nout;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < tot;
       q += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(q / nout), j = (int)(q % nout);
    float acc = __bfloat162float(bias[j]);
    const __nv_bfloat16* x = X + (long long)b * nin;
    for (int i = 0; i < nin; ++i)
      acc = fmaf(__bfloat162float(x[i]), __bfloat162float(W[i * nout + j]), acc);
    const float r = act ? tanhf(acc) : acc;
    if (Yb) Yb[q] = __float2bfloat16(r);
    if (Yf) Yf[q] = r;
  }
}

// dY = (Y - T) / B and per-block partial sums of (Y - T)^2 / (2 B).
__global__ void mse_grad_k(const float* Y, const float* T, long long n, int B, float* dY,
                           float* partial) {
  __shared__ float sh[32];
  float s = 0.f;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const float r = Y[q] - T[q];
    dY[q] = r / B;
    s = fmaf(r, r, s);
  }
  s = wsum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.f;
    v = wsum(v);
    if (threadIdx.x == 0) partial[blockIdx.x] = v / (2.0f * B);
  }
}

// dZ = dA * (1 - A^2) in place (tanh layers).
__global__ void tanh_bwd_k(const float* A, float* dA, long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x)
    dA[q] *= (1.f - A[q] * A[q]);
}

// gW[i, j] = sum_b X[b, i] dZ[b, j] (one block per (i, j), fixed-order tree);
// row i == nin gives the bias gradient (X = 1).
__global__ void dense_wgrad_k(const float* X, const float* dZ, int B, int nin, int nout,
                              float* gW, float* gb) {
  __shared__ float sh[32];
  const int i = blockIdx.x / nout, j = blockIdx.x % nout;
  float s = 0.f;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const float x = (i < nin) ? X[(long long)b * nin + i] : 1.f;
    s = fmaf(x, dZ[(long long)b * nout + j], s);
  }
  s = wsum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.f;
    v = wsum(v);
    if (threadIdx.x == 0) {
      if (i < nin) gW[i * nout + j] = v;
      else gb[j] = v;
    }
  }
}

// dX[b, i] = sum_j dZ[b, j] W[i, j]
__global__ void dense_xgrad_k(const float* dZ, const float* W, int B, int nin, int nout, float* dX) {
  const long long tot = (long long)B * nin;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < tot;
       q += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(q / nin), i = (int)(q % nin);
    float acc = 0.f;
    for (int j = 0; j < nout; ++j) acc = fmaf(dZ[(long long)b * nout + j], W[i * nout + j], acc);
    dX[q] = acc;
  }
}

__global__ void adam_k(float* theta, const float* g, float* m, float* v, int n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.f - b1) * gq;
    const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    theta[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
  }
}

// column mean and standard deviation of a [B][ncol] matrix (one block per column)
__global__ void col_stats_k(const float* X, int B, int ncol, float* mean, float* stdv) {
  __shared__ float sh[32];
  const int c = blockIdx.x;
  float s = 0.f;
  for (int b = threadIdx.x; b < B; b += blockDim.x) s += X[(long long)b * ncol + c];
  s = wsum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  float mu = 0.f;
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.f;
    v = wsum(v);
    if (threadIdx.x == 0) sh[0] = v / B;
  }
  __syncthreads();
  mu = sh[0];
  __syncthreads();
  float q = 0.f;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const float d = X[(long long)b * ncol + c] - mu;
    q = fmaf(d, d, q);
  }
  q = wsum(q);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = q;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.f;
    v = wsum(v);
    if (threadIdx.x == 0) {
      mean[c] = mu;
      stdv[c] = fmaxf(sqrtf(v / B), 1e-6f);   // constant columns keep a unit scale
    }
  }
}

// Z = (X - mean) / std (scale = 1) or X = Z * std + mean (scale = 0)
__global__ void normalize_k(const float* X, long long n, int ncol, const float* mean,
                            const float* stdv, int forward, float* Z) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(q % ncol);
    Z[q] = forward ? (X[q] - mean[c]) / stdv[c] : fmaf(X[q], stdv[c], mean[c]);
  }
}

__global__ void to_bf16_k(const float* x, long long n, __nv_bfloat16* y) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x)
    y[q] = __float2bfloat16(x[q]);
}

// Field features: anisotropy-weighted histogram (16 bins over [-pi/2, pi/2))
// of the principal direction 1/2 atan2(2 Dxy, Dxx - Dyy), the extreme
// eigenvalues max lambda_1, min lambda_2 of D over the cells and, when
// advection fields are given, max |a| over the cells.  out: hist[16],
// lmax, lmin, amax (non-negative floats order like their bit patterns).
__global__ void field_features_k(const double* Dxx, const double* Dxy, const double* Dyy,
                                 const double* ax, const double* ay, long long n, float* out) {
  __shared__ float sh[16];
  __shared__ float smax[kT], smin[kT], samax[kT];
  if (threadIdx.x < 16) sh[threadIdx.x] = 0.f;
  __syncthreads();
  float mx = 0.f, mn = 3.4e38f, am = 0.f;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const float a = (float)Dxx[q], c = (float)Dxy[q], b = (float)Dyy[q];
    const float tr = 0.5f * (a + b), dd = sqrtf(0.25f * (a - b) * (a - b) + c * c);
    const float l1 = tr + dd, l2 = tr - dd;
    mx = fmaxf(mx, l1);
    mn = fminf(mn, l2);
    const float w = (l1 + l2) > 0.f ? (l1 - l2) / (l1 + l2) : 0.f;
    const float th = 0.5f * atan2f(2.f * c, a - b);            // (-pi/2, pi/2]
    int bin = (int)floorf((th + 1.57079633f) * (16.f / 3.14159265f));
    bin = bin < 0 ? 0 : (bin > 15 ? 15 : bin);
    atomicAdd(&sh[bin], w);
    if (ax || ay) {
      const float vx = ax ? (float)ax[q] : 0.f, vy = ay ? (float)ay[q] : 0.f;
      am = fmaxf(am, sqrtf(vx * vx + vy * vy));
    }
  }
  smax[threadIdx.x] = mx;
  smin[threadIdx.x] = mn;
  samax[threadIdx.x] = am;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      smax[threadIdx.x] = fmaxf(smax[threadIdx.x], smax[threadIdx.x + s]);
      smin[threadIdx.x] = fminf(smin[threadIdx.x], smin[threadIdx.x + s]);
      samax[threadIdx.x] = fmaxf(samax[threadIdx.x], samax[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x < 16) atomicAdd(&out[threadIdx.x], sh[threadIdx.x]);
  if (threadIdx.x == 0) {
    atomicMax((int*)&out[16], __float_as_int(smax[0]));
    atomicMin((int*)&out[17], __float_as_int(fmaxf(smin[0], 0.f)));
    atomicMax((int*)&out[18], __float_as_int(samax[0]));
  }
}

// Accumulators of the feature reduction: one small device array shared by
// every call (calls are serialised on the host), so no call allocates.
__device__ float g_feature_acc[19];

int grid_for(long long n) {
  long long g = (n + kT - 1) / kT;
  return (int)(g < 1 ? 1 : (g > 152 * 8 ? 152 * 8 : g));
}

}  // namespace

struct ad_mlp {
  int n_in = 0, h = 0, n_out = 0, np = 0;
  cudaStream_t stream = nullptr;
  float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  float *xm = nullptr, *xs = nullptr, *ym = nullptr, *ys = nullptr;
  __nv_bfloat16* theta16 = nullptr;
  int step = 0;
  // activation workspace for `cap` rows
  int cap = 0;
  float *X = nullptr, *A1 = nullptr, *A2 = nullptr, *Y = nullptr, *T = nullptr, *dY = nullptr,
        *dA = nullptr, *dB = nullptr, *partial = nullptr, *Xin = nullptr;
  __nv_bfloat16 *Xb = nullptr, *A1b = nullptr, *A2b = nullptr;
  float* scratch = nullptr;
};

namespace {

int mfail(int code, const std::string& m) {
  set_error_message(m.c_str());
  return code;
}

#define M_CUDA(expr)                                                                     \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      cudaGetLastError();                                                                \
      return mfail(AD_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));     \
    }                                                                                    \
  } while (0)

// parameter block offsets: W1, b1, W2, b2, W3, b3
void offsets(const ad_mlp* M, int o[6]) {
  o[0] = 0;
  o[1] = o[0] + M->n_in * M->h;
  o[2] = o[1] + M->h;
  o[3] = o[2] + M->h * M->h;
  o[4] = o[3] + M->h;
  o[5] = o[4] + M->h * M->n_out;
}

int ensure_cap(ad_mlp* M, int B) {
  if (B <= M->cap) return AD_OK;
  for (float** p : {&M->X, &M->A1, &M->A2, &M->Y, &M->T, &M->dY, &M->dA, &M->dB, &M->partial,
                    &M->Xin})
    if (*p) { cudaFree(*p); *p = nullptr; }
  for (__nv_bfloat16** p : {&M->Xb, &M->A1b, &M->A2b})
    if (*p) { cudaFree(*p); *p = nullptr; }
  const size_t h = M->h;
  M_CUDA(cudaMalloc(&M->X, sizeof(float) * B * M->n_in));
  M_CUDA(cudaMalloc(&M->Xin, sizeof(float) * B * M->n_in));
  M_CUDA(cudaMalloc(&M->A1, sizeof(float) * B * h));
  M_CUDA(cudaMalloc(&M->A2, sizeof(float) * B * h));
  M_CUDA(cudaMalloc(&M->Y, sizeof(float) * B * M->n_out));
  M_CUDA(cudaMalloc(&M->T, sizeof(float) * B * M->n_out));
  M_CUDA(cudaMalloc(&M->dY, sizeof(float) * B * M->n_out));
  M_CUDA(cudaMalloc(&M->dA, sizeof(float) * B * h));
  M_CUDA(cudaMalloc(&M->dB, sizeof(float) * B * h));
  M_CUDA(cudaMalloc(&M->partial, sizeof(float) * 152 * 8));
  M_CUDA(cudaMalloc(&M->Xb, sizeof(__nv_bfloat16) * B * M->n_in));
  M_CUDA(cudaMalloc(&M->A1b, sizeof(__nv_bfloat16) * B * h));
  M_CUDA(cudaMalloc(&M->A2b, sizeof(__nv_bfloat16) * B * h));
  M->cap = B;
  return AD_OK;
}

// forward (FP32) on normalised inputs already in M->X; outputs normalised in M->Y
void forward_f32(ad_mlp* M, int B) {
  int o[6];
  offsets(M, o);
  const float* th = M->theta;
  cudaStream_t s = M->stream;
  ++launch_counter();
  dense_fwd_k<<<grid_for((long long)B * M->h), kT, 0, s>>>(M->X, B, M->n_in, th + o[0], th + o[1], M->h, 1, M->A1);
  ++launch_counter();
  dense_fwd_k<<<grid_for((long long)B * M->h), kT, 0, s>>>(M->A1, B, M->h, th + o[2], th + o[3], M->h, 1, M->A2);
  ++launch_counter();
  dense_fwd_k<<<grid_for((long long)B * M->n_out), kT, 0, s>>>(M->A2, B, M->h, th + o[4], th + o[5], M->n_out, 0, M->Y);
}

// loss and gradient into M->grad for normalised targets in M->T; returns the
// loss partial count (sum of M->partial[0..nb) is the loss)
int backward(ad_mlp* M, int B) {
  int o[6];
  offsets(M, o);
  cudaStream_t s = M->stream;
  const long long ny = (long long)B * M->n_out;
  const int nb = grid_for(ny);
  ++launch_counter();
  mse_grad_k<<<nb, kT, 0, s>>>(M->Y, M->T, ny, B, M->dY, M->partial);
  float* g = M->grad;
  const float* th = M->theta;
  // layer 3 (linear)
  ++launch_counter();
  dense_wgrad_k<<<(M->h + 1) * M->n_out, kT, 0, s>>>(M->A2, M->dY, B, M->h, M->n_out, g + o[4], g + o[5]);
  ++launch_counter();
  dense_xgrad_k<<<grid_for((long long)B * M->h), kT, 0, s>>>(M->dY, th + o[4], B, M->h, M->n_out, M->dA);
  ++launch_counter();
  tanh_bwd_k<<<grid_for((long long)B * M->h), kT, 0, s>>>(M->A2, M->dA, (long long)B * M->h);
  // layer 2
  ++launch_counter();
  dense_wgrad_k<<<(M->h + 1) * M->h, kT, 0, s>>>(M->A1, M->dA, B, M->h, M->h, g + o[2], g + o[3]);
  ++launch_counter();
  dense_xgrad_k<<<grid_for((long long)B * M->h), kT, 0, s>>>(M->dA, th + o[2], B, M->h, M->h, M->dB);
  ++launch_counter();
  tanh_bwd_k<<<grid_for((long long)B * M->h), kT, 0, s>>>(M->A1, M->dB, (long long)B * M->h);
  // layer 1
  ++launch_counter();
  dense_wgrad_k<<<(M->n_in + 1) * M->h, kT, 0, s>>>(M->X, M->dB, B, M->n_in, M->h, g + o[0], g + o[1]);
  return nb;
}

// normalise X (device, [B][n_in]), run the network, de-standardise into Y (device)
int predict_device(ad_mlp* M, const float* X, int B, int bf16, float* Y) {
  cudaStream_t s = M->stream;
  ++launch_counter();
  normalize_k<<<grid_for((long long)B * M->n_in), kT, 0, s>>>(X, (long long)B * M->n_in, M->n_in, M->xm, M->xs, 1, M->X);
  if (bf16) {
    int o[6];
    offsets(M, o);
    ++launch_counter();
    to_bf16_k<<<grid_for(M->np), kT, 0, s>>>(M->theta, M->np, M->theta16);
    ++launch_counter();
    to_bf16_k<<<grid_for((long long)B * M->n_in), kT, 0, s>>>(M->X, (long long)B * M->n_in, M->Xb);
    const __nv_bfloat16* t = M->theta16;
    ++launch_counter();
    dense_fwd_bf16_k<<<grid_for((long long)B * M->h), kT, 0, s>>>(M->Xb, B, M->n_in, t + o[0], t + o[1], M->h, 1, M->A1b, nullptr);
    ++launch_counter();
    dense_fwd_bf16_k<<<grid_for((long long)B * M->h), kT, 0, s>>>(M->A1b, B, M->h, t + o[2], t + o[3], M->h, 1, M->A2b, nullptr);
    ++launch_counter();
    dense_fwd_bf16_k<<<grid_for((long long)B * M->n_out), kT, 0, s>>>(M->A2b, B, M->h, t + o[4], t + o[5], M->n_out, 0, nullptr, M->Y);
  } else {
    forward_f32(M, B);
  }
  ++launch_counter();
  normalize_k<<<grid_for((long long)B * M->n_out), kT, 0, s>>>(M->Y, (long long)B * M->n_out, M->n_out, M->ym, M->ys, 0, Y);
  M_CUDA(cudaGetLastError());
  return AD_OK;
}

}  // namespace

namespace ad {

int field_features(long long n, double dxmin, const double* Dxx, const double* Dxy,
                   const double* Dyy, const double* ax, const double* ay, double max_a,
                   cudaStream_t s, float* out21) {
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  const float init[19] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0.f, 3.0e38f, 0.f};
  if (cudaMemcpyToSymbolAsync(g_feature_acc, init, sizeof(init), 0, cudaMemcpyHostToDevice, s) !=
      cudaSuccess)
    return 1;
  float* d = nullptr;
  if (cudaGetSymbolAddress((void**)&d, g_feature_acc) != cudaSuccess) return 1;
  ++launch_counter();
  field_features_k<<<grid_for(n), kT, 0, s>>>(Dxx, Dxy, Dyy, ax, ay, n, d);
  float h[19];
  if (cudaMemcpyFromSymbolAsync(h, g_feature_acc, sizeof(h), 0, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return 1;
  double tot = 0.0;
  for (int k = 0; k < 16; ++k) tot += h[k];
  const double amax = (ax || ay) ? (double)h[18] : max_a;
  out21[0] = (float)std::log(std::max((double)h[16], 1e-30));          // log D_par
  out21[1] = (float)std::log(std::max((double)h[17], 1e-30));          // log D_perp
  out21[2] = (float)std::log(amax + 1e-6);                              // log max|a|
  out21[3] = (float)std::log(dxmin);                                    // log dx
  out21[4] = 0.f;                                                       // log dt: per call
  for (int k = 0; k < 16; ++k) out21[5 + k] = tot > 0 ? (float)(h[k] / tot) : 1.f / 16.f;
  return 0;
}

int mlp_predict_host(ad_mlp* M, const float* X, int B, int bf16, float* Y) {
  if (!M || !X || !Y || B < 1) return mfail(AD_ERR_INVALID, "bad arguments");
  if (M->n_in != kFeatures || M->n_out != 2)
    return mfail(AD_ERR_INVALID, "the bound model must have 21 inputs and 2 outputs");
  {
    const int r = ensure_cap(M, B);
    if (r != AD_OK) return r;
  }
  cudaStream_t s = M->stream;
  M_CUDA(cudaMemcpyAsync(M->Xin, X, sizeof(float) * B * M->n_in, cudaMemcpyHostToDevice, s));
  {
    const int r = predict_device(M, M->Xin, B, bf16, M->T);
    if (r != AD_OK) return r;
  }
  M_CUDA(cudaMemcpyAsync(Y, M->T, sizeof(float) * B * M->n_out, cudaMemcpyDeviceToHost, s));
  M_CUDA(cudaStreamSynchronize(s));
  return AD_OK;
}

}  // namespace ad

extern "C" {

int ad_mlp_create(int n_in, int n_hidden, int n_out, unsigned long long seed, void* stream,
                  ad_mlp** out) {
  set_error_message("");
  if (!out || n_in < 1 || n_hidden < 1 || n_out < 1 || n_in > 4096 || n_hidden > 4096 || n_out > 4096)
    return mfail(AD_ERR_INVALID, "bad MLP sizes");
  ad_mlp* M = new ad_mlp();
  M->n_in = n_in;
  M->h = n_hidden;
  M->n_out = n_out;
  M->stream = (cudaStream_t)stream;
  M->np = n_in * n_hidden + n_hidden + n_hidden * n_hidden + n_hidden + n_hidden * n_out + n_out;
  const size_t bytes = sizeof(float) * M->np;
  bool ok = cudaMalloc(&M->theta, bytes) == cudaSuccess && cudaMalloc(&M->grad, bytes) == cudaSuccess &&
            cudaMalloc(&M->m, bytes) == cudaSuccess && cudaMalloc(&M->v, bytes) == cudaSuccess &&
            cudaMalloc(&M->theta16, sizeof(__nv_bfloat16) * M->np) == cudaSuccess &&
            cudaMalloc(&M->xm, sizeof(float) * n_in) == cudaSuccess &&
            cudaMalloc(&M->xs, sizeof(float) * n_in) == cudaSuccess &&
            cudaMalloc(&M->ym, sizeof(float) * n_out) == cudaSuccess &&
            cudaMalloc(&M->ys, sizeof(float) * n_out) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    ad_mlp_destroy(M);
    return mfail(AD_ERR_NOMEM, "MLP allocation failed");
  }
  // Glorot-uniform weights from SplitMix64, zero biases; identity normalisation
  std::vector<float> h(M->np, 0.f);
  int o[6];
  offsets(M, o);
  unsigned long long k = 0;
  auto uni = [&]() {
    unsigned long long z = seed + (++k) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1.0p-53;
  };
  const int fan[3][2] = {{n_in, n_hidden}, {n_hidden, n_hidden}, {n_hidden, n_out}};
  for (int l = 0; l < 3; ++l) {
    const double lim = std::sqrt(6.0 / (fan[l][0] + fan[l][1]));
    for (int q = 0; q < fan[l][0] * fan[l][1]; ++q) h[o[2 * l] + q] = (float)((2.0 * uni() - 1.0) * lim);
  }
  std::vector<float> zeros(std::max(n_in, n_out), 0.f), ones(std::max(n_in, n_out), 1.f);
  cudaMemcpy(M->theta, h.data(), bytes, cudaMemcpyHostToDevice);
  cudaMemset(M->m, 0, bytes);
  cudaMemset(M->v, 0, bytes);
  cudaMemcpy(M->xm, zeros.data(), sizeof(float) * n_in, cudaMemcpyHostToDevice);
  cudaMemcpy(M->xs, ones.data(), sizeof(float) * n_in, cudaMemcpyHostToDevice);
  cudaMemcpy(M->ym, zeros.data(), sizeof(float) * n_out, cudaMemcpyHostToDevice);
  cudaMemcpy(M->ys, ones.data(), sizeof(float) * n_out, cudaMemcpyHostToDevice);
  if (cudaGetLastError() != cudaSuccess) {
    ad_mlp_destroy(M);
    return mfail(AD_ERR_CUDA, "MLP initialisation failed");
  }
  *out = M;
  return AD_OK;
}

int ad_mlp_destroy(ad_mlp* M) {
  if (!M) return AD_OK;
  if (M->stream) cudaStreamSynchronize(M->stream);
  for (float* p : {M->theta, M->grad, M->m, M->v, M->xm, M->xs, M->ym, M->ys, M->X, M->A1, M->A2,
                   M->Y, M->T, M->dY, M->dA, M->dB, M->partial, M->Xin})
    if (p) cudaFree(p);
  for (__nv_bfloat16* p : {M->theta16, M->Xb, M->A1b, M->A2b})
    if (p) cudaFree(p);
  delete M;
  return AD_OK;
}

int ad_mlp_num_params(const ad_mlp* M, int* n) {
  if (!M || !n) return mfail(AD_ERR_INVALID, "NULL argument");
  *n = M->np;
  return AD_OK;
}

int ad_mlp_params(ad_mlp* M, float* host, int n, int set) {
  set_error_message("");
  if (!M || !host || n != M->np) return mfail(AD_ERR_INVALID, "parameter count mismatch");
  if (set) {
    M_CUDA(cudaMemcpy(M->theta, host, sizeof(float) * n, cudaMemcpyHostToDevice));
    M->step = 0;
    M_CUDA(cudaMemset(M->m, 0, sizeof(float) * n));
    M_CUDA(cudaMemset(M->v, 0, sizeof(float) * n));
  } else {
    M_CUDA(cudaMemcpy(host, M->theta, sizeof(float) * n, cudaMemcpyDeviceToHost));
  }
  return AD_OK;
}

int ad_mlp_normalization(ad_mlp* M, float* x_mean, float* x_std, float* y_mean, float* y_std,
                         int set) {
  set_error_message("");
  if (!M || !x_mean || !x_std || !y_mean || !y_std) return mfail(AD_ERR_INVALID, "NULL argument");
  const cudaMemcpyKind k = set ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
  const size_t ni = sizeof(float) * M->n_in, no = sizeof(float) * M->n_out;
  M_CUDA(cudaMemcpy(set ? (void*)M->xm : (void*)x_mean, set ? (void*)x_mean : (void*)M->xm, ni, k));
  M_CUDA(cudaMemcpy(set ? (void*)M->xs : (void*)x_std, set ? (void*)x_std : (void*)M->xs, ni, k));
  M_CUDA(cudaMemcpy(set ? (void*)M->ym : (void*)y_mean, set ? (void*)y_mean : (void*)M->ym, no, k));
  M_CUDA(cudaMemcpy(set ? (void*)M->ys : (void*)y_std, set ? (void*)y_std : (void*)M->ys, no, k));
  return AD_OK;
}

int ad_mlp_loss_grad(ad_mlp* M, const float* X, const float* Y, int B, float* loss,
                     float* host_grad) {
  set_error_message("");
  if (!M || !X || !Y || B < 1) return mfail(AD_ERR_INVALID, "bad arguments");
  {
    const int r = ensure_cap(M, B);
    if (r != AD_OK) return r;
  }
  cudaStream_t s = M->stream;
  ++launch_counter();
  normalize_k<<<grid_for((long long)B * M->n_in), kT, 0, s>>>(X, (long long)B * M->n_in, M->n_in, M->xm, M->xs, 1, M->X);
  ++launch_counter();
  normalize_k<<<grid_for((long long)B * M->n_out), kT, 0, s>>>(Y, (long long)B * M->n_out, M->n_out, M->ym, M->ys, 1, M->T);
  forward_f32(M, B);
  const int nb = backward(M, B);
  std::vector<float> part(nb);
  M_CUDA(cudaMemcpyAsync(part.data(), M->partial, sizeof(float) * nb, cudaMemcpyDeviceToHost, s));
  if (host_grad)
    M_CUDA(cudaMemcpyAsync(host_grad, M->grad, sizeof(float) * M->np, cudaMemcpyDeviceToHost, s));
  M_CUDA(cudaStreamSynchronize(s));
  double L = 0.0;
  for (float p : part) L += p;
  if (loss) *loss = (float)L;
  return AD_OK;
}

int ad_mlp_train(ad_mlp* M, const float* X, const float* Y, int B, int epochs, float lr,
                 int fit_normalization, float* final_loss) {
  set_error_message("");
  if (!M || !X || !Y || B < 1 || epochs < 0 || !(lr > 0)) return mfail(AD_ERR_INVALID, "bad arguments");
  {
    const int r = ensure_cap(M, B);
    if (r != AD_OK) return r;
  }
  cudaStream_t s = M->stream;
  if (fit_normalization) {
    ++launch_counter();
    col_stats_k<<<M->n_in, kT, 0, s>>>(X, B, M->n_in, M->xm, M->xs);
    ++launch_counter();
    col_stats_k<<<M->n_out, kT, 0, s>>>(Y, B, M->n_out, M->ym, M->ys);
  }
  ++launch_counter();
  normalize_k<<<grid_for((long long)B * M->n_in), kT, 0, s>>>(X, (long long)B * M->n_in, M->n_in, M->xm, M->xs, 1, M->X);
  ++launch_counter();
  normalize_k<<<grid_for((long long)B * M->n_out), kT, 0, s>>>(Y, (long long)B * M->n_out, M->n_out, M->ym, M->ys, 1, M->T);
  int nb = 1;
  for (int e = 0; e < epochs; ++e) {
    forward_f32(M, B);
    nb = backward(M, B);
    ++M->step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)M->step), c2 = 1.f - std::pow(b2, (float)M->step);
    ++launch_counter();
    adam_k<<<grid_for(M->np), kT, 0, s>>>(M->theta, M->grad, M->m, M->v, M->np, lr, b1, b2, 1e-8f, c1, c2);
  }
  M_CUDA(cudaGetLastError());
  if (final_loss) {
    forward_f32(M, B);
    nb = backward(M, B);
    std::vector<float> part(nb);
    M_CUDA(cudaMemcpyAsync(part.data(), M->partial, sizeof(float) * nb, cudaMemcpyDeviceToHost, s));
    M_CUDA(cudaStreamSynchronize(s));
    double L = 0.0;
    for (float p : part) L += p;
    *final_loss = (float)L;
  }
  M_CUDA(cudaStreamSynchronize(s));
  return AD_OK;
}

int ad_mlp_predict(ad_mlp* M, const float* X, int B, int bf16, float* Y) {
  set_error_message("");
  if (!M || !X || !Y || B < 1) return mfail(AD_ERR_INVALID, "bad arguments");
  {
    const int r = ensure_cap(M, B);
    if (r != AD_OK) return r;
  }
  {
    const int r = predict_device(M, X, B, bf16, Y);
    if (r != AD_OK) return r;
  }
  M_CUDA(cudaStreamSynchronize(M->stream));
  return AD_OK;
}

int ad_field_features(const ad_grid* grid, const double* Dxx, const double* Dxy,
                      const double* Dyy, double max_a, double dt, void* stream, float* out21) {
  set_error_message("");
  if (!grid || !Dxx || !Dxy || !Dyy || !out21 || grid->nx < 1 || grid->ny < 1 || !(dt > 0))
    return mfail(AD_ERR_INVALID, "bad arguments");
  const double dx = (grid->x1 - grid->x0) / grid->nx, dy = (grid->y1 - grid->y0) / grid->ny;
  const long long n = (long long)grid->nx * grid->ny;
  if (field_features(n, std::min(dx, dy), Dxx, Dxy, Dyy, nullptr, nullptr, max_a,
                     (cudaStream_t)stream, out21) != 0)
    return mfail(AD_ERR_CUDA, "field features kernel failed");
  out21[4] = (float)std::log(dt);                                       // log dt
  return AD_OK;
}

}  // extern "C"
