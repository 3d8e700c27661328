// Internal declarations shared by the library's translation units.
// Not part of the public ABI (that is include/anidiff.h).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace ad {

constexpr int kMaxIters = 500;      // cap on Leja iterations per series
constexpr int kMaxSources = 16;     // separable source terms per step
constexpr int kThreads = 256;       // threads per block of the streaming kernels
constexpr int kMaxGmres = 200;      // largest GMRES restart length

// Per-iteration scalars of the Newton series, uploaded once per series
// configuration.  Iteration m (0-based) produces term m+1.
struct LejaCoef {
  double xi;      // xi_m
  double d;       // d_{m+1}
  double absd;    // |d_{m+1}|
  double e1;      // eta1_m / gamma  (augmented coupling with w2)
  double e2;      // eta2_m / gamma  (augmented coupling with w1)
  double pad[3];
};

// Device-side control block of one Newton series.
struct Ctrl {
  int m;          // iteration about to run (0-based)
  int stop;       // 1 once the series has finished
  int iters;      // iterations done
  int status;     // 0 ok, 3 not converged
  int force;      // > 0: exact iteration count, no stopping test
  int max_iters;
  unsigned int ticket;  // blocks of the running iteration that have finished
  unsigned int gen;     // grid-barrier generation of the persistent series kernel;
                        // batched persistent iteration: passes the slice has completed
  double tol;
  double err_est;
  double ynorm2;  // last ||y_{m+1}||^2
  double pnorm2;  // last ||p_{m+1}||^2
};

struct Sources {
  const void* g[kMaxSources];
  double a[kMaxSources];    // coefficients of the first combination
  double b[kMaxSources];    // coefficients of the second combination
  int n;
};

struct GridDev {
  int nx, ny, bc;
  long long n;
};

// ---------------------------------------------------------------- FP64 path
// W: 9 planes [9][n] of folded stencil weights, slot k = (dj+1)*3 + (di+1).
void pack_weights_f64(const GridDev& g, double dx, double dy, const double* Dxx, const double* Dxy,
                      const double* Dyy, const double* ax, const double* ay, double ax_c,
                      double ay_c, double* W, cudaStream_t s);
void scale_weights_f64(const GridDev& g, const double* W, double c, double gamma, double* Ws,
                       cudaStream_t s);
void gershgorin_partials_f64(const GridDev& g, const double* W, double* partials, int nblocks,
                             cudaStream_t s);
// out1 = A u + sum_k a_k g_k ; if out2: out2 = sum_k b_k g_k.
void apply_f64(const GridDev& g, const double* W, const double* u, double* out1, double* out2,
               const Sources& src, cudaStream_t s);

// ---------------------------------------------------------------- FP32 storage path
// F: packed fields float [3][n] = Dxx/(2 dx^2), Dyy/(2 dy^2), Dxy/(8 dx dy) (the factors 1/2
// of the face means are folded in), plus [2][n] = ax/(4 dx), ay/(4 dy) when advection is a field.
// adv: 0 none, 1 constant (abx = ax/(2 dx), aby = ay/(2 dy)), 2 fields.
void pack_fields_f32(const GridDev& g, double dx, double dy, const double* Dxx, const double* Dxy,
                     const double* Dyy, const double* ax, const double* ay, double ax_c,
                     double ay_c, float* F, cudaStream_t s);
void gershgorin_partials_f32(const GridDev& g, const float* F, int adv, float abx, float aby,
                             double* partials, int nblocks, cudaStream_t s);
void apply_f32(const GridDev& g, const float* F, int adv, float abx, float aby, const float* u,
               float* out1, float* out2, const Sources& src, cudaStream_t s);
void apply_shifted_f64(const GridDev& g, const double* W, const double* u, double* out, double s0,
                       double s1, cudaStream_t s);

// ---------------------------------------------------------------- Leja series
// Tensor maps of the FP32 two-iteration kernel's TMA row loader: the two
// Newton-basis buffers, p and the three coefficient fields, each [ny][nx]
// float32 with a box of 128 columns x 1 row (zero-Dirichlet grids, nx % 4 == 0).
struct PairTmaMaps {     // aligned as CUtensorMap
  CUtensorMap y[2];
  CUtensorMap p, xx, yy, xy;
};
// Encode the maps (false when the driver offers no encoder or refuses a map).
bool encode_pair_tma(const GridDev& g, const void* y0, const void* y1, const void* p,
                     const float* F, PairTmaMaps* out);

struct SeriesArgs {
  GridDev g;
  int prec;                 // 0 fp64, 1 fp32
  const void* coef;         // Ws (fp64) or F (fp32)
  double c, gamma;          // spectral shift/scale (fp32 path applies them per cell)
  void* y[2];               // ping-pong Newton basis vectors
  void* p;                  // partial sum
  const void* w1;           // augmented couplings (may be null)
  const void* w2;
  const LejaCoef* lc;       // device [kMaxIters]
  Ctrl* ctrl;               // device
  double* partials;         // device [2 * nblocks]
  int nblocks;
  int aug;
  int adv;                  // fp32 advection mode (see pack_fields_f32)
  float abx, aby;
  unsigned long long handle;  // CUDA graph conditional of the WHILE loop
  int has_handle;             // 1 when run inside the graph loop
  int f32k;                   // FP32 iteration kernel: 0 tile, 1 bulk-copy pipeline, 2 register
                            // marching, 3 register marching fed by cp.async rings
  const PairTmaMaps* tma;     // host: the operator's TMA maps, or null (two-iteration
                              // kernel on the cp.async ring)
};
// y[0] = src (or 0 if src == null), p = d0 * y[0]; resets ctrl.
void series_init(const SeriesArgs& a, const void* src, double d0, int force, int max_iters,
                 double tol, cudaStream_t s);
// FP32 phi_1 series start from u: y[0] = A u + sum_k a_k g_k (S, at most two
// terms), p = d0 * y[0], ctrl reset -- one pass of the ring kernel.  false
// (nothing enqueued) where the ring kernels do not apply.
bool series_start_f32(const SeriesArgs& a, const void* u, const Sources& S, double d0, int force,
                      int max_iters, double tol, cudaStream_t s);
// One fused Leja iteration over the grid (a.nblocks blocks).  The last block to
// finish reduces the norm partials in a fixed order, applies the stopping rule,
// advances ctrl->m and, with a.has_handle, sets the graph loop condition.
void series_iteration(const SeriesArgs& a, cudaStream_t s);
// FP32 phi_1 series on the ring kernel run two iterations per launch
// (series_iteration then launches leja_iter2_f32_ring_k); after such a
// series, series_flush_pair adds the pending last term to p.
bool series_pair(const SeriesArgs& a);
// ... and its row records come in by TMA (zero-Dirichlet grids with maps).
bool series_pair_tma(const SeriesArgs& a);
// Marching of the two-iteration kernels: 1 one row of lookahead in registers
// (default), 0 without, 2 as 1 with packed FP32 pair arithmetic.
int pair_march();
// The marching set by AD_F32_MARCH (0, 1 or 2), -1 when it is not set.
int pair_march_env();
void series_flush_pair(const SeriesArgs& a, cudaStream_t s);
// Pair mode, after the series: u += b (p + the pending term), FP32, one pass
// (the flush and the update axpby together; p is not written).
void series_finish_pair_update(const SeriesArgs& a, void* u, double b, cudaStream_t s);
// Whole Newton series in one cooperative launch (FP64, n <= kPersistMaxCells).
// gen: device barrier generation counter (persists across calls).  Returns
// false if not applicable or refused; nothing was launched then.
constexpr long long kPersistMaxCells = 152LL * 2048;
// Device scratch of the neighbour-synchronised persistent kernel: write-once
// norm slots [kMaxIters][nsync_max_blocks()][2] and one flag per block.
struct NsyncScratch {
  double* slots;
  unsigned int* flags;
};
size_t nsync_slots_bytes();
int nsync_max_blocks();
// Totals of asynchronous steps, accumulated on the device (one thread).
struct AsyncTotals {
  long long iters;         // Leja iterations of all series
  long long timed_iters;   // ... of the series that ran with timing events
  long long launches;      // graph-body kernel launches (known on the device only)
  int series;
  int status;              // worst: 0 ok, 3 not converged, 4 no stop state / timeout
  double err_est;          // largest error estimate
};

// A whole exponential step in the persistent tile kernel (fixed rule, one
// substep, FP64).  Prologue: w1 = A u + sum a_k g_k (to global w1) and
// w2 = sum b_k g_k, as the apply kernel forms them, then the series start of
// series_init (s = 2: y_0 = 0, p_0 = d0 y_0; s = 1: y_0 = w1, p_0 = d0 w1);
// epilogue: u = u + b P in place of the axpby (b = 1 for s = 2, dt for s = 1).
// With totals set, block 0 also adds the series to them (asynchronous steps).
struct StepFuse {
  int s;                   // 1 or 2
  const double* W;         // unscaled weights of A
  double* u;               // the step's state (read by the prologue, updated by the epilogue)
  double* w1;              // global scratch for w1
  Sources src;
  double d0, b;
  int force, max_iters;
  double tol;
  AsyncTotals* totals;     // null: synchronous step
  int timed;
};

// ns == nullptr selects the grid-barrier kernel.  Returns 7 (tile kernel),
// 2 (row kernel), 1 (grid-barrier kernel) when launched, or 0.  With fuse,
// only the tile kernel is tried (0: the caller runs the step unfused).
int series_run_persistent(const SeriesArgs& a, unsigned int* gen, const NsyncScratch* ns,
                          cudaStream_t s, const StepFuse* fuse = nullptr);

// grid size of the fused iteration kernel (FP64: by cell count; FP32: by tile count)
int series_blocks(int prec, long long n);
int series_blocks_grid(int prec, int nx, int ny);
// FP32 iteration kernel for this grid: 3 cp.async-ring marching (default, nx % 4 == 0),
// 2 register marching, 1 bulk-copy pipeline, 0 tile (any nx);
// AD_F32_KERNEL=ring|vec|bulk|tile overrides.
int series_f32_kernel(int prec, int nx);

// ---------------------------------------------------------------- vector helpers
// z = a*x + b*y (x or y may be null = 0), elementwise, storage type prec.
void axpby(int prec, long long n, double a, const void* x, double b, const void* y, void* z,
           cudaStream_t s);
// partial sums of squares of x into partials[nblocks]; then finalize to out[0] = sqrt(sum).
void norm2_partials(int prec, long long n, const void* x, double* partials, int nblocks,
                    cudaStream_t s);
void reduce_partials(const double* partials, int nblocks, int op /*0 sum,1 min,2 sqrt-sum*/,
                     double* out, cudaStream_t s);
// x = y / dev_scalar[0] (power iteration normalisation).
void scale_by_inv(int prec, long long n, const void* y, const double* dev_scalar, void* x,
                  cudaStream_t s);
void splitmix_fill(int prec, long long n, unsigned long long seed, void* x, cudaStream_t s);

// ---------------------------------------------------------------- GMRES (FP64)
// h[i] = <V_i, w> for i < k (partials per block: [k][nblocks]).
void multi_dot_partials(long long n, const double* V, long long ldv, int k, const double* w,
                        double* partials, int nblocks, cudaStream_t s);
void multi_dot_finalize(const double* partials, int nblocks, int k, double* h, cudaStream_t s);
// w -= sum_i h[i] V_i ; also partial sums of ||w||^2 into partials.
void multi_axpy_norm(long long n, const double* V, long long ldv, int k, const double* h,
                     double* w, double* partials, int nblocks, cudaStream_t s);
// x += sum_i y[i] V_i
void multi_axpy_add(long long n, const double* V, long long ldv, int k, const double* y, double* x,
                    cudaStream_t s);

int stream_blocks(long long n);   // grid size of the streaming kernels

// Read-only view of an operator's buffers and spectral state (capi.cu).
struct OperatorView {
  GridDev g;
  int prec;
  const void* coef;
  void *y0, *y1, *p, *w1, *w2;
  double alpha, c, gamma, rho_max;
  int max_iters;
  int adv;
  float abx, aby;
  cudaStream_t stream;
};
}  // namespace ad
struct ad_operator;
struct ad_mlp;
namespace ad {
bool operator_view(const ad_operator* op, OperatorView* v);

// FP64 FMA rate of the device (TFLOP/s) from a timed launch of `blocks` blocks of
// independent DFMA chains, `iters` per chain; 0, or 2 on a CUDA error.
int fp64_fma_rate(int blocks, int iters, cudaStream_t s, double* tflops);

// One-block kernel whose bounded wait must run out (failure-detection test).
int wait_timeout_probe(unsigned long long timeout_ns, int* status_dev, cudaStream_t s);

// Set the thread-local message returned by ad_last_error().
void set_error_message(const char* msg);

// Kernels enqueued from the host by this thread (every launcher adds one);
// kernels run inside graph loops are counted by the caller.
long long& launch_counter();
// ---------------------------------------------------------------- penalised IMEX step
// One conjugate-gradient iteration on (I - c L) x = b (L: 5-point Laplacian of
// the flux form with the grid's boundary rule); scal[3] holds <r, r> on entry
// (set by a reduction of the initial residual) and on exit.
void penalty_cg_iteration(const GridDev& g, double dx, double dy, double c, double* x, double* r,
                          double* p, double* Mp, double* partials, int nblocks, double* scal,
                          cudaStream_t s);
// max over cells of lambda_max(D), reduced on the device with no scratch
// buffer; synchronises s.  Returns 0, or 1 on a CUDA error.
int lambda_max_reduce(long long n, const double* Dxx, const double* Dxy, const double* Dyy,
                      int nblocks, cudaStream_t s, double* out);

// ---------------------------------------------------------------- learned bound
constexpr int kFeatures = 21;
// The 21 inputs of the bound model for one field (slot 4, log dt, is left 0):
// log max lambda_1(D), log min lambda_2(D), log(max|a| + 1e-6) (max over the
// advection fields when given, else max_a), log dxmin, -, and the
// anisotropy-weighted 16-bin histogram of the principal direction of D.
// Reduced on the device in a fixed accumulator (no scratch buffer); host
// threads are serialised; synchronises s.  Returns 0, or 1 on a CUDA error.
int field_features(long long n, double dxmin, const double* Dxx, const double* Dxy,
                   const double* Dyy, const double* ax, const double* ay, double max_a,
                   cudaStream_t s, float* out21);
// Y[B][2] = model(X[B][21]) with host X and Y (BF16 kernels when bf16 != 0);
// synchronises the model's stream.
int mlp_predict_host(ad_mlp* M, const float* X, int B, int bf16, float* Y);

}  // namespace ad
