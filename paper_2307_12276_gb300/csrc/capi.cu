// C ABI of the library (include/anidiff.h): operator lifecycle, spectral
// bounds, the Leja phi_1 action, exponential quadrature steps and the
// Crank-Nicolson comparison step.  Host code here does only the scalar work
// of the method (Leja points, divided differences, the scalar eta recurrence
// of the augmented matrix, the GMRES Hessenberg solve) and orchestration;
// every per-cell pass runs in the kernels of stencil_kernels.cu and
// vec_kernels.cu.
//
// Each Newton series (Section 2) runs as one CUDA graph launch: a
// conditional WHILE node whose body is the fused Leja iteration kernel.  The
// last block of each launch evaluates the stopping rule on the device and
// sets the loop condition, so the host neither polls nor syncs per
// iteration; the loop is bounded by the iteration cap (<= 500).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "anidiff.h"
#include "ad_internal.h"
#include "cluster_f64.h"
#include "leja_host.h"

using namespace ad;

namespace {

constexpr int kGraphUnroll = 4;   // iteration kernels per body of the graph loop

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

// On failure the runtime's pending (non-sticky) error is cleared so that it is
// not reported again by a later, unrelated call.
#define CUDA_TRY(expr)                                                                    \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      cudaGetLastError();                                                                 \
      return fail(AD_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));       \
    }                                                                                     \
  } while (0)

#define AD_TRY(expr)              \
  do {                            \
    int r_ = (expr);              \
    if (r_ != AD_OK) return r_;   \
  } while (0)

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

namespace ad {
void set_error_message(const char* msg) { g_err = msg; }
}  // namespace ad

struct SeriesGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool ok = false;
  bool tried = false;
};

struct ad_operator {
  ad_grid grid{};
  GridDev g{};
  int prec = 0;
  size_t esz = 8;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  int dev = 0;
  // coefficients
  double* W = nullptr;   // fp64 [9][n]
  double* Ws = nullptr;  // fp64 [9][n], (W - c)/gamma
  float* F = nullptr;    // fp32 [3 or 5][n]
  int adv = 0;
  double ax_c = 0, ay_c = 0;
  float abx = 0, aby = 0;
  // workspace vectors (storage type)
  void* Y0 = nullptr; void* Y1 = nullptr; void* P = nullptr;
  void* W1 = nullptr; void* W2 = nullptr;
  void* T1 = nullptr; void* T2 = nullptr; void* T3 = nullptr;
  void* S0 = nullptr; void* S1 = nullptr;      // host staging (allocated at creation)
  double* Vk = nullptr; int vk_cols = 0;       // GMRES basis (ad_reserve_gmres)
  LejaCoef* lc = nullptr;
  Ctrl* ctrl = nullptr;
  double* partials = nullptr;                  // >= 2 * nblocks and >= kMaxGmres+1 rows for GMRES
  size_t partials_len = 0;
  double* dscal = nullptr;                     // device scalars [64]
  NsyncScratch nsync{nullptr, nullptr};        // persistent-kernel scratch (FP64, small grids)
  int nblocks = 1;
  // asynchronous steps (ad_expquad_step_async): what the device knows is
  // accumulated there by async_collect_k, what the host knows here
  AsyncTotals* totals = nullptr;               // device
  AsyncTotals* h_totals = nullptr;             // pinned mirror
  ad_stats async_host{};
  int async_worst = 0;                         // worst status of synchronous fallbacks
  bool ctrl_dirty = false;                     // a series gave up: reset ctrl before a fused step
  std::vector<cudaEvent_t> atev;               // event pairs around async series (timing)
  int atev_used = 0;
  // series timing (ad_time_series)
  bool time_series = false;
  cudaEvent_t tev[2] = {nullptr, nullptr};
  double t_ms = 0.0;
  int t_series = 0;
  long long t_iters = 0;
  int t_path = 0;
  // pinned host mirrors
  LejaCoef* h_lc = nullptr;
  Ctrl* h_ctrl = nullptr;
  double* h_scal = nullptr;                    // [4 * (kMaxGmres + 2)]
  // learned bound: the model's inputs of this operator's fields (slot 4,
  // log dt, is filled per prediction), and the model ad_spectral_bound uses
  PairTmaMaps tma{};                           // TMA maps of the FP32 two-iteration kernel
  bool has_tma = false;
  float feat[kFeatures] = {};
  double dxmin = 0.0;
  ad_mlp* bound_model = nullptr;
  double bound_margin = 1.1, bound_dt = 0.0;
  // method state
  double alpha = 0.0, c = 0.0, gamma = 0.0;
  bool have_alpha = false;
  double rho_max = 200.0;
  int max_iters = kMaxIters;
  int adaptive = 0;                            // substep control: 0 fixed, 1 adaptive
  SeriesGraph graphs[2];                       // [aug]
  // cache of the coefficient upload
  int cache_kind = -1;
  double cache_h = 0.0, cache_alpha = 0.0;
  double cache_eta[2] = {0.0, 0.0};            // eta_0 of the uploaded table (augmented)
  std::vector<double> d_host;                  // divided differences of the current series
};

namespace ad {
bool operator_view(const ad_operator* op, OperatorView* v) {
  if (!op || !v) return false;
  v->g = op->g;
  v->prec = op->prec;
  v->coef = op->prec == 0 ? (const void*)op->Ws : (const void*)op->F;
  v->y0 = op->Y0;
  v->y1 = op->Y1;
  v->p = op->P;
  v->w1 = op->W1;
  v->w2 = op->W2;
  v->alpha = op->alpha;
  v->c = op->c;
  v->gamma = op->gamma;
  v->rho_max = op->rho_max;
  v->max_iters = op->max_iters;
  v->adv = op->adv;
  v->abx = op->abx;
  v->aby = op->aby;
  v->stream = op->stream;
  return true;
}
}  // namespace ad

namespace {

SeriesArgs series_args(ad_operator* op, int aug) {
  SeriesArgs a{};
  a.g = op->g;
  a.prec = op->prec;
  a.coef = op->prec == 0 ? (const void*)op->Ws : (const void*)op->F;
  a.c = op->c;
  a.gamma = op->gamma;
  a.y[0] = op->Y0;
  a.y[1] = op->Y1;
  a.p = op->P;
  a.w1 = op->W1;
  a.w2 = op->W2;
  a.lc = op->lc;
  a.ctrl = op->ctrl;
  a.partials = op->partials;
  a.nblocks = series_blocks_grid(op->prec, op->g.nx, op->g.ny);
  a.f32k = series_f32_kernel(op->prec, op->g.nx);
  a.aug = aug;
  a.adv = op->adv;
  a.abx = op->abx;
  a.aby = op->aby;
  a.tma = op->has_tma ? &op->tma : nullptr;
  return a;
}

void destroy_graphs(ad_operator* op) {
  for (auto& sg : op->graphs) {
    if (sg.exec) cudaGraphExecDestroy(sg.exec);
    if (sg.graph) cudaGraphDestroy(sg.graph);
    sg = SeriesGraph{};
  }
}

// Build the WHILE-loop graph of one series variant.  Returns false (and the
// caller falls back to launching iterations from the host) if the runtime
// refuses any step.
bool build_graph(ad_operator* op, int aug) {
  SeriesGraph& sg = op->graphs[aug];
  sg.tried = true;
  if (getenv("AD_NO_GRAPH")) return false;
  if (!op->cap_stream && cudaStreamCreateWithFlags(&op->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaGraph_t graph = nullptr;
  if (cudaGraphCreate(&graph, 0) != cudaSuccess) { cudaGetLastError(); return false; }
  cudaGraphConditionalHandle handle;
  if (cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(graph);
    return false;
  }
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp) != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(graph);
    return false;
  }
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if (cudaStreamBeginCaptureToGraph(op->cap_stream, body, nullptr, nullptr, 0,
                                    cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(graph);
    return false;
  }
  // The loop body holds kGraphUnroll iteration kernels: each body execution of a
  // conditional node costs a few microseconds of scheduling on this driver, so
  // it is amortised over several iterations.  Kernels after the one that stops
  // the series return at once (they see ctrl->stop).
  SeriesArgs a = series_args(op, aug);
  a.handle = (unsigned long long)handle;
  a.has_handle = 1;
  for (int u = 0; u < kGraphUnroll; ++u) series_iteration(a, op->cap_stream);
  // A launch the runtime refused during capture adds no node: a loop body
  // without its iteration kernels would never clear the loop condition, so
  // the graph is only kept when every launch was taken.
  const cudaError_t launched = cudaGetLastError();
  cudaGraph_t captured = nullptr;
  const cudaError_t ended = cudaStreamEndCapture(op->cap_stream, &captured);
  size_t body_nodes = 0;
  if (launched != cudaSuccess || ended != cudaSuccess ||
      cudaGraphGetNodes(body, nullptr, &body_nodes) != cudaSuccess ||
      body_nodes < (size_t)kGraphUnroll) {
    cudaGetLastError();
    cudaGraphDestroy(graph);
    return false;
  }
  cudaGraphExec_t exec = nullptr;
  if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(graph);
    return false;
  }
  sg.graph = graph;
  sg.exec = exec;
  sg.ok = true;
  return true;
}

int set_alpha(ad_operator* op, double alpha) {
  if (!(alpha < 0.0) || !std::isfinite(alpha))
    return fail(AD_ERR_INVALID, "spectral bound alpha must be finite and negative");
  op->alpha = alpha;
  op->c = alpha / 2.0;       // Section 2: c = alpha/2, gamma = -alpha/4
  op->gamma = -alpha / 4.0;
  op->have_alpha = true;
  op->cache_kind = -1;
  if (op->prec == 0) {
    scale_weights_f64(op->g, op->W, op->c, op->gamma, op->Ws, op->stream);
    CUDA_TRY(cudaGetLastError());
  }
  destroy_graphs(op);        // kernel arguments hold c and gamma
  return AD_OK;
}

int gershgorin(ad_operator* op, double* out) {
  if (op->prec == 0)
    gershgorin_partials_f64(op->g, op->W, op->partials, op->nblocks, op->stream);
  else
    gershgorin_partials_f32(op->g, op->F, op->adv, op->abx, op->aby, op->partials, op->nblocks,
                            op->stream);
  reduce_partials(op->partials, op->nblocks, 1, op->dscal, op->stream);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(op->h_scal, op->dscal, sizeof(double), cudaMemcpyDeviceToHost, op->stream));
  CUDA_TRY(cudaStreamSynchronize(op->stream));
  *out = op->h_scal[0];
  return AD_OK;
}

// A x (+ sources) in the storage type.
void apply(ad_operator* op, const void* u, void* out1, void* out2, const Sources& src) {
  if (op->prec == 0)
    apply_f64(op->g, op->W, (const double*)u, (double*)out1, (double*)out2, src, op->stream);
  else
    apply_f32(op->g, op->F, op->adv, op->abx, op->aby, (const float*)u, (float*)out1,
              (float*)out2, src, op->stream);
}

// Upload the per-iteration scalars of a series.
//   kind 0: phi_1 at step h (no augmented coupling);
//   kind 1: exp at step h, augmented coupling from eta0 (e1_m, e2_m filled).
// Returns d_0 in *d0 and, for kind 1, the eta part of the series sum in eta_out.
int upload_series(ad_operator* op, int kind, double h, const double eta0[2], double* d0,
                  double eta_out[2]) {
  const std::vector<double>& xi = leja_points();
  const int M = kMaxIters + 1;
  const bool cached = op->cache_kind == kind && op->cache_h == h && op->cache_alpha == op->alpha;
  // the device table already holds exactly these coefficients
  const bool same_table =
      cached && (kind == 0 || (op->cache_eta[0] == eta0[0] && op->cache_eta[1] == eta0[1]));
  if (!cached) {
    std::vector<double> f(M);
    for (int m = 0; m < M; ++m) {
      const double z = (op->c + op->gamma * xi[m]) * h;
      f[m] = kind == 0 ? phi1(z) : std::exp(z);
    }
    op->d_host.assign(M, 0.0);
    divided_differences(xi.data(), f.data(), M, op->d_host.data());
  }
  const std::vector<double>& d = op->d_host;
  double e1 = 0.0, e2 = 0.0, pe1 = 0.0, pe2 = 0.0;
  if (kind == 1) {
    e1 = eta0[0];
    e2 = eta0[1];
    pe1 = d[0] * e1;
    pe2 = d[0] * e2;
  }
  *d0 = d[0];
  if (kind == 1) {
    eta_out[0] = pe1;
    eta_out[1] = pe2;
  }
  if (same_table) return AD_OK;
  for (int m = 0; m < kMaxIters; ++m) {
    LejaCoef& L = op->h_lc[m];
    L.xi = xi[m];
    L.d = d[m + 1];
    L.absd = std::fabs(d[m + 1]);
    L.e1 = kind == 1 ? e1 / op->gamma : 0.0;
    L.e2 = kind == 1 ? e2 / op->gamma : 0.0;
    if (kind == 1) {
      // eta_{m+1} = ((J - c)/gamma - xi_m) eta_m with J = [[0, 1], [0, 0]]
      const double n1 = (e2 - op->c * e1) / op->gamma - xi[m] * e1;
      const double n2 = (-op->c * e2) / op->gamma - xi[m] * e2;
      e1 = n1;
      e2 = n2;
    }
  }
  CUDA_TRY(cudaMemcpyAsync(op->lc, op->h_lc, sizeof(LejaCoef) * kMaxIters, cudaMemcpyHostToDevice,
                           op->stream));
  op->cache_kind = kind;
  op->cache_h = h;
  op->cache_alpha = op->alpha;
  if (kind == 1) {
    op->cache_eta[0] = eta0[0];
    op->cache_eta[1] = eta0[1];
  }
  return AD_OK;
}

// Vector updates that need no host decision, enqueued right after a series
// and before the synchronisation that reads its result, so that the device
// does not wait for the host between the series and them.
struct Tail {
  struct Op {
    double a;
    const void* x;
    double b;
    const void* y;
    void* z;
  };
  int k = 0;
  Op op[3];
  void add(double a, const void* x, double b, const void* y, void* z) { op[k++] = Op{a, x, b, y, z}; }
  void add(const Tail* t) {
    if (t)
      for (int i = 0; i < t->k; ++i) op[k++] = t->op[i];
  }
};

void enqueue_tail(const ad_operator* op, const Tail* t) {
  if (!t) return;
  for (int i = 0; i < t->k; ++i)
    axpby(op->prec, op->g.n, t->op[i].a, t->op[i].x, t->op[i].b, t->op[i].y, t->op[i].z,
          op->stream);
}

// Run one Newton series from src (device vector of the storage type, or null
// for a zero start); the result is left in op->P.  *iters receives the
// number of iterations; the eta part (augmented series) is accumulated on
// the host into eta_sum using the uploaded d.  tail (optional) is enqueued
// after the series and before the synchronisation.  async: no
// synchronisation; async_collect_k adds the series to the device totals and
// *iters_out is -1 (unknown to the host).
__global__ void async_collect_k(const Ctrl* c, AsyncTotals* t, int per_launch, int timed) {
  const int it = c->iters;
  t->iters += it;
  if (timed) t->timed_iters += it;
  if (per_launch > 0) t->launches += (it + per_launch - 1) / per_launch;
  t->series += 1;
  const int st = c->stop ? (c->status == 4 ? 4 : c->status) : 4;
  if (st > t->status) t->status = st;
  // the estimate as the synchronous path forms it on the host
  const double e = c->pnorm2 > 0.0 ? c->err_est * sqrt(c->ynorm2 / c->pnorm2)
                                   : (c->ynorm2 > 0.0 ? INFINITY : 0.0);
  if (e > t->err_est) t->err_est = e;
}

constexpr int kNotFused = -100;   // run_series: the fused step did not launch

// fuse (optional): run the whole step in the tile kernel (see StepFuse); src
// and tail are then unused, and kNotFused is returned when it cannot launch
// (nothing was enqueued: the caller runs the step unfused).
// started: the series start (y_0, p_0, ctrl reset) is already enqueued.
// update_u (FP32 pair mode only): the tail is u += update_b P, done with the
// pending term in one pass (series_finish_pair_update); tail is then unused.
int run_series(ad_operator* op, int aug, const void* src, double d0, int force, double tol,
               ad_stats* st, int* iters_out, const Tail* tail = nullptr, bool async = false,
               const StepFuse* fuse = nullptr, bool started = false, void* update_u = nullptr,
               double update_b = 0.0) {
  SeriesArgs a = series_args(op, aug);
  if (fuse && (force == 0 || getenv("AD_NO_PERSIST") || getenv("AD_NO_FUSE"))) return kNotFused;
  if (fuse && op->ctrl_dirty) {   // the fused kernel relies on a clean barrier ticket
    CUDA_TRY(cudaMemsetAsync(op->ctrl, 0, sizeof(Ctrl), op->stream));
    op->ctrl_dirty = false;
  }
  if (!fuse && !started) series_init(a, src, d0, force, op->max_iters, tol, op->stream);
  CUDA_TRY(cudaGetLastError());
  int iters = 0;
  bool graph_used = false;
  if (force == 0) {
    iters = 0;
    op->h_ctrl->status = 0;
    op->h_ctrl->err_est = 0.0;
    enqueue_tail(op, tail);
  } else {
    SeriesGraph& sg = op->graphs[aug];
    cudaEvent_t ev[2] = {op->tev[0], op->tev[1]};
    if (op->time_series && async) {   // one event pair per series, read by ad_async_totals
      while ((int)op->atev.size() < 2 * (op->atev_used + 1)) {
        cudaEvent_t e = nullptr;
        CUDA_TRY(cudaEventCreate(&e));
        op->atev.push_back(e);
      }
      ev[0] = op->atev[2 * op->atev_used];
      ev[1] = op->atev[2 * op->atev_used + 1];
      ++op->atev_used;
    }
    if (op->time_series) CUDA_TRY(cudaEventRecord(ev[0], op->stream));
    // small FP64 grids: the whole series in one thread-block cluster; small and
    // medium ones: in one cooperative launch
    int pk = getenv("AD_NO_PERSIST") ? 0 : series_run_cluster(a, op->stream, fuse);
    if (!pk && !getenv("AD_NO_PERSIST"))
      pk = series_run_persistent(a, &op->ctrl->gen, &op->nsync, op->stream, fuse);
    if (fuse && !pk) {
      if (op->time_series && async) --op->atev_used;   // the event pair is reused
      return kNotFused;
    }
    const bool persist = pk != 0;
    if (!persist && !sg.tried) build_graph(op, aug);
    if (persist) {
      // launched; the kernel counted itself
    } else if (sg.ok) {
      CUDA_TRY(cudaGraphLaunch(sg.exec, op->stream));
      graph_used = true;
    } else {  // host-driven fallback: chunks of iterations, poll the stop flag
      int launched = 0;
      for (;;) {
        const int chunk = 16;
        for (int k = 0; k < chunk; ++k) series_iteration(a, op->stream);
        launched += chunk;
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaMemcpyAsync(op->h_ctrl, op->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, op->stream));
        CUDA_TRY(cudaStreamSynchronize(op->stream));
        if (op->h_ctrl->stop || launched >= kMaxIters + chunk) break;
      }
    }
    const bool finish_update = update_u && !persist && series_pair(a);
    if (!persist && series_pair(a) && !finish_update)
      series_flush_pair(a, op->stream);                                  // the pending last term
    CUDA_TRY(cudaGetLastError());
    if (op->time_series) CUDA_TRY(cudaEventRecord(ev[1], op->stream));
    if (finish_update) series_finish_pair_update(a, update_u, update_b, op->stream);
    else enqueue_tail(op, tail);
    if (async) {
      if (!fuse) {   // (the fused kernel reports to the totals itself)
        const int per_launch = graph_used ? (series_pair(a) ? 2 : 1) : 0;
        async_collect_k<<<1, 1, 0, op->stream>>>(op->ctrl, op->totals, per_launch,
                                                 op->time_series ? 1 : 0);
        ++launch_counter();
      }
      CUDA_TRY(cudaGetLastError());
      if (op->time_series) op->t_path = persist ? pk : (graph_used ? 3 : 4) + (series_pair(a) ? (series_pair_tma(a) ? 5 : 2) : 0);
      *iters_out = -1;
      return AD_OK;
    }
    CUDA_TRY(cudaMemcpyAsync(op->h_ctrl, op->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, op->stream));
    CUDA_TRY(cudaStreamSynchronize(op->stream));
    iters = op->h_ctrl->iters;
    if (op->time_series) {
      float ms = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&ms, op->tev[0], op->tev[1]));
      op->t_ms += ms;
      op->t_series += 1;
      op->t_iters += iters;
      op->t_path = persist ? pk : (graph_used ? 3 : 4) + (series_pair(a) ? (series_pair_tma(a) ? 5 : 2) : 0);
    }
    if (!op->h_ctrl->stop || op->h_ctrl->status == 4) op->ctrl_dirty = true;
    if (!op->h_ctrl->stop) return fail(AD_ERR_TIMEOUT, "Leja series did not reach its stop state");
    {  // the device stores |d_{m+1}| and the squared norms; form the estimate here
      const Ctrl& h = *op->h_ctrl;
      op->h_ctrl->err_est = h.pnorm2 > 0.0 ? h.err_est * std::sqrt(h.ynorm2 / h.pnorm2)
                                           : (h.ynorm2 > 0.0 ? INFINITY : 0.0);
    }
    // graph bodies: one fused iteration kernel per iteration, or per two in
    // pair mode (host launches are counted by the launchers themselves)
    if (st && graph_used) st->kernel_launches += series_pair(a) ? (iters + 1) / 2 : iters;
    if (op->h_ctrl->status == 4) return fail(AD_ERR_TIMEOUT, "a grid barrier wait gave up");
  }
  if (st) {
    st->iters += iters;
    st->matvecs += iters;
    st->err_est = std::max(st->err_est, op->h_ctrl->err_est);
    if (op->h_ctrl->status != 0) st->converged = 0;
  }
  *iters_out = iters;
  return op->h_ctrl->status == 0 ? AD_OK : AD_ERR_NOT_CONVERGED;
}

int n_substeps(const ad_operator* op, double dt) {
  const double rho = op->gamma * dt;
  if (rho <= op->rho_max) return 1;
  return (int)std::ceil(rho / op->rho_max);
}

// Bring a caller vector to the device: returns the device pointer to use and
// whether the result must be copied back.
int stage_in(ad_operator* op, const void* user, int which, const void** dev, bool copy) {
  if (is_device_ptr(user)) { *dev = user; return AD_OK; }
  void* slot = which == 0 ? op->S0 : (which == 1 ? op->S1 : op->T3);
  if (copy)
    CUDA_TRY(cudaMemcpyAsync(slot, user, (size_t)op->g.n * op->esz, cudaMemcpyHostToDevice, op->stream));
  *dev = slot;
  return AD_OK;
}

int finish_out(ad_operator* op, void* user, const void* dev) {
  if (dev != user)
    CUDA_TRY(cudaMemcpyAsync(user, dev, (size_t)op->g.n * op->esz, cudaMemcpyDeviceToHost, op->stream));
  CUDA_TRY(cudaStreamSynchronize(op->stream));
  return AD_OK;
}

int fill_sources(const ad_source* src, int nterms_max, Sources* out) {
  *out = Sources{};
  if (!src) return AD_OK;
  if (src->nterms < 0 || src->nterms > nterms_max)
    return fail(AD_ERR_INVALID, "source: nterms out of range [0, 16]");
  if (src->nterms > 0 && !src->g) return fail(AD_ERR_INVALID, "source: g is NULL");
  for (int k = 0; k < src->nterms; ++k) {
    if (!is_device_ptr(src->g[k])) return fail(AD_ERR_INVALID, "source: g[k] must be a device pointer");
    out->g[k] = src->g[k];
  }
  out->n = src->nterms;
  return AD_OK;
}

double h_at(const ad_source* src, int k, double t) {
  return (src && src->h) ? src->h(k, t, src->ctx) : 1.0;
}

// The eta part of an augmented series sum, sum_m d_m eta_m (host scalars),
// after `it` iterations from eta (d: the divided differences last uploaded).
void advance_eta(const ad_operator* op, int it, double eta[2]) {
  const std::vector<double>& d = op->d_host;
  const std::vector<double>& xi = leja_points();
  double e1 = eta[0], e2 = eta[1];
  double s1 = d[0] * e1, s2 = d[0] * e2;
  for (int m = 0; m < it; ++m) {
    const double n1 = (e2 - op->c * e1) / op->gamma - xi[m] * e1;
    const double n2 = (-op->c * e2) / op->gamma - xi[m] * e2;
    e1 = n1;
    e2 = n2;
    s1 += d[m + 1] * e1;
    s2 += d[m + 1] * e2;
  }
  eta[0] = s1;
  eta[1] = s2;
}

// Adaptive substep control (the paper fixes none).  Starting from the substep
// of the rho_max rule, a substep whose series reaches the iteration budget
// (max_iters) without meeting the stopping rule is rejected and retried at
// half the size; after an accepted substep of m iterations the next one
// doubles when 4 m <= budget, unless the attempt before was rejected; the
// last substep is the remainder of the step.  More than kMaxRejects
// rejections or kMaxSubsteps accepted substeps give up.
constexpr int kMaxRejects = 40;
constexpr int kMaxSubsteps = 4096;

struct SubstepCtl {
  double dt, done = 0.0, h;
  int budget, accepted = 0, rejected = 0;
  bool grow = true;
  SubstepCtl(double dt_, int K0, int budget_) : dt(dt_), h(dt_ / K0), budget(budget_) {}
  // size of the next attempt; *last: it ends the step
  double next(bool* last) const {
    const double rem = dt - done;
    *last = h >= rem || rem - h <= 1e-12 * dt;
    return *last ? rem : h;
  }
  // false: give up
  bool reject(double hs) {
    ++rejected;
    h = hs / 2.0;
    grow = false;
    return rejected <= kMaxRejects;
  }
  // after an accepted attempt that was not the last; false: give up
  bool accept(double hs, int iters) {
    ++accepted;
    done += hs;
    if (accepted >= kMaxSubsteps) return false;
    h = (grow && 4 * iters <= budget) ? 2.0 * hs : hs;
    grow = true;
    return true;
  }
};

// Work of one series attempt: iterations always count; the error estimate
// only for accepted attempts.
void add_attempt(ad_stats* st, const ad_stats& at, bool accepted) {
  if (!st) return;
  st->iters += at.iters;
  st->matvecs += at.matvecs;
  st->kernel_launches += at.kernel_launches;
  if (accepted) st->err_est = std::max(st->err_est, at.err_est);
}

// phi_1 under adaptive substep control: w_{k+1} = w_k + h_k phi_1(h_k A)(A w_k + v),
// out = w / dt (a single substep: the series itself).  On giving up, out is not
// written and AD_ERR_NOT_CONVERGED is returned.
int phi1_device_adaptive(ad_operator* op, const void* v_dev, void* out_dev, double dt,
                         double tol, ad_stats* st) {
  const long long n = op->g.n;
  SubstepCtl ctl(dt, n_substeps(op, dt), op->max_iters);
  Sources none{};
  const void* rhs = v_dev;
  bool have_w = false;
  for (;;) {
    bool last;
    const double hs = ctl.next(&last);
    double d0;
    AD_TRY(upload_series(op, 0, hs, nullptr, &d0, nullptr));
    ad_stats at{};
    at.converged = 1;
    int it = 0;
    const int r = run_series(op, 0, rhs, d0, -1, tol, &at, &it);
    if (r != AD_OK && r != AD_ERR_NOT_CONVERGED) return r;
    add_attempt(st, at, r == AD_OK);
    if (r != AD_OK) {
      if (!ctl.reject(hs)) break;
      continue;
    }
    if (last) {
      ++ctl.accepted;
      if (!have_w) {
        axpby(op->prec, n, 1.0, op->P, 0.0, nullptr, out_dev, op->stream);
      } else {
        axpby(op->prec, n, 1.0, op->T2, hs, op->P, op->T2, op->stream);
        axpby(op->prec, n, 1.0 / dt, op->T2, 0.0, nullptr, out_dev, op->stream);
      }
      if (st) { st->substeps = ctl.accepted; st->rejected = ctl.rejected; }
      CUDA_TRY(cudaGetLastError());
      return AD_OK;
    }
    if (!have_w) {   // v kept in T1, w in T2
      axpby(op->prec, n, 1.0, v_dev, 0.0, nullptr, op->T1, op->stream);
      axpby(op->prec, n, hs, op->P, 0.0, nullptr, op->T2, op->stream);
      have_w = true;
    } else {
      axpby(op->prec, n, 1.0, op->T2, hs, op->P, op->T2, op->stream);
    }
    apply(op, op->T2, op->T3, nullptr, none);
    axpby(op->prec, n, 1.0, op->T3, 1.0, op->T1, op->T3, op->stream);
    if (st) st->matvecs += 1;
    rhs = op->T3;
    if (!ctl.accept(hs, it)) break;
  }
  if (st) { st->substeps = ctl.accepted; st->rejected = ctl.rejected; st->converged = 0; }
  CUDA_TRY(cudaGetLastError());
  return AD_ERR_NOT_CONVERGED;
}

// out_dev (storage type) = phi_1(dt A) v_dev; v_dev must not alias T1/T2/T3.
// post (optional, fixed substeps only): the caller's own updates after out,
// enqueued with the last series.  async: one substep only (see run_series).
int phi1_device(ad_operator* op, const void* v_dev, void* out_dev, double dt, double tol,
                int force, ad_stats* st, const Tail* post = nullptr, bool async = false) {
  if (op->adaptive && force < 0) return phi1_device_adaptive(op, v_dev, out_dev, dt, tol, st);
  const int K = n_substeps(op, dt);
  const double h = dt / K;
  double d0;
  AD_TRY(upload_series(op, 0, h, nullptr, &d0, nullptr));
  if (st) st->substeps = K;
  int status = AD_OK, it = 0;
  const long long n = op->g.n;
  if (K == 1) {
    Tail tail;
    tail.add(1.0, op->P, 0.0, nullptr, out_dev);
    tail.add(post);
    int r = run_series(op, 0, v_dev, d0, force, tol, st, &it, &tail, async);
    if (r != AD_OK && r != AD_ERR_NOT_CONVERGED) return r;
    status = r;
  } else {
    // w_{k+1} = w_k + h phi_1(h A)(A w_k + v), w_0 = 0; out = w_K / dt
    axpby(op->prec, n, 1.0, v_dev, 0.0, nullptr, op->T1, op->stream);   // v
    axpby(op->prec, n, 0.0, nullptr, 0.0, nullptr, op->T2, op->stream); // w
    Sources none{};
    for (int k = 0; k < K; ++k) {
      const void* rhs = op->T1;
      if (k > 0) {
        apply(op, op->T2, op->T3, nullptr, none);
        axpby(op->prec, n, 1.0, op->T3, 1.0, op->T1, op->T3, op->stream);
        rhs = op->T3;
        if (st) st->matvecs += 1;
      }
      Tail tail;
      tail.add(1.0, op->T2, h, op->P, op->T2);
      if (k == K - 1) {
        tail.add(1.0 / dt, op->T2, 0.0, nullptr, out_dev);
        tail.add(post);
      }
      int r = run_series(op, 0, rhs, d0, force, tol, st, &it, &tail);
      if (r != AD_OK && r != AD_ERR_NOT_CONVERGED) return r;
      if (r != AD_OK) status = r;
    }
  }
  CUDA_TRY(cudaGetLastError());
  return status;
}

}  // namespace

extern "C" {

int ad_version(void) { return 10000; }

const char* ad_last_error(void) { return g_err.c_str(); }

int ad_create_operator(const ad_grid* grid, const double* Dxx, const double* Dxy, const double* Dyy,
                       const double* ax, const double* ay, double ax_c, double ay_c, int precision,
                       void* cuda_stream, ad_operator** out) {
  g_err.clear();
  cudaGetLastError();  // a pending error of the caller's own runtime use is not ours
  if (!out) return fail(AD_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!grid || !Dxx || !Dxy || !Dyy) return fail(AD_ERR_INVALID, "grid or D field is NULL");
  if (grid->nx < 1 || grid->ny < 1) return fail(AD_ERR_INVALID, "grid: nx, ny must be >= 1");
  if ((long long)grid->nx * grid->ny > (1LL << 31) - 1) return fail(AD_ERR_INVALID, "grid: too many cells");
  if (!(grid->x1 > grid->x0) || !(grid->y1 > grid->y0)) return fail(AD_ERR_INVALID, "grid: empty domain");
  if (grid->bc != AD_BC_PERIODIC && grid->bc != AD_BC_DIRICHLET0) return fail(AD_ERR_INVALID, "grid: bad bc");
  if (precision != AD_FP64 && precision != AD_FP32_STORAGE) return fail(AD_ERR_INVALID, "bad precision");
  for (const void* p : {(const void*)Dxx, (const void*)Dxy, (const void*)Dyy})
    if (!is_device_ptr(p)) return fail(AD_ERR_INVALID, "coefficient fields must be device pointers");
  if ((ax && !is_device_ptr(ax)) || (ay && !is_device_ptr(ay)))
    return fail(AD_ERR_INVALID, "advection fields must be device pointers");
  if (!std::isfinite(ax_c) || !std::isfinite(ay_c)) return fail(AD_ERR_INVALID, "advection constants");

  ad_operator* op = new ad_operator();
  op->grid = *grid;
  op->g.nx = grid->nx;
  op->g.ny = grid->ny;
  op->g.bc = grid->bc;
  op->g.n = (long long)grid->nx * grid->ny;
  op->prec = precision;
  op->esz = precision == AD_FP64 ? 8 : 4;
  op->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&op->dev);
  const double dx = (grid->x1 - grid->x0) / grid->nx, dy = (grid->y1 - grid->y0) / grid->ny;
  const long long n = op->g.n;
  op->nblocks = stream_blocks(n);
  op->ax_c = ax_c;
  op->ay_c = ay_c;
  op->adv = (ax || ay) ? 2 : ((ax_c != 0.0 || ay_c != 0.0) ? 1 : 0);
  op->abx = (float)(ax_c / (2.0 * dx));
  op->aby = (float)(ay_c / (2.0 * dy));

  auto alloc = [&](void** p, size_t bytes) -> bool {
    if (cudaMalloc(p, bytes) != cudaSuccess) { cudaGetLastError(); return false; }
    return true;
  };
  bool ok = true;
  if (precision == AD_FP64) {
    ok = ok && alloc((void**)&op->W, sizeof(double) * 9 * n);
    ok = ok && alloc((void**)&op->Ws, sizeof(double) * 9 * n);
  } else {
    ok = ok && alloc((void**)&op->F, sizeof(float) * (op->adv == 2 ? 5 : 3) * n);
  }
  // S0, S1: staging of host-pointer vectors, allocated here so that no step allocates
  for (void** v : {&op->Y0, &op->Y1, &op->P, &op->W1, &op->W2, &op->T1, &op->T2, &op->T3,
                   &op->S0, &op->S1})
    ok = ok && alloc(v, op->esz * n);
  op->partials_len = std::max<size_t>(2 * (size_t)op->nblocks, (size_t)(kMaxGmres + 2) * op->nblocks);
  ok = ok && alloc((void**)&op->partials, sizeof(double) * op->partials_len);
  ok = ok && alloc((void**)&op->lc, sizeof(LejaCoef) * kMaxIters);
  ok = ok && alloc((void**)&op->ctrl, sizeof(Ctrl));
  ok = ok && alloc((void**)&op->totals, sizeof(AsyncTotals));
  ok = ok && alloc((void**)&op->dscal, sizeof(double) * 4 * (kMaxGmres + 2));
  if (precision == AD_FP64 && n <= kPersistMaxCells) {
    ok = ok && alloc((void**)&op->nsync.slots, nsync_slots_bytes());
    ok = ok && alloc((void**)&op->nsync.flags, sizeof(unsigned int) * nsync_max_blocks());
  }
  if (ok) ok = cudaMallocHost((void**)&op->h_lc, sizeof(LejaCoef) * kMaxIters) == cudaSuccess;
  if (ok) ok = cudaMallocHost((void**)&op->h_ctrl, sizeof(Ctrl)) == cudaSuccess;
  if (ok) ok = cudaMallocHost((void**)&op->h_totals, sizeof(AsyncTotals)) == cudaSuccess;
  if (ok) ok = cudaMallocHost((void**)&op->h_scal, sizeof(double) * 4 * (kMaxGmres + 2)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    ad_destroy_operator(op);
    return fail(AD_ERR_NOMEM, "device allocation failed");
  }
  std::memset(op->h_ctrl, 0, sizeof(Ctrl));
  cudaMemsetAsync(op->ctrl, 0, sizeof(Ctrl), op->stream);
  cudaMemsetAsync(op->totals, 0, sizeof(AsyncTotals), op->stream);
  if (precision == AD_FP64)
    pack_weights_f64(op->g, dx, dy, Dxx, Dxy, Dyy, ax, ay, ax_c, ay_c, op->W, op->stream);
  else
    pack_fields_f32(op->g, dx, dy, Dxx, Dxy, Dyy, ax, ay, ax_c, ay_c, op->F, op->stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ad_destroy_operator(op);
    return fail(AD_ERR_CUDA, std::string("pack kernel: ") + cudaGetErrorString(e));
  }
  // FP32 zero-Dirichlet grids with nx % 4 == 0: the two-iteration kernel's
  // rows come in by TMA (the maps cover this operator's own buffers)
  if (precision != AD_FP64 && grid->bc == AD_BC_DIRICHLET0 && series_f32_kernel(1, grid->nx) == 3)
    op->has_tma = encode_pair_tma(op->g, op->Y0, op->Y1, op->P, op->F, &op->tma);
  // inputs of the learned bound, from the fields while they are at hand
  op->dxmin = std::min(dx, dy);
  if (field_features(n, op->dxmin, Dxx, Dxy, Dyy, ax, ay, std::hypot(ax_c, ay_c), op->stream,
                     op->feat) != 0) {
    cudaGetLastError();
    ad_destroy_operator(op);
    return fail(AD_ERR_CUDA, "field features kernel failed");
  }
  (void)leja_points();  // computed once per process
  double alpha = 0.0;
  int r = gershgorin(op, &alpha);
  if (r == AD_OK) {
    if (!(alpha < 0.0)) alpha = -1.0;  // A == 0: any negative bound serves
    r = set_alpha(op, alpha);
  }
  if (r != AD_OK) {
    std::string msg = g_err;
    ad_destroy_operator(op);
    return fail(r, msg);
  }
  *out = op;
  return AD_OK;
}

int ad_destroy_operator(ad_operator* op) {
  if (!op) return AD_OK;
  if (op->stream) cudaStreamSynchronize(op->stream);
  destroy_graphs(op);
  if (op->cap_stream) cudaStreamDestroy(op->cap_stream);
  for (void* p : {(void*)op->W, (void*)op->Ws, (void*)op->F, op->Y0, op->Y1, op->P, op->W1, op->W2,
                  op->T1, op->T2, op->T3, op->S0, op->S1, (void*)op->Vk, (void*)op->lc,
                  (void*)op->ctrl, (void*)op->totals, (void*)op->partials, (void*)op->dscal,
                  (void*)op->nsync.slots, (void*)op->nsync.flags})
    if (p) cudaFree(p);
  for (cudaEvent_t e : op->tev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : op->atev)
    if (e) cudaEventDestroy(e);
  if (op->h_lc) cudaFreeHost(op->h_lc);
  if (op->h_ctrl) cudaFreeHost(op->h_ctrl);
  if (op->h_totals) cudaFreeHost(op->h_totals);
  if (op->h_scal) cudaFreeHost(op->h_scal);
  delete op;
  return AD_OK;
}

int ad_set_options(ad_operator* op, double rho_max, int max_iters) {
  g_err.clear();
  if (!op) return fail(AD_ERR_INVALID, "op is NULL");
  if (max_iters > kMaxIters) return fail(AD_ERR_INVALID, "max_iters > 500");
  if (rho_max > 0) op->rho_max = rho_max;
  if (max_iters > 0) op->max_iters = max_iters;
  return AD_OK;
}

int ad_set_substep_control(ad_operator* op, int adaptive) {
  g_err.clear();
  if (!op) return fail(AD_ERR_INVALID, "op is NULL");
  if (adaptive != 0 && adaptive != 1) return fail(AD_ERR_INVALID, "adaptive must be 0 or 1");
  op->adaptive = adaptive;
  return AD_OK;
}

int ad_set_spectral_bound(ad_operator* op, double alpha) {
  g_err.clear();
  if (!op) return fail(AD_ERR_INVALID, "op is NULL");
  return set_alpha(op, alpha);
}

int ad_get_spectral_bound(const ad_operator* op, double* alpha) {
  if (!op || !alpha) return fail(AD_ERR_INVALID, "NULL argument");
  *alpha = op->alpha;
  return AD_OK;
}

int ad_spectral_bound(ad_operator* op, int method, const void* x0, unsigned long long seed,
                      int power_iters, double safety, double* alpha) {
  g_err.clear();
  if (!op || !alpha) return fail(AD_ERR_INVALID, "NULL argument");
  double a = 0.0;
  if (method == AD_BOUND_GERSHGORIN) {
    AD_TRY(gershgorin(op, &a));
  } else if (method == AD_BOUND_POWER) {
    if (power_iters < 1 || !(safety > 0)) return fail(AD_ERR_INVALID, "power_iters >= 1, safety > 0");
    const long long n = op->g.n;
    const void* x0d = nullptr;
    if (x0) AD_TRY(stage_in(op, x0, 2, &x0d, true));
    if (x0d) axpby(op->prec, n, 1.0, x0d, 0.0, nullptr, op->T1, op->stream);
    else splitmix_fill(op->prec, n, seed, op->T1, op->stream);
    // x <- x0 / ||x0||
    norm2_partials(op->prec, n, op->T1, op->partials, op->nblocks, op->stream);
    reduce_partials(op->partials, op->nblocks, 2, op->dscal, op->stream);
    scale_by_inv(op->prec, n, op->T1, op->dscal, op->T1, op->stream);
    Sources none{};
    for (int it = 0; it < power_iters; ++it) {
      apply(op, op->T1, op->T2, nullptr, none);                          // y = A x
      norm2_partials(op->prec, n, op->T2, op->partials, op->nblocks, op->stream);
      reduce_partials(op->partials, op->nblocks, 2, op->dscal, op->stream);  // est = ||y||
      scale_by_inv(op->prec, n, op->T2, op->dscal, op->T1, op->stream);      // x = y / est
    }
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(op->h_scal, op->dscal, sizeof(double), cudaMemcpyDeviceToHost, op->stream));
    CUDA_TRY(cudaStreamSynchronize(op->stream));
    a = -safety * op->h_scal[0];
  } else if (method == AD_BOUND_LEARNED) {
    if (!op->bound_model)
      return fail(AD_ERR_INVALID, "no bound model: call ad_set_bound_model first");
    ad_operator* one[1] = {op};
    AD_TRY(ad_learned_bounds(op->bound_model, one, 1, &op->bound_dt, op->bound_margin, 1, &a,
                             nullptr));
  } else {
    return fail(AD_ERR_INVALID, "unknown spectral bound method");
  }
  if (!(a < 0.0)) return fail(AD_ERR_INVALID, "spectral bound is not negative (A == 0?)");
  AD_TRY(set_alpha(op, a));
  *alpha = a;
  return AD_OK;
}

int ad_set_bound_model(ad_operator* op, ad_mlp* m, double margin, double dt) {
  g_err.clear();
  if (!op) return fail(AD_ERR_INVALID, "NULL argument");
  if (m && (!(margin >= 1.0) || !std::isfinite(margin) || !(dt > 0) || !std::isfinite(dt)))
    return fail(AD_ERR_INVALID, "margin must be >= 1 and dt positive");
  op->bound_model = m;
  op->bound_margin = margin;
  op->bound_dt = dt;
  return AD_OK;
}

int ad_learned_bounds(ad_mlp* m, ad_operator* const* ops, int nops, const double* dt,
                      double margin, int bf16, double* alpha_out, double* iters_out) {
  g_err.clear();
  if (!m || !ops || !dt || nops < 1) return fail(AD_ERR_INVALID, "NULL argument or nops < 1");
  if (!(margin >= 1.0) || !std::isfinite(margin)) return fail(AD_ERR_INVALID, "margin must be >= 1");
  std::vector<float> X((size_t)nops * kFeatures), Y((size_t)nops * 2);
  for (int k = 0; k < nops; ++k) {
    if (!ops[k]) return fail(AD_ERR_INVALID, "NULL operator");
    if (!(dt[k] > 0) || !std::isfinite(dt[k])) return fail(AD_ERR_INVALID, "dt must be positive");
    std::copy(ops[k]->feat, ops[k]->feat + kFeatures, X.begin() + (size_t)k * kFeatures);
    X[(size_t)k * kFeatures + 4] = (float)std::log(dt[k]);
  }
  AD_TRY(mlp_predict_host(m, X.data(), nops, bf16, Y.data()));
  // outputs: t0 = log(|alpha| dx^2 / D_par) and t1 = log(iterations); the
  // bound is inflated by the margin
  std::vector<double> alpha(nops);
  for (int k = 0; k < nops; ++k) {
    const ad_operator* op = ops[k];
    const double dpar = std::exp((double)op->feat[0]);
    alpha[k] = -margin * std::exp((double)Y[2 * k]) * dpar / (op->dxmin * op->dxmin);
    if (!(alpha[k] < 0.0) || !std::isfinite(alpha[k]))
      return fail(AD_ERR_INVALID, "the model predicted no usable bound (not finite or not negative)");
  }
  for (int k = 0; k < nops; ++k) {
    AD_TRY(set_alpha(ops[k], alpha[k]));
    if (alpha_out) alpha_out[k] = alpha[k];
    if (iters_out) iters_out[k] = std::exp((double)Y[2 * k + 1]);
  }
  return AD_OK;
}

int ad_bound_training_sample(ad_operator* op, double dt, unsigned long long seed, int power_iters,
                             double safety, double tol, float* x21, float* t2,
                             double* power_estimate) {
  g_err.clear();
  if (!op || !x21 || !t2) return fail(AD_ERR_INVALID, "NULL argument");
  if (op->prec != AD_FP64) return fail(AD_ERR_INVALID, "training labels need an AD_FP64 operator");
  if (!(dt > 0) || !std::isfinite(dt) || !(tol > 0) || !(safety >= 1.0))
    return fail(AD_ERR_INVALID, "dt, tol must be positive and safety >= 1");
  double a = 0.0;
  AD_TRY(ad_spectral_bound(op, AD_BOUND_POWER, nullptr, seed + 1, power_iters, 1.0, &a));
  const double est = -a;                       // power-iteration estimate of |lambda|max
  AD_TRY(set_alpha(op, -safety * est));
  // iterations of phi_1(dt A) v at tol for a SplitMix64 vector v
  splitmix_fill(op->prec, op->g.n, seed, op->S0, op->stream);
  ad_stats st{};
  st.converged = 1;
  const int r = phi1_device(op, op->S0, op->S1, dt, tol, -1, &st);
  if (r != AD_OK && r != AD_ERR_NOT_CONVERGED) return r;
  CUDA_TRY(cudaStreamSynchronize(op->stream));
  std::copy(op->feat, op->feat + kFeatures, x21);
  x21[4] = (float)std::log(dt);
  const double dpar = std::exp((double)op->feat[0]);
  t2[0] = (float)std::log(est * op->dxmin * op->dxmin / dpar);
  t2[1] = (float)std::log((double)std::max(st.iters, 1));
  if (power_estimate) *power_estimate = est;
  return AD_OK;
}

int ad_apply(ad_operator* op, const void* u, void* Au) {
  g_err.clear();
  if (!op || !u || !Au) return fail(AD_ERR_INVALID, "NULL argument");
  const void* ud;
  AD_TRY(stage_in(op, u, 2, &ud, true));
  void* od = is_device_ptr(Au) ? Au : nullptr;
  if (!od) od = op->S1;
  Sources none{};
  apply(op, ud, od, nullptr, none);
  CUDA_TRY(cudaGetLastError());
  return finish_out(op, Au, od);
}

int ad_leja_phi1(ad_operator* op, const void* v, void* out, double dt, double tol, int force_iters,
                 ad_stats* stats) {
  g_err.clear();
  if (!op || !v || !out) return fail(AD_ERR_INVALID, "NULL argument");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(AD_ERR_INVALID, "dt must be positive");
  if (force_iters < 0 && !(tol > 0)) return fail(AD_ERR_INVALID, "tol must be positive");
  if (force_iters > op->max_iters) return fail(AD_ERR_INVALID, "force_iters > max_iters");
  ad_stats st{};
  st.converged = 1;
  st.alpha = op->alpha;
  const long long l0 = launch_counter();
  const void* vd;
  AD_TRY(stage_in(op, v, 0, &vd, true));
  void* od = is_device_ptr(out) ? out : nullptr;
  if (!od) od = op->S1;
  int r = phi1_device(op, vd, od, dt, tol, force_iters < 0 ? -1 : force_iters, &st);
  if (r != AD_OK && r != AD_ERR_NOT_CONVERGED) return r;
  if (r != AD_OK && op->adaptive && force_iters < 0) {   // gave up: out is not written
    CUDA_TRY(cudaStreamSynchronize(op->stream));
  } else {
    AD_TRY(finish_out(op, out, od));
  }
  st.kernel_launches += (int)(launch_counter() - l0);
  if (stats) *stats = st;
  if (r == AD_ERR_NOT_CONVERGED) return fail(r, "Leja series reached max_iters");
  return AD_OK;
}

}  // extern "C"

namespace {

// One step (ad_expquad_step).  async (device u, fixed rule, one substep): no
// synchronisation; the series report to the operator's async totals.
int expquad_impl(ad_operator* op, void* u, double t, double dt, int s, const double* c,
                 const ad_source* src, double tol, int force_iters, ad_stats* stats, bool async) {
  if (!op || !u || !c) return fail(AD_ERR_INVALID, "NULL argument");
  if (!(dt > 0) || !std::isfinite(dt) || !std::isfinite(t)) return fail(AD_ERR_INVALID, "bad t or dt");
  if (s != 1 && s != 2) return fail(AD_ERR_INVALID, "s must be 1 or 2");
  if (s == 2 && !(c[0] != c[1])) return fail(AD_ERR_INVALID, "s = 2 needs c[0] != c[1]");
  if (force_iters < 0 && !(tol > 0)) return fail(AD_ERR_INVALID, "tol must be positive");
  if (force_iters > op->max_iters) return fail(AD_ERR_INVALID, "force_iters > max_iters");
  Sources S;
  AD_TRY(fill_sources(src, kMaxSources, &S));
  ad_stats st{};
  st.converged = 1;
  st.alpha = op->alpha;
  const long long l0 = launch_counter();
  const void* ud_c;
  AD_TRY(stage_in(op, u, 0, &ud_c, true));
  void* ud = const_cast<void*>(ud_c);
  const long long n = op->g.n;
  const int force = force_iters < 0 ? -1 : force_iters;
  int status = AD_OK;
  // FP64 steps of one substep under the fixed rule: the whole step in one
  // launch of the tile kernel when it fits (apply, series start, series and
  // update fused); false if it cannot run, with nothing enqueued.
  auto try_fused = [&](int kind, double b, int* r_out) -> bool {
    if (op->prec != 0 || (op->adaptive && force < 0) || n_substeps(op, dt) != 1) return false;
    double d0 = 0.0, eta0[2] = {0.0, 1.0}, eta_next[2];
    if (upload_series(op, kind, dt, eta0, &d0, eta_next) != AD_OK) return false;
    StepFuse F{};
    F.s = kind == 1 ? 2 : 1;
    F.W = op->W;
    F.u = static_cast<double*>(ud);
    F.w1 = static_cast<double*>(op->W1);
    F.src = S;
    F.d0 = d0;
    F.b = b;
    F.force = force;
    F.max_iters = op->max_iters;
    F.tol = tol;
    F.totals = async ? op->totals : nullptr;
    F.timed = op->time_series ? 1 : 0;
    int it = 0;
    const int r = run_series(op, kind, nullptr, d0, force, tol, &st, &it, nullptr, async, &F);
    if (r == kNotFused) return false;
    st.matvecs += 1;
    st.substeps = 1;
    *r_out = r;
    return true;
  };
  // FP32 midpoint steps of one substep under the fixed rule: the series start
  // y_0 = A u + sources, p_0 = d0 y_0 in one ring pass (series_start_f32)
  // instead of the apply and start kernels, and u += dt P as the tail.
  auto try_started_f32 = [&](int* r_out) -> bool {
    if (op->prec != 1 || (op->adaptive && force < 0) || n_substeps(op, dt) != 1 || force == 0)
      return false;
    double d0 = 0.0, eta_next[2];
    if (upload_series(op, 0, dt, nullptr, &d0, eta_next) != AD_OK) return false;
    if (!series_start_f32(series_args(op, 0), ud, S, d0, force, op->max_iters, tol, op->stream))
      return false;
    Tail tail;
    tail.add(1.0, ud, dt, op->P, ud);
    int it = 0;
    *r_out = run_series(op, 0, nullptr, d0, force, tol, &st, &it, &tail, async, nullptr, true,
                        ud, dt);
    st.matvecs += 1;
    st.substeps = 1;
    return true;
  };
  int rf = AD_OK;
  if (s == 1) {
    // v = A u + S(t + c1 dt);  u += dt phi_1(dt A) v   (Eq. exp_midpoint for c1 = 1/2)
    for (int k = 0; k < S.n; ++k) S.a[k] = h_at(src, k, t + c[0] * dt);
  }
  if (s == 1 && (try_fused(0, dt, &rf) || try_started_f32(&rf))) {
    if (rf != AD_OK && rf != AD_ERR_NOT_CONVERGED) return rf;
    status = rf;
  } else if (s == 1) {
    apply(op, ud, op->W1, nullptr, S);
    st.matvecs += 1;
    // a non-converged fixed step is still applied (with the last series);
    // adaptive control that gave up leaves u unchanged
    const bool fixed = !(op->adaptive && force < 0);
    Tail post;
    post.add(1.0, ud, dt, op->W2, ud);
    const int r =
        phi1_device(op, op->W1, op->W2, dt, tol, force, &st, fixed ? &post : nullptr, async);
    if (r != AD_OK && r != AD_ERR_NOT_CONVERGED) return r;
    status = r;
    if (!fixed && r == AD_OK) axpby(op->prec, n, 1.0, ud, dt, op->W2, ud, op->stream);
  } else {
    // w1 = A u + (c2 S1 - c1 S2)/(c2 - c1), w2 = (S2 - S1)/((c2 - c1) dt);
    // u += top block of exp(dt [[A, W], [0, J]]) [0; 0; 1]
    const double c1 = c[0], c2 = c[1];
    for (int k = 0; k < S.n; ++k) {
      const double h1 = h_at(src, k, t + c1 * dt), h2 = h_at(src, k, t + c2 * dt);
      S.a[k] = (c2 * h1 - c1 * h2) / (c2 - c1);
      S.b[k] = (h2 - h1) / ((c2 - c1) * dt);
    }
    const bool fused = try_fused(1, 1.0, &rf);
    if (fused && rf != AD_OK && rf != AD_ERR_NOT_CONVERGED) return rf;
    if (fused) status = rf;
    if (!fused) {
      apply(op, ud, op->W1, op->W2, S);
      st.matvecs += 1;
    }
    double eta[2] = {0.0, 1.0};
    if (fused) {
      // done in the tile kernel
    } else if (op->adaptive && force < 0) {
      // adaptive substep control: exp(h_k Atilde) applied to the accepted state
      SubstepCtl ctl(dt, n_substeps(op, dt), op->max_iters);
      bool have_x = false, finished = false;
      for (;;) {
        bool last;
        const double hs = ctl.next(&last);
        double d0, eta_next[2];
        AD_TRY(upload_series(op, 1, hs, eta, &d0, eta_next));
        ad_stats at{};
        at.converged = 1;
        int it = 0;
        const int r = run_series(op, 1, have_x ? op->T2 : nullptr, d0, -1, tol, &at, &it);
        if (r != AD_OK && r != AD_ERR_NOT_CONVERGED) return r;
        add_attempt(&st, at, r == AD_OK);
        if (r != AD_OK) {
          if (!ctl.reject(hs)) break;
          continue;
        }
        advance_eta(op, it, eta);
        if (last) {
          ++ctl.accepted;
          finished = true;
          break;
        }
        axpby(op->prec, n, 1.0, op->P, 0.0, nullptr, op->T2, op->stream);
        have_x = true;
        if (!ctl.accept(hs, it)) break;
      }
      st.substeps = ctl.accepted;
      st.rejected = ctl.rejected;
      if (finished) {
        axpby(op->prec, n, 1.0, ud, 1.0, op->P, ud, op->stream);
      } else {   // gave up: u is left unchanged
        status = AD_ERR_NOT_CONVERGED;
        st.converged = 0;
      }
    } else {
      const int K = n_substeps(op, dt);
      const double h = dt / K;
      st.substeps = K;
      for (int k = 0; k < K; ++k) {
        double d0, eta_next[2];
        AD_TRY(upload_series(op, 1, h, eta, &d0, eta_next));
        int it = 0;
        // the next substep starts from P (copied: its series rewrites P); the
        // last one adds P to u
        Tail tail;
        if (k + 1 < K) tail.add(1.0, op->P, 0.0, nullptr, op->T2);
        else tail.add(1.0, ud, 1.0, op->P, ud);
        const int r = run_series(op, 1, k == 0 ? nullptr : op->T2, d0, force, tol, &st, &it,
                                 &tail, async);
        if (r != AD_OK && r != AD_ERR_NOT_CONVERGED) return r;
        if (r != AD_OK) status = r;
        if (k + 1 < K) advance_eta(op, it, eta);
      }
    }
  }
  CUDA_TRY(cudaGetLastError());
  if (!async) AD_TRY(finish_out(op, u, ud));
  st.kernel_launches += (int)(launch_counter() - l0);
  if (stats) *stats = st;
  if (status == AD_ERR_NOT_CONVERGED) return fail(status, "Leja series reached max_iters");
  return AD_OK;
}

}  // namespace

extern "C" {

int ad_expquad_step(ad_operator* op, void* u, double t, double dt, int s, const double* c,
                    const ad_source* src, double tol, int force_iters, ad_stats* stats) {
  g_err.clear();
  return expquad_impl(op, u, t, dt, s, c, src, tol, force_iters, stats, false);
}

int ad_expquad_step_async(ad_operator* op, void* u, double t, double dt, int s, const double* c,
                          const ad_source* src, double tol) {
  g_err.clear();
  if (!op || !u) return fail(AD_ERR_INVALID, "NULL argument");
  const bool async = is_device_ptr(u) && !op->adaptive && std::isfinite(dt) && dt > 0 &&
                     n_substeps(op, dt) == 1;
  ad_stats st{};
  const int r = expquad_impl(op, u, t, dt, s, c, src, tol, -1, &st, async);
  if (r != AD_OK && r != AD_ERR_NOT_CONVERGED) return r;
  // what the host knows of this step (the device adds the series)
  ad_stats& h = op->async_host;
  h.iters += st.iters;
  h.matvecs += st.matvecs;
  h.substeps += st.substeps;
  h.rejected += st.rejected;
  h.kernel_launches += st.kernel_launches;
  h.err_est = std::max(h.err_est, st.err_est);
  if (r == AD_ERR_NOT_CONVERGED) op->async_worst = std::max(op->async_worst, (int)AD_ERR_NOT_CONVERGED);
  g_err.clear();
  return AD_OK;
}

int ad_async_totals(ad_operator* op, ad_stats* stats) {
  g_err.clear();
  if (!op) return fail(AD_ERR_INVALID, "op is NULL");
  CUDA_TRY(cudaMemcpyAsync(op->h_totals, op->totals, sizeof(AsyncTotals), cudaMemcpyDeviceToHost,
                           op->stream));
  CUDA_TRY(cudaStreamSynchronize(op->stream));
  const AsyncTotals T = *op->h_totals;
  ad_stats r = op->async_host;
  r.iters += (int)T.iters;
  r.matvecs += (int)T.iters;
  r.kernel_launches += (int)T.launches;
  r.err_est = std::max(r.err_est, T.err_est);
  r.alpha = op->alpha;
  const int worst = std::max(op->async_worst, T.status);
  r.converged = worst == 0 ? 1 : 0;
  if (op->time_series) {   // the event pairs of the series enqueued with timing
    for (int k = 0; k < op->atev_used; ++k) {
      float ms = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&ms, op->atev[2 * k], op->atev[2 * k + 1]));
      op->t_ms += ms;
    }
    op->t_series += op->atev_used;
    op->t_iters += T.timed_iters;
  }
  op->atev_used = 0;
  op->async_host = ad_stats{};
  op->async_worst = 0;
  CUDA_TRY(cudaMemsetAsync(op->totals, 0, sizeof(AsyncTotals), op->stream));
  if (stats) *stats = r;
  if (worst == 4) op->ctrl_dirty = true;
  if (worst == 4) return fail(AD_ERR_TIMEOUT, "an asynchronous series did not reach its stop state");
  if (worst == 3) return fail(AD_ERR_NOT_CONVERGED, "an asynchronous series reached max_iters");
  return AD_OK;
}

int ad_penalty_beta(const ad_grid* grid, const double* Dxx, const double* Dxy, const double* Dyy,
                    void* cuda_stream, double* beta) {
  g_err.clear();
  if (!grid || !Dxx || !Dxy || !Dyy || !beta) return fail(AD_ERR_INVALID, "NULL argument");
  if (grid->nx < 1 || grid->ny < 1) return fail(AD_ERR_INVALID, "grid: nx, ny must be >= 1");
  for (const void* p : {(const void*)Dxx, (const void*)Dxy, (const void*)Dyy})
    if (!is_device_ptr(p)) return fail(AD_ERR_INVALID, "D fields must be device pointers");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const long long n = (long long)grid->nx * grid->ny;
  const int nb = stream_blocks(n);
  double v = 0.0;
  if (lambda_max_reduce(n, Dxx, Dxy, Dyy, nb, s, &v) != 0) {
    cudaGetLastError();
    return fail(AD_ERR_CUDA, "ad_penalty_beta: reduction failed");
  }
  *beta = v;
  return AD_OK;
}

int ad_penalised_step(ad_operator* op, void* u, double t, double dt, const ad_source* src,
                      double beta, double cg_tol, int max_cg, ad_stats* stats) {
  g_err.clear();
  if (!op || !u) return fail(AD_ERR_INVALID, "NULL argument");
  if (op->prec != AD_FP64) return fail(AD_ERR_INVALID, "ad_penalised_step needs an AD_FP64 operator");
  if (!(dt > 0) || !std::isfinite(dt) || !std::isfinite(t)) return fail(AD_ERR_INVALID, "bad t or dt");
  if (!(beta >= 0) || !std::isfinite(beta)) return fail(AD_ERR_INVALID, "beta must be finite and >= 0");
  if (!(cg_tol > 0)) return fail(AD_ERR_INVALID, "cg_tol must be positive");
  if (max_cg < 1) return fail(AD_ERR_INVALID, "max_cg must be >= 1");
  Sources S;
  AD_TRY(fill_sources(src, kMaxSources, &S));
  for (int k = 0; k < S.n; ++k) S.a[k] = h_at(src, k, t);
  ad_stats st{};
  st.converged = 1;
  st.alpha = op->alpha;
  st.substeps = 1;
  const long long l0 = launch_counter();
  const void* ud_c;
  AD_TRY(stage_in(op, u, 0, &ud_c, true));
  void* ud = const_cast<void*>(ud_c);
  const long long n = op->g.n;
  double* r = static_cast<double*>(op->T1);
  double* pdir = static_cast<double*>(op->T2);
  double* Mp = static_cast<double*>(op->T3);
  double* x = static_cast<double*>(op->W1);
  // b = dt (A u + S(t)); x = 0, r = b, p = b
  apply(op, ud, r, nullptr, S);
  axpby(0, n, dt, r, 0.0, nullptr, r, op->stream);
  axpby(0, n, 0.0, nullptr, 0.0, nullptr, x, op->stream);
  axpby(0, n, 1.0, r, 0.0, nullptr, pdir, op->stream);
  st.matvecs += 1;
  norm2_partials(0, n, r, op->partials, op->nblocks, op->stream);
  reduce_partials(op->partials, op->nblocks, 0, op->dscal + 3, op->stream);
  CUDA_TRY(cudaMemcpyAsync(op->h_scal, op->dscal + 3, sizeof(double), cudaMemcpyDeviceToHost,
                           op->stream));
  CUDA_TRY(cudaStreamSynchronize(op->stream));
  const double rr0 = op->h_scal[0];
  double rr = rr0;
  int it = 0;
  const double dx = (op->grid.x1 - op->grid.x0) / op->grid.nx;
  const double dy = (op->grid.y1 - op->grid.y0) / op->grid.ny;
  const int chunk = 8;                  // CG iterations between host reads of <r, r>
  while (rr0 > 0.0 && !(std::sqrt(rr) <= cg_tol * std::sqrt(rr0)) && it < max_cg) {
    const int q = std::min(chunk, max_cg - it);
    for (int k = 0; k < q; ++k)
      penalty_cg_iteration(op->g, dx, dy, dt * beta, x, r, pdir, Mp, op->partials, op->nblocks,
                           op->dscal, op->stream);
    it += q;
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(op->h_scal, op->dscal + 3, sizeof(double), cudaMemcpyDeviceToHost,
                             op->stream));
    CUDA_TRY(cudaStreamSynchronize(op->stream));
    rr = op->h_scal[0];
    if (!std::isfinite(rr)) break;
  }
  st.iters = it;
  st.matvecs += it;
  st.err_est = rr0 > 0.0 ? std::sqrt(rr / rr0) : 0.0;
  const bool ok = rr0 == 0.0 || std::sqrt(rr) <= cg_tol * std::sqrt(rr0);
  if (ok) axpby(0, n, 1.0, ud, 1.0, x, ud, op->stream);     // u += delta
  else st.converged = 0;                                     // u is left unchanged
  CUDA_TRY(cudaGetLastError());
  AD_TRY(finish_out(op, u, ud));
  st.kernel_launches = (int)(launch_counter() - l0);
  if (stats) *stats = st;
  if (!ok) return fail(AD_ERR_NOT_CONVERGED, "conjugate gradients did not reach cg_tol");
  return AD_OK;
}

int ad_reserve_gmres(ad_operator* op, int max_restart) {
  g_err.clear();
  if (!op) return fail(AD_ERR_INVALID, "NULL argument");
  if (op->prec != AD_FP64) return fail(AD_ERR_INVALID, "GMRES needs an AD_FP64 operator");
  if (max_restart < 1 || max_restart > kMaxGmres)
    return fail(AD_ERR_INVALID, "max_restart must be in [1, 200]");
  if (op->vk_cols >= max_restart + 1) return AD_OK;
  if (op->stream) CUDA_TRY(cudaStreamSynchronize(op->stream));
  if (op->Vk) cudaFree(op->Vk);
  op->Vk = nullptr;
  op->vk_cols = 0;
  if (cudaMalloc(&op->Vk, sizeof(double) * (size_t)(max_restart + 1) * op->g.n) != cudaSuccess) {
    cudaGetLastError();
    return fail(AD_ERR_NOMEM, "GMRES basis");
  }
  op->vk_cols = max_restart + 1;
  return AD_OK;
}

int ad_cn_step(ad_operator* op, void* u, double t, double dt, const ad_source* src,
               double gmres_tol, int restart, int force_iters, ad_stats* stats) {
  g_err.clear();
  if (!op || !u) return fail(AD_ERR_INVALID, "NULL argument");
  if (op->prec != AD_FP64) return fail(AD_ERR_INVALID, "ad_cn_step needs an AD_FP64 operator");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(AD_ERR_INVALID, "dt must be positive");
  if (restart < 1 || restart > kMaxGmres) return fail(AD_ERR_INVALID, "restart must be in [1, 200]");
  if (force_iters > restart) return fail(AD_ERR_INVALID, "force_iters > restart");
  if (force_iters <= 0 && !(gmres_tol > 0)) return fail(AD_ERR_INVALID, "gmres_tol must be positive");
  Sources S;
  AD_TRY(fill_sources(src, kMaxSources, &S));
  const long long n = op->g.n;
  const int m = force_iters > 0 ? force_iters : restart;
  if (op->vk_cols < m + 1)
    return fail(AD_ERR_INVALID, "GMRES basis too small for this restart: call "
                                "ad_reserve_gmres(op, restart) first");
  ad_stats st{};
  st.converged = 1;
  st.alpha = op->alpha;
  const long long l0 = launch_counter();
  const void* ud_c;
  AD_TRY(stage_in(op, u, 0, &ud_c, true));
  double* x = (double*)const_cast<void*>(ud_c);
  double* b = (double*)op->T1;
  double* w = (double*)op->T2;
  double* V = op->Vk;
  const int nb = op->nblocks;
  cudaStream_t s = op->stream;
  // b = u + dt/2 A u + dt/2 (S(t) + S(t + dt))
  for (int k = 0; k < S.n; ++k) S.a[k] = 0.5 * dt * (h_at(src, k, t) + h_at(src, k, t + dt));
  {
    apply_shifted_f64(op->g, op->W, x, b, 1.0, 0.5 * dt, s);
    if (S.n > 0) {
      // add the source combination: b += sum a_k g_k  (apply with zero field -> sources only)
      for (int k = 0; k < S.n; ++k)
        axpby(0, n, S.a[k], S.g[k], 1.0, b, b, s);
    }
  }
  st.matvecs += 1;
  auto read_scalars = [&](int count) -> int {
    CUDA_TRY(cudaMemcpyAsync(op->h_scal, op->dscal, sizeof(double) * count, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return AD_OK;
  };
  norm2_partials(0, n, b, op->partials, nb, s);
  reduce_partials(op->partials, nb, 2, op->dscal, s);
  AD_TRY(read_scalars(1));
  const double bnorm = op->h_scal[0];
  if (bnorm == 0.0) {
    axpby(0, n, 0.0, nullptr, 0.0, nullptr, x, s);
    AD_TRY(finish_out(op, u, x));
    if (stats) *stats = st;
    return AD_OK;
  }
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  auto Hc = [&](int i, int k) -> double& { return H[(size_t)i * m + k]; };
  int total_iters = 0;
  const int max_total = force_iters > 0 ? force_iters : 5000;
  for (;;) {
    // r = b - M x, M = I - dt/2 A
    apply_shifted_f64(op->g, op->W, x, w, 1.0, -0.5 * dt, s);
    axpby(0, n, 1.0, b, -1.0, w, V, s);
    st.matvecs += 1;
    norm2_partials(0, n, V, op->partials, nb, s);
    reduce_partials(op->partials, nb, 2, op->dscal, s);
    AD_TRY(read_scalars(1));
    const double beta = op->h_scal[0];
    st.err_est = beta / bnorm;
    if (force_iters <= 0 && (beta / bnorm <= gmres_tol || total_iters >= max_total)) {
      st.converged = beta / bnorm <= gmres_tol;
      break;
    }
    axpby(0, n, 1.0 / beta, V, 0.0, nullptr, V, s);
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int kused = 0;
    for (int k = 0; k < m; ++k) {
      double* Vk = V + (size_t)k * n;
      double* Vn = V + (size_t)(k + 1) * n;
      apply_shifted_f64(op->g, op->W, Vk, Vn, 1.0, -0.5 * dt, s);
      st.matvecs += 1;
      ++total_iters;
      // classical Gram-Schmidt, twice
      multi_dot_partials(n, V, n, k + 1, Vn, op->partials, nb, s);
      multi_dot_finalize(op->partials, nb, k + 1, op->dscal, s);
      multi_axpy_norm(n, V, n, k + 1, op->dscal, Vn, op->partials, nb, s);
      multi_dot_partials(n, V, n, k + 1, Vn, op->partials, nb, s);
      multi_dot_finalize(op->partials, nb, k + 1, op->dscal + (k + 1), s);
      multi_axpy_norm(n, V, n, k + 1, op->dscal + (k + 1), Vn, op->partials, nb, s);
      reduce_partials(op->partials, nb, 2, op->dscal + 2 * (k + 1), s);
      CUDA_TRY(cudaGetLastError());
      AD_TRY(read_scalars(2 * (k + 1) + 1));
      for (int i = 0; i <= k; ++i) Hc(i, k) = op->h_scal[i] + op->h_scal[k + 1 + i];
      const double hk1 = op->h_scal[2 * (k + 1)];
      Hc(k + 1, k) = hk1;
      if (hk1 != 0.0) axpby(0, n, 1.0 / hk1, Vn, 0.0, nullptr, Vn, s);
      for (int i = 0; i < k; ++i) {
        const double tmp = cs[i] * Hc(i, k) + sn[i] * Hc(i + 1, k);
        Hc(i + 1, k) = -sn[i] * Hc(i, k) + cs[i] * Hc(i + 1, k);
        Hc(i, k) = tmp;
      }
      const double den = std::hypot(Hc(k, k), Hc(k + 1, k));
      cs[k] = Hc(k, k) / den;
      sn[k] = Hc(k + 1, k) / den;
      Hc(k, k) = den;
      Hc(k + 1, k) = 0.0;
      g[k + 1] = -sn[k] * g[k];
      g[k] = cs[k] * g[k];
      kused = k + 1;
      if (force_iters <= 0 && (std::fabs(g[k + 1]) <= gmres_tol * bnorm || total_iters >= max_total))
        break;
    }
    for (int i = kused - 1; i >= 0; --i) {      // back substitution
      double r = g[i];
      for (int j = i + 1; j < kused; ++j) r -= Hc(i, j) * y[j];
      y[i] = r / Hc(i, i);
    }
    CUDA_TRY(cudaMemcpyAsync(op->dscal, y.data(), sizeof(double) * kused, cudaMemcpyHostToDevice, s));
    multi_axpy_add(n, V, n, kused, op->dscal, x, s);
    CUDA_TRY(cudaStreamSynchronize(s));     // y lives on the host stack
    if (force_iters > 0) {
      st.err_est = std::fabs(g[kused]) / bnorm;
      break;
    }
  }
  st.iters = total_iters;
  CUDA_TRY(cudaGetLastError());
  AD_TRY(finish_out(op, u, x));
  st.kernel_launches += (int)(launch_counter() - l0);
  if (stats) *stats = st;
  if (!st.converged) return fail(AD_ERR_NOT_CONVERGED, "GMRES reached its iteration cap");
  return AD_OK;
}

int ad_fp64_fma_rate(int blocks_per_sm, int iters, void* cuda_stream, double* tflops) {
  g_err.clear();
  if (!tflops || blocks_per_sm < 1 || blocks_per_sm > 8 || iters < 1024 || iters > (1 << 24))
    return fail(AD_ERR_INVALID, "blocks_per_sm in [1, 8], iters in [1024, 2^24]");
  int dev = 0, sms = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (fp64_fma_rate(blocks_per_sm * sms, iters, (cudaStream_t)cuda_stream, tflops) != 0) {
    cudaGetLastError();
    return fail(AD_ERR_CUDA, "FP64 rate probe failed");
  }
  return AD_OK;
}

int ad_check_wait_timeout(double timeout_ms, void* cuda_stream) {
  g_err.clear();
  if (!(timeout_ms > 0) || timeout_ms > 1000.0) return fail(AD_ERR_INVALID, "timeout_ms in (0, 1000]");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int* d = nullptr;
  CUDA_TRY(cudaMalloc(&d, sizeof(int)));
  int h = -1;
  const int r = wait_timeout_probe((unsigned long long)(timeout_ms * 1e6), d, s);
  cudaError_t e1 = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  cudaFree(d);
  if (r != 0 || e1 != cudaSuccess || e2 != cudaSuccess) {
    cudaGetLastError();
    return fail(AD_ERR_CUDA, "wait probe launch failed");
  }
  if (h == 4) return fail(AD_ERR_TIMEOUT, "bounded device wait gave up (expected)");
  return fail(AD_ERR_INVALID, "the wait completed although nothing released it");
}

int ad_time_series(ad_operator* op, int enable) {
  g_err.clear();
  if (!op) return fail(AD_ERR_INVALID, "op is NULL");
  if (enable) {
    for (cudaEvent_t& e : op->tev)
      if (!e) CUDA_TRY(cudaEventCreate(&e));
    op->t_ms = 0.0;
    op->t_series = 0;
    op->t_iters = 0;
    op->t_path = 0;
  }
  op->time_series = enable != 0;
  return AD_OK;
}

int ad_series_timing(const ad_operator* op, double* ms, int* series, long long* iters,
                     int* kernel) {
  g_err.clear();
  if (!op || !ms || !series || !iters) return fail(AD_ERR_INVALID, "NULL argument");
  *ms = op->t_ms;
  *series = op->t_series;
  *iters = op->t_iters;
  if (kernel) *kernel = op->t_path;
  return AD_OK;
}

int ad_profile_leja_iteration(ad_operator* op, int aug, int reps, double* ms_per_launch) {
  g_err.clear();
  if (!op || !ms_per_launch) return fail(AD_ERR_INVALID, "NULL argument");
  if (aug != 0 && aug != 1) return fail(AD_ERR_INVALID, "aug must be 0 or 1");
  if (reps < 1 || reps > kMaxIters) return fail(AD_ERR_INVALID, "reps must be in [1, 500]");
  // a forced series on a SplitMix64 start vector with couplings w1 = w2 = start
  double d0 = 0.0, eta[2] = {0.0, 1.0}, eta_out[2];
  AD_TRY(upload_series(op, aug, 1e-3 / op->gamma, eta, &d0, eta_out));
  splitmix_fill(op->prec, op->g.n, 7ULL, op->W1, op->stream);
  splitmix_fill(op->prec, op->g.n, 8ULL, op->W2, op->stream);
  SeriesArgs a = series_args(op, aug);
  series_init(a, op->W1, d0, reps, op->max_iters, 0.0, op->stream);
  if (!getenv("AD_NO_PERSIST") && op->prec == 0 && op->g.n <= kPersistMaxCells) {
    // the persistent kernel runs the whole series: one launch of `reps` iterations
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    CUDA_TRY(cudaEventRecord(e0, op->stream));
    const bool ok = series_run_persistent(a, &op->ctrl->gen, &op->nsync, op->stream) != 0;
    CUDA_TRY(cudaEventRecord(e1, op->stream));
    CUDA_TRY(cudaStreamSynchronize(op->stream));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ok) {
      op->cache_kind = -1;
      *ms_per_launch = ms / reps;
      return AD_OK;
    }
    series_init(a, op->W1, d0, reps, op->max_iters, 0.0, op->stream);
  }
  // pair mode: each launch runs two iterations
  const int per = series_pair(a) ? 2 : 1;
  const int launches = (reps + per - 1) / per;
  std::vector<cudaEvent_t> ev(2 * launches);
  for (auto& e : ev) CUDA_TRY(cudaEventCreate(&e));
  for (int r = 0; r < launches; ++r) {
    CUDA_TRY(cudaEventRecord(ev[2 * r], op->stream));
    series_iteration(a, op->stream);
    CUDA_TRY(cudaEventRecord(ev[2 * r + 1], op->stream));
  }
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(op->stream));
  double total = 0.0;
  for (int r = 0; r < launches; ++r) {
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, ev[2 * r], ev[2 * r + 1]));
    total += ms;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  op->cache_kind = -1;
  *ms_per_launch = total / ((double)launches * per);
  return AD_OK;
}

}  // extern "C"
