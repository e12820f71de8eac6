// The inner self-consistency loop of GF2 (the supplement's steps 2.a-2.b) as
// one CUDA graph that decides everything on the device.
//
// Graph:  WHILE (inner) {
//           moment basis of the tail at the current F           (FP64 GEMMs)
//           mu search: start + WHILE (one count evaluation)      (step 2.a)
//           F_out = Fock(P)                                      (step 2.b, Eq. FockMatrix)
//           R = F_out - F;  R.R and R.R_k for the stored residuals
//           controller (one thread): converged / damped step / Pulay step
//           update of F and of the residual history
//         }
//         moment basis + mu search at the converged F
//
// The schedule of the next F is the one the host loop takes: while |R| exceeds
// diis_from, the damped step F + mix R (the history restarts); below it, the
// Pulay (DIIS) combination of the last `diis` rebuilt matrices F_out, whose
// weights minimise |sum_k c_k R_k| under sum_k c_k = 1.  The host reads one
// block of scalars after the graph.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "gf2_internal.cuh"

namespace {

constexpr int kDiisMax = 8;
constexpr int kThreads = 256;

struct InnerState {
  // read by the mu search's start kernel: {mu0, n_elec, tol, max_iter}
  double mu, n_elec, mu_tol, mu_max_iter;
  double r_norm;
  int status;      // 0 running, 1 converged, 2 iteration cap, 3 mu search failed, 4 non-finite residual
  int mu_status;   // the failed search's own status (gf2_mu_state::status)
  int iter, mu_evals;
  // inputs
  double tol, mix, diis_from;
  int max_iter, diis;
  // the residual history: m entries ending at ring slot `head`
  int m, head;
  int mode;        // update of F: 0 damped step, 1 Pulay combination, 2 F = F_out, 3 none
  int store;       // the new (F_out, R) goes into slot `head`
  double gram[kDiisMax][kDiisMax];  // R_a . R_b by ring slot
  double coef[kDiisMax];            // Pulay weights by ring slot
};

// the host reads this block after the graph
constexpr size_t kResultBytes = offsetof(InnerState, tol);
static_assert(kResultBytes <= 8 * sizeof(double), "result block fits the pinned scalars");

__global__ void inner_init_kernel(InnerState *st, double mu0, double n_elec, double mu_tol, int mu_max_iter,
                                  double tol, int max_iter, int diis, double mix, double diis_from) {
  if (threadIdx.x != 0) return;
  st->mu = mu0;
  st->n_elec = n_elec;
  st->mu_tol = mu_tol;
  st->mu_max_iter = (double)mu_max_iter;
  st->r_norm = 0.0;
  st->status = 0;
  st->mu_status = 0;
  st->iter = 0;
  st->mu_evals = 0;
  st->tol = tol;
  st->mix = mix;
  st->diis_from = diis_from;
  st->max_iter = max_iter;
  st->diis = diis;
  st->m = 0;
  st->head = 0;
  st->mode = 3;
  st->store = 0;
}

__global__ void inner_resid_kernel(int n, const double *__restrict__ F_out, const double *__restrict__ F,
                                   double *__restrict__ R) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) R[e] = F_out[e] - F[e];
}

// block k < diis: R . R_k (ring slot k); block kDiisMax: R . R.  Fixed order.
__global__ void inner_dots_kernel(const InnerState *st, int n, const double *__restrict__ R,
                                  const double *__restrict__ ringR, double *__restrict__ dots) {
  __shared__ double red[kThreads];
  const int k = blockIdx.x;
  if (k < kDiisMax && k >= st->diis) return;
  const double *other = k == kDiisMax ? R : ringR + (size_t)k * n;
  double acc = 0.0;
  for (int e = threadIdx.x; e < n; e += kThreads) acc += R[e] * other[e];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) dots[k] = red[0];
}

// Pulay weights of the m stored residuals (slots oldest first): the bordered
// system [B -1; -1 0] [c; lambda] = [0; -1] with B_ab = R_a . R_b scaled by its
// largest diagonal entry, by Gaussian elimination with partial pivoting.  A
// (numerically) singular system drops the oldest residual and tries again.
// Returns the number of residuals used (1: take the newest F_out).
__device__ int pulay_weights(InnerState *st) {
  const int d = st->diis;
  while (st->m > 1) {
    const int m = st->m, n = m + 1;
    int slot[kDiisMax];
    for (int j = 0; j < m; ++j) slot[j] = (st->head - (m - 1) + j + d) % d;
    double scale = 0.0;
    for (int j = 0; j < m; ++j) scale = fmax(scale, st->gram[slot[j]][slot[j]]);
    if (!(scale > 0.0) || !isfinite(scale)) return 1;
    double A[kDiisMax + 1][kDiisMax + 2];
    for (int i = 0; i < m; ++i) {
      for (int j = 0; j < m; ++j) A[i][j] = st->gram[slot[i]][slot[j]] / scale;
      A[i][m] = -1.0;
      A[i][n] = 0.0;
    }
    for (int j = 0; j < m; ++j) A[m][j] = -1.0;
    A[m][m] = 0.0;
    A[m][n] = -1.0;
    bool singular = false;
    for (int c = 0; c < n && !singular; ++c) {
      int p = c;
      for (int r = c + 1; r < n; ++r)
        if (fabs(A[r][c]) > fabs(A[p][c])) p = r;
      if (fabs(A[p][c]) < 1e-14) {
        singular = true;
        break;
      }
      if (p != c)
        for (int j = 0; j <= n; ++j) {
          const double t = A[c][j];
          A[c][j] = A[p][j];
          A[p][j] = t;
        }
      for (int r = c + 1; r < n; ++r) {
        const double f = A[r][c] / A[c][c];
        for (int j = c; j <= n; ++j) A[r][j] -= f * A[c][j];
      }
    }
    if (!singular) {
      double x[kDiisMax + 1];
      for (int r = n - 1; r >= 0; --r) {
        double s = A[r][n];
        for (int j = r + 1; j < n; ++j) s -= A[r][j] * x[j];
        x[r] = s / A[r][r];
      }
      for (int j = 0; j < m; ++j) st->coef[slot[j]] = x[j];
      return m;
    }
    --st->m;  // the oldest residual leaves the history
  }
  return 1;
}

__global__ void inner_control_kernel(InnerState *st, const gf2_mu_state *ms, const double *dots,
                                     cudaGraphConditionalHandle loop) {
  if (threadIdx.x != 0) return;
  ++st->iter;
  st->mu_evals += ms->evals;
  st->store = 0;
  st->mode = 3;
  if (ms->status != 1) {
    st->status = 3;
    st->mu_status = ms->status;
    cudaGraphSetConditional(loop, 0u);
    return;
  }
  st->mu = ms->mu_out;
  const double r = sqrt(dots[kDiisMax]);
  st->r_norm = r;
  if (!isfinite(r)) {
    st->status = 4;
  } else if (r < st->tol) {
    st->mode = 2;
    st->status = 1;
  } else if (r > st->diis_from || st->diis <= 0) {
    st->m = 0;
    st->mode = 0;
  } else {
    const int d = st->diis;
    const int slot = st->m == 0 ? 0 : (st->head + 1) % d;
    if (st->m < d) ++st->m;
    st->head = slot;
    st->store = 1;
    for (int k = 0; k < d; ++k) st->gram[slot][k] = st->gram[k][slot] = dots[k];
    st->gram[slot][slot] = dots[kDiisMax];
    st->mode = pulay_weights(st) > 1 ? 1 : 2;
  }
  if (st->status == 0 && st->iter >= st->max_iter) st->status = 2;
  cudaGraphSetConditional(loop, st->status == 0 ? 1u : 0u);
}

__global__ void inner_update_kernel(const InnerState *st, int n, double *__restrict__ F,
                                    const double *__restrict__ F_out, const double *__restrict__ R,
                                    double *__restrict__ ringF, double *__restrict__ ringR) {
  const int mode = st->mode, head = st->head, m = st->m, d = st->diis;
  const bool store = st->store;
  const double mix = st->mix;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const double fo = F_out[e];
    if (store) {
      ringF[(size_t)head * n + e] = fo;
      ringR[(size_t)head * n + e] = R[e];
    }
    if (mode == 0) {
      F[e] += mix * R[e];
    } else if (mode == 1) {
      double acc = 0.0;  // oldest first
      for (int j = 0; j < m; ++j) {
        const int s = (head - (m - 1) + j + d) % d;
        acc += st->coef[s] * (s == head ? fo : ringF[(size_t)s * n + e]);
      }
      F[e] = acc;
    } else if (mode == 2) {
      F[e] = fo;
    }
  }
}

__global__ void inner_finish_kernel(InnerState *st, const gf2_mu_state *ms) {
  if (threadIdx.x != 0) return;
  st->mu_evals += ms->evals;
  if (st->status != 1) return;
  if (ms->status != 1) {
    st->status = 3;
    st->mu_status = ms->status;
  } else {
    st->mu = ms->mu_out;
  }
}

// device workspace of the loop, in doubles
struct InnerWs {
  InnerState *st;
  double *F_out, *R, *ringF, *ringR, *dots;
};

InnerWs inner_ws(gf2_ctx *ctx) {
  const size_t n = (size_t)ctx->N * ctx->N;
  uint8_t *base = static_cast<uint8_t *>(ctx->d_inner_ws);
  double *d = reinterpret_cast<double *>(base + ((sizeof(InnerState) + 255) / 256) * 256);
  InnerWs w;
  w.st = reinterpret_cast<InnerState *>(base);
  w.F_out = d;
  w.R = w.F_out + n;
  w.ringF = w.R + n;
  w.ringR = w.ringF + kDiisMax * n;
  w.dots = w.ringR + kDiisMax * n;
  return w;
}

size_t inner_ws_bytes(int N) {
  const size_t n = (size_t)N * N;
  return ((sizeof(InnerState) + 255) / 256) * 256 + sizeof(double) * ((2 + 2 * kDiisMax) * n + kDiisMax + 1);
}

// launches through the library's helpers go to ctx->stream: point it at a
// capturing stream (and keep the event profiler off) for the guard's lifetime
struct StreamSwap {
  gf2_ctx *ctx;
  cudaStream_t saved;
  bool prof;
  long long launches;
  StreamSwap(gf2_ctx *c, cudaStream_t s) : ctx(c), saved(c->stream), prof(c->prof_on), launches(c->launches) {
    c->stream = s;
    c->prof_on = false;
  }
  long long counted() const { return ctx->launches - launches; }
  ~StreamSwap() {
    ctx->stream = saved;
    ctx->prof_on = prof;
    ctx->launches = launches;  // captured, not launched: counted when the graph runs
  }
};

gf2_status capture_fail(gf2_ctx *ctx, cudaStream_t s, cudaError_t e, const char *what) {
  cudaGraph_t g = nullptr;
  cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cst) == cudaSuccess && cst != cudaStreamCaptureStatusNone) {
    cudaStreamEndCapture(s, &g);
  }
  (void)cudaGetLastError();
  return gf2_cuda_fail(ctx, e, what);
}

// the loop body, captured on s2 (its nested mu search body on s3)
gf2_status capture_body(gf2_ctx *ctx, cudaStream_t s2, cudaStream_t s3, const double *S, const double *h,
                        double *F, const double *Sig, const double *sig12, double *G, double *P,
                        cudaGraphConditionalHandle loop, long long *kernels) {
  const InnerWs w = inner_ws(ctx);
  const int n = ctx->N * ctx->N;
  const int blocks = std::min((n + kThreads - 1) / kThreads, 2 * ctx->num_sms);
  StreamSwap swap(ctx, s2);
  gf2_status st;
  if ((st = gf2_build_moment_basis(ctx, S, F, sig12, false)) != GF2_OK) return st;
  if ((st = gf2_capture_mu_search(ctx, s2, s3, S, F, Sig, G, P, &w.st->mu)) != GF2_OK) return st;
  if ((st = gf2_fock(ctx, h, P, w.F_out)) != GF2_OK) return st;
  inner_resid_kernel<<<blocks, kThreads, 0, s2>>>(n, w.F_out, F, w.R);
  inner_dots_kernel<<<kDiisMax + 1, kThreads, 0, s2>>>(w.st, n, w.R, w.ringR, w.dots);
  inner_control_kernel<<<1, 32, 0, s2>>>(w.st, static_cast<const gf2_mu_state *>(ctx->d_mu_state), w.dots, loop);
  inner_update_kernel<<<blocks, kThreads, 0, s2>>>(w.st, n, F, w.F_out, w.R, w.ringF, w.ringR);
  GF2_CK(ctx, cudaGetLastError());
  *kernels = swap.counted() + 1 + 4;  // + the search's start kernel and the four above
  return GF2_OK;
}

gf2_status build_inner_graph(gf2_ctx *ctx, const double *S, const double *h, double *F, const double *Sig,
                             const double *sig12, double *G, double *P) {
  const void *key[7] = {S, h, F, Sig, sig12, G, P};
  if (ctx->inner_graph_exec && std::equal(key, key + 7, ctx->inner_graph_key)) return GF2_OK;
  if (ctx->inner_graph_exec) cudaGraphExecDestroy(ctx->inner_graph_exec);
  if (ctx->inner_graph) cudaGraphDestroy(ctx->inner_graph);
  ctx->inner_graph_exec = nullptr;
  ctx->inner_graph = nullptr;
  if (!ctx->d_mu_state) GF2_CK(ctx, cudaMalloc(&ctx->d_mu_state, sizeof(gf2_mu_state)));
  for (cudaStream_t *s : {&ctx->capture_stream, &ctx->capture_stream2, &ctx->capture_stream3})
    if (!*s) GF2_CK(ctx, cudaStreamCreateWithFlags(s, cudaStreamNonBlocking));
  cudaStream_t s1 = ctx->capture_stream2, s2 = ctx->capture_stream3, s3 = ctx->capture_stream;
  const InnerWs w = inner_ws(ctx);

  cudaGraph_t top = nullptr;
  GF2_CK(ctx, cudaGraphCreate(&top, 0));
  ctx->inner_graph = top;
  cudaGraphConditionalHandle loop;
  GF2_CK(ctx, cudaGraphConditionalHandleCreate(&loop, top, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = loop;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t loop_node;
  GF2_CK(ctx, cudaGraphAddNode(&loop_node, top, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];

  cudaError_t e = cudaStreamBeginCaptureToGraph(s2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return capture_fail(ctx, s2, e, "inner loop graph: begin body capture");
  long long per_iter = 0;
  gf2_status st = capture_body(ctx, s2, s3, S, h, F, Sig, sig12, G, P, loop, &per_iter);
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(s2, &captured);
  if (st != GF2_OK) return st;
  if (e != cudaSuccess) return capture_fail(ctx, s2, e, "inner loop graph: end of body capture");

  // after the loop: the search at the converged F
  e = cudaStreamBeginCaptureToGraph(s1, top, &loop_node, nullptr, 1, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return capture_fail(ctx, s1, e, "inner loop graph: begin tail capture");
  long long tail = 0;
  {
    StreamSwap swap(ctx, s1);
    st = gf2_build_moment_basis(ctx, S, F, sig12, false);
    if (st == GF2_OK) st = gf2_capture_mu_search(ctx, s1, s3, S, F, Sig, G, P, &w.st->mu);
    if (st == GF2_OK) {
      inner_finish_kernel<<<1, 32, 0, s1>>>(w.st, static_cast<const gf2_mu_state *>(ctx->d_mu_state));
      e = cudaGetLastError();
      if (e != cudaSuccess) st = gf2_cuda_fail(ctx, e, "inner_finish_kernel capture");
    }
    tail = swap.counted() + 2;
  }
  e = cudaStreamEndCapture(s1, &captured);
  if (st != GF2_OK) return st;
  if (e != cudaSuccess) return capture_fail(ctx, s1, e, "inner loop graph: end of tail capture");
  GF2_CK(ctx, cudaGraphInstantiate(&ctx->inner_graph_exec, top, 0));
  std::copy(key, key + 7, ctx->inner_graph_key);
  ctx->inner_kernels_per_iter = per_iter;
  ctx->inner_kernels_tail = tail;
  return GF2_OK;
}

}  // namespace

extern "C" gf2_status gf2_inner_loop(gf2_ctx *ctx, const double *d_S, const double *d_h, double *d_F,
                                     const double *d_Sigma_iw, const double *d_sig12, double n_elec,
                                     double *mu_inout, double *d_G_iw, double *d_P, double tol, int max_iter,
                                     double mu_tol, int diis, double mix, double diis_from, int *n_iter,
                                     int *n_mu_eval) {
  if (!ctx) return GF2_ERR_ARG;
  if (!d_S || !d_h || !d_F || !mu_inout || !d_G_iw || !d_P)
    return gf2_fail(ctx, GF2_ERR_ARG, "gf2_inner_loop: NULL pointer");
  if (!ctx->have_integrals) return gf2_fail(ctx, GF2_ERR_ARG, "gf2_inner_loop: gf2_set_integrals not called");
  if (!(tol > 0.0) || max_iter < 1 || !(mu_tol > 0.0) || diis < 0 || diis > kDiisMax ||
      !(mix > 0.0) || !std::isfinite(mix) || !(diis_from >= 0.0) || !std::isfinite(*mu_inout) ||
      !(n_elec > 0.0) || !(n_elec < 2.0 * ctx->N))
    return gf2_fail(ctx, GF2_ERR_ARG, "gf2_inner_loop: bad tol, max_iter, mu_tol, diis, mix, diis_from, mu or n_elec");
  const double *ptrs[] = {d_F, d_h, d_S};
  for (const double *q : ptrs)
    if (q == d_P || q == d_G_iw) return gf2_fail(ctx, GF2_ERR_ARG, "gf2_inner_loop: outputs alias inputs");
  if (!ctx->d_inner_ws) GF2_CK(ctx, cudaMalloc(&ctx->d_inner_ws, inner_ws_bytes(ctx->N)));
  gf2_status st = gf2_inverse_spd(ctx, d_S, ctx->d_small + (size_t)GF2_SL_SINV * ctx->N * ctx->N);  // fixed for the loop
  if (st != GF2_OK) return st;
  if ((st = build_inner_graph(ctx, d_S, d_h, d_F, d_Sigma_iw, d_sig12, d_G_iw, d_P)) != GF2_OK) return st;
  const InnerWs w = inner_ws(ctx);
  inner_init_kernel<<<1, 32, 0, ctx->stream>>>(w.st, *mu_inout, n_elec, mu_tol, 100, tol, max_iter, diis, mix,
                                               diis_from);
  GF2_CK_LAUNCH(ctx, "inner_init_kernel");
  GF2_PROF(ctx, GF2_K_INNER, GF2_CK(ctx, cudaGraphLaunch(ctx->inner_graph_exec, ctx->stream)));
  // the one host synchronization: the result block
  GF2_CK(ctx, cudaMemcpyAsync(ctx->h_pinned, w.st, kResultBytes, cudaMemcpyDeviceToHost, ctx->stream));
  GF2_CK(ctx, cudaStreamSynchronize(ctx->stream));
  InnerState r;
  std::memcpy(&r, ctx->h_pinned, kResultBytes);
  ctx->launches += r.iter * ctx->inner_kernels_per_iter + ctx->inner_kernels_tail + 7LL * r.mu_evals;
  if (n_iter) *n_iter = r.iter;
  if (n_mu_eval) *n_mu_eval = r.mu_evals;
  if (r.status == 3) {
    if (r.mu_status == 4) return gf2_fail(ctx, GF2_ERR_NONFINITE, "gf2_inner_loop: vanishing Dyson pivot");
    if (r.mu_status == 3) return gf2_fail(ctx, GF2_ERR_NONFINITE, "gf2_inner_loop: non-finite count");
    return gf2_fail(ctx, GF2_ERR_NOT_CONVERGED, "gf2_inner_loop: mu search did not reach its tolerance");
  }
  if (r.status == 4) return gf2_fail(ctx, GF2_ERR_NONFINITE, "gf2_inner_loop: non-finite Fock residual");
  *mu_inout = r.mu;
  if (r.status != 1) return gf2_fail(ctx, GF2_ERR_NOT_CONVERGED, "gf2_inner_loop: iteration cap reached");
  return GF2_OK;
}
