// Eq. Sigma for a batch of independent systems of uneven size on one GPU.
//
// Each instance keeps its own context (integrals, split planes, workspace).
// An autotuner times the candidate paths of every instance on a sample of its
// own time grid -- the FP64 staged contraction on the CUDA cores, and the split
// tensor-core pipeline (64-wide tiles, time points packed for N <= 32) with 32
// or 16 time-point slots per launch when N <= 64 -- and keeps the fastest; the
// FP64 path is always admissible, being the more accurate.  Instances are then
// spread over a few worker streams by longest estimated time first, and the
// whole batched build is recorded once into a CUDA graph: a fork on a private
// stream of the batch, every instance's launches on its lane, a join back; each
// replay is ordered after the caller's stream and before its later work by
// events.  Later calls with the same buffers replay the graph with one launch;
// the error words of the split kernels are read once afterwards.
//
// Shared tiles.  With a BF16 split, an instance with 32 < N <= 64 pays the
// whole 64-wide tile set whatever its N.  The tuner pairs each such instance
// with the largest unpaired instance of the same time grid that fits beside
// it (N_a + N_b <= 64) and runs the two as one block-diagonal system: v, S and
// G(tau) are block-diagonal, every term of Eq. Sigma keeps its indices inside
// one block (v couples i, m, q, k; W couples l, p, n, j; G links k-l, m-n,
// p-q), so the Sigma of the pair is block-diagonal with the two Sigmas on its
// diagonal and the smaller instance costs nothing extra.  Each pair owns a
// context; the graph gathers the two G(tau) into its block-diagonal input and
// scatters the two Sigma blocks back.  FP16 splits are not paired: their
// power-of-two scales are per time point and would be shared by the two.
#include <algorithm>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "gf2_internal.cuh"

struct gf2_batch {
  int n = 0;
  std::vector<gf2_ctx *> ctx;
  std::vector<int> N, n_tau;
  cudaStream_t origin = nullptr;  // the caller's stream (may be the legacy stream, which cannot be captured)
  cudaStream_t cap = nullptr;     // private stream the graph is recorded on and launched on
  std::vector<cudaStream_t> lanes;
  std::vector<cudaEvent_t> ev_join;
  cudaEvent_t ev_fork = nullptr, ev_in = nullptr, ev_out = nullptr;
  // autotuner result
  int tuned_prec = -1;
  std::vector<int> path;       // precision code each instance runs with
  std::vector<int> chunk;      // split pipeline: time-point slots per launch
  std::vector<double> est_ms;  // estimated ms of one full-grid Sigma build
  std::vector<int> lane_of;
  // instances sharing one block-diagonal system (see the header comment)
  struct Pair {
    int big = -1, small = -1;
    gf2_ctx *ctx = nullptr;
    double *G = nullptr, *Sig = nullptr;  // [n_tau][N_big + N_small]^2 gather / result buffers
  };
  std::vector<Pair> pairs;
  std::vector<int> pair_of;            // index into pairs, or -1
  std::vector<double *> S_copy;        // the overlap given to gf2_batch_set_system (or NULL)
  // recorded graph and the buffers it was recorded with
  cudaGraphExec_t exec = nullptr;
  int graph_prec = -1;
  std::vector<const double *> graph_g;
  std::vector<double *> graph_s;
  std::string last_error;
};

namespace {

constexpr int kMaxLanes = 4;
constexpr int kTcMaxN = 64;

gf2_status bfail(gf2_batch *b, gf2_status s, const std::string &m) {
  if (b) b->last_error = m;
  return s;
}

gf2_status from_ctx(gf2_batch *b, int i, gf2_status s) {
  if (s != GF2_OK) b->last_error = "instance " + std::to_string(i) + ": " + gf2_last_error(b->ctx[i]);
  return s;
}

bool split_prec(int p) {
  return p == GF2_PREC_BF16X3 || p == GF2_PREC_BF16X6 || p == GF2_PREC_FP16X3 || p == GF2_PREC_FP16X6;
}

// out[t] = blockdiag(A[t], B[t]) for t < count (A: na x na, B: nb x nb)
__global__ void blockdiag2_kernel(int na, int nb, int count, const double *__restrict__ A,
                                  const double *__restrict__ B, double *__restrict__ out) {
  const int ns = na + nb;
  const long long total = (long long)count * ns * ns;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long t = e / ((long long)ns * ns);
    const int r = (int)(e - t * ns * ns), i = r / ns, j = r - i * ns;
    double x = 0.0;
    if (i < na && j < na) x = A[(t * na + i) * na + j];
    else if (i >= na && j >= na) x = B[(t * nb + (i - na)) * nb + (j - na)];
    out[e] = x;
  }
}

// A[t] = in[t][:na, :na], B[t] = in[t][na:, na:]
__global__ void blocksplit2_kernel(int na, int nb, int count, const double *__restrict__ in,
                                   double *__restrict__ A, double *__restrict__ B) {
  const int ns = na + nb;
  const long long total = (long long)count * ns * ns;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long t = e / ((long long)ns * ns);
    const int r = (int)(e - t * ns * ns), i = r / ns, j = r - i * ns;
    if (i < na && j < na) A[(t * na + i) * na + j] = in[e];
    else if (i >= na && j >= na) B[(t * nb + (i - na)) * nb + (j - na)] = in[e];
  }
}

// v[i][j][k][l] of the pair: A's when all four indices lie in the first block,
// B's when all lie in the second, zero otherwise
__global__ void blockdiag4_kernel(int na, int nb, const double *__restrict__ A, const double *__restrict__ B,
                                  double *__restrict__ out) {
  const long long ns = na + nb, total = ns * ns * ns * ns;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int l = (int)(e % ns), k = (int)((e / ns) % ns), j = (int)((e / (ns * ns)) % ns), i = (int)(e / (ns * ns * ns));
    double x = 0.0;
    if (i < na && j < na && k < na && l < na) x = A[(((long long)i * na + j) * na + k) * na + l];
    else if (i >= na && j >= na && k >= na && l >= na)
      x = B[(((long long)(i - na) * nb + (j - na)) * nb + (k - na)) * nb + (l - na)];
    out[e] = x;
  }
}

int grid_of(long long total) { return (int)std::min<long long>((total + 255) / 256, 4096); }

void drop_pairs(gf2_batch *b) {
  for (auto &p : b->pairs) {
    if (p.ctx) gf2_destroy(p.ctx);
    if (p.G) cudaFree(p.G);
    if (p.Sig) cudaFree(p.Sig);
  }
  b->pairs.clear();
  b->pair_of.assign(b->n, -1);
}

void drop_graph(gf2_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->graph_prec = -1;
  b->graph_g.clear();
  b->graph_s.clear();
}

void release(gf2_batch *b) {
  drop_graph(b);
  drop_pairs(b);
  for (auto p : b->S_copy)
    if (p) cudaFree(p);
  for (auto c : b->ctx)
    if (c) gf2_destroy(c);
  for (auto s : b->lanes) cudaStreamDestroy(s);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (auto e : b->ev_join) cudaEventDestroy(e);
  for (auto e : {b->ev_fork, b->ev_in, b->ev_out})
    if (e) cudaEventDestroy(e);
}

// time one call of `prec` on instance i over `count` points from k0 (second of two calls)
gf2_status time_path(gf2_batch *b, int i, const double *d_G, double *d_out, int k0, int count, int prec,
                     double *ms) {
  gf2_ctx *c = b->ctx[i];
  gf2_set_stream(c, b->origin);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return bfail(b, GF2_ERR_CUDA, "autotuner: cudaEventCreate");
  gf2_status st = gf2_sigma_tau_points(c, d_G, k0, count, d_out, prec);  // also allocates the workspace
  if (st == GF2_OK) {
    cudaEventRecord(e0, b->origin);
    st = gf2_sigma_tau_points(c, d_G, k0, count, d_out, prec);
    cudaEventRecord(e1, b->origin);
  }
  float t = 0.f;
  if (st == GF2_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
    st = bfail(b, GF2_ERR_CUDA, "autotuner: event timing");
  else if (st != GF2_OK)
    from_ctx(b, i, st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = t;
  return st;
}

// Pairs every split-path instance with 32 < N <= 64 (which pays the whole
// 64-wide tile set) with the largest unpaired instance of the same time grid
// and overlap kind that fits beside it, builds the block-diagonal system of
// each pair and runs it once on the tune input (so the graph recording that
// follows allocates nothing).  BF16 splits only.
gf2_status make_pairs(gf2_batch *b, const double *const *d_G_tau, int prec) {
  drop_pairs(b);
  if (prec != GF2_PREC_BF16X3 && prec != GF2_PREC_BF16X6) return GF2_OK;
  std::vector<int> bigs;
  for (int i = 0; i < b->n; ++i)
    if (b->path[i] == prec && b->N[i] > 32 && b->N[i] <= kTcMaxN) bigs.push_back(i);
  std::stable_sort(bigs.begin(), bigs.end(), [&](int x, int y) { return b->est_ms[x] > b->est_ms[y]; });
  for (int big : bigs) {
    if (b->pair_of[big] >= 0) continue;
    int best = -1;
    for (int j = 0; j < b->n; ++j) {
      if (j == big || b->pair_of[j] >= 0 || b->N[j] + b->N[big] > kTcMaxN || b->n_tau[j] != b->n_tau[big] ||
          (b->S_copy[j] == nullptr) != (b->S_copy[big] == nullptr))
        continue;
      if (best < 0 || b->est_ms[j] > b->est_ms[best]) best = j;
    }
    if (best < 0) continue;
    gf2_batch::Pair p;
    p.big = big;
    p.small = best;
    const int na = b->N[big], nb = b->N[best], ns = na + nb, nt = b->n_tau[big];
    gf2_status st = gf2_create(&p.ctx, ns, nt, 8, 1.0, b->origin);
    if (st != GF2_OK) return bfail(b, st, "shared-tile pair: context");
    double *tmp = nullptr;
    const size_t n4 = (size_t)ns * ns * ns * ns;
    if (cudaMalloc(&tmp, sizeof(double) * std::max(n4, (size_t)ns * ns)) != cudaSuccess) {
      gf2_destroy(p.ctx);
      return bfail(b, GF2_ERR_NOMEM, "shared-tile pair: integrals");
    }
    blockdiag4_kernel<<<grid_of((long long)n4), 256, 0, b->origin>>>(na, nb, b->ctx[big]->d_v, b->ctx[best]->d_v, tmp);
    st = gf2_set_integrals(p.ctx, tmp);
    if (st == GF2_OK && b->S_copy[big]) {
      blockdiag2_kernel<<<grid_of((long long)ns * ns), 256, 0, b->origin>>>(na, nb, 1, b->S_copy[big],
                                                                           b->S_copy[best], tmp);
      st = gf2_set_overlap(p.ctx, tmp);
    }
    cudaStreamSynchronize(b->origin);
    cudaFree(tmp);
    const size_t grid_bytes = sizeof(double) * (size_t)nt * ns * ns;
    if (st == GF2_OK && (cudaMalloc(&p.G, grid_bytes) != cudaSuccess || cudaMalloc(&p.Sig, grid_bytes) != cudaSuccess))
      st = GF2_ERR_NOMEM;
    b->pairs.push_back(p);  // owned by the batch from here on (released with it)
    if (st != GF2_OK) return bfail(b, st, "shared-tile pair: set-up");
    p.ctx->tc_chunk_max = b->chunk[big];
    // one run on the tune input: builds the split planes and the workspace
    blockdiag2_kernel<<<grid_of((long long)nt * ns * ns), 256, 0, b->origin>>>(na, nb, nt, d_G_tau[big],
                                                                              d_G_tau[best], p.G);
    st = gf2_sigma_tau_points(p.ctx, p.G, 0, std::min(nt, 2), p.Sig, prec);
    if (st != GF2_OK) return bfail(b, st, std::string("shared-tile pair: ") + gf2_last_error(p.ctx));
    if (cudaStreamSynchronize(b->origin) != cudaSuccess) return bfail(b, GF2_ERR_CUDA, "shared-tile pair: sync");
    const int k = (int)b->pairs.size() - 1;
    b->pair_of[big] = b->pair_of[best] = k;
    // the smaller instance's own workspace is no longer used
    gf2_tc_release(b->ctx[best]);
    if (b->ctx[best]->d_ws) {
      cudaFree(b->ctx[best]->d_ws);
      b->ctx[best]->d_ws = nullptr;
      b->ctx[best]->ws_elems = 0;
    }
    b->path[best] = prec;
    b->chunk[best] = b->chunk[big];
    b->est_ms[best] = 0.0;  // runs inside its partner's build
  }
  return GF2_OK;
}

}  // namespace

extern "C" gf2_status gf2_batch_create(gf2_batch **out, int n_inst, const int *n_bf, const int *n_tau, void *stream) {
  if (!out) return GF2_ERR_ARG;
  *out = nullptr;
  if (n_inst < 1 || n_inst > 4096 || !n_bf || !n_tau) return GF2_ERR_ARG;
  for (int i = 0; i < n_inst; ++i) {  // the gf2_create rules, checked before any context touches the device
    const int M = n_tau[i] - 1;
    if (n_bf[i] < 1 || n_bf[i] > GF2_MAX_N || M < 8 || M > 8192 || (M & (M - 1)) != 0) return GF2_ERR_ARG;
  }
  gf2_batch *b = new (std::nothrow) gf2_batch();
  if (!b) return GF2_ERR_NOMEM;
  b->n = n_inst;
  b->origin = reinterpret_cast<cudaStream_t>(stream);
  b->ctx.assign(n_inst, nullptr);
  b->N.assign(n_bf, n_bf + n_inst);
  b->n_tau.assign(n_tau, n_tau + n_inst);
  b->S_copy.assign(n_inst, nullptr);
  b->pair_of.assign(n_inst, -1);
  gf2_status st = GF2_OK;
  for (int i = 0; i < n_inst && st == GF2_OK; ++i)
    st = gf2_create(&b->ctx[i], n_bf[i], n_tau[i], 8, 1.0, stream);  // Sigma(tau) uses no frequency grid
  const int L = std::min(kMaxLanes, n_inst);
  for (int l = 0; l < L && st == GF2_OK; ++l) {
    cudaStream_t s;
    cudaEvent_t e;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) st = GF2_ERR_CUDA;
    else b->lanes.push_back(s);
    if (st == GF2_OK && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) st = GF2_ERR_CUDA;
    else if (st == GF2_OK) b->ev_join.push_back(e);
  }
  for (cudaEvent_t *e : {&b->ev_fork, &b->ev_in, &b->ev_out})
    if (st == GF2_OK && cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) st = GF2_ERR_CUDA;
  if (st == GF2_OK && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) st = GF2_ERR_CUDA;
  if (st != GF2_OK) {
    release(b);
    delete b;
    return st;
  }
  *out = b;
  return GF2_OK;
}

extern "C" gf2_status gf2_batch_destroy(gf2_batch *b) {
  if (!b) return GF2_ERR_ARG;
  cudaStreamSynchronize(b->origin);
  release(b);
  delete b;
  return GF2_OK;
}

extern "C" const char *gf2_batch_last_error(const gf2_batch *b) { return b ? b->last_error.c_str() : ""; }

extern "C" gf2_status gf2_batch_set_system(gf2_batch *b, int inst, const double *d_v, const double *d_S) {
  if (!b) return GF2_ERR_ARG;
  if (inst < 0 || inst >= b->n || !d_v) return bfail(b, GF2_ERR_ARG, "gf2_batch_set_system: bad instance or NULL v");
  drop_graph(b);
  drop_pairs(b);
  b->tuned_prec = -1;
  gf2_ctx *c = b->ctx[inst];
  gf2_set_stream(c, b->origin);
  gf2_status st = gf2_set_integrals(c, d_v);
  if (st == GF2_OK && d_S) st = gf2_set_overlap(c, d_S);
  // a copy of S for a block-diagonal pair built by the tuner
  if (b->S_copy[inst]) {
    cudaFree(b->S_copy[inst]);
    b->S_copy[inst] = nullptr;
  }
  if (st == GF2_OK && d_S) {
    const size_t bytes = sizeof(double) * b->N[inst] * b->N[inst];
    if (cudaMalloc(&b->S_copy[inst], bytes) != cudaSuccess ||
        cudaMemcpyAsync(b->S_copy[inst], d_S, bytes, cudaMemcpyDeviceToDevice, b->origin) != cudaSuccess)
      return bfail(b, GF2_ERR_NOMEM, "gf2_batch_set_system: copy of S");
  }
  return from_ctx(b, inst, st);
}

extern "C" gf2_status gf2_batch_tune(gf2_batch *b, const double *const *d_G_tau, int prec) {
  if (!b) return GF2_ERR_ARG;
  if (!d_G_tau) return bfail(b, GF2_ERR_ARG, "gf2_batch_tune: NULL pointer array");
  if (prec != GF2_PREC_FP64 && !split_prec(prec)) return bfail(b, GF2_ERR_ARG, "gf2_batch_tune: unknown precision");
  for (int i = 0; i < b->n; ++i) {
    if (!d_G_tau[i]) return bfail(b, GF2_ERR_ARG, "gf2_batch_tune: NULL G(tau) of an instance");
    if (!b->ctx[i]->have_integrals) return bfail(b, GF2_ERR_ARG, "gf2_batch_tune: gf2_batch_set_system not called");
  }
  drop_graph(b);
  drop_pairs(b);
  b->path.assign(b->n, GF2_PREC_FP64);
  b->chunk.assign(b->n, 32);
  b->est_ms.assign(b->n, 0.0);
  b->lane_of.assign(b->n, 0);
  // the sample: 32 points for FP64, one chunk (up to 32 slots of tc_pack points) for the split pipeline
  size_t out_elems = 0;
  for (int i = 0; i < b->n; ++i)
    out_elems = std::max(out_elems, (size_t)std::min(b->n_tau[i], 32 * std::max(1, b->ctx[i]->tc_pack)) *
                                        b->N[i] * b->N[i]);
  double *d_out = nullptr;
  if (cudaMalloc(&d_out, out_elems * sizeof(double)) != cudaSuccess)
    return bfail(b, GF2_ERR_NOMEM, "gf2_batch_tune: sample buffer");
  gf2_status st = GF2_OK;
  for (int i = 0; i < b->n && st == GF2_OK; ++i) {
    const int count = std::min(32, b->n_tau[i]);
    gf2_ctx *c = b->ctx[i];
    // candidates: FP64, and the split pipeline with 32 or 16 slots per launch
    // (16 halves its 4.3 GB of intermediates and doubles its launches)
    struct Cand { int prec, chunk; };
    std::vector<Cand> cands{{GF2_PREC_FP64, 32}};
    if (split_prec(prec) && b->N[i] <= kTcMaxN) {
      cands.push_back({prec, 32});
      cands.push_back({prec, 16});
    }
    double best = 0.0;
    for (size_t k = 0; k < cands.size() && st == GF2_OK; ++k) {
      const Cand cd = cands[k];
      if (cd.prec != GF2_PREC_FP64) {  // a fresh workspace of this chunk size
        if (cudaStreamSynchronize(b->origin) != cudaSuccess) st = bfail(b, GF2_ERR_CUDA, "autotuner: sync");
        gf2_tc_release(c);
        c->tc_chunk_max = cd.chunk;
      }
      // one whole chunk of this candidate
      const int cnt = std::min(b->n_tau[i], cd.prec == GF2_PREC_FP64 ? count : cd.chunk * c->tc_pack);
      double ms = 0.0;
      if (st == GF2_OK && (st = time_path(b, i, d_G_tau[i], d_out, 0, cnt, cd.prec, &ms)) != GF2_OK) break;
      const double full = ms * b->n_tau[i] / cnt;
      if (k == 0 || full < best) {
        best = full;
        b->path[i] = cd.prec;
        b->chunk[i] = cd.chunk;
      }
    }
    b->est_ms[i] = best;
    if (st != GF2_OK) break;
    // keep only the workspace of the chosen path and chunk size, allocated now:
    // the graph recording that follows must not allocate
    if (cudaStreamSynchronize(b->origin) != cudaSuccess) st = bfail(b, GF2_ERR_CUDA, "autotuner: sync");
    gf2_tc_release(c);
    c->tc_chunk_max = b->chunk[i];
    if (st == GF2_OK && b->path[i] != GF2_PREC_FP64) {
      if (c->d_ws) {
        cudaFree(c->d_ws);
        c->d_ws = nullptr;
        c->ws_elems = 0;
      }
      st = from_ctx(b, i, gf2_sigma_tau_points(c, d_G_tau[i], 0, std::min(b->n_tau[i], 2), d_out, b->path[i]));
    }
  }
  cudaFree(d_out);
  if (st != GF2_OK) return st;
  if ((st = make_pairs(b, d_G_tau, prec)) != GF2_OK) return st;
  // longest estimated time first, each to the least-loaded lane
  std::vector<int> order(b->n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->est_ms[x] > b->est_ms[y]; });
  std::vector<double> load(b->lanes.size(), 0.0);
  for (int i : order) {
    const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->lane_of[i] = l;
    load[l] += b->est_ms[i];
  }
  b->tuned_prec = prec;
  return GF2_OK;
}

extern "C" gf2_status gf2_batch_plan(const gf2_batch *b, int inst, int *path, double *est_ms, int *lane,
                                     int *chunk) {
  if (!b || inst < 0 || inst >= b->n || b->tuned_prec < 0) return GF2_ERR_ARG;
  if (path) *path = b->path[inst];
  if (chunk) *chunk = b->chunk[inst];
  if (est_ms) *est_ms = b->est_ms[inst];
  if (lane) *lane = b->lane_of[inst];
  return GF2_OK;
}

extern "C" gf2_status gf2_batch_partner(const gf2_batch *b, int inst, int *partner) {
  if (!b || inst < 0 || inst >= b->n || b->tuned_prec < 0 || !partner) return GF2_ERR_ARG;
  const int k = b->pair_of[inst];
  *partner = k < 0 ? -1 : (b->pairs[k].big == inst ? b->pairs[k].small : b->pairs[k].big);
  return GF2_OK;
}

extern "C" gf2_status gf2_sigma_tau_batched(gf2_batch *b, const double *const *d_G_tau, double *const *d_Sigma_tau,
                                            int prec) {
  if (!b) return GF2_ERR_ARG;
  if (!d_G_tau || !d_Sigma_tau) return bfail(b, GF2_ERR_ARG, "gf2_sigma_tau_batched: NULL pointer array");
  for (int i = 0; i < b->n; ++i)
    if (!d_G_tau[i] || !d_Sigma_tau[i]) return bfail(b, GF2_ERR_ARG, "gf2_sigma_tau_batched: NULL buffer");
  gf2_status st;
  if (b->tuned_prec != prec && (st = gf2_batch_tune(b, d_G_tau, prec)) != GF2_OK) return st;
  const bool same = b->exec && b->graph_prec == prec &&
                    std::equal(b->graph_g.begin(), b->graph_g.end(), d_G_tau) &&
                    std::equal(b->graph_s.begin(), b->graph_s.end(), d_Sigma_tau);
  if (!same) {
    drop_graph(b);
    // relaxed: the recorded calls set kernel attributes, which the stricter modes refuse
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed);
    st = e == cudaSuccess ? GF2_OK : bfail(b, GF2_ERR_CUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
    if (st == GF2_OK) cudaEventRecord(b->ev_fork, b->cap);
    for (size_t l = 0; l < b->lanes.size() && st == GF2_OK; ++l) {
      cudaStreamWaitEvent(b->lanes[l], b->ev_fork, 0);
      for (int i = 0; i < b->n && st == GF2_OK; ++i) {
        if (b->lane_of[i] != (int)l) continue;
        if (b->pair_of[i] >= 0) {  // the pair runs on its larger instance's lane
          const gf2_batch::Pair &p = b->pairs[b->pair_of[i]];
          if (i != p.big) continue;
          const int na = b->N[p.big], nb = b->N[p.small], ns = na + nb, nt = b->n_tau[p.big];
          const int grid = grid_of((long long)nt * ns * ns);
          blockdiag2_kernel<<<grid, 256, 0, b->lanes[l]>>>(na, nb, nt, d_G_tau[p.big], d_G_tau[p.small], p.G);
          gf2_set_stream(p.ctx, b->lanes[l]);
          p.ctx->defer_error_check = true;
          gf2_status sp = gf2_sigma_tau(p.ctx, p.G, p.Sig, b->path[i]);
          p.ctx->defer_error_check = false;
          if (sp != GF2_OK) st = bfail(b, sp, "shared-tile pair of instances " + std::to_string(p.big) + " and " +
                                                  std::to_string(p.small) + ": " + gf2_last_error(p.ctx));
          blocksplit2_kernel<<<grid, 256, 0, b->lanes[l]>>>(na, nb, nt, p.Sig, d_Sigma_tau[p.big],
                                                           d_Sigma_tau[p.small]);
          continue;
        }
        gf2_ctx *c = b->ctx[i];
        gf2_set_stream(c, b->lanes[l]);
        c->defer_error_check = true;
        st = from_ctx(b, i, gf2_sigma_tau(c, d_G_tau[i], d_Sigma_tau[i], b->path[i]));
        c->defer_error_check = false;
      }
      cudaEventRecord(b->ev_join[l], b->lanes[l]);
      cudaStreamWaitEvent(b->cap, b->ev_join[l], 0);
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(b->cap, &graph);
    if (st == GF2_OK && e != cudaSuccess)
      st = bfail(b, GF2_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    if (st == GF2_OK) {
      e = cudaGraphInstantiate(&b->exec, graph, 0);
      if (e != cudaSuccess) {
        b->exec = nullptr;
        st = bfail(b, GF2_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
      }
    }
    if (graph) cudaGraphDestroy(graph);
    for (int i = 0; i < b->n; ++i) gf2_set_stream(b->ctx[i], b->origin);
    for (auto &p : b->pairs) gf2_set_stream(p.ctx, b->origin);
    if (st != GF2_OK) return st;
    b->graph_prec = prec;
    b->graph_g.assign(d_G_tau, d_G_tau + b->n);
    b->graph_s.assign(d_Sigma_tau, d_Sigma_tau + b->n);
  }
  // the graph runs on the private stream, after everything queued on the caller's stream
  cudaEventRecord(b->ev_in, b->origin);
  cudaStreamWaitEvent(b->cap, b->ev_in, 0);
  cudaError_t e = cudaGraphLaunch(b->exec, b->cap);
  if (e != cudaSuccess) return bfail(b, GF2_ERR_CUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
  cudaEventRecord(b->ev_out, b->cap);
  cudaStreamWaitEvent(b->origin, b->ev_out, 0);
  if ((e = cudaStreamSynchronize(b->origin)) != cudaSuccess)
    return bfail(b, GF2_ERR_CUDA, std::string("batched Sigma: ") + cudaGetErrorString(e));
  for (int i = 0; i < b->n; ++i) {
    if (!split_prec(b->path[i])) continue;
    const gf2_ctx *c = b->pair_of[i] >= 0 ? b->pairs[b->pair_of[i]].ctx : b->ctx[i];
    int flag = 0;
    if (cudaMemcpy(&flag, c->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      return bfail(b, GF2_ERR_CUDA, "batched Sigma: reading an error word");
    if (flag) return bfail(b, GF2_ERR_TIMEOUT, "instance " + std::to_string(i) + ": a pipeline wait timed out");
  }
  return GF2_OK;
}
