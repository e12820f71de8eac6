// Context management, argument checking and dispatch of the C-ABI.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <cstdio>
#include <new>

#include "gf2_internal.cuh"

gf2_status gf2_fail(gf2_ctx *ctx, gf2_status s, const std::string &msg) {
  if (ctx) ctx->last_error = msg;
  return s;
}

gf2_status gf2_cuda_fail(gf2_ctx *ctx, cudaError_t e, const char *what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return gf2_fail(ctx, GF2_ERR_NOMEM, m);
  return gf2_fail(ctx, GF2_ERR_CUDA, m);
}

namespace {

// Wt[n][p][l][j] = W[l][p][n][j] = 2 v[l][p][n][j] - v[n][p][l][j]
__global__ void build_wt_kernel(int N, const double *__restrict__ v, double *__restrict__ Wt) {
  const long long N2 = (long long)N * N, N3 = N2 * N, N4 = N3 * N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < N4;
       idx += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(idx % N);
    const int l = (int)((idx / N) % N);
    const int p = (int)((idx / N2) % N);
    const int n = (int)(idx / N3);
    const double a = v[(long long)l * N3 + (long long)p * N2 + (long long)n * N + j];
    const double b = v[(long long)n * N3 + (long long)p * N2 + (long long)l * N + j];
    Wt[idx] = 2.0 * a - b;
  }
}

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

const char *kKernelNames[GF2_K_COUNT] = {"sigma_sandwich", "sigma_xform", "sigma_contract", "sigma_split_g",
                                         "dgemm_fp64", "dyson_inverse", "density_reduce", "fft_iw_to_tau",
                                         "fft_tau_to_iw", "fock_build", "energy_reduce", "small",
                                         "inner_loop_graph"};

void prof_drain(gf2_ctx *c) {
  for (auto &r : c->prof_recs) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      c->prof_ms[r.id] += ms;
      c->prof_n[r.id] += 1;
    }
    c->prof_pool.push_back(r.a);
    c->prof_pool.push_back(r.b);
  }
  c->prof_recs.clear();
}

void free_all(gf2_ctx *c) {
  if (c->mu_graph_exec) cudaGraphExecDestroy(c->mu_graph_exec);
  if (c->mu_graph) cudaGraphDestroy(c->mu_graph);
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  if (c->inner_graph_exec) cudaGraphExecDestroy(c->inner_graph_exec);
  if (c->inner_graph) cudaGraphDestroy(c->inner_graph);
  if (c->capture_stream2) cudaStreamDestroy(c->capture_stream2);
  if (c->capture_stream3) cudaStreamDestroy(c->capture_stream3);
  if (c->d_inner_ws) cudaFree(c->d_inner_ws);
  if (c->d_mu_state) cudaFree(c->d_mu_state);
  for (auto &r : c->prof_recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->prof_pool) cudaEventDestroy(e);
  c->prof_recs.clear();
  c->prof_pool.clear();
  void *ptrs[] = {c->d_v, c->d_Wt, c->d_Shalf, c->d_orth_ws, c->d_v_split, c->d_wt_split, c->d_v_split16, c->d_wt_split16, c->d_twiddle, c->d_iw_pole,
                  c->d_tau_pole, c->d_pole_resum, c->d_t2w_w, c->d_t2w_corr, c->d_ws,
                  c->d_err, c->d_small, c->d_red, c->d_df_B, c->d_df_ws, c->d_tau_index, c->d_fine_a, c->d_grid_lag, c->d_grid_mu, c->d_iw_pole_fold};
  gf2_tc_release(c);
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
}

}  // namespace

int gf2_prof_begin(gf2_ctx *ctx, int id) {
  if (!ctx->prof_on) return -1;
  if (ctx->prof_recs.size() > 4096) prof_drain(ctx);
  gf2_prof_rec r;
  r.id = id;
  for (cudaEvent_t *e : {&r.a, &r.b}) {
    if (!ctx->prof_pool.empty()) {
      *e = ctx->prof_pool.back();
      ctx->prof_pool.pop_back();
    } else if (cudaEventCreate(e) != cudaSuccess) {
      return -1;
    }
  }
  cudaEventRecord(r.a, ctx->stream);
  ctx->prof_recs.push_back(r);
  return (int)ctx->prof_recs.size() - 1;
}

void gf2_prof_end(gf2_ctx *ctx, int rec) {
  if (rec < 0 || rec >= (int)ctx->prof_recs.size()) return;
  cudaEventRecord(ctx->prof_recs[rec].b, ctx->stream);
}

extern "C" gf2_status gf2_profile(gf2_ctx *ctx, int enable) {
  if (!ctx) return GF2_ERR_ARG;
  prof_drain(ctx);
  for (int k = 0; k < GF2_K_COUNT; ++k) {
    ctx->prof_ms[k] = 0.0;
    ctx->prof_n[k] = 0;
  }
  ctx->prof_on = enable != 0;
  ctx->launches = 0;
  return GF2_OK;
}

extern "C" gf2_status gf2_profile_report(gf2_ctx *ctx, char *buf, int buflen, long long *launches) {
  if (!ctx || !buf || buflen < 1) return GF2_ERR_ARG;
  prof_drain(ctx);
  std::string out;
  for (int k = 0; k < GF2_K_COUNT; ++k) {
    if (!ctx->prof_n[k]) continue;
    char line[128];
    snprintf(line, sizeof line, "%s %lld %.6f\n", kKernelNames[k], ctx->prof_n[k], ctx->prof_ms[k]);
    out += line;
  }
  if ((int)out.size() >= buflen) return gf2_fail(ctx, GF2_ERR_ARG, "gf2_profile_report: buffer too small");
  memcpy(buf, out.c_str(), out.size() + 1);
  if (launches) *launches = ctx->launches;
  return GF2_OK;
}

extern "C" const char *gf2_status_string(gf2_status s) {
  switch (s) {
    case GF2_OK: return "ok";
    case GF2_ERR_ARG: return "invalid argument";
    case GF2_ERR_CUDA: return "CUDA error";
    case GF2_ERR_NOMEM: return "out of device memory";
    case GF2_ERR_NOT_CONVERGED: return "not converged";
    case GF2_ERR_TIMEOUT: return "device wait timed out";
    case GF2_ERR_NONFINITE: return "non-finite or singular value";
    case GF2_ERR_UNSUPPORTED: return "unsupported size or option";
  }
  return "unknown status";
}

extern "C" const char *gf2_last_error(const gf2_ctx *ctx) {
  return ctx ? ctx->last_error.c_str() : "no context";
}

// a context on the uniform grid (tau_index == nullptr, n_tau = M + 1) or on the
// grid of n_tau points tau_k = tau_index[k] beta / M (validated by the caller)
static gf2_status create_impl(gf2_ctx **out, int n_bf, int M, int n_tau, const int *tau_index, int n_iw,
                              double beta, void *stream) {
  gf2_ctx *c = new (std::nothrow) gf2_ctx();
  if (!c) return GF2_ERR_NOMEM;
  c->N = n_bf;
  c->n_tau = n_tau;
  c->n_iw = n_iw;
  c->M = M;
  c->log2M = 0;
  while ((1 << c->log2M) < M) ++c->log2M;
  c->beta = beta;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  gf2_status st = GF2_OK;
  auto ck = [&](cudaError_t e, const char *w) {
    if (e != cudaSuccess && st == GF2_OK) st = gf2_cuda_fail(c, e, w);
  };
  ck(cudaGetDevice(&c->device), "cudaGetDevice");
  ck(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device), "cudaDeviceGetAttribute");
  const size_t N2 = (size_t)n_bf * n_bf;
  ck(cudaMalloc(&c->d_small, sizeof(double) * N2 * GF2_SL_COUNT), "cudaMalloc(small)");
  const size_t nchunks = (n_iw + 255) / 256;
  c->red_elems = std::max(nchunks * N2, (size_t)n_iw) + 64;
  ck(cudaMalloc(&c->d_red, sizeof(double) * c->red_elems), "cudaMalloc(red)");
  ck(cudaMalloc(&c->d_err, sizeof(int) * 16), "cudaMalloc(err)");
  ck(cudaMallocHost(&c->h_pinned, sizeof(double) * 8), "cudaMallocHost");
  if (tau_index && st == GF2_OK) {
    ck(cudaMalloc(&c->d_tau_index, sizeof(int) * n_tau), "cudaMalloc(tau_index)");
    ck(cudaMemcpy(c->d_tau_index, tau_index, sizeof(int) * n_tau, cudaMemcpyHostToDevice), "tau_index upload");
  }
  if (st == GF2_OK) st = gf2_tables_build(c, tau_index);
  if (st == GF2_OK) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) st = gf2_cuda_fail(c, e, "gf2_create sync");
  }
  if (st != GF2_OK) {
    free_all(c);
    delete c;
    return st;
  }
  *out = c;
  return GF2_OK;
}

extern "C" gf2_status gf2_create(gf2_ctx **out, int n_bf, int n_tau, int n_iw, double beta, void *stream) {
  if (!out) return GF2_ERR_ARG;
  *out = nullptr;
  const int M = n_tau - 1;
  if (n_bf < 1 || n_bf > GF2_MAX_N || !is_pow2(M) || M < 8 || M > 8192 || n_iw < 1 ||
      n_iw > (1 << 20) || !(beta > 0.0) || !std::isfinite(beta))
    return GF2_ERR_ARG;
  return create_impl(out, n_bf, M, n_tau, nullptr, n_iw, beta, stream);
}

extern "C" gf2_status gf2_create_grid(gf2_ctx **out, int n_bf, int M, int n_tau, const int *tau_index, int n_iw,
                                      double beta, void *stream) {
  if (!out) return GF2_ERR_ARG;
  *out = nullptr;
  if (n_bf < 1 || n_bf > GF2_MAX_N || !is_pow2(M) || M < 8 || M > 8192 || n_tau < 8 || n_tau > M + 1 ||
      !tau_index || n_iw < 1 || n_iw > (1 << 20) || !(beta > 0.0) || !std::isfinite(beta))
    return GF2_ERR_ARG;
  if (tau_index[0] != 0 || tau_index[n_tau - 1] != M) return GF2_ERR_ARG;
  for (int k = 0; k < n_tau; ++k) {
    if (k > 0 && tau_index[k] <= tau_index[k - 1]) return GF2_ERR_ARG;   // strictly increasing
    if (tau_index[k] + tau_index[n_tau - 1 - k] != M) return GF2_ERR_ARG;  // symmetric about beta / 2
  }
  if (gf2_grid_smem_bytes(M, n_tau) > 227 * 1024) return GF2_ERR_UNSUPPORTED;
  return create_impl(out, n_bf, M, n_tau, tau_index, n_iw, beta, stream);
}

extern "C" gf2_status gf2_destroy(gf2_ctx *ctx) {
  if (!ctx) return GF2_ERR_ARG;
  cudaStreamSynchronize(ctx->stream);
  free_all(ctx);
  delete ctx;
  return GF2_OK;
}

extern "C" gf2_status gf2_set_stream(gf2_ctx *ctx, void *stream) {
  if (!ctx) return GF2_ERR_ARG;
  ctx->stream = reinterpret_cast<cudaStream_t>(stream);
  return GF2_OK;
}

extern "C" gf2_status gf2_set_integrals(gf2_ctx *ctx, const double *d_v) {
  if (!ctx) return GF2_ERR_ARG;
  if (!d_v) return gf2_fail(ctx, GF2_ERR_ARG, "gf2_set_integrals: NULL pointer");
  const size_t N4 = (size_t)ctx->N * ctx->N * ctx->N * ctx->N;
  if (!ctx->d_v) GF2_CK(ctx, cudaMalloc(&ctx->d_v, N4 * sizeof(double)));
  GF2_CK(ctx, cudaMemcpyAsync(ctx->d_v, d_v, N4 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  ctx->df_m = 0;  // a density-fitted factor no longer matches these integrals
  return gf2_integrals_ready(ctx);
}

gf2_status gf2_integrals_ready(gf2_ctx *ctx) {
  const size_t N4 = (size_t)ctx->N * ctx->N * ctx->N * ctx->N;
  if (!ctx->d_Wt) GF2_CK(ctx, cudaMalloc(&ctx->d_Wt, N4 * sizeof(double)));
  build_wt_kernel<<<std::max(1, std::min<int>((int)((N4 + 255) / 256), 8 * ctx->num_sms)), 256, 0,
                    ctx->stream>>>(ctx->N, ctx->d_v, ctx->d_Wt);
  GF2_CK_LAUNCH(ctx, "build_wt_kernel");
  ctx->have_integrals = true;
  gf2_status st = gf2_tc_prepare_integrals(ctx);
  if (st != GF2_OK && st != GF2_ERR_UNSUPPORTED) return st;
  return GF2_OK;
}

static gf2_status sigma_dispatch(gf2_ctx *ctx, const double *d_G, int k0, int count, double *d_out, int prec) {
  if (!ctx->have_integrals) return gf2_fail(ctx, GF2_ERR_ARG, "gf2_sigma_tau: gf2_set_integrals not called");
  if (prec == GF2_PREC_FP64) return gf2_sigma_fp64(ctx, d_G, k0, count, d_out);
  if (prec == GF2_PREC_BF16X3 || prec == GF2_PREC_BF16X6 || prec == GF2_PREC_FP16X3 || prec == GF2_PREC_FP16X6)
    return gf2_sigma_tc(ctx, d_G, k0, count, d_out, prec);
  return gf2_fail(ctx, GF2_ERR_ARG, "gf2_sigma_tau: unknown precision");
}

extern "C" gf2_status gf2_sigma_tau(gf2_ctx *ctx, const double *d_G_tau, double *d_Sigma_tau, int prec) {
  if (!ctx) return GF2_ERR_ARG;
  if (!d_G_tau || !d_Sigma_tau) return gf2_fail(ctx, GF2_ERR_ARG, "gf2_sigma_tau: NULL pointer");
  return sigma_dispatch(ctx, d_G_tau, 0, ctx->n_tau, d_Sigma_tau, prec);
}

extern "C" gf2_status gf2_sigma_tau_points(gf2_ctx *ctx, const double *d_G_tau, int k0, int count,
                                           double *d_Sigma_out, int prec) {
  if (!ctx) return GF2_ERR_ARG;
  if (!d_G_tau || !d_Sigma_out) return gf2_fail(ctx, GF2_ERR_ARG, "gf2_sigma_tau_points: NULL pointer");
  if (k0 < 0 || count < 0 || k0 + count > ctx->n_tau)
    return gf2_fail(ctx, GF2_ERR_ARG, "gf2_sigma_tau_points: range outside the grid");
  if (count == 0) return GF2_OK;
  return sigma_dispatch(ctx, d_G_tau, k0, count, d_Sigma_out, prec);
}
