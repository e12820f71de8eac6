// Internal declarations shared by the translation units of libgf2.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/gf2.h"

// Real pole (hartree) about which the four-moment tail is resummed:
// T(z) = sum_r c_r (z - a)^-r with the moments G1..G4 of Eq. GF.
#define GF2_TAIL_POLE 1.0
#define GF2_MAX_N 128

// slots of ctx->d_small, each N*N doubles
enum {
  GF2_SL_SINV = 0, GF2_SL_A1, GF2_SL_A2, GF2_SL_A3, GF2_SL_B1, GF2_SL_B2, GF2_SL_B3,
  GF2_SL_T1, GF2_SL_TMP, GF2_SL_MOM = 9, GF2_SL_COEF = 13, GF2_SL_MISC = 17, GF2_SL_COUNT = 20
};

// kernels timed by the optional per-launch profiler (gf2_profile)
enum gf2_kernel_id {
  GF2_K_SANDWICH = 0, GF2_K_XFORM, GF2_K_CONTRACT, GF2_K_SPLIT, GF2_K_DGEMM, GF2_K_DYSON,
  GF2_K_DENSITY, GF2_K_IW2TAU, GF2_K_TAU2IW, GF2_K_FOCK, GF2_K_ENERGY, GF2_K_SMALL, GF2_K_INNER, GF2_K_COUNT
};

// State of the device-resident chemical-potential search (step 2.a): the point
// to evaluate next and the bracket / Brent variables, updated by one thread
// after every count evaluation (mu_control_kernel in dyson.cu).
struct gf2_mu_state {
  double n_elec, tol, tol_coarse;   // inputs
  int max_iter, cap_coarse, n_iw, n_coarse;
  double mu;                        // next point to evaluate
  int nf;                           // frequencies of that evaluation
  int stage;                        // 0 coarse, 1 full, 2 done
  int status;                       // 0 running, 1 found, 2 not converged, 3 non-finite count, 4 vanishing pivot
  int evals;
  double mu_out;
  int phase;                        // 0 first point, 1 bracketing upward, 2 downward, 3 Brent
  int n, cap, have_prev;
  double slope_hint, tol_f, step, lo, hi, flo, fhi, a, b, c, fa, fb, fc, d, e;
  double last_mu, last_f, prev_mu, prev_f;
};

struct gf2_prof_rec {
  int id;
  cudaEvent_t a, b;
};

struct gf2_ctx {
  int N = 0, n_tau = 0, n_iw = 0, M = 0, log2M = 0;
  double beta = 0.0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  std::string last_error;

  // integrals (FP64, owned copies)
  double *d_v = nullptr;    // v[i][j][k][l] = (ij|kl)
  double *d_Shalf = nullptr;   // S^{1/2} and S^{-1/2} (gf2_set_overlap), [2][N][N]
  double *d_orth_ws = nullptr; // orthogonal-basis G(tau), Sigma, scratch for the split path
  double *d_Wt = nullptr;   // Wt[n][p][l][j] = W[l][p][n][j] = 2 v_lpnj - v_nplj
  bool have_integrals = false;

  // tensor-core operands (split planes), built by gf2_set_integrals
  void *d_v_split = nullptr;    // [terms][N^4] bf16: v[i][m][q][k]
  void *d_wt_split = nullptr;   // [terms][N^4] bf16: Wt4[j][l][n][p] = W[l][p][n][j]
  void *d_v_split16 = nullptr;  // the same as FP16 terms of 2^e_v16 v
  void *d_wt_split16 = nullptr; // the same as FP16 terms of 2^e_w16 W
  int e_v16 = 0, e_w16 = 0;
  double vmax16 = 0.0;          // largest |v| after its FP16 scale
  int split_terms = 0;
  bool tc_pair_sym = false;     // v[i][m][q][k] = v[q][k][i][m] to rounding: the sandwich computes half the tiles
  bool tc_planes_stale = false; // N > 64: the 128-wide planes are built by the first split-precision call

  // grid tables (built at create)
  double2 *d_twiddle = nullptr;   // e^{-2 pi i k / M}, k < M/2
  double2 *d_iw_pole = nullptr;   // [n_iw][4]: (i w_n - a)^-(r+1)
  double2 *d_iw_pole_fold = nullptr;  // [M][4]: sum over n = j mod M, n < n_iw, of (i w_n - a)^-(r+1)
  double *d_tau_pole = nullptr;   // [n_tau][4]: tau image of (z - a)^-(r+1)
  double *d_pole_resum = nullptr; // [8]: sum_{n<n_iw}, then sum_{n<n_coarse}, of Re (i w_n - a)^-(r+1)
  int n_coarse = 0;               // frequencies of a coarse particle count (0: none)
  double2 *d_t2w_w = nullptr;     // [n_iw]: h W(theta_n), attenuation factor
  double2 *d_t2w_corr = nullptr;  // [n_iw][8]: end corrections, nodes 0..3, M-3..M

  // non-equidistant time grid (gf2_create_grid): the n_tau points as indices
  // into the uniform grid of M intervals (nullptr: the uniform grid itself,
  // n_tau = M + 1); the tables of the local-cubic Fourier integral on it
  int *d_tau_index = nullptr;
  int *d_fine_a = nullptr;         // [M]: the grid interval holding uniform interval f
  double *d_grid_lag = nullptr;    // [n_tau - 1][4 nodes][4 powers]: local cubics in x = (tau - tau_a) / h_a
  double2 *d_grid_mu = nullptr;    // [n_iw][4]: (beta / M) mu_q(w_n beta / M)
  double grid_dw[8] = {};          // Sig2 weights: slopes at tau = 0 (nodes 0..3) and at beta (n_tau-4..n_tau-1)

  // density-fitted integrals (gf2_set_df_integrals): the factor B [df_m][N][N]
  // and the FP64 workspace of the factor-order Sigma (C, X, U: 3 df_chunk m N^2)
  double *d_df_B = nullptr;
  int df_m = 0, df_cap = 0;
  double *d_df_ws = nullptr;
  int df_chunk = 0;

  // FP64 Sigma workspace (two ping-pong buffers of chunk * N^4 doubles)
  double *d_ws = nullptr;
  size_t ws_elems = 0;
  int fp64_chunk = 0;

  // tensor-core Sigma workspace (host-side state owning device buffers)
  void *d_tc_ws = nullptr;
  void *d_tc128_ws = nullptr;     // the same for the 128-wide tile pipeline
  size_t tc_ws_bytes = 0;
  int tc_chunk = 0;
  int tc_chunk_max = 32;           // slots per split-pipeline launch (even, 2..32; the batch tuner sets it)
  int tc_pack = 1;                // time points per 64-wide tile slot (floor(64/N) for N <= 32)
  int *d_err = nullptr;           // device error word (timeouts in tcgen05 kernels)
  bool defer_error_check = false; // set while a batch records this context into a CUDA graph:
                                  // the split path then skips its closing read of d_err

  // device-resident chemical-potential search: its state and the CUDA graph
  // (a WHILE conditional node around one count evaluation) that runs it
  void *d_mu_state = nullptr;
  cudaGraph_t mu_graph = nullptr;
  cudaGraphExec_t mu_graph_exec = nullptr;
  cudaStream_t capture_stream = nullptr;
  const void *mu_graph_key[5] = {};

  // device-resident inner loop (steps 2.a-2.b, inner.cu): its state, residual
  // history and graph (a WHILE node whose body nests the mu search's)
  void *d_inner_ws = nullptr;
  cudaGraph_t inner_graph = nullptr;
  cudaGraphExec_t inner_graph_exec = nullptr;
  cudaStream_t capture_stream2 = nullptr, capture_stream3 = nullptr;
  const void *inner_graph_key[7] = {};
  long long inner_kernels_per_iter = 0, inner_kernels_tail = 0;

  // small scratch
  double *d_small = nullptr;      // Sinv, basis(7), coef(4), misc: 16 N^2
  double *d_red = nullptr;        // reduction partials
  size_t red_elems = 0;
  double *h_pinned = nullptr;     // host-pinned scalars (8 doubles)

  // launch accounting and the optional event profiler
  long long launches = 0;
  bool prof_on = false;
  std::vector<gf2_prof_rec> prof_recs;
  std::vector<cudaEvent_t> prof_pool;
  double prof_ms[GF2_K_COUNT] = {};
  long long prof_n[GF2_K_COUNT] = {};
};

// profiler hooks: begin returns a record index (or -1 when off)
int gf2_prof_begin(gf2_ctx *ctx, int kernel_id);
void gf2_prof_end(gf2_ctx *ctx, int rec);

// ---- error helpers (host) ----
gf2_status gf2_fail(gf2_ctx *ctx, gf2_status s, const std::string &msg);
gf2_status gf2_cuda_fail(gf2_ctx *ctx, cudaError_t e, const char *what);

#define GF2_CK(ctx, call)                                                  \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) return gf2_cuda_fail((ctx), e_, #call);         \
  } while (0)

#define GF2_CK_LAUNCH(ctx, what)                                           \
  do {                                                                     \
    ++(ctx)->launches;                                                     \
    cudaError_t e_ = cudaGetLastError();                                   \
    if (e_ != cudaSuccess) return gf2_cuda_fail((ctx), e_, (what));        \
  } while (0)

// time one launch statement under the profiler
#define GF2_PROF(ctx, id, stmt)                                            \
  do {                                                                     \
    int r_ = gf2_prof_begin((ctx), (id));                                  \
    stmt;                                                                  \
    gf2_prof_end((ctx), r_);                                               \
  } while (0)

// ---- FP64 strided batched GEMM: C = alpha * A B + beta_c * C ----
struct Dgemm {
  int M, N, K;
  const double *A; long long a_rs, a_cs, a_b0, a_b1;
  const double *B; long long b_rs, b_cs, b_b0, b_b1;
  double *C;       long long c_rs, c_cs, c_b0, c_b1;
  int nb0, nb1;
  double alpha, beta_c;
  int split_k;   // > 1: partial products added with atomics (C must hold beta_c*C already)
};
gf2_status gf2_dgemm(gf2_ctx *ctx, const Dgemm &g);

// inverse of a real symmetric positive-definite matrix (Gauss-Jordan, one CTA)
gf2_status gf2_inverse_spd(gf2_ctx *ctx, const double *d_A, double *d_Ainv);

// ---- internal entry points between translation units ----
gf2_status gf2_tables_build(gf2_ctx *ctx, const int *h_tau_index);
// shared memory of the tau -> iw kernel of a non-equidistant grid
size_t gf2_grid_smem_bytes(int M, int n_tau);
gf2_status gf2_pole_coefficients(gf2_ctx *ctx, const double *d_moments, double *d_coef);
// W and the tensor-core copies of the integrals now in ctx->d_v
gf2_status gf2_integrals_ready(gf2_ctx *ctx);
gf2_status gf2_sigma_fp64(gf2_ctx *ctx, const double *d_G_tau, int k0, int count, double *d_out);
gf2_status gf2_sigma_tc(gf2_ctx *ctx, const double *d_G_tau, int k0, int count, double *d_out,
                        int prec);
gf2_status gf2_tc_prepare_integrals(gf2_ctx *ctx);
gf2_status gf2_tc_build_planes(gf2_ctx *ctx, int P);
void gf2_tc_release(gf2_ctx *ctx);
// 128-wide tile pipeline (64 < N <= 128)
gf2_status gf2_tc128_workspace(gf2_ctx *ctx);
gf2_status gf2_tc128_run(gf2_ctx *ctx, const double *d_G, int k0, int count, double *d_out, int prec);
void gf2_tc128_release(gf2_ctx *ctx);
gf2_status gf2_orth_transform_g(gf2_ctx *ctx, const double *d_G, int k0, int count, double **d_Gorth);
gf2_status gf2_orth_transform_v(gf2_ctx *ctx, double *d_vorth);
gf2_status gf2_symmetrize(gf2_ctx *ctx, double *d_X, int count);
// the moment basis of Eq. GF's tail (A1..A3 from S^-1 F, B1..B3 from Sig1, Sig2)
// into the small slots; S^-1 is recomputed only when invert_S is set
gf2_status gf2_build_moment_basis(gf2_ctx *ctx, const double *S, const double *F, const double *sig12,
                                  bool invert_S);
// Appends to the graph being captured on `parent` one whole mu search (step
// 2.a): its start, with prm = {mu0, n_elec, tol, max_iter} read from device
// memory when it runs, and a WHILE node around one count evaluation whose body
// is captured on body_stream.  The result is in ctx->d_mu_state.  Seven kernels
// per evaluation plus the start.
gf2_status gf2_capture_mu_search(gf2_ctx *ctx, cudaStream_t parent, cudaStream_t body_stream, const double *S,
                                 const double *F, const double *Sig, double *G, double *P, const double *prm);

// ---- small device helpers ----
__host__ __device__ inline double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ inline double2 crecip(double2 a) {
  double d = a.x * a.x + a.y * a.y;
  return make_double2(a.x / d, -a.y / d);
}
