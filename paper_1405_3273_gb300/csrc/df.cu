// Eq. Sigma on density-fitted integrals, v_ijkl = sum_Q B[Q][i][j] B[Q][k][l]
// (the O(n^3 m) route of the paper's computational details, m auxiliary
// functions).
//
// gf2_set_df_integrals keeps a copy of the factor B and writes the fitted v
// into the context (one FP64 GEMM, v = B^T B over the pair index), so every
// Sigma path, the Fock build and the energy then run on the fitted integrals.
//
// gf2_sigma_tau_df evaluates Eq. Sigma in the factor order, with no N^4
// intermediate per time point.  Substituting v_imqk = sum_Q B^Q_im B^Q_qk:
//   C[i][Q][n] = sum_m B[Q][i][m] G[m][n]            C^Q = B^Q G        2 m N^3
//   X[Q][p][l] = sum_q Gbar[p][q] C[q][Q][l]          X^Q = Gbar C^Q     2 m N^3
//   U[Q][n][j] = sum_(p,l) X[Q][p][l] W[l][p][n][j]                      2 m N^4
//   Sigma[i][j] = - sum_(Q,n) C[i][Q][n] U[Q][n][j]                      2 m N^3
// with W = 2v - v' of the fitted v (its copy Wt[n][p][l][j] = W[l][p][n][j],
// so for fixed n the (p,l) x j block of Wt is a row-major matrix).  Every
// step is one strided batched FP64 GEMM (dgemm.cu); the three intermediates
// take 3 m N^2 doubles per time point.
#include <algorithm>

#include "gf2_internal.cuh"

extern "C" gf2_status gf2_set_df_integrals(gf2_ctx *ctx, const double *d_B, int m) {
  if (!ctx) return GF2_ERR_ARG;
  if (!d_B) return gf2_fail(ctx, GF2_ERR_ARG, "gf2_set_df_integrals: NULL pointer");
  if (m < 1 || m > 65535) return gf2_fail(ctx, GF2_ERR_ARG, "gf2_set_df_integrals: m outside 1..65535");
  const long long N = ctx->N, N2 = N * N, N4 = N2 * N2;
  if (m > ctx->df_cap) {
    if (ctx->d_df_B) cudaFree(ctx->d_df_B);
    ctx->d_df_B = nullptr;
    ctx->df_cap = 0;
    GF2_CK(ctx, cudaMalloc(&ctx->d_df_B, sizeof(double) * (size_t)m * N2));
    ctx->df_cap = m;
  }
  if (ctx->d_df_ws) cudaFree(ctx->d_df_ws);  // sized for the previous m
  ctx->d_df_ws = nullptr;
  ctx->df_chunk = 0;
  GF2_CK(ctx, cudaMemcpyAsync(ctx->d_df_B, d_B, sizeof(double) * (size_t)m * N2, cudaMemcpyDeviceToDevice,
                              ctx->stream));
  if (!ctx->d_v) GF2_CK(ctx, cudaMalloc(&ctx->d_v, sizeof(double) * (size_t)N4));
  // v[(i,j)][(k,l)] = sum_Q B[Q][(i,j)] B[Q][(k,l)]
  Dgemm g{};
  g.M = (int)N2; g.N = (int)N2; g.K = m;
  g.A = ctx->d_df_B;  g.a_rs = 1;  g.a_cs = N2; g.a_b0 = 0; g.a_b1 = 0;
  g.B = ctx->d_df_B;  g.b_rs = N2; g.b_cs = 1;  g.b_b0 = 0; g.b_b1 = 0;
  g.C = ctx->d_v;     g.c_rs = N2; g.c_cs = 1;  g.c_b0 = 0; g.c_b1 = 0;
  g.nb0 = 1; g.nb1 = 1; g.alpha = 1.0; g.beta_c = 0.0; g.split_k = 1;
  gf2_status st = gf2_dgemm(ctx, g);
  if (st != GF2_OK) return st;
  ctx->df_m = 0;
  st = gf2_integrals_ready(ctx);
  if (st != GF2_OK) return st;
  ctx->df_m = m;
  return GF2_OK;
}

static gf2_status sigma_df_fp64(gf2_ctx *ctx, const double *d_G, int k0, int count, double *d_out) {
  const long long N = ctx->N, N2 = N * N, N3 = N2 * N;
  const long long m = ctx->df_m, mN = m * N, mN2 = m * N2;
  const int Mt = ctx->n_tau - 1;  // G(-tau_k) = -G(tau_{Mt-k}): the grid is symmetric about beta/2
  if (!ctx->d_df_ws) {
    const size_t budget = (size_t)1 << 30;  // bytes for C, X and U of one chunk
    long long chunk = std::max<long long>(1, (long long)(budget / (3 * mN2 * sizeof(double))));
    chunk = std::min<long long>({chunk, (long long)ctx->n_tau, 65535LL, (long long)(0x7fffffff / m)});
    ctx->df_chunk = (int)chunk;
    GF2_CK(ctx, cudaMalloc(&ctx->d_df_ws, sizeof(double) * 3 * (size_t)chunk * mN2));
  }
  double *wC = ctx->d_df_ws;
  double *wX = wC + (size_t)ctx->df_chunk * mN2;
  double *wU = wX + (size_t)ctx->df_chunk * mN2;
  for (int c0 = 0; c0 < count; c0 += ctx->df_chunk) {
    const int Bc = std::min(ctx->df_chunk, count - c0);
    const int kb = k0 + c0;
    gf2_status st;

    // C[b][i][Q][n] = sum_m B[Q][i][m] G_b[m][n]: batches (i, b)
    Dgemm g1{};
    g1.M = (int)m; g1.N = (int)N; g1.K = (int)N;
    g1.A = ctx->d_df_B;   g1.a_rs = N2; g1.a_cs = 1; g1.a_b0 = N;   g1.a_b1 = 0;
    g1.B = d_G + kb * N2; g1.b_rs = N;  g1.b_cs = 1; g1.b_b0 = 0;   g1.b_b1 = N2;
    g1.C = wC;            g1.c_rs = N;  g1.c_cs = 1; g1.c_b0 = mN;  g1.c_b1 = mN2;
    g1.nb0 = (int)N; g1.nb1 = Bc; g1.alpha = 1.0; g1.beta_c = 0.0; g1.split_k = 1;
    if ((st = gf2_dgemm(ctx, g1)) != GF2_OK) return st;

    // X[b][Q][p][l] = - sum_q G(tau_{Mt-k})[p][q] C[b][q][Q][l]: batches (Q, b)
    Dgemm g2{};
    g2.M = (int)N; g2.N = (int)N; g2.K = (int)N;
    g2.A = d_G + (long long)(Mt - kb) * N2; g2.a_rs = N; g2.a_cs = 1; g2.a_b0 = 0; g2.a_b1 = -N2;
    g2.B = wC;            g2.b_rs = mN; g2.b_cs = 1; g2.b_b0 = N;   g2.b_b1 = mN2;
    g2.C = wX;            g2.c_rs = N;  g2.c_cs = 1; g2.c_b0 = N2;  g2.c_b1 = mN2;
    g2.nb0 = (int)m; g2.nb1 = Bc; g2.alpha = -1.0; g2.beta_c = 0.0; g2.split_k = 1;
    if ((st = gf2_dgemm(ctx, g2)) != GF2_OK) return st;

    // U[(b,Q)][n][j] = sum_(p,l) X[(b,Q)][(p,l)] Wt[n][(p,l)][j]: batches n
    Dgemm g3{};
    g3.M = (int)(Bc * m); g3.N = (int)N; g3.K = (int)N2;
    g3.A = wX;            g3.a_rs = N2; g3.a_cs = 1; g3.a_b0 = 0;   g3.a_b1 = 0;
    g3.B = ctx->d_Wt;     g3.b_rs = N;  g3.b_cs = 1; g3.b_b0 = N3;  g3.b_b1 = 0;
    g3.C = wU;            g3.c_rs = N2; g3.c_cs = 1; g3.c_b0 = N;   g3.c_b1 = 0;
    g3.nb0 = (int)N; g3.nb1 = 1; g3.alpha = 1.0; g3.beta_c = 0.0; g3.split_k = 1;
    if ((st = gf2_dgemm(ctx, g3)) != GF2_OK) return st;

    // Sigma_b[i][j] = - sum_(Q,n) C[b][i][(Q,n)] U[b][(Q,n)][j], split over K
    double *out = d_out + (long long)c0 * N2;
    GF2_CK(ctx, cudaMemsetAsync(out, 0, sizeof(double) * Bc * N2, ctx->stream));
    Dgemm g4{};
    g4.M = (int)N; g4.N = (int)N; g4.K = (int)mN;
    g4.A = wC;            g4.a_rs = mN; g4.a_cs = 1; g4.a_b0 = mN2; g4.a_b1 = 0;
    g4.B = wU;            g4.b_rs = N;  g4.b_cs = 1; g4.b_b0 = mN2; g4.b_b1 = 0;
    g4.C = out;           g4.c_rs = N;  g4.c_cs = 1; g4.c_b0 = N2;  g4.c_b1 = 0;
    g4.nb0 = Bc; g4.nb1 = 1; g4.alpha = -1.0; g4.beta_c = 0.0;
    const int tiles = (int)((N + 63) / 64) * (int)((N + 63) / 64);
    const int want = std::max(1, (2 * ctx->num_sms) / std::max(1, Bc * tiles));
    g4.split_k = (int)std::min<long long>(want, std::max<long long>(1, mN / 256));
    if ((st = gf2_dgemm(ctx, g4)) != GF2_OK) return st;
  }
  return GF2_OK;
}

extern "C" gf2_status gf2_sigma_tau_df(gf2_ctx *ctx, const double *d_G_tau, int k0, int count, double *d_Sigma_out,
                                       int prec) {
  if (!ctx) return GF2_ERR_ARG;
  if (!d_G_tau || !d_Sigma_out) return gf2_fail(ctx, GF2_ERR_ARG, "gf2_sigma_tau_df: NULL pointer");
  if (ctx->df_m < 1) return gf2_fail(ctx, GF2_ERR_ARG, "gf2_sigma_tau_df: gf2_set_df_integrals not called");
  if (k0 < 0 || count < 0 || k0 + count > ctx->n_tau)
    return gf2_fail(ctx, GF2_ERR_ARG, "gf2_sigma_tau_df: range outside the grid");
  if (prec != GF2_PREC_FP64) return gf2_fail(ctx, GF2_ERR_UNSUPPORTED, "gf2_sigma_tau_df: FP64 only");
  if (count == 0) return GF2_OK;
  return sigma_df_fp64(ctx, d_G_tau, k0, count, d_Sigma_out);
}
