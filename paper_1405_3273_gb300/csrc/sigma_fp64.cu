// Eq. Sigma in FP64 as four successive single-index contractions per time
// point (the O(n_tau N^5) route of the paper's cost discussion):
//   T1[i,m,q,l] = sum_k v[i,m,q,k] G[k,l]
//   T2[i,n,q,l] = sum_m G[m,n] T1[i,m,q,l]
//   T3[i,n,p,l] = sum_q Gbar[p,q] T2[i,n,q,l],      Gbar = G(-tau) = -G(tau_{M-k})
//   Sigma[i,j]  = - sum_{(n,p,l)} T3[i,(n,p,l)] Wt[(n,p,l),j],  Wt[n,p,l,j] = W[l,p,n,j]
// Time points are processed in chunks so that two N^4 intermediates per point
// fit the workspace; every stage is one strided batched DGEMM launch.
#include <algorithm>

#include "gf2_internal.cuh"

gf2_status gf2_sigma_fp64(gf2_ctx *ctx, const double *d_G, int k0, int count, double *d_out) {
  const long long N = ctx->N, N2 = N * N, N3 = N2 * N, N4 = N3 * N;
  const int M = ctx->n_tau - 1;  // last grid point (tau = beta); the grid is symmetric about beta/2
  if (!ctx->d_ws) {
    size_t budget = (size_t)2 << 30;  // bytes for the two ping-pong buffers
    long long chunk = std::max<long long>(1, (long long)(budget / (2 * N4 * sizeof(double))));
    chunk = std::min<long long>(chunk, ctx->n_tau);
    chunk = std::min<long long>(chunk, 65535);
    ctx->fp64_chunk = (int)chunk;
    ctx->ws_elems = (size_t)(2 * chunk * N4);
    GF2_CK(ctx, cudaMalloc(&ctx->d_ws, ctx->ws_elems * sizeof(double)));
  }
  double *bufA = ctx->d_ws;
  double *bufB = ctx->d_ws + (size_t)ctx->fp64_chunk * N4;

  for (int c0 = 0; c0 < count; c0 += ctx->fp64_chunk) {
    const int B = std::min(ctx->fp64_chunk, count - c0);
    const int kb = k0 + c0;  // first grid point of the chunk
    gf2_status st;

    // stage 1: T1[b] (N^3 x N) = v (N^3 x N) * G_b
    Dgemm g1{};
    g1.M = (int)N3; g1.N = (int)N; g1.K = (int)N;
    g1.A = ctx->d_v;          g1.a_rs = N;  g1.a_cs = 1;  g1.a_b0 = 0;       g1.a_b1 = 0;
    g1.B = d_G + kb * N2;     g1.b_rs = N;  g1.b_cs = 1;  g1.b_b0 = N2;      g1.b_b1 = 0;
    g1.C = bufA;              g1.c_rs = N;  g1.c_cs = 1;  g1.c_b0 = N4;      g1.c_b1 = 0;
    g1.nb0 = B; g1.nb1 = 1; g1.alpha = 1.0; g1.beta_c = 0.0; g1.split_k = 1;
    if ((st = gf2_dgemm(ctx, g1)) != GF2_OK) return st;

    // stage 2: T2[b][i] (N x N^2) = G_b^T (N x N) * T1[b][i] (N x N^2)
    Dgemm g2{};
    g2.M = (int)N; g2.N = (int)N2; g2.K = (int)N;
    g2.A = d_G + kb * N2;     g2.a_rs = 1;  g2.a_cs = N;  g2.a_b0 = 0;       g2.a_b1 = N2;
    g2.B = bufA;              g2.b_rs = N2; g2.b_cs = 1;  g2.b_b0 = N3;      g2.b_b1 = N4;
    g2.C = bufB;              g2.c_rs = N2; g2.c_cs = 1;  g2.c_b0 = N3;      g2.c_b1 = N4;
    g2.nb0 = (int)N; g2.nb1 = B; g2.alpha = 1.0; g2.beta_c = 0.0; g2.split_k = 1;
    if ((st = gf2_dgemm(ctx, g2)) != GF2_OK) return st;

    // stage 3: T3[b][i][n] (N x N) = Gbar_b (N x N) * T2[b][i][n] (N x N);
    // Gbar_b = -G(tau_{M-kb-b}) : negative batch stride, sign folded into alpha
    Dgemm g3{};
    g3.M = (int)N; g3.N = (int)N; g3.K = (int)N;
    g3.A = d_G + (long long)(M - kb) * N2; g3.a_rs = N; g3.a_cs = 1; g3.a_b0 = 0; g3.a_b1 = -N2;
    g3.B = bufB;              g3.b_rs = N;  g3.b_cs = 1;  g3.b_b0 = N2;      g3.b_b1 = N4;
    g3.C = bufA;              g3.c_rs = N;  g3.c_cs = 1;  g3.c_b0 = N2;      g3.c_b1 = N4;
    g3.nb0 = (int)N2; g3.nb1 = B; g3.alpha = -1.0; g3.beta_c = 0.0; g3.split_k = 1;
    if ((st = gf2_dgemm(ctx, g3)) != GF2_OK) return st;

    // stage 4: Sigma_b (N x N) = - T3[b] (N x N^3) * Wt (N^3 x N), split over K
    double *out = d_out + (long long)c0 * N2;
    GF2_CK(ctx, cudaMemsetAsync(out, 0, sizeof(double) * B * N2, ctx->stream));
    Dgemm g4{};
    g4.M = (int)N; g4.N = (int)N; g4.K = (int)N3;
    g4.A = bufA;              g4.a_rs = N3; g4.a_cs = 1;  g4.a_b0 = N4;      g4.a_b1 = 0;
    g4.B = ctx->d_Wt;         g4.b_rs = N;  g4.b_cs = 1;  g4.b_b0 = 0;       g4.b_b1 = 0;
    g4.C = out;               g4.c_rs = N;  g4.c_cs = 1;  g4.c_b0 = N2;      g4.c_b1 = 0;
    g4.nb0 = B; g4.nb1 = 1; g4.alpha = -1.0; g4.beta_c = 0.0;
    int tiles = (int)((N + 63) / 64) * (int)((N + 63) / 64);
    int want = std::max(1, (2 * ctx->num_sms) / std::max(1, B * tiles));
    g4.split_k = (int)std::min<long long>(want, std::max<long long>(1, N3 / 256));
    if ((st = gf2_dgemm(ctx, g4)) != GF2_OK) return st;
  }
  return GF2_OK;
}
