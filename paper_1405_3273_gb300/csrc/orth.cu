// Symmetric (Loewdin) orthogonalisation used by the split-precision Sigma path.
//
// Eq. Sigma is covariant under a change of basis: with X = S^{-1/2},
//   G' = S^{1/2} G S^{1/2},  v'_ijkl = sum X_ai X_bj X_ck X_dl v_abcd,
//   Sigma = S^{1/2} Sigma'[G', v'] S^{1/2}.
// In the orthonormal basis |G'_ij| <= 1, while in a nearly linearly dependent
// AO basis S^{-1} has large entries and G(tau -> 0) inherits them; the FP32
// accumulation of the tensor cores then loses the digits those cancel.  The
// transforms themselves are FP64 (CUDA cores): S^{1/2} and S^{-1/2} by the
// coupled Newton-Schulz iteration (Y -> (S/c)^{1/2}, Z -> (S/c)^{-1/2},
// T = (3I - ZY)/2, Y <- YT, Z <- TZ, c = ||S||_F so that the spectrum of S/c
// lies in (0, 1]), v by four single-index transforms, G by two matrix
// products per time point.  Of Sigma's back transform, the split path folds
// the right factor into its W operand and applies the left one as a single
// FP64 product per time point.
#include <algorithm>
#include <cmath>

#include "gf2_internal.cuh"

namespace {

__global__ void frob_scale_kernel(int N, const double *S, double *Y, double *Z, double *scal) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) acc += S[e] * S[e];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const double c = sqrt(red[0]);
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    Y[e] = S[e] / c;
    Z[e] = (e / N == e % N) ? 1.0 : 0.0;
  }
  if (threadIdx.x == 0) scal[0] = c;
}

// T = (3I - P) / 2
__global__ void ns_step_kernel(int N, const double *P, double *T) {
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) T[e] = 0.5 * ((e / N == e % N ? 3.0 : 0.0) - P[e]);
}

// Shalf = sqrt(c) Y, Smhalf = Z / sqrt(c)
__global__ void ns_finish_kernel(int N, const double *Y, const double *Z, const double *scal, double *out) {
  const double r = sqrt(scal[0]);
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    out[e] = r * Y[e];
    out[N * N + e] = Z[e] / r;
  }
}

Dgemm sq(int N, const double *A, const double *B, double *C) {
  Dgemm g{};
  g.M = N; g.N = N; g.K = N;
  g.A = A; g.a_rs = N; g.a_cs = 1;
  g.B = B; g.b_rs = N; g.b_cs = 1;
  g.C = C; g.c_rs = N; g.c_cs = 1;
  g.nb0 = 1; g.nb1 = 1; g.alpha = 1.0; g.beta_c = 0.0; g.split_k = 1;
  return g;
}

// out[b] = L * A[b] * R for `count` matrices (stride N*N), via tmp
gf2_status sandwich_batch(gf2_ctx *ctx, const double *L, const double *A, const double *R, double *tmp,
                          double *out, int count) {
  const long long N = ctx->N, N2 = N * N;
  for (int b0 = 0; b0 < count; b0 += 65535) {
    const int nb = std::min(65535, count - b0);
    Dgemm g1 = sq((int)N, L, A + b0 * N2, tmp + b0 * N2);
    g1.a_b0 = 0; g1.b_b0 = N2; g1.c_b0 = N2; g1.nb0 = nb;
    gf2_status st = gf2_dgemm(ctx, g1);
    if (st != GF2_OK) return st;
    Dgemm g2 = sq((int)N, tmp + b0 * N2, R, out + b0 * N2);
    g2.a_b0 = N2; g2.b_b0 = 0; g2.c_b0 = N2; g2.nb0 = nb;
    st = gf2_dgemm(ctx, g2);
    if (st != GF2_OK) return st;
  }
  return GF2_OK;
}

}  // namespace

extern "C" gf2_status gf2_set_overlap(gf2_ctx *ctx, const double *d_S) {
  if (!ctx) return GF2_ERR_ARG;
  if (!d_S) return gf2_fail(ctx, GF2_ERR_ARG, "gf2_set_overlap: NULL pointer");
  const int N = ctx->N;
  const size_t N2 = (size_t)N * N;
  if (!ctx->d_Shalf) GF2_CK(ctx, cudaMalloc(&ctx->d_Shalf, 2 * N2 * sizeof(double)));
  double *w = ctx->d_small + (size_t)GF2_SL_MOM * N2;  // 4 slots: Y, Z, P, T
  double *Y = w, *Z = w + N2, *P = w + 2 * N2, *T = w + 3 * N2, *Y2 = ctx->d_small + (size_t)GF2_SL_COEF * N2,
         *Z2 = Y2 + N2, *scal = ctx->d_small + (size_t)GF2_SL_MISC * N2;
  frob_scale_kernel<<<1, 256, 0, ctx->stream>>>(N, d_S, Y, Z, scal);
  GF2_CK_LAUNCH(ctx, "frob_scale_kernel");
  gf2_status st;
  for (int it = 0; it < 80; ++it) {
    if ((st = gf2_dgemm(ctx, sq(N, Z, Y, P))) != GF2_OK) return st;
    ns_step_kernel<<<1, 256, 0, ctx->stream>>>(N, P, T);
    GF2_CK_LAUNCH(ctx, "ns_step_kernel");
    if ((st = gf2_dgemm(ctx, sq(N, Y, T, Y2))) != GF2_OK) return st;
    if ((st = gf2_dgemm(ctx, sq(N, T, Z, Z2))) != GF2_OK) return st;
    std::swap(Y, Y2);
    std::swap(Z, Z2);
  }
  ns_finish_kernel<<<1, 256, 0, ctx->stream>>>(N, Y, Z, scal, ctx->d_Shalf);
  GF2_CK_LAUNCH(ctx, "ns_finish_kernel");
  if (ctx->have_integrals) {
    st = gf2_tc_prepare_integrals(ctx);
    if (st != GF2_OK && st != GF2_ERR_UNSUPPORTED) return st;
  }
  return GF2_OK;
}

// v'[i][j][k][l] = sum X_ai X_bj X_ck X_dl v[a][b][c][d], X = S^{-1/2} (symmetric)
gf2_status gf2_orth_transform_v(gf2_ctx *ctx, double *d_vorth) {
  const long long N = ctx->N, N2 = N * N, N3 = N2 * N, N4 = N3 * N;
  const double *X = ctx->d_Shalf + N2;
  double *tmp = nullptr;
  GF2_CK(ctx, cudaMalloc(&tmp, N4 * sizeof(double)));
  gf2_status st = GF2_OK;
  // l: tmp[(a,b,c), l] = v[(a,b,c), d] X[d, l]
  Dgemm g{};
  g.M = (int)N3; g.N = (int)N; g.K = (int)N;
  g.A = ctx->d_v; g.a_rs = N; g.a_cs = 1;
  g.B = X; g.b_rs = N; g.b_cs = 1;
  g.C = tmp; g.c_rs = N; g.c_cs = 1;
  g.nb0 = 1; g.nb1 = 1; g.alpha = 1.0; g.split_k = 1;
  if ((st = gf2_dgemm(ctx, g)) != GF2_OK) goto done;
  {  // k: out[a,b][k, l] = X^T[k, c] tmp[a,b][c, l]   (batch over (a,b))
    Dgemm h{};
    h.M = (int)N; h.N = (int)N; h.K = (int)N;
    h.A = X; h.a_rs = 1; h.a_cs = N;
    h.B = tmp; h.b_rs = N; h.b_cs = 1; h.b_b0 = N2;
    h.C = d_vorth; h.c_rs = N; h.c_cs = 1; h.c_b0 = N2;
    h.nb0 = (int)N2; h.nb1 = 1; h.alpha = 1.0; h.split_k = 1;
    if ((st = gf2_dgemm(ctx, h)) != GF2_OK) goto done;
  }
  {  // j: tmp[a][j, (k,l)] = X^T[j, b] out[a][b, (k,l)]   (batch over a)
    Dgemm h{};
    h.M = (int)N; h.N = (int)N2; h.K = (int)N;
    h.A = X; h.a_rs = 1; h.a_cs = N;
    h.B = d_vorth; h.b_rs = N2; h.b_cs = 1; h.b_b0 = N3;
    h.C = tmp; h.c_rs = N2; h.c_cs = 1; h.c_b0 = N3;
    h.nb0 = (int)N; h.nb1 = 1; h.alpha = 1.0; h.split_k = 1;
    if ((st = gf2_dgemm(ctx, h)) != GF2_OK) goto done;
  }
  {  // i: out[i, (j,k,l)] = X^T[i, a] tmp[a, (j,k,l)]
    Dgemm h{};
    h.M = (int)N; h.N = (int)N3; h.K = (int)N;
    h.A = X; h.a_rs = 1; h.a_cs = N;
    h.B = tmp; h.b_rs = N3; h.b_cs = 1;
    h.C = d_vorth; h.c_rs = N3; h.c_cs = 1;
    h.nb0 = 1; h.nb1 = 1; h.alpha = 1.0; h.split_k = 1;
    st = gf2_dgemm(ctx, h);
  }
done:
  cudaStreamSynchronize(ctx->stream);
  cudaFree(tmp);
  return st;
}

// G'(tau_k) = S^{1/2} G(tau_k) S^{1/2} for k in [k0, k0+count) and the mirrored
// points M-k used for G(-tau); *d_Gorth points at a full-grid array.
gf2_status gf2_orth_transform_g(gf2_ctx *ctx, const double *d_G, int k0, int count, double **d_Gorth) {
  const long long N2 = (long long)ctx->N * ctx->N;
  const size_t grid = (size_t)ctx->n_tau * N2;
  if (!ctx->d_orth_ws) GF2_CK(ctx, cudaMalloc(&ctx->d_orth_ws, 3 * grid * sizeof(double)));
  double *Go = ctx->d_orth_ws, *tmp = ctx->d_orth_ws + grid;
  const double *Sh = ctx->d_Shalf;
  const int m0 = (ctx->n_tau - 1) - (k0 + count - 1);  // G(-tau) = -G(beta - tau): the mirrored points
  gf2_status st;
  if (m0 <= k0 + count && k0 <= m0 + count) {  // the two ranges touch: one pass over the union
    const int lo = std::min(k0, m0), hi = std::max(k0, m0) + count;
    st = sandwich_batch(ctx, Sh, d_G + lo * N2, Sh, tmp, Go + lo * N2, hi - lo);
  } else {
    st = sandwich_batch(ctx, Sh, d_G + k0 * N2, Sh, tmp, Go + k0 * N2, count);
    if (st == GF2_OK) st = sandwich_batch(ctx, Sh, d_G + m0 * N2, Sh, tmp, Go + m0 * N2, count);
  }
  if (st != GF2_OK) return st;
  *d_Gorth = Go;
  return GF2_OK;
}

namespace {
// X <- (X + X^T)/2 for `count` N x N matrices
__global__ void symmetrize_kernel(int N, long long count, double *X) {
  const long long N2 = (long long)N * N;
  const long long total = count * N2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / N2;
    const int r = (int)(e % N2), i = r / N, j = r % N;
    if (i >= j) continue;
    double *m = X + b * N2;
    const double avg = 0.5 * (m[i * N + j] + m[j * N + i]);
    m[i * N + j] = avg;
    m[j * N + i] = avg;
  }
}
}  // namespace

gf2_status gf2_symmetrize(gf2_ctx *ctx, double *d_X, int count) {
  const long long total = (long long)count * ctx->N * ctx->N;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 16LL * ctx->num_sms);
  symmetrize_kernel<<<std::max(blocks, 1), 256, 0, ctx->stream>>>(ctx->N, count, d_X);
  GF2_CK_LAUNCH(ctx, "symmetrize_kernel");
  return GF2_OK;
}
