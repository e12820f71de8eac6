// FP64 building blocks: a strided, doubly-batched GEMM on the CUDA cores and a
// one-CTA Gauss-Jordan inverse for the (symmetric positive-definite) overlap.
//
// The GEMM computes, for every batch index (b0, b1),
//   C[b] = alpha * A[b] B[b] + beta_c * C[b]
// with arbitrary row/column/batch strides, so that every single-index
// contraction of a 4-index tensor by an N x N matrix maps onto it without
// copies.  64x64 output tile per CTA, 256 threads with 4x4 outputs each,
// K consumed in slabs of 16 staged through shared memory.  FP64 FMA on
// GB300 is the bound, not memory.
#include "gf2_internal.cuh"

namespace {

constexpr int TM = 64, TN = 64, TK = 16;

__global__ void __launch_bounds__(256) dgemm_kernel(Dgemm g, int tiles_m, int tiles_n) {
  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TN + 1];
  const int tile = blockIdx.x;
  const int ks = g.split_k > 1 ? g.split_k : 1;
  const int kpart = tile % ks;
  const int t = tile / ks;
  const int tm = t / tiles_n, tn = t % tiles_n;
  const int b0 = blockIdx.y, b1 = blockIdx.z;
  const double *A = g.A + b0 * g.a_b0 + b1 * g.a_b1;
  const double *B = g.B + b0 * g.b_b0 + b1 * g.b_b1;
  double *C = g.C + b0 * g.c_b0 + b1 * g.c_b1;

  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int row0 = tm * TM, col0 = tn * TN;
  double acc[4][4] = {};

  long long kchunk = ((long long)g.K + ks - 1) / ks;
  kchunk = ((kchunk + TK - 1) / TK) * TK;
  const long long kbeg = kpart * kchunk;
  const long long kend = min((long long)g.K, kbeg + kchunk);

  for (long long k0 = kbeg; k0 < kend; k0 += TK) {
    // stage A[row0:+64, k0:+16] and B[k0:+16, col0:+64]
    for (int e = threadIdx.x; e < TM * TK; e += 256) {
      int r = e / TK, kk = e % TK;
      long long gr = row0 + r, gk = k0 + kk;
      As[kk][r] = (gr < g.M && gk < kend) ? A[gr * g.a_rs + gk * g.a_cs] : 0.0;
    }
    for (int e = threadIdx.x; e < TK * TN; e += 256) {
      int kk = e / TN, c = e % TN;
      long long gc = col0 + c, gk = k0 + kk;
      Bs[kk][c] = (gc < g.N && gk < kend) ? B[gk * g.b_rs + gc * g.b_cs] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    long long gr = row0 + ty + 16 * i;
    if (gr >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      long long gc = col0 + tx + 16 * j;
      if (gc >= g.N) continue;
      double *c = C + gr * g.c_rs + gc * g.c_cs;
      if (ks > 1) {
        atomicAdd(c, g.alpha * acc[i][j]);
      } else {
        double prev = g.beta_c != 0.0 ? g.beta_c * (*c) : 0.0;
        *c = g.alpha * acc[i][j] + prev;
      }
    }
  }
}

// In-place Gauss-Jordan inversion of an SPD matrix (no pivoting needed).
__global__ void inverse_spd_kernel(const double *A, double *Ainv, int n) {
  extern __shared__ double sm[];
  double *a = sm;            // n*n
  double *col = sm + n * n;  // n
  double *row = col + n;     // n
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) a[e] = A[e];
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] = a[i * n + k];
    __syncthreads();
    const double p = 1.0 / col[k];
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      double r = (j == k) ? p : a[k * n + j] * p;
      row[j] = r;
      a[k * n + j] = r;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      int i = e / n, j = e % n;
      if (i == k) continue;
      if (j == k) a[e] = -col[i] * p;
      else a[e] -= col[i] * row[j];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) Ainv[e] = a[e];
}

}  // namespace

gf2_status gf2_dgemm(gf2_ctx *ctx, const Dgemm &g) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0 || g.nb0 <= 0 || g.nb1 <= 0) return GF2_OK;
  if (g.nb0 > 65535 || g.nb1 > 65535) return gf2_fail(ctx, GF2_ERR_UNSUPPORTED, "dgemm batch too large");
  const int tiles_m = (g.M + TM - 1) / TM, tiles_n = (g.N + TN - 1) / TN;
  const int ks = g.split_k > 1 ? g.split_k : 1;
  dim3 grid(tiles_m * tiles_n * ks, g.nb0, g.nb1);
  GF2_PROF(ctx, GF2_K_DGEMM, (dgemm_kernel<<<grid, 256, 0, ctx->stream>>>(g, tiles_m, tiles_n)));
  GF2_CK_LAUNCH(ctx, "dgemm_kernel");
  return GF2_OK;
}

gf2_status gf2_inverse_spd(gf2_ctx *ctx, const double *d_A, double *d_Ainv) {
  const int n = ctx->N;
  size_t smem = sizeof(double) * (size_t)(n * n + 2 * n);
  if (smem > 48 * 1024)
    GF2_CK(ctx, cudaFuncSetAttribute(inverse_spd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  inverse_spd_kernel<<<1, 256, smem, ctx->stream>>>(d_A, d_Ainv, n);
  GF2_CK_LAUNCH(ctx, "inverse_spd_kernel");
  return GF2_OK;
}
