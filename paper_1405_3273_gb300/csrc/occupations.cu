// Natural occupation numbers, the observable of the paper's H32 lattice
// results: n_k = eig(S^1/2 P S^1/2) / 2, sorted from largest to smallest.
//
// X = S^1/2 P S^1/2 by two FP64 GEMMs, then the eigenvalues of the symmetric
// N x N matrix by the cyclic Jacobi method in one CTA, the matrix resident in
// shared memory (N <= 128: 130 KB).  Each sweep visits every pair (p, q) once
// in N' - 1 rounds of the round-robin ordering (N' = N rounded up to even):
// the pairs of a round are disjoint, so their rotations commute and are applied
// together -- all row updates, then all column updates.  Rotation per Golub &
// Van Loan, "Matrix Computations", symmetric Schur decomposition: with
// theta = (a_qq - a_pp) / (2 a_pq), t = sign(theta) / (|theta| + sqrt(1 + theta^2)),
// c = 1 / sqrt(1 + t^2), s = t c, the (p, q) entry of J^T A J vanishes.
// Sweeps stop when the off-diagonal Frobenius norm is below 1e-15 of the
// whole norm, or after kMaxSweeps (error word set).
#include <algorithm>

#include "gf2_internal.cuh"

namespace {

constexpr int kMaxSweeps = 60;
constexpr int kJacobiThreads = 512;

__global__ void __launch_bounds__(kJacobiThreads)
    jacobi_occupations_kernel(int N, const double *__restrict__ X, double *__restrict__ occ, int *err) {
  extern __shared__ double A[];  // [N][N], then the rotations of a round
  const int Np = (N + 1) & ~1, npairs = Np / 2;
  double *cs = A + N * N;        // [npairs][2]: c, s
  int *pp = reinterpret_cast<int *>(cs + 2 * npairs);  // [npairs][2]: p, q (q = N: dummy)
  __shared__ double red[kJacobiThreads / 32];
  __shared__ int done;
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int i = e / N, j = e % N;
    A[e] = 0.5 * (X[i * N + j] + X[j * N + i]);
  }
  if (threadIdx.x == 0) done = 0;
  __syncthreads();
  int sweep = 0;
  for (; sweep < kMaxSweeps; ++sweep) {
    // convergence test: off-diagonal against total Frobenius norm
    double off = 0.0, all = 0.0;
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
      const double a2 = A[e] * A[e];
      all += a2;
      if (e / N != e % N) off += a2;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      all += __shfl_xor_sync(0xffffffffu, all, o);
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = off;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s_off = 0.0;
      for (int w = 0; w < (int)blockDim.x / 32; ++w) s_off += red[w];
      red[0] = s_off;
    }
    __syncthreads();
    const double off_tot = red[0];
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = all;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s_all = 0.0;
      for (int w = 0; w < (int)blockDim.x / 32; ++w) s_all += red[w];
      done = !(off_tot > 1e-30 * s_all);  // off-diagonal norm below 1e-15 of the total
    }
    __syncthreads();
    if (done) break;
    for (int r = 0; r < Np - 1; ++r) {
      // round r of the circle method: (r, Np-1) and ((r+k) mod (Np-1), (r-k) mod (Np-1))
      for (int k = threadIdx.x; k < npairs; k += blockDim.x) {
        int p, q;
        if (k == 0) {
          p = r;
          q = Np - 1;
        } else {
          p = (r + k) % (Np - 1);
          q = (r - k + (Np - 1)) % (Np - 1);
        }
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        double c = 1.0, s = 0.0;
        if (q < N) {
          const double apq = A[p * N + q];
          if (apq != 0.0) {
            const double theta = (A[q * N + q] - A[p * N + p]) / (2.0 * apq);
            const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        }
        cs[2 * k] = c;
        cs[2 * k + 1] = s;
        pp[2 * k] = p;
        pp[2 * k + 1] = q;
      }
      __syncthreads();
      // rows p, q of every pair:  A <- J^T A
      for (int w = threadIdx.x; w < npairs * N; w += blockDim.x) {
        const int k = w / N, j = w % N, p = pp[2 * k], q = pp[2 * k + 1];
        if (q >= N) continue;
        const double c = cs[2 * k], s = cs[2 * k + 1], ap = A[p * N + j], aq = A[q * N + j];
        A[p * N + j] = c * ap - s * aq;
        A[q * N + j] = s * ap + c * aq;
      }
      __syncthreads();
      // columns p, q of every pair:  A <- A J
      for (int w = threadIdx.x; w < npairs * N; w += blockDim.x) {
        const int k = w / N, i = w % N, p = pp[2 * k], q = pp[2 * k + 1];
        if (q >= N) continue;
        const double c = cs[2 * k], s = cs[2 * k + 1], ap = A[i * N + p], aq = A[i * N + q];
        A[i * N + p] = c * ap - s * aq;
        A[i * N + q] = s * ap + c * aq;
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    if (!done) atomicExch(err, 1);
    // eigenvalues from the diagonal, sorted largest first (insertion sort), halved
    for (int i = 0; i < N; ++i) cs[i] = A[i * N + i];
    for (int i = 1; i < N; ++i) {
      const double x = cs[i];
      int j = i - 1;
      while (j >= 0 && cs[j] < x) {
        cs[j + 1] = cs[j];
        --j;
      }
      cs[j + 1] = x;
    }
    for (int i = 0; i < N; ++i) occ[i] = 0.5 * cs[i];
  }
}

Dgemm square(int N, const double *A, const double *B, double *C) {
  Dgemm g{};
  g.M = N; g.N = N; g.K = N;
  g.A = A; g.a_rs = N; g.a_cs = 1;
  g.B = B; g.b_rs = N; g.b_cs = 1;
  g.C = C; g.c_rs = N; g.c_cs = 1;
  g.nb0 = 1; g.nb1 = 1; g.alpha = 1.0; g.beta_c = 0.0; g.split_k = 1;
  return g;
}

}  // namespace

extern "C" gf2_status gf2_natural_occupations(gf2_ctx *ctx, const double *d_P, double *d_occ) {
  if (!ctx) return GF2_ERR_ARG;
  if (!d_P || !d_occ) return gf2_fail(ctx, GF2_ERR_ARG, "gf2_natural_occupations: NULL pointer");
  if (!ctx->d_Shalf) return gf2_fail(ctx, GF2_ERR_ARG, "gf2_natural_occupations: gf2_set_overlap not called");
  const int N = ctx->N;
  const size_t N2 = (size_t)N * N;
  double *T = ctx->d_small + (size_t)GF2_SL_TMP * N2, *X = ctx->d_small + (size_t)GF2_SL_T1 * N2;
  gf2_status st;
  if ((st = gf2_dgemm(ctx, square(N, ctx->d_Shalf, d_P, T))) != GF2_OK) return st;
  if ((st = gf2_dgemm(ctx, square(N, T, ctx->d_Shalf, X))) != GF2_OK) return st;
  const int npairs = (N + 1) / 2;
  const size_t smem = N2 * sizeof(double) + 2 * npairs * sizeof(double) + 2 * npairs * sizeof(int);
  GF2_CK(ctx, cudaFuncSetAttribute(jacobi_occupations_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  GF2_CK(ctx, cudaMemsetAsync(ctx->d_err + 1, 0, sizeof(int), ctx->stream));
  jacobi_occupations_kernel<<<1, kJacobiThreads, smem, ctx->stream>>>(N, X, d_occ, ctx->d_err + 1);
  GF2_CK_LAUNCH(ctx, "jacobi_occupations_kernel");
  int flag = 0;
  GF2_CK(ctx, cudaMemcpyAsync(&flag, ctx->d_err + 1, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  GF2_CK(ctx, cudaStreamSynchronize(ctx->stream));
  if (flag) return gf2_fail(ctx, GF2_ERR_NOT_CONVERGED, "gf2_natural_occupations: Jacobi sweeps did not converge");
  return GF2_OK;
}
