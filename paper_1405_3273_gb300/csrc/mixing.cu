// Linear combinations and Gram matrices of device arrays: the damping of P
// and Sigma(tau) named in the supplement's remarks on convergence, and the
// Pulay (DIIS) extrapolation of F used by the inner loop.
#include <algorithm>

#include "gf2_internal.cuh"

namespace {

constexpr int kMaxTerms = 16;

struct CombineArgs {
  int n;
  double coef[kMaxTerms];
  const double *src[kMaxTerms];
};

__global__ void combine_kernel(CombineArgs a, long long count, double *__restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < a.n; ++k) acc += a.coef[k] * a.src[k][e];
    out[e] = acc;
  }
}

struct GramArgs {
  int n;
  const double *vec[kMaxTerms];
};

// one CTA per pair (a <= b), fixed reduction order
__global__ void gram_kernel(GramArgs g, long long count, double *__restrict__ out) {
  __shared__ double red[256];
  int p = blockIdx.x, a = 0;
  while (p >= g.n - a) { p -= g.n - a; ++a; }
  const int b = a + p;
  double acc = 0.0;
  for (long long e = threadIdx.x; e < count; e += blockDim.x) acc += g.vec[a][e] * g.vec[b][e];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[a * g.n + b] = red[0];
    out[b * g.n + a] = red[0];
  }
}

}  // namespace

extern "C" gf2_status gf2_combine(gf2_ctx *ctx, int n, const double *coef, const double *const *d_src,
                                  long long count, double *d_out) {
  if (!ctx) return GF2_ERR_ARG;
  if (n < 1 || n > kMaxTerms || !coef || !d_src || !d_out || count < 0)
    return gf2_fail(ctx, GF2_ERR_ARG, "gf2_combine: bad arguments");
  CombineArgs a{};
  a.n = n;
  for (int k = 0; k < n; ++k) {
    if (!d_src[k]) return gf2_fail(ctx, GF2_ERR_ARG, "gf2_combine: NULL source");
    a.coef[k] = coef[k];
    a.src[k] = d_src[k];
  }
  if (count == 0) return GF2_OK;
  const int blocks = (int)std::min<long long>((count + 255) / 256, 8LL * ctx->num_sms);
  combine_kernel<<<blocks, 256, 0, ctx->stream>>>(a, count, d_out);
  GF2_CK_LAUNCH(ctx, "combine_kernel");
  return GF2_OK;
}

extern "C" gf2_status gf2_gram(gf2_ctx *ctx, int n, const double *const *d_vecs, long long count,
                               double *gram_out) {
  if (!ctx) return GF2_ERR_ARG;
  if (n < 1 || n > kMaxTerms || !d_vecs || !gram_out || count < 0)
    return gf2_fail(ctx, GF2_ERR_ARG, "gf2_gram: bad arguments");
  if ((size_t)n * n > ctx->red_elems) return gf2_fail(ctx, GF2_ERR_UNSUPPORTED, "gf2_gram: too many vectors");
  GramArgs g{};
  g.n = n;
  for (int k = 0; k < n; ++k) {
    if (!d_vecs[k]) return gf2_fail(ctx, GF2_ERR_ARG, "gf2_gram: NULL vector");
    g.vec[k] = d_vecs[k];
  }
  gram_kernel<<<n * (n + 1) / 2, 256, 0, ctx->stream>>>(g, count, ctx->d_red);
  GF2_CK_LAUNCH(ctx, "gram_kernel");
  GF2_CK(ctx, cudaMemcpyAsync(gram_out, ctx->d_red, sizeof(double) * n * n, cudaMemcpyDeviceToHost, ctx->stream));
  GF2_CK(ctx, cudaStreamSynchronize(ctx->stream));
  return GF2_OK;
}
