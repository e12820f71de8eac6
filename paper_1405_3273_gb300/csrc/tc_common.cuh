// Pieces shared by the split-precision Sigma pipelines of both tile widths
// (a 64- and a 128-wide padded basis): the products of a T-term split, the
// rounding of FP32 values to 16-bit terms (BF16 or FP16 with power-of-two
// scales), the splitting of the FP64 inputs into term planes, compensated
// FP32 sums, and tensor-map encoding.  Included by one translation unit per
// tile width; everything here has internal linkage.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "tc_ptx.cuh"

namespace {

constexpr int TMAX = 3;
constexpr int kErrTimeout = 1;

// product list (a, b) with a + b < T, smallest terms first
template <int T>
struct Products;
template <>
struct Products<2> {
  static constexpr int n = 3;
  __device__ static int a(int k) { return k == 0 ? 1 : 0; }
  __device__ static int b(int k) { return k == 1 ? 1 : 0; }
};
template <>
struct Products<3> {
  static constexpr int n = 6;
  __device__ static int a(int k) { const int t[6] = {2, 1, 0, 1, 0, 0}; return t[k]; }
  __device__ static int b(int k) { const int t[6] = {0, 1, 2, 0, 1, 0}; return t[k]; }
};

// rounding of two FP32 values to a packed pair of 16-bit terms; `back` gets the
// rounded values in FP32, so the caller can form the next residual
template <int F>
__device__ __forceinline__ uint32_t pack2(float a, float b, float2 &back) {
  if constexpr (F == 0) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(a, b);
    back = __bfloat1622float2(p);
    return *reinterpret_cast<const uint32_t *>(&p);
  } else {
    const __half2 p = __floats2half2_rn(a, b);
    back = __half22float2(p);
    return *reinterpret_cast<const uint32_t *>(&p);
  }
}

// instruction descriptor of a kind::f16 MMA with BF16 (F = 0) or FP16 (F = 1) operands
__host__ __device__ constexpr uint32_t idesc_fmt(int F, int M, int N, int a_mn_major, int b_mn_major) {
  return F == 0 ? tc::idesc_bf16(M, N, a_mn_major, b_mn_major) : tc::idesc_f16(M, N, a_mn_major, b_mn_major);
}

// exponent e with 2^e * amax in [2^13, 2^14) (0 for an all-zero operand)
__host__ __device__ inline int fp16_exponent(double amax) {
  if (!(amax > 0.0)) return 0;
  int E;
  frexp(amax, &E);  // amax = f 2^E, f in [0.5, 1)
  return 14 - E;
}

// FP16 scale exponents per time point of a chunk, [kExpSets][C] ints:
// eg (G(tau)^T), egb (Gbar(tau)), r1 (T1 operand), max|T2| and max|T3| (float bits)
enum { kExpG = 0, kExpGbar = 1, kExpT1 = 2, kMaxT2 = 3, kMaxT3 = 4, kExpSets = 5 };

__device__ __forceinline__ float exp2_scale(int e) { return ldexpf(1.0f, e); }

// scale that brings the largest |value| of a stored T2 or T3 (float bits) into [2^13, 2^14)
__device__ __forceinline__ int fp16_exponent_bits(int bits) { return fp16_exponent((double)__int_as_float(bits)); }

// largest |x| of a warp into slot[0] (nonnegative floats order like their bits)
__device__ __forceinline__ void warp_absmax_to(int *slot, float m) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(slot, __float_as_int(m));
}

__device__ __forceinline__ uint8_t *align1024(uint8_t *p) {
  return reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

__device__ __forceinline__ void raise_abort(volatile int *abort, int *err) {
  *abort = 1;
  atomicExch(err, kErrTimeout);
}

// eight consecutive fp32 values (times `scale`, FP16 only) -> T 16-bit terms,
// 16 bytes per term at dst + t * plane
template <int T, int F>
__device__ __forceinline__ void split8_store(const float *v, uint8_t *dst, uint32_t plane, float scale) {
  float x[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) x[e] = F == 0 ? v[e] : v[e] * scale;
#pragma unroll
  for (int t = 0; t < T; ++t) {
    uint32_t w[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float2 f;
      w[e] = pack2<F>(x[2 * e], x[2 * e + 1], f);
      x[2 * e] -= f.x;
      x[2 * e + 1] -= f.y;
    }
    *reinterpret_cast<uint4 *>(dst + t * plane) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// Split one row of 64 fp32 values (a TMEM lane of an A operand, times
// `scale` for FP16) into T 16-bit terms and write term t as 32 packed columns
// at column taddr + 32 t.
template <int T, int F>
__device__ __forceinline__ void split_row_to_tmem(float *x, uint32_t taddr, float scale) {
  if constexpr (F != 0) {
#pragma unroll
    for (int c = 0; c < 64; ++c) x[c] *= scale;
  }
#pragma unroll
  for (int t = 0; t < T; ++t) {
    uint32_t w[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      float2 f;
      w[c] = pack2<F>(x[2 * c], x[2 * c + 1], f);
      x[2 * c] -= f.x;
      x[2 * c + 1] -= f.y;
    }
    tc::tmem_st_32x32b_x32(taddr + 32 * t, w);
  }
}

// x (already scaled) -> TMAX 16-bit terms of format F, as raw bits
template <int F>
__device__ __forceinline__ void split_f64(double x, uint16_t *p) {
  double r = x;
#pragma unroll
  for (int t = 0; t < TMAX; ++t) {
    if constexpr (F == 0) {
      const __nv_bfloat16 h = __double2bfloat16(r);
      p[t] = *reinterpret_cast<const uint16_t *>(&h);
      r -= (double)__bfloat162float(h);
    } else {
      const __half h = __double2half(r);
      p[t] = *reinterpret_cast<const uint16_t *>(&h);
      r -= (double)__half2float(h);
    }
  }
}


// Vs[t][i][q][m][k] = split_t (2^e v[i][m][q][k]), block-diagonal with B
// blocks of N (zero outside them)
template <int NP, int F>
__global__ void split_v_kernel(int N, int B, const double *__restrict__ v, int e, uint16_t *__restrict__ Vs) {
  const size_t plane = (size_t)NP * NP * NP * NP;
  const double sc = ldexp(1.0, e);
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < plane;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int k = idx % NP, m = (idx / NP) % NP, q = (idx / (NP * NP)) % NP, i = idx / (NP * NP * NP);
    const int b = i / N, o = b * N;
    double x = 0.0;
    if (b < B && m / N == b && q / N == b && k / N == b)
      x = v[(((size_t)(i - o) * N + (m - o)) * N + (q - o)) * N + (k - o)] * sc;
    uint16_t p[TMAX];
    split_f64<F>(x, p);
    for (int t = 0; t < TMAX; ++t) Vs[t * plane + idx] = p[t];
  }
}

// Ws[t][j][l][n][p] = split_t (2^e W[l][p][n][j]),  W_lpnj = 2 v_lpnj - v_nplj,
// block-diagonal with B blocks of N
template <int NP, int F>
__global__ void split_w_kernel(int N, int B, const double *__restrict__ v, int e, uint16_t *__restrict__ Ws) {
  const size_t plane = (size_t)NP * NP * NP * NP;
  const double sc = ldexp(1.0, e);
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < plane;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int p = idx % NP, n = (idx / NP) % NP, l = (idx / (NP * NP)) % NP, j = idx / (NP * NP * NP);
    const int bk = j / N, o = bk * N;
    double x = 0.0;
    if (bk < B && l / N == bk && n / N == bk && p / N == bk) {
      const int jj = j - o, ll = l - o, nn = n - o, pp = p - o;
      const double a = v[(((size_t)ll * N + pp) * N + nn) * N + jj];
      const double b = v[(((size_t)nn * N + pp) * N + ll) * N + jj];
      x = (2.0 * a - b) * sc;
    }
    uint16_t p3[TMAX];
    split_f64<F>(x, p3);
    for (int t = 0; t < TMAX; ++t) Ws[t * plane + idx] = p3[t];
  }
}

// Gs[set][t][c][r][s]: set 0 = G(tau)^T (GT[l][k] = G[k][l]),
//                      set 1 = Gbar = G(-tau) = -G(tau_{M-k}) (Gbar[p][q]).
// Slot c holds the time points c*B + b (b < B) of the chunk in its diagonal
// blocks of N.  FP16: every slot matrix is scaled by its own 2^ex[set][c];
// block (c, 0) also sets the T1 exponent ex[kExpT1][c] from the bound
// |T1| <= vmax_s * max_l sum_k |G_s[k][l]| (vmax_s: largest |v| after its
// scale) and clears the T2/T3 maxima of slot c.
template <int NP, int F>
__global__ void split_g_kernel(int N, int B, int M, int k0, int count, int C, const double *__restrict__ G,
                               uint16_t *__restrict__ Gs, int *__restrict__ ex, double vmax_s) {
  const int c = blockIdx.x, set = blockIdx.y;
  const size_t plane = (size_t)C * NP * NP;
  auto elem = [&](int r, int s) -> double {  // entry (r, s) of the slot matrix
    const int b = r / N;
    if (b >= B || s / N != b || c * B + b >= count) return 0.0;
    const int k = k0 + c * B + b, rr = r - b * N, ss = s - b * N;
    return set == 0 ? G[(size_t)k * N * N + (size_t)ss * N + rr] : -G[(size_t)(M - k) * N * N + (size_t)rr * N + ss];
  };
  double sc = 1.0;
  if constexpr (F != 0) {
    __shared__ double red[2][32];
    double m = 0.0, cs = 0.0;  // largest |entry|, largest row sum of |GT| (a column sum of |G|)
    for (int r4 = threadIdx.x; r4 < NP * 4; r4 += blockDim.x) {  // four threads per row, NP / 4 entries each
      const int r = r4 >> 2, q0 = (r4 & 3) * (NP / 4);
      double a = 0.0;
      for (int q = q0; q < q0 + NP / 4; ++q) {
        const double x = fabs(elem(r, q));
        a += x;
        m = fmax(m, x);
      }
      a += __shfl_xor_sync(0xffffffffu, a, 1);
      a += __shfl_xor_sync(0xffffffffu, a, 2);
      cs = fmax(cs, a);
    }
    for (int o = 16; o > 0; o >>= 1) {
      m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
      cs = fmax(cs, __shfl_xor_sync(0xffffffffu, cs, o));
    }
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x / 32] = m;
      red[1][threadIdx.x / 32] = cs;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)blockDim.x / 32; ++w) {
        m = fmax(m, red[0][w]);
        cs = fmax(cs, red[1][w]);
      }
      red[0][0] = m;
      red[1][0] = cs;
    }
    __syncthreads();
    const int e = fp16_exponent(red[0][0]);
    sc = ldexp(1.0, e);
    if (threadIdx.x == 0) {
      ex[set * C + c] = e;
      if (set == 0) {
        ex[kExpT1 * C + c] = fp16_exponent(vmax_s * red[1][0] * sc);
        ex[kMaxT2 * C + c] = 0;
        ex[kMaxT3 * C + c] = 0;
      }
    }
  }
  for (int e = threadIdx.x; e < NP * NP; e += blockDim.x) {
    uint16_t p[TMAX];
    split_f64<F>(elem(e / NP, e % NP) * sc, p);
    for (int t = 0; t < TMAX; ++t) Gs[(size_t)(set * TMAX + t) * plane + (size_t)c * NP * NP + e] = p[t];
  }
}

__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bp = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
  hi = s;
  lo = __fadd_rn(lo, e);
}


PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// bf16 operand tiles use the 128-byte swizzle of the MMA layouts; fp32 tiles
// (split on chip) are plain row-major
bool make_map(CUtensorMap *m, const void *base, int rank, const uint64_t *dims, const uint64_t *strides_bytes,
              const uint32_t *box, bool fp32 = false, bool fp32_swizzle = false) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  CUresult r = fn(m, fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, rank,
                  const_cast<void *>(base), reinterpret_cast<const cuuint64_t *>(dims),
                  reinterpret_cast<const cuuint64_t *>(strides_bytes), reinterpret_cast<const cuuint32_t *>(box), es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE,
                  (fp32 && !fp32_swizzle) ? CU_TENSOR_MAP_SWIZZLE_NONE : CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}


}  // namespace
