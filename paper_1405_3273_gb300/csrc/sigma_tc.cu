// Eq. Sigma on the sm_103a tensor cores (tcgen05 + TMEM, TMA-fed), with every
// operand split into T 16-bit terms and the products sum_{a+b<T} x_a y_b
// accumulated in FP32 (T = 2: three products, T = 3: six).  The terms are BF16
// (F = 0: 8-bit significand, FP32 exponent range) or FP16 (F = 1: 11-bit
// significand, so two terms carry 22 bits).  An FP16 term must stay inside
// [2^-14, 2^15] to keep its bits, so every FP16 operand is scaled by a power of
// two that puts its largest entry in [2^13, 2^14): one exponent for v, one for
// W, one per G(tau) and per Gbar(tau); the T1 operand of the second MMA by a
// bound per time point (max|v| times the largest column sum of |G|); T2 and T3
// by their measured maximum per time point (the producing kernel reduces it
// with atomicMax).  Each stage removes its own operand scale in its epilogue,
// so the stored intermediates carry only the scales of v and G, and the last
// stage removes those.  All scales are powers of two, hence exact.
//
// The basis is padded to NP = 64 (zero rows and columns contribute nothing).
// For N <= 32, B = floor(64 / N) time points share one 64-wide tile: G, Gbar,
// v and W are block-diagonal with B copies of N x N blocks (block b of G holds
// time point b of the group), and Eq. Sigma of a block-diagonal system is the
// block-diagonal of the per-block Sigmas -- every index of a nonzero term lies
// in one block, since G links k-l, m-n, p-q and v, W keep i, m, q, k (and
// l, p, n, j) in one block.  The tile pipeline is unchanged; only the splits of
// the inputs and the output mapping know about B.
// Per chunk of C time points three kernels run back to back:
//
//  sandwich   stages 1+2 fused.  Unit (tau pair, i, q pair): the v tile
//             V[(q,m), k] (128 x 64) is loaded once and used for both time
//             points.  MMA1  D1[(q,m), l]   = sum_k V[(q,m),k] G[k,l]
//             (TMEM) -> split by eight epilogue warps into an MN-major smem
//             operand A2[(q,l), m] -> MMA2  D2[(q,l), n] = sum_m A2 G[m,n]
//             -> four more warps stage T2[tau][i][q][l][n] in FP32 for TMA
//             tile stores (two staging tiles at T = 2).
//  xform      stage 3.  D3[(l,n), p] = sum_q T2[tau][i][q][(l,n)] Gbar[p,q]
//             with the FP32 T2 tile read by TMA and split on chip into the
//             MN-major bf16 operand; stores T3[tau][i][l][n][p] in FP32.
//  contract   stage 4.  Sigma[(tau,i), j] -= sum_K T3[(tau,i), K] Wt4[j, K],
//             K = (l,n,p) of length NP^3, rows = two time points x 64 i;
//             T3 tiles are split on chip like T2.  Split over K in slices of
//             NP^2 (FP32 accumulation in TMEM in groups of two K steps, two
//             accumulators at T = 2, compensated group sums) and reduced into
//             the FP64 output with atomics.
//
// The intermediates T2 and T3 live in HBM as FP32 (4 bytes per value instead
// of 2T for stored bf16 terms).  T bf16 terms of an FP32 value are formed by
// the same rounding on either side of the store, so the operands the tensor
// cores see are the same as if the terms had been stored.  In xform and
// contract the split A operand is written to TMEM by converter warps (one
// thread per row, tcgen05.st) and read from there by tcgen05.mma, so shared
// memory carries only the FP32 tiles and the B operand.
//
// All three are persistent, warp-specialised: one TMA producer thread, one
// MMA-issuing thread, converter warps where an FP32 tile is split, and
// epilogue warps that own the TMEM lane quarters (warp w reads lanes
// 32*(w%4) .. +31).  Waits are bounded; a timeout raises the context error
// word and the kernel drains and exits.
#include <algorithm>
#include <cstring>
#include <new>

#include <cudaTypedefs.h>

#include "gf2_internal.cuh"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int NP = 64;
constexpr uint32_t TILE128 = 128 * NP * 2;  // 16 KB: 128 rows x 64 bf16
constexpr uint32_t TILE64 = 64 * NP * 2;    //  8 KB: 64 rows x 64 bf16
constexpr uint32_t kIdescKK = tc::idesc_bf16(128, 64, 0, 0);
constexpr uint32_t kIdescMK = tc::idesc_bf16(128, 64, 1, 0);
// 64-wide K steps per FP32 group in stage 4 (four doubled the BF16x6 error)
template <int T>
constexpr int contract_group() { return 2; }
// stage-4 ring depths (32 KB T3 tiles, T x 8 KB W stages) within 227 KB of shared memory
template <int T>
constexpr int contract_stages_f() { return T == 2 ? 5 : 4; }
template <int T>
constexpr int contract_stages_w() { return 4; }

constexpr uint32_t kF32Tile = 128 * NP * 4;  // one FP32 tile of 128 x 64 values (32 KB)

// ---------------------------------------------------------------------------
// splitting of the FP64 inputs
// ---------------------------------------------------------------------------
// largest |v| as the bit pattern of a non-negative double (atomicMax on the bits)
__global__ void absmax_kernel(size_t n, const double *__restrict__ x, unsigned long long *out) {
  double m = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// largest |v[i][m][q][k] - v[q][k][i][m]| (the pair symmetry (im|qk) = (qk|im)),
// as the bit pattern of a non-negative double
__global__ void pair_asym_kernel(int N, const double *__restrict__ v, unsigned long long *out) {
  const size_t n2 = (size_t)N * N, n4 = n2 * n2;
  double m = 0.0;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n4; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t a = idx / n2, b = idx % n2;  // a = (i, m), b = (q, k)
    m = fmax(m, fabs(v[idx] - v[b * n2 + a]));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// v <- the pair-symmetric part (v[i][m][q][k] + v[q][k][i][m]) / 2, in place
// (each unordered pair of (i,m), (q,k) handled by one thread)
__global__ void pair_symmetrize_kernel(int N, double *__restrict__ v) {
  const size_t n2 = (size_t)N * N, n4 = n2 * n2;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n4; idx += (size_t)gridDim.x * blockDim.x) {
    const size_t a = idx / n2, b = idx % n2;
    if (a < b) {
      const double x = 0.5 * (v[idx] + v[b * n2 + a]);
      v[idx] = x;
      v[b * n2 + a] = x;
    }
  }
}

// ---------------------------------------------------------------------------
// stage 3: T3[c][i][l][n][p] = sum_q Gbar_c[p][q] T2[c][i][q][l][n]
//
// Unit (c, i, 128 rows m of (l,n)).  The FP32 tile F[q][m] = T2[c][i][q][(l,n)]
// arrives by TMA; each converter thread owns one row m (one TMEM lane), reads
// its 64 values of q, splits them into T bf16 terms and writes them to TMEM as
// the A operand (lane m, q packed two per column).  The MMA warp multiplies
// A (TMEM) by the Gbar planes (shared memory); four epilogue warps store the
// FP32 rows T3[c][i][(l,n)][p].  Keeping A in TMEM leaves shared memory to the
// FP32 tiles and B, whose traffic otherwise bounds this kernel.
// 320 threads: warp 0 TMA, warp 1 MMA, warps 2-5 epilogue, warps 6-9 convert.
// TMEM: accumulators at columns 0 and 64, A stages from column 128.
// ---------------------------------------------------------------------------
template <int T, int F>
__global__ void __launch_bounds__(320, 1)
    xform_kernel(const __grid_constant__ CUtensorMap map_t2, const __grid_constant__ CUtensorMap map_g,
                 const __grid_constant__ CUtensorMap map_t3s, int C, int S, int sl0, int n_units, int *__restrict__ ex,
                 int *err) {
  constexpr int SF = 4, SA = 4;
  constexpr int OS = 2;  // output staging tiles: a TMA store reads one while the next is written
  // Gbar sets: two at T = 2; one at T = 3, where the room goes to the second
  // staging tile (a CTA's contiguous block of units meets one or two time points)
  constexpr int GB = (T == 2) ? 2 : 1;
  constexpr uint32_t B_SET = T * TILE64, A_COLS = T * 32;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = align1024(smem_raw);
  uint8_t *sF = smem;
  uint8_t *sB = sF + SF * kF32Tile;
  uint8_t *sO = sB + GB * B_SET;  // OS output tiles [2 halves of 32 p][128 rows], 128-byte swizzle
  uint64_t *bar = reinterpret_cast<uint64_t *>(sO + OS * kF32Tile);
  uint64_t *f_full = bar, *f_empty = bar + SF, *a_full = bar + 2 * SF, *a_empty = a_full + SA;
  uint64_t *b_full = a_empty + SA, *b_empty = b_full + 2, *d_full = b_full + 4, *d_empty = b_full + 6;
  uint64_t *o_full = b_full + 8, *o_empty = b_full + 10;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(b_full + 12);
  __shared__ int s_abort;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int s = 0; s < SF; ++s) {
      tc::mbar_init(&f_full[s], 1);
      tc::mbar_init(&f_empty[s], 4);
    }
    for (int s = 0; s < SA; ++s) {
      tc::mbar_init(&a_full[s], 4);
      tc::mbar_init(&a_empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      tc::mbar_init(&b_full[s], 1);
      tc::mbar_init(&b_empty[s], 1);
      tc::mbar_init(&d_full[s], 1);
      tc::mbar_init(&d_empty[s], 4);
      tc::mbar_init(&o_full[s], 4);
      tc::mbar_init(&o_empty[s], 1);
    }
    tc::fence_barrier_init();
    s_abort = 0;
    tc::prefetch_tmap(&map_t2);
    tc::prefetch_tmap(&map_g);
    tc::prefetch_tmap(&map_t3s);
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, 512);
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  volatile int *abort = &s_abort;
  // a contiguous block of units per CTA (balanced to within one unit)
  const int u_begin = (int)((long long)blockIdx.x * n_units / gridDim.x);
  const int u_end = (int)((long long)(blockIdx.x + 1) * n_units / gridDim.x);

  if (warp == 0 && lane == 0) {
    const uint64_t stream_pol = tc::policy_evict_first();
    int it = 0, cur_c = -1, gcount = 0;
    for (int u = u_begin; u < u_end; ++u, ++it) {
      const int c = u / (NP * 32), i = (u / 32) % NP, mt = u % 32;
      if (c != cur_c) {
        const int gs = gcount % GB;
        if (gcount >= GB && !tc::mbar_wait(&b_empty[gs], ((gcount / GB) - 1) & 1, abort)) { raise_abort(abort, err); break; }
        tc::mbar_arrive_expect_tx(&b_full[gs], B_SET);
        for (int t = 0; t < T; ++t)
          tc::tma_load_3d(sB + gs * B_SET + t * TILE64, &map_g, &b_full[gs], 0, 0, (TMAX + t) * S + sl0 + c);
        cur_c = c;
        ++gcount;
      }
      const int s = it % SF;
      if (it >= SF && !tc::mbar_wait(&f_empty[s], ((it / SF) - 1) & 1, abort)) { raise_abort(abort, err); break; }
      tc::mbar_arrive_expect_tx(&f_full[s], kF32Tile);
      tc::tma_load_3d_hint(sF + s * kF32Tile, &map_t2, &f_full[s], mt * 128, 0, c * NP + i, stream_pol);
    }
  } else if (warp == 1 && lane == 0) {
    int it = 0, cur_c = -1, gcount = 0, gs = 0;
    for (int u = u_begin; u < u_end; ++u, ++it) {
      const int c = u / (NP * 32);
      if (c != cur_c) {
        if (cur_c >= 0) tc::mma_commit(&b_empty[gs]);
        gs = gcount % GB;
        if (!tc::mbar_wait(&b_full[gs], (gcount / GB) & 1, abort)) { raise_abort(abort, err); break; }
        cur_c = c;
        ++gcount;
      }
      const int sa = it % SA, d = it & 1;
      if (!tc::mbar_wait(&a_full[sa], (it / SA) & 1, abort)) { raise_abort(abort, err); break; }
      if (it >= 2 && !tc::mbar_wait(&d_empty[d], ((it >> 1) - 1) & 1, abort)) { raise_abort(abort, err); break; }
      tc::tc_fence_after();
      const uint32_t a0 = tmem + 128 + sa * A_COLS, b0 = tc::smem_u32(sB + gs * B_SET);
      for (int pr = 0; pr < Products<T>::n; ++pr) {
        const int ta = Products<T>::a(pr), tb = Products<T>::b(pr);
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t bd = tc::smem_desc(b0 + tb * TILE64 + kk * 32, 16, 1024);
          tc::mma_bf16_ts(tmem + d * 64, a0 + ta * 32 + kk * 8, bd, idesc_fmt(F, 128, 64, 0, 0), (pr | kk) ? 1u : 0u);
        }
      }
      tc::mma_commit(&a_empty[sa]);
      tc::mma_commit(&d_full[d]);
    }
  } else if (warp >= 2 && warp < 6) {
    // epilogue: D row -> the swizzled output tile (16-byte chunk j of row r of
    // half h at chunk j ^ (r % 8)); warp 2 lane 0 stores the tile with TMA
    const int wq = warp & 3, row = wq * 32 + lane;
    int it = 0;
    float run_mx = 0.f;  // FP16: largest |T3| of time point run_c seen by this thread
    int run_c = -1;
    for (int u = u_begin; u < u_end; ++u, ++it) {
      const int c = u / (NP * 32), i = (u / 32) % NP, mt = u % 32;
      const int d = it & 1;
      if (!tc::mbar_wait(&d_full[d], (it >> 1) & 1, abort)) { raise_abort(abort, err); break; }
      tc::tc_fence_after();
      float v[64];
      const uint32_t taddr = tmem + ((uint32_t)(wq * 32) << 16) + d * 64;
      tc::tmem_ld_32x32b_x32(taddr, v);
      tc::tmem_ld_32x32b_x32(taddr + 32, v + 32);
      tc::tmem_ld_wait();
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&d_empty[d]);
      if constexpr (F != 0) {  // remove the T2 operand scale; record max |T3| of the time point
        const float un = exp2_scale(-fp16_exponent_bits(ex[kMaxT2 * S + sl0 + c]));
        if (c != run_c) {  // one atomic per warp and time point, not per unit
          if (run_c >= 0) warp_absmax_to(&ex[kMaxT3 * S + sl0 + run_c], run_mx);
          run_c = c;
          run_mx = 0.f;
        }
#pragma unroll
        for (int k = 0; k < 64; ++k) {
          v[k] *= un;
          run_mx = fmaxf(run_mx, fabsf(v[k]));
        }
      }
      const int ob = it % OS;
      if (it >= OS && !tc::mbar_wait(&o_empty[ob], ((it / OS) - 1) & 1, abort)) { raise_abort(abort, err); break; }
      uint8_t *otile = sO + ob * kF32Tile, *orow = otile + row * 128;
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < 8; ++j)
          *reinterpret_cast<float4 *>(orow + h * (kF32Tile / 2) + ((j ^ (row & 7)) << 4)) =
              make_float4(v[32 * h + 4 * j], v[32 * h + 4 * j + 1], v[32 * h + 4 * j + 2], v[32 * h + 4 * j + 3]);
      tc::fence_proxy_async_smem();  // these writes are read by the TMA store
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&o_full[ob]);
      if (warp == 2) {  // the whole warp waits (uniform exit on a timeout); lane 0 issues
        if (!tc::mbar_wait(&o_full[ob], (it / OS) & 1, abort)) { raise_abort(abort, err); break; }
        if (lane == 0) {
          for (int h = 0; h < 2; ++h)
            tc::tma_store_3d(&map_t3s, otile + h * (kF32Tile / 2), 32 * h, mt * 128, c * NP + i);
          tc::tma_store_commit();
          if constexpr (OS == 1) {
            tc::tma_store_wait_read();
            tc::mbar_arrive(&o_empty[0]);
          } else {  // the store of unit it - 1 has read its tile once at most this one is pending
            tc::tma_store_wait_read_but_one();
            if (it >= 1) tc::mbar_arrive(&o_empty[(it - 1) % OS]);
          }
        }
        __syncwarp();
      }
    }
    if (F != 0 && run_c >= 0) warp_absmax_to(&ex[kMaxT3 * S + sl0 + run_c], run_mx);
    if (warp == 2 && lane == 0) tc::tma_store_wait_all();
  } else if (warp >= 6) {
    // converter: row m = 32 (warp % 4) + lane of the tile, the TMEM lane this warp may access
    const int wq = warp & 3, m = wq * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(wq * 32) << 16) + 128;
    int it = 0;
    for (int u = u_begin; u < u_end; ++u, ++it) {
      const int s = it % SF, sa = it % SA;
      const float scale = F == 0 ? 1.0f : exp2_scale(fp16_exponent_bits(ex[kMaxT2 * S + sl0 + u / (NP * 32)]));
      if (!tc::mbar_wait(&f_full[s], (it / SF) & 1, abort)) { raise_abort(abort, err); break; }
      float x[64];
      const float *src = reinterpret_cast<const float *>(sF + s * kF32Tile) + m;
#pragma unroll
      for (int q = 0; q < 64; ++q) x[q] = src[q * 128];
      // the next TMA write to this stage (async proxy) must follow these reads
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&f_empty[s]);
      if (it >= SA && !tc::mbar_wait(&a_empty[sa], ((it / SA) - 1) & 1, abort)) { raise_abort(abort, err); break; }
      tc::tc_fence_after();
      split_row_to_tmem<T, F>(x, lane_base + sa * A_COLS, scale);
      tc::tmem_st_wait();
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&a_full[sa]);
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------------------
// stage 4: Sigma[c][i][j] -= sum_K T3[c][i][K] Ws[j][K],  split over K slices
//
// Each slice of NP*NP values of K is accumulated in groups of KSUB 64-wide
// steps: the tensor cores sum one group in FP32 (TMEM), and the epilogue adds
// every group into a compensated FP32 pair (TwoSum), so that the long sum never
// runs through a single FP32 accumulator.  The slice total enters the FP64
// output through atomics.  The split products are issued as one MMA per A
// term: A_a times the W planes 0 .. T-1-a stacked along N (N = 64 (T - a)), so
// column block b of the accumulator collects A_a W_b for all a + b < T and the
// epilogue adds the T blocks -- half the MMA instructions of one product per
// instruction, with wider N.
// ---------------------------------------------------------------------------
template <int T, int KSUB, int F>
__global__ void __launch_bounds__(448, 1)
    contract_kernel(const __grid_constant__ CUtensorMap map_t3, const __grid_constant__ CUtensorMap map_w,
                    double *__restrict__ out, int N, int B, int count, int C, int S, int sl0, int n_units,
                    const int *__restrict__ ex, int e_fixed, int *err) {
  // T3 tile and W stages: the producer is held back by whichever ring frees last,
  // and a W stage is released only when the MMA of its K step is done, so the
  // W ring must be as deep as the T3 ring for the HBM loads to run ahead
  constexpr int SF = contract_stages_f<T>(), SW = contract_stages_w<T>(), SA = (T == 3) ? 3 : 4;
  constexpr uint32_t D_COLS = T * 64;  // column block b accumulates sum_a A_a W_b
  // two accumulators where TMEM holds them next to the A stages (T = 2), else one
  constexpr int DB = (2 * D_COLS + SA * T * 32 <= 512) ? 2 : 1;
  constexpr int KSTEPS = NP;  // 64-wide steps per slice of NP*NP
  constexpr int NGROUP = KSTEPS / KSUB;
  constexpr uint32_t W_STAGE = T * TILE64, A_COLS = T * 32;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = align1024(smem_raw);
  uint8_t *sF = smem;                  // FP32 tiles [2 halves of 32 k][128 rows], 128-byte swizzle
  uint8_t *sW = sF + SF * kF32Tile;    // W planes
  uint64_t *bar = reinterpret_cast<uint64_t *>(sW + SW * W_STAGE);
  uint64_t *f_full = bar, *f_empty = bar + SF, *w_full = bar + 2 * SF, *w_empty = w_full + SW;
  uint64_t *a_full = w_empty + SW, *a_empty = a_full + SA, *d_full = a_empty + SA, *d_empty = d_full + DB;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(d_empty + DB);
  __shared__ int s_abort;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int s = 0; s < SF; ++s) {
      tc::mbar_init(&f_full[s], 1);
      tc::mbar_init(&f_empty[s], 4);
    }
    for (int s = 0; s < SW; ++s) {
      tc::mbar_init(&w_full[s], 1);
      tc::mbar_init(&w_empty[s], 1);
    }
    for (int s = 0; s < SA; ++s) {
      tc::mbar_init(&a_full[s], 4);
      tc::mbar_init(&a_empty[s], 1);
    }
    for (int s = 0; s < DB; ++s) {
      tc::mbar_init(&d_full[s], 1);
      tc::mbar_init(&d_empty[s], 8);
    }
    tc::fence_barrier_init();
    s_abort = 0;
    tc::prefetch_tmap(&map_t3);
    tc::prefetch_tmap(&map_w);
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, 512);
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;  // accumulators at columns 0 .. DB * D_COLS - 1, A stages after them
  volatile int *abort = &s_abort;
  const int npairs = n_units / NP;

  if (warp == 0 && lane == 0) {
    const uint64_t stream_pol = tc::policy_evict_first(), keep_pol = tc::policy_evict_last();
    int g = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
      const int l = u / npairs, cp = u % npairs;
      for (int ks = 0; ks < KSTEPS; ++ks, ++g) {
        const int k0 = l * NP * NP + ks * NP;
        const int s = g % SF, sw = g % SW;
        if (g >= SF && !tc::mbar_wait(&f_empty[s], ((g / SF) - 1) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
        tc::mbar_arrive_expect_tx(&f_full[s], kF32Tile);
        for (int h = 0; h < 2; ++h)
          tc::tma_load_3d_hint(sF + s * kF32Tile + h * (kF32Tile / 2), &map_t3, &f_full[s], k0 + 32 * h, cp * 128, 0,
                               stream_pol);
        if (g >= SW && !tc::mbar_wait(&w_empty[sw], ((g / SW) - 1) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
        tc::mbar_arrive_expect_tx(&w_full[sw], W_STAGE);
        for (int t = 0; t < T; ++t)
          tc::tma_load_3d_hint(sW + sw * W_STAGE + t * TILE64, &map_w, &w_full[sw], k0, 0, t, keep_pol);
      }
    }
  } else if (warp == 1 && lane == 0) {
    int g = 0, grp = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
      for (int gi = 0; gi < NGROUP && ok; ++gi, ++grp) {
        const int db = grp % DB;
        if (grp >= DB && !tc::mbar_wait(&d_empty[db], ((grp / DB) - 1) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
        tc::tc_fence_after();
        const uint32_t dacc = tmem + db * D_COLS;
        for (int kq = 0; kq < KSUB; ++kq, ++g) {
          const int sa = g % SA, sw = g % SW;
          if (!tc::mbar_wait(&a_full[sa], (g / SA) & 1, abort) || !tc::mbar_wait(&w_full[sw], (g / SW) & 1, abort)) {
            raise_abort(abort, err);
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const uint32_t a0 = tmem + DB * D_COLS + sa * A_COLS, b0 = tc::smem_u32(sW + sw * W_STAGE);
          // A_a times the W planes 0 .. T-1-a stacked along N: columns of plane b
          // receive A_a W_b, so each block sums exactly the products a + b < T.
          // The a = 0 product spans every column and opens the group.
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t bd = tc::smem_desc(b0 + kk * 32, 16, 1024);
            if (kq == 0 && kk == 0) tc::mma_bf16_ts(dacc, a0, bd, idesc_fmt(F, 128, T * 64, 0, 0), 0u);
            for (int ta = T - 1; ta >= ((kq == 0 && kk == 0) ? 1 : 0); --ta)
              tc::mma_bf16_ts(dacc, a0 + ta * 32 + kk * 8, bd, idesc_fmt(F, 128, (T - ta) * 64, 0, 0), 1u);
          }
          tc::mma_commit(&a_empty[sa]);
          tc::mma_commit(&w_empty[sw]);
        }
        if (ok) tc::mma_commit(&d_full[db]);
      }
    }
  } else if (warp >= 2 && warp < 10) {
    // epilogue: warp w reads TMEM lane quarter w % 4, columns 32 * ((w - 2) / 4) .. +31
    const int wq = warp & 3, row = wq * 32 + lane, col = 32 * ((warp - 2) >> 2);
    int grp = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
      const int cp = u % npairs;
      float hi[32], lo[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) hi[j] = lo[j] = 0.f;
      for (int gi = 0; gi < NGROUP; ++gi, ++grp) {
        const int db = grp % DB;
        if (!tc::mbar_wait(&d_full[db], (grp / DB) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
        tc::tc_fence_after();
        // sum the column blocks (smallest terms first), 16 columns at a time; the
        // T loads of a half are in flight together
        const uint32_t dl = tmem + ((uint32_t)(wq * 32) << 16) + db * D_COLS + col;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          // blocks T-1 and T-2 in flight together, then (T = 3) block 0
          float v[16], w[16];
          tc::tmem_ld_32x32b_x16(dl + 64 * (T - 1) + 16 * hh, v);
          tc::tmem_ld_32x32b_x16(dl + 64 * (T - 2) + 16 * hh, w);
          tc::tmem_ld_wait();
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) v[jj] += w[jj];
          if constexpr (T == 3) {
            tc::tmem_ld_32x32b_x16(dl + 16 * hh, w);
            tc::tmem_ld_wait();
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) v[jj] += w[jj];
          }
          if (hh == 1) {  // every column of this accumulator is in registers
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&d_empty[db]);
          }
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) two_sum_acc(hi[16 * hh + jj], lo[16 * hh + jj], v[jj]);
        }
      }
      if (!ok) break;
      // row (slot c, i) of the tile is row i - bN of time point c B + b, b = i / N;
      // only the columns of the same block are nonzero
      const int c = 2 * cp + row / NP, ib = row % NP, b = ib / N, t = c * B + b;
      if (b < B && t < count) {
        // FP16: remove the scales of v, W, G(tau) (twice), Gbar(tau) and the T3 operand
        const double unscale =
            F == 0 ? 1.0
                   : ldexp(1.0, -(e_fixed + 2 * ex[kExpG * S + sl0 + c] + ex[kExpGbar * S + sl0 + c] +
                                  fp16_exponent_bits(ex[kMaxT3 * S + sl0 + c])));
        double *o = out + ((long long)t * N + (ib - b * N)) * N + (col - b * N);
        const int j0 = b * N - col, j1 = j0 + N;  // this thread's columns j0 <= j < j1 lie in block b
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (j >= j0 && j < j1) atomicAdd(o + j, -((double)hi[j] + (double)lo[j]) * unscale);
      }
    }
  } else if (warp >= 10) {
    // converter: row r = 32 (warp % 4) + lane (the TMEM lane this warp may access).
    // Half h of the FP32 tile holds k = 32 h .. +31 of all rows, 128 bytes a row,
    // with 16-byte chunk c of row r stored at chunk c ^ (r % 8).
    const int wq = warp & 3, r = wq * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(wq * 32) << 16) + DB * D_COLS;
    int g = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x) {
      const int c = 2 * (u % npairs) + r / NP;
      const float scale = F == 0 ? 1.0f : exp2_scale(fp16_exponent_bits(ex[kMaxT3 * S + sl0 + c]));
      for (int ks = 0; ks < KSTEPS; ++ks, ++g) {
        const int s = g % SF, sa = g % SA;
        if (!tc::mbar_wait(&f_full[s], (g / SF) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
        float x[64];
        const uint8_t *row_base = sF + s * kF32Tile + r * 128;
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int cch = 0; cch < 8; ++cch) {
            const float4 q = *reinterpret_cast<const float4 *>(row_base + h * (kF32Tile / 2) + ((cch ^ (r & 7)) << 4));
            x[32 * h + 4 * cch] = q.x;
            x[32 * h + 4 * cch + 1] = q.y;
            x[32 * h + 4 * cch + 2] = q.z;
            x[32 * h + 4 * cch + 3] = q.w;
          }
        // the next TMA write to this stage (async proxy) must follow these reads
        tc::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&f_empty[s]);
        if (g >= SA && !tc::mbar_wait(&a_empty[sa], ((g / SA) - 1) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
        tc::tc_fence_after();
        split_row_to_tmem<T, F>(x, lane_base + sa * A_COLS, scale);
        tc::tmem_st_wait();
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&a_full[sa]);
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------------------
// Units of the sandwich.  With the pair symmetry of the integrals,
// v[i][m][q][k] = v[q][k][i][m] ((im|qk) = (qk|im)), the stage-2 intermediate is
// symmetric under the simultaneous exchange i <-> q, l <-> n:
//   T2[i][q][l][n] = sum_{m,k} v[i][m][q][k] G[k][l] G[m][n]
//                  = sum_{m,k} v[q][k][i][m] G[k][l] G[m][n] = T2[q][i][n][l],
// so the 64 x 64 (l, n) tile of (i, q) is the transpose of the tile of (q, i).
// A symmetric run computes only the units (i, q pair) with q pair >= i / 2
// (1056 of 2048 per time-point pair): each writes its two tiles in place and,
// when q pair > i / 2, also their transposes as the tiles of (q, i); every tile
// of T2 is then written exactly once.
// ---------------------------------------------------------------------------
constexpr int kSymUnitsPerPair = NP * (NP / 2) - (NP / 2) * (NP / 2 - 1);  // 1056 for NP = 64

__device__ __forceinline__ void sandwich_unit(int u, int sym, int &cp, int &i, int &qp) {
  if (!sym) {
    cp = u / (NP * 32);
    i = (u / 32) % NP;
    qp = u % 32;
    return;
  }
  cp = u / kSymUnitsPerPair;
  int w = u % kSymUnitsPerPair, a = 0;
  // the i pair (2a, 2a+1) owns 2 (32 - a) units, i.e. 64 a - a (a - 1) before it
  while (a < NP / 2 - 1 && w >= 2 * (NP / 2 - a)) {
    w -= 2 * (NP / 2 - a);
    ++a;
  }
  const int per_i = NP / 2 - a;
  i = 2 * a + w / per_i;
  qp = a + w % per_i;
}

// ---------------------------------------------------------------------------
// stages 1+2 fused: T2[c][i][q][l][n] = sum_{m,k} G[m][n] v[i][m][q][k] G[k][l]
//
// Unit = (tau pair, i, q pair).  MMA1 covers both time points at once: its B
// operand stacks G(tau_a)^T and G(tau_b)^T (N = 128), so D1 holds
// [(q,m), (s,l)] for s = 0, 1.  Each half becomes one job for epilogue 1
// (D1 -> A2 smem, MN-major; warps 2-5 and 10-13, one column half each) and
// MMA2 (N = 64, one time point); epilogue 2 (warps 6-9) stores each D2 tile with
// TMA through a swizzled shared staging tile, two of them alternating at T = 2.
// TMEM: D1 buffers at columns 0 and 128 (128 wide), D2 buffers at 256, 320.
// ---------------------------------------------------------------------------
template <int T, int F>
__global__ void __launch_bounds__(448, 1)
    sandwich_kernel(const __grid_constant__ CUtensorMap map_v, const __grid_constant__ CUtensorMap map_g,
                    const __grid_constant__ CUtensorMap map_t2s, int C, int S, int sl0, int n_units,
                    int *__restrict__ ex, int *err, int sym, float *__restrict__ t2) {
  constexpr int GS = 1;                  // buffered G sets (a tau pair each; a CTA meets one or two)
  constexpr int A1S = (T == 2) ? 2 : 1;  // buffered v tiles (MMA1 consumes them first)
  constexpr int A2S = 2;                 // buffered MMA2 operands: epilogue 1 overlaps MMA2
  constexpr int OS = (T == 2) ? 2 : 1;   // output staging tiles: a TMA store reads one while the next is written
  constexpr uint32_t A1_STAGE = T * TILE128, G_SET = 2 * T * TILE64, A2_BUF = T * TILE128;
  constexpr uint32_t kIdescKK128 = idesc_fmt(F, 128, 128, 0, 0), kIdescMK64 = idesc_fmt(F, 128, 64, 1, 0);
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = align1024(smem_raw);
  uint8_t *sA1 = smem;
  uint8_t *sG = sA1 + A1S * A1_STAGE;  // per set: [t][s][64][64]
  uint8_t *sA2 = sG + GS * G_SET;
  uint8_t *sO = sA2 + A2S * A2_BUF;  // OS output tiles [2 halves of 32 n][128 rows], 128-byte swizzle
  uint64_t *bar = reinterpret_cast<uint64_t *>(sO + OS * kF32Tile);
  uint64_t *a1_full = bar, *a1_empty = bar + 2, *g_full = bar + 4, *g_empty = bar + 6;
  uint64_t *d1_full = bar + 8, *d1_empty = bar + 10, *a2_full = bar + 12, *a2_empty = bar + 14;
  uint64_t *d2_full = bar + 16, *d2_empty = bar + 18, *o_full = bar + 20, *o_empty = bar + 22;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 24);
  __shared__ int s_abort;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      tc::mbar_init(&a1_full[s], 1);
      tc::mbar_init(&a1_empty[s], 1);
      tc::mbar_init(&g_full[s], 1);
      tc::mbar_init(&g_empty[s], 1);
      tc::mbar_init(&d1_full[s], 1);
      tc::mbar_init(&d1_empty[s], 8);
      tc::mbar_init(&a2_full[s], 8);
      tc::mbar_init(&a2_empty[s], 1);
      tc::mbar_init(&d2_full[s], 1);
      tc::mbar_init(&d2_empty[s], 4);
      tc::mbar_init(&o_full[s], 4);
      tc::mbar_init(&o_empty[s], 1);
    }
    tc::fence_barrier_init();
    s_abort = 0;
    tc::prefetch_tmap(&map_v);
    tc::prefetch_tmap(&map_g);
    tc::prefetch_tmap(&map_t2s);
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, 512);
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  volatile int *abort = &s_abort;
  // a contiguous block of units per CTA (balanced to within one unit)
  const int u_begin = (int)((long long)blockIdx.x * n_units / gridDim.x);
  const int u_end = (int)((long long)(blockIdx.x + 1) * n_units / gridDim.x);

  if (warp == 0 && lane == 0) {
    const uint64_t keep_pol = tc::policy_evict_last();
    int it = 0, cur_cp = -1, gcount = 0;
    for (int u = u_begin; u < u_end; ++u, ++it) {
      int cp, i, qp;
      sandwich_unit(u, sym, cp, i, qp);
      if (cp != cur_cp) {
        const int gs = gcount % GS;
        if (gcount >= GS && !tc::mbar_wait(&g_empty[gs], ((gcount / GS) - 1) & 1, abort)) { raise_abort(abort, err); break; }
        tc::mbar_arrive_expect_tx(&g_full[gs], G_SET);
        for (int t = 0; t < T; ++t)
          for (int s = 0; s < 2; ++s)
            tc::tma_load_3d(sG + gs * G_SET + (t * 2 + s) * TILE64, &map_g, &g_full[gs], 0, 0,
                            t * S + sl0 + 2 * cp + s);
        cur_cp = cp;
        ++gcount;
      }
      const int st = it % A1S;
      if (it >= A1S && !tc::mbar_wait(&a1_empty[st], ((it / A1S) - 1) & 1, abort)) { raise_abort(abort, err); break; }
      tc::mbar_arrive_expect_tx(&a1_full[st], A1_STAGE);
      for (int t = 0; t < T; ++t)
        tc::tma_load_5d_hint(sA1 + st * A1_STAGE + t * TILE128, &map_v, &a1_full[st], 0, 0, 2 * qp, i, t, keep_pol);
    }
  } else if (warp == 1 && lane == 0) {
    int it = 0, cur_cp = -1, gcount = 0, gs = 0;
    int pend_u = -1, pend_gs = 0;  // unit whose two MMA2 jobs are not yet issued
    bool ok = true;
    auto issue_mma2 = [&](int jj, int jgs) -> bool {
      const int ab = jj % A2S, db = jj & 1, js = jj & 1;
      if (!tc::mbar_wait(&a2_full[ab], (jj / A2S) & 1, abort)) return false;
      if (jj >= 2 && !tc::mbar_wait(&d2_empty[db], ((jj >> 1) - 1) & 1, abort)) return false;
      tc::tc_fence_after();
      const uint64_t a0 = tc::smem_desc(tc::smem_u32(sA2 + ab * A2_BUF), TILE64, 1024);
      const uint64_t b0 = tc::smem_desc(tc::smem_u32(sG + jgs * G_SET + js * TILE64), 16, 1024);
#pragma unroll
      for (int pr = 0; pr < Products<T>::n; ++pr) {
        const int ta = Products<T>::a(pr), tb = Products<T>::b(pr);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          // descriptors advance in 16-byte units: A by 2048 B (16 K rows), B by 32 B
          const uint64_t ad = a0 + (uint64_t)((ta * TILE128 + kk * 2048) >> 4);
          const uint64_t bd = b0 + (uint64_t)((tb * 2 * TILE64 + kk * 32) >> 4);
          tc::mma_bf16(tmem + 256 + db * 64, ad, bd, kIdescMK64, (pr | kk) ? 1u : 0u);
        }
      }
      tc::mma_commit(&a2_empty[ab]);
      tc::mma_commit(&d2_full[db]);
      return true;
    };
    const int upp = sym ? kSymUnitsPerPair : NP * 32;  // units per time-point pair
    for (int u = u_begin; u < u_end && ok; ++u, ++it) {
      const int cp = u / upp;
      if (cp != cur_cp) {
        if (pend_u >= 0) {  // finish the previous pair before its G set can be recycled
          if (!issue_mma2(2 * pend_u, pend_gs) || !issue_mma2(2 * pend_u + 1, pend_gs)) {
            raise_abort(abort, err);
            ok = false;
            break;
          }
          pend_u = -1;
          tc::mma_commit(&g_empty[gs]);
        }
        gs = gcount % GS;
        if (!tc::mbar_wait(&g_full[gs], (gcount / GS) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
        cur_cp = cp;
        ++gcount;
      }
      const int st = it % A1S, b = it & 1;
      if (!tc::mbar_wait(&a1_full[st], (it / A1S) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
      if (it >= 2 && !tc::mbar_wait(&d1_empty[b], ((it >> 1) - 1) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
      tc::tc_fence_after();
      const uint64_t a0 = tc::smem_desc(tc::smem_u32(sA1 + st * A1_STAGE), 16, 1024);
      const uint64_t b0 = tc::smem_desc(tc::smem_u32(sG + gs * G_SET), 16, 1024);
#pragma unroll
      for (int pr = 0; pr < Products<T>::n; ++pr) {
        const int ta = Products<T>::a(pr), tb = Products<T>::b(pr);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t ad = a0 + (uint64_t)((ta * TILE128 + kk * 32) >> 4);
          const uint64_t bd = b0 + (uint64_t)((tb * 2 * TILE64 + kk * 32) >> 4);
          tc::mma_bf16(tmem + b * 128, ad, bd, kIdescKK128, (pr | kk) ? 1u : 0u);
        }
      }
      tc::mma_commit(&d1_full[b]);
      tc::mma_commit(&a1_empty[st]);
      if (pend_u >= 0) {
        if (!issue_mma2(2 * pend_u, pend_gs) || !issue_mma2(2 * pend_u + 1, pend_gs)) {
          raise_abort(abort, err);
          ok = false;
          break;
        }
      }
      pend_u = it;
      pend_gs = gs;
    }
    if (ok && pend_u >= 0 && (!issue_mma2(2 * pend_u, pend_gs) || !issue_mma2(2 * pend_u + 1, pend_gs)))
      raise_abort(abort, err);
  } else if ((warp >= 2 && warp < 6) || warp >= 10) {
    // epilogue 1: D1[(q,m), (s,l)] -> A2_j[(q,l), m] (MN-major, 128-byte swizzle), j = 2 it + s;
    // a warp holds 32 consecutive m of one q, so its 16-byte stores hit distinct banks.
    // Warps 2-5 convert l = 0..31, warps 10-13 l = 32..63 of the same rows.
    const int wq = warp & 3, row = wq * 32 + lane, hf = warp >= 10 ? 1 : 0;
    const int m = row & 63, ql = row >> 6;
    const int upp = sym ? kSymUnitsPerPair : NP * 32;
    int it = 0;
    bool ok = true;
    for (int u = u_begin; u < u_end && ok; ++u, ++it) {
      const int b = it & 1, cp = u / upp;
      if (!tc::mbar_wait(&d1_full[b], (it >> 1) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
      tc::tc_fence_after();
      for (int s = 0; s < 2; ++s) {
        const int j = 2 * it + s;
        const float scale = F == 0 ? 1.0f : exp2_scale(ex[kExpT1 * S + sl0 + 2 * cp + s]);
        float v[32];
        tc::tmem_ld_32x32b_x32(tmem + ((uint32_t)(wq * 32) << 16) + b * 128 + s * 64 + 32 * hf, v);
        tc::tmem_ld_wait();
        if (s == 1) {
          tc::tc_fence_before();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&d1_empty[b]);
        }
        const int ab = j % A2S;
        if (j >= A2S && !tc::mbar_wait(&a2_empty[ab], ((j / A2S) - 1) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
        uint8_t *dst = sA2 + ab * A2_BUF + ql * TILE64 + m * 128;
#pragma unroll
        for (int cch = 0; cch < 4; ++cch)
          split8_store<T, F>(v + 8 * cch, dst + (((4 * hf + cch) ^ (m & 7)) << 4), TILE128, scale);
        tc::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&a2_full[ab]);
      }
    }
  } else if (warp >= 6 && warp < 10) {
    // epilogue 2: D2[(q,l), n] -> T2[c][i][q][l][n]
    const int wq = warp & 3, row = wq * 32 + lane;
    int j = 0;
    bool ok = true;
    float run_mx[2] = {0.f, 0.f};  // FP16: largest |T2| of time points 2 run_cp + s seen by this thread
    int run_cp = -1;
    for (int u = u_begin; u < u_end && ok; ++u) {
      int cp, i, qp;
      sandwich_unit(u, sym, cp, i, qp);
      const bool mirror = sym && qp > i / 2;  // also write the transposed tiles (q, i)
      if (F != 0 && cp != run_cp) {  // one atomic per warp and time point, not per job
        if (run_cp >= 0)
          for (int s = 0; s < 2; ++s) warp_absmax_to(&ex[kMaxT2 * S + sl0 + 2 * run_cp + s], run_mx[s]);
        run_cp = cp;
        run_mx[0] = run_mx[1] = 0.f;
      }
      for (int s = 0; s < 2; ++s, ++j) {
        const int b = j & 1;
        if (!tc::mbar_wait(&d2_full[b], (j >> 1) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
        tc::tc_fence_after();
        float v[64];
        const uint32_t taddr = tmem + ((uint32_t)(wq * 32) << 16) + 256 + b * 64;
        tc::tmem_ld_32x32b_x32(taddr, v);
        tc::tmem_ld_32x32b_x32(taddr + 32, v + 32);
        tc::tmem_ld_wait();
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&d2_empty[b]);
        if constexpr (F != 0) {  // remove the T1 operand scale; record max |T2| of the time point
          const float un = exp2_scale(-ex[kExpT1 * S + sl0 + 2 * cp + s]);
          float mx = run_mx[s];
#pragma unroll
          for (int k = 0; k < 64; ++k) {
            v[k] *= un;
            mx = fmaxf(mx, fabsf(v[k]));
          }
          run_mx[s] = mx;
        }
        // row (ql, l) of the tile is row 128 qp + row of T2[c][i]; 16-byte chunk
        // k of row r in half h sits at chunk k ^ (r % 8)
        const int ob = j % OS;
        if (j >= OS && !tc::mbar_wait(&o_empty[ob], ((j / OS) - 1) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
        uint8_t *otile = sO + ob * kF32Tile, *orow = otile + row * 128;
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int k = 0; k < 8; ++k)
            *reinterpret_cast<float4 *>(orow + h * (kF32Tile / 2) + ((k ^ (row & 7)) << 4)) =
                make_float4(v[32 * h + 4 * k], v[32 * h + 4 * k + 1], v[32 * h + 4 * k + 2], v[32 * h + 4 * k + 3]);
        tc::fence_proxy_async_smem();  // these writes are read by the TMA store
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&o_full[ob]);
        if (mirror) {
          // the transposed tile: T2[c][q][i][n][l] = D2[(ql, l), n], q = 2 qp + ql.
          // For each n a warp writes 32 consecutive l, one 128-byte line.
          const int q = 2 * qp + (row >> 6), l = row & 63;
          float *dst = t2 + ((((size_t)(2 * cp + s) * NP + q) * NP + i) * NP) * NP + l;
#pragma unroll
          for (int n = 0; n < 64; ++n) dst[(size_t)n * NP] = v[n];
        }
        if (warp == 6) {  // the whole warp waits (uniform exit on a timeout); lane 0 issues
          if (!tc::mbar_wait(&o_full[ob], (j / OS) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
          if (lane == 0) {
            const int c = 2 * cp + s;
            for (int h = 0; h < 2; ++h) tc::tma_store_3d(&map_t2s, otile + h * (kF32Tile / 2), 32 * h, qp * 128, c * NP + i);
            tc::tma_store_commit();
            if constexpr (OS == 1) {
              tc::tma_store_wait_read();
              tc::mbar_arrive(&o_empty[0]);
            } else {  // the store of job j - 1 has read its tile once at most this one is pending
              tc::tma_store_wait_read_but_one();
              if (j >= 1) tc::mbar_arrive(&o_empty[(j - 1) % OS]);
            }
          }
          __syncwarp();
        }
      }
    }
    if (F != 0 && run_cp >= 0)
      for (int s = 0; s < 2; ++s) warp_absmax_to(&ex[kMaxT2 * S + sl0 + 2 * run_cp + s], run_mx[s]);
    if (warp == 6 && lane == 0) tc::tma_store_wait_all();
  }
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------------------
// single-tile check of the operand layouts (test hook)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128, 1)
    umma_tile_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                     int a_mn_major, float *__restrict__ D, int *err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = align1024(smem_raw);
  uint8_t *sA = smem, *sB = smem + TILE128;
  uint64_t *bar = reinterpret_cast<uint64_t *>(sB + TILE64);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 2);
  __shared__ int s_abort;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::fence_barrier_init();
    s_abort = 0;
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, 64);
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  volatile int *abort = &s_abort;
  if (threadIdx.x == 0) {
    tc::mbar_arrive_expect_tx(&bar[0], TILE128 + TILE64);
    if (a_mn_major) {
      tc::tma_load_3d(sA, &map_a, &bar[0], 0, 0, 0);
      tc::tma_load_3d(sA + TILE64, &map_a, &bar[0], 64, 0, 0);
    } else {
      tc::tma_load_3d(sA, &map_a, &bar[0], 0, 0, 0);
    }
    tc::tma_load_3d(sB, &map_b, &bar[0], 0, 0, 0);
    if (tc::mbar_wait(&bar[0], 0, abort)) {
      tc::tc_fence_after();
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t ad = a_mn_major ? tc::smem_desc(tc::smem_u32(sA) + kk * 2048, TILE64, 1024)
                                       : tc::smem_desc(tc::smem_u32(sA) + kk * 32, 16, 1024);
        const uint64_t bd = tc::smem_desc(tc::smem_u32(sB) + kk * 32, 16, 1024);
        tc::mma_bf16(tmem, ad, bd, a_mn_major ? kIdescMK : kIdescKK, kk ? 1u : 0u);
      }
      tc::mma_commit(&bar[1]);
    } else {
      raise_abort(abort, err);
    }
  }
  __syncwarp();
  const bool done = tc::mbar_wait(&bar[1], 0, abort);
  if (done) {
    tc::tc_fence_after();
    float v[64];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    tc::tmem_ld_32x32b_x32(taddr, v);
    tc::tmem_ld_32x32b_x32(taddr + 32, v + 32);
    tc::tmem_ld_wait();
    const int row = warp * 32 + lane;
    for (int j = 0; j < 64; ++j) D[row * 64 + j] = v[j];
  } else if (lane == 0) {
    raise_abort(abort, err);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 64);
  }
}

// the same tile with A taken from TMEM: each thread writes its row of A
// (64 bf16 = 32 packed columns) into TMEM, then one thread issues the MMAs
__global__ void __launch_bounds__(128, 1)
    umma_tile_ts_kernel(const __nv_bfloat16 *__restrict__ A, const __grid_constant__ CUtensorMap map_b,
                        float *__restrict__ D, int *err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = align1024(smem_raw);
  uint8_t *sB = smem;
  uint64_t *bar = reinterpret_cast<uint64_t *>(sB + TILE64);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 2);
  __shared__ int s_abort;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, row = warp * 32 + lane;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::fence_barrier_init();
    s_abort = 0;
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, 128);
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;  // D at columns 0..63, A at 64..95
  volatile int *abort = &s_abort;
  uint32_t w[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) w[c] = reinterpret_cast<const uint32_t *>(A + row * 64)[c];
  tc::tmem_st_32x32b_x32(tmem + ((uint32_t)(warp * 32) << 16) + 64, w);
  tc::tmem_st_wait();
  tc::tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    tc::tc_fence_after();
    tc::mbar_arrive_expect_tx(&bar[0], TILE64);
    tc::tma_load_3d(sB, &map_b, &bar[0], 0, 0, 0);
    if (tc::mbar_wait(&bar[0], 0, abort)) {
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t bd = tc::smem_desc(tc::smem_u32(sB) + kk * 32, 16, 1024);
        tc::mma_bf16_ts(tmem, tmem + 64 + kk * 8, bd, kIdescKK, kk ? 1u : 0u);
      }
      tc::mma_commit(&bar[1]);
    } else {
      raise_abort(abort, err);
    }
  }
  __syncwarp();
  if (tc::mbar_wait(&bar[1], 0, abort)) {
    tc::tc_fence_after();
    float v[64];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    tc::tmem_ld_32x32b_x32(taddr, v);
    tc::tmem_ld_32x32b_x32(taddr + 32, v + 32);
    tc::tmem_ld_wait();
    for (int j = 0; j < 64; ++j) D[row * 64 + j] = v[j];
  } else if (lane == 0) {
    raise_abort(abort, err);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 128);
  }
}

// a wait that nothing satisfies: the bounded wait gives up and raises the error word
__global__ void wait_timeout_kernel(int *err) {
  __shared__ uint64_t bar;
  __shared__ int s_abort;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_barrier_init();
    s_abort = 0;
  }
  __syncthreads();
  volatile int *abort = &s_abort;
  if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0, abort)) raise_abort(abort, err);
  __syncthreads();
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct TcState {
  int C = 0;                           // slots per chunk (one launch of each tile kernel)
  int S = 0;                           // slots of the whole grid (a multiple of C)
  uint16_t *Gs = nullptr;              // split G sets of every slot of the grid (BF16 or FP16 bits)
  int *gexp = nullptr;                 // [kExpSets][S] FP16 scale exponents and maxima per slot
  float *T2 = nullptr, *T3 = nullptr;  // FP32 intermediates, C * NP^4 each
  CUtensorMap map_v, map_g, map_t2, map_t2s, map_t3, map_t3s, map_w;
  CUtensorMap map_v16, map_w16;        // the FP16 planes of v and W
};

constexpr size_t kPlane4 = (size_t)NP * NP * NP * NP;

template <int T>
size_t smem_sandwich() {
  const int GS = 1, A1S = (T == 2) ? 2 : 1, A2S = 2, OS = (T == 2) ? 2 : 1;
  return 1024 + A1S * T * TILE128 + GS * 2 * T * TILE64 + A2S * T * TILE128 + OS * kF32Tile + 256;
}
template <int T>
size_t smem_xform() {  // 4 input tiles, 2 output tiles, Gbar sets (two at T = 2, one at T = 3)
  return 1024 + 6 * (size_t)kF32Tile + (T == 2 ? 2 : 1) * T * TILE64 + 256;
}
template <int T>
size_t smem_contract() {
  return 1024 + contract_stages_f<T>() * (size_t)kF32Tile + contract_stages_w<T>() * T * TILE64 + 256;
}

template <int T, int F>
gf2_status run_chunks(gf2_ctx *ctx, TcState *s, const double *d_G, int k0, int count, double *d_out) {
  const int N = ctx->N, C = s->C, sms = ctx->num_sms;
  const size_t ssw = smem_sandwich<T>(), sxf = smem_xform<T>(), sct = smem_contract<T>();
  GF2_CK(ctx, cudaFuncSetAttribute(sandwich_kernel<T, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssw));
  GF2_CK(ctx, cudaFuncSetAttribute(xform_kernel<T, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sxf));
  GF2_CK(ctx, cudaFuncSetAttribute(contract_kernel<T, contract_group<T>(), F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)sct));
  const CUtensorMap &map_v = F == 0 ? s->map_v : s->map_v16, &map_w = F == 0 ? s->map_w : s->map_w16;
  const int e_fixed = F == 0 ? 0 : ctx->e_v16 + ctx->e_w16;
  const int B = ctx->tc_pack;  // time points per tile slot
  const int S = s->S;          // slot stride of the split G planes and the exponents
  if (count <= 0) return GF2_OK;
  // every slot of the call split in one launch, the whole output cleared once
  const int n_chunks = (count + C * B - 1) / (C * B);
  GF2_PROF(ctx, GF2_K_SPLIT, (split_g_kernel<NP, F><<<dim3(n_chunks * C, 2), 256, 0, ctx->stream>>>(
                                 N, B, ctx->n_tau - 1, k0, count, S, d_G, s->Gs, s->gexp, ctx->vmax16)));
  GF2_CK_LAUNCH(ctx, "split_g_kernel");
  GF2_CK(ctx, cudaMemsetAsync(d_out, 0, sizeof(double) * (size_t)count * N * N, ctx->stream));
  for (int c0 = 0, sl0 = 0; c0 < count; c0 += C * B, sl0 += C) {
    const int cnt = std::min(C * B, count - c0);
    const int ce = (((cnt + B - 1) / B) + 1) & ~1;  // slots, rounded up to whole pairs
    double *out = d_out + (size_t)c0 * N * N;
    const int sym = ctx->tc_pair_sym ? 1 : 0;
    const int u1 = (ce / 2) * (sym ? kSymUnitsPerPair : NP * 32);
    GF2_PROF(ctx, GF2_K_SANDWICH,
             (sandwich_kernel<T, F><<<std::min(u1, sms), 448, ssw, ctx->stream>>>(
                 map_v, s->map_g, s->map_t2s, C, S, sl0, u1, s->gexp, ctx->d_err, sym, s->T2)));
    GF2_CK_LAUNCH(ctx, "sandwich_kernel");
    const int u2 = ce * NP * 32;
    GF2_PROF(ctx, GF2_K_XFORM,
             (xform_kernel<T, F><<<std::min(u2, sms), 320, sxf, ctx->stream>>>(s->map_t2, s->map_g, s->map_t3s, C, S, sl0,
                                                                               u2, s->gexp, ctx->d_err)));
    GF2_CK_LAUNCH(ctx, "xform_kernel");
    const int u3 = (ce / 2) * NP;
    GF2_PROF(ctx, GF2_K_CONTRACT,
             (contract_kernel<T, contract_group<T>(), F><<<std::min(u3, sms), 448, sct, ctx->stream>>>(
                 s->map_t3, map_w, out, N, B, cnt, C, S, sl0, u3, s->gexp, e_fixed, ctx->d_err)));
    GF2_CK_LAUNCH(ctx, "contract_kernel");
  }
  return GF2_OK;
}

TcState *tc_state(gf2_ctx *ctx) { return reinterpret_cast<TcState *>(ctx->d_tc_ws); }

}  // namespace

gf2_status gf2_tc_prepare_integrals(gf2_ctx *ctx) {
  if (ctx->N > 2 * NP) return GF2_ERR_UNSUPPORTED;
  if (!encode_fn()) return gf2_fail(ctx, GF2_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled unavailable");
  if (ctx->N > NP) {  // 128-wide planes (several GB): built by the first split-precision call
    ctx->tc_planes_stale = true;
    return GF2_OK;
  }
  return gf2_tc_build_planes(ctx, NP);
}

// The split term planes of v and W (BF16 and FP16) for tiles of width P (64 or 128)
gf2_status gf2_tc_build_planes(gf2_ctx *ctx, int P) {
  ctx->tc_pack = (P == NP && ctx->N <= NP / 2) ? NP / ctx->N : 1;
  const size_t plane4 = (size_t)P * P * P * P;
  const size_t bytes = TMAX * plane4 * sizeof(uint16_t);
  if (!ctx->d_v_split) GF2_CK(ctx, cudaMalloc(&ctx->d_v_split, bytes));
  if (!ctx->d_wt_split) GF2_CK(ctx, cudaMalloc(&ctx->d_wt_split, bytes));
  if (!ctx->d_v_split16) GF2_CK(ctx, cudaMalloc(&ctx->d_v_split16, bytes));
  if (!ctx->d_wt_split16) GF2_CK(ctx, cudaMalloc(&ctx->d_wt_split16, bytes));
  const int blocks = 8 * ctx->num_sms;
  // With the overlap known the contraction runs in the orthonormal (Loewdin)
  // basis: v' = (S^-1/2)^{x4} v, G' = S^1/2 G S^1/2.  Of the back transform
  // Sigma = S^1/2 Sigma' S^1/2 the right factor (Sigma's column index j) is
  // folded into W: vw = v' x_4 S^1/2 and W = 2 vw_lpnj - vw_nplj, so the tile
  // kernels return Sigma' S^1/2 and one FP64 product per time point supplies
  // the left factor.  (Folding the left factor into v as well saved 3.6 ms more
  // but raised the energy error three- to fourfold: measured.)
  const int N = ctx->N;
  const size_t n4 = (size_t)N * N * N * N;
  double *vs = ctx->d_v, *vw = ctx->d_v, *vorth = nullptr, *vfold = nullptr;
  if (ctx->d_Shalf) {
    GF2_CK(ctx, cudaMalloc(&vorth, n4 * sizeof(double)));
    if (cudaMalloc(&vfold, n4 * sizeof(double)) != cudaSuccess) {
      cudaFree(vorth);
      return gf2_fail(ctx, GF2_ERR_NOMEM, "gf2_set_integrals: folded integrals");
    }
    gf2_status st = gf2_orth_transform_v(ctx, vorth);
    const long long N3 = (long long)N * N * N;
    if (st == GF2_OK) {  // vw[(l,p,n), b] = sum_j v'[(l,p,n), j] Sh[j, b]
      Dgemm g{};
      g.M = (int)N3; g.N = N; g.K = N;
      g.A = vorth; g.a_rs = N; g.a_cs = 1;
      g.B = ctx->d_Shalf; g.b_rs = N; g.b_cs = 1;
      g.C = vfold; g.c_rs = N; g.c_cs = 1;
      g.nb0 = 1; g.nb1 = 1; g.alpha = 1.0; g.beta_c = 0.0; g.split_k = 1;
      st = gf2_dgemm(ctx, g);
    }
    if (st != GF2_OK) {
      cudaStreamSynchronize(ctx->stream);
      cudaFree(vorth);
      cudaFree(vfold);
      return st;
    }
    vs = vorth;
    vw = vfold;
  }
  // The symmetric sandwich needs (im|qk) = (qk|im).  Integrals of real orbitals
  // have it; the orthonormal-basis integrals have it mathematically, so their
  // rounding-level asymmetry (from the order of the four index transforms) is
  // removed by averaging the pair-transposed entries.
  unsigned long long *d_amax = reinterpret_cast<unsigned long long *>(ctx->d_red);
  GF2_CK(ctx, cudaMemsetAsync(d_amax, 0, 3 * sizeof(unsigned long long), ctx->stream));
  absmax_kernel<<<blocks, 256, 0, ctx->stream>>>(n4, ctx->d_v, d_amax);
  GF2_CK_LAUNCH(ctx, "absmax_kernel");
  pair_asym_kernel<<<blocks, 256, 0, ctx->stream>>>(N, ctx->d_v, d_amax + 2);
  GF2_CK_LAUNCH(ctx, "pair_asym_kernel");
  {
    unsigned long long b3[3] = {0, 0, 0};
    GF2_CK(ctx, cudaMemcpyAsync(b3, d_amax, sizeof(b3), cudaMemcpyDeviceToHost, ctx->stream));
    GF2_CK(ctx, cudaStreamSynchronize(ctx->stream));
    double v0max, asym;
    std::memcpy(&v0max, &b3[0], sizeof(v0max));
    std::memcpy(&asym, &b3[2], sizeof(asym));
    ctx->tc_pair_sym = asym <= 1e-12 * v0max;
  }
  if (ctx->tc_pair_sym && vorth) {
    pair_symmetrize_kernel<<<blocks, 256, 0, ctx->stream>>>(N, vorth);
    GF2_CK_LAUNCH(ctx, "pair_symmetrize_kernel");
  }
  const int B = ctx->tc_pack;
  if (P == NP)
    split_v_kernel<NP, 0><<<blocks, 256, 0, ctx->stream>>>(N, B, vs, 0, (uint16_t *)ctx->d_v_split);
  else
    split_v_kernel<2 * NP, 0><<<blocks, 256, 0, ctx->stream>>>(N, 1, vs, 0, (uint16_t *)ctx->d_v_split);
  GF2_CK_LAUNCH(ctx, "split_v_kernel");
  if (P == NP)
    split_w_kernel<NP, 0><<<blocks, 256, 0, ctx->stream>>>(N, B, vw, 0, (uint16_t *)ctx->d_wt_split);
  else
    split_w_kernel<2 * NP, 0><<<blocks, 256, 0, ctx->stream>>>(N, 1, vw, 0, (uint16_t *)ctx->d_wt_split);
  GF2_CK_LAUNCH(ctx, "split_w_kernel");
  // FP16 planes: v scaled so that its largest entry lies in [2^13, 2^14); W
  // (|W| <= 3 max|vw|) by the exponent of 3 max|vw|
  GF2_CK(ctx, cudaMemsetAsync(d_amax, 0, 2 * sizeof(unsigned long long), ctx->stream));
  absmax_kernel<<<blocks, 256, 0, ctx->stream>>>(n4, vs, d_amax);
  GF2_CK_LAUNCH(ctx, "absmax_kernel");
  absmax_kernel<<<blocks, 256, 0, ctx->stream>>>(n4, vw, d_amax + 1);
  GF2_CK_LAUNCH(ctx, "absmax_kernel");
  unsigned long long bits[2] = {0, 0};
  GF2_CK(ctx, cudaMemcpyAsync(bits, d_amax, sizeof(bits), cudaMemcpyDeviceToHost, ctx->stream));
  GF2_CK(ctx, cudaStreamSynchronize(ctx->stream));
  double vmax, wmax;
  std::memcpy(&vmax, &bits[0], sizeof(vmax));
  std::memcpy(&wmax, &bits[1], sizeof(wmax));
  ctx->e_v16 = fp16_exponent(vmax);
  ctx->e_w16 = fp16_exponent(3.0 * wmax);
  ctx->vmax16 = ldexp(vmax, ctx->e_v16);
  if (P == NP)
    split_v_kernel<NP, 1><<<blocks, 256, 0, ctx->stream>>>(N, B, vs, ctx->e_v16, (uint16_t *)ctx->d_v_split16);
  else
    split_v_kernel<2 * NP, 1><<<blocks, 256, 0, ctx->stream>>>(N, 1, vs, ctx->e_v16, (uint16_t *)ctx->d_v_split16);
  GF2_CK_LAUNCH(ctx, "split_v_kernel");
  if (P == NP)
    split_w_kernel<NP, 1><<<blocks, 256, 0, ctx->stream>>>(N, B, vw, ctx->e_w16, (uint16_t *)ctx->d_wt_split16);
  else
    split_w_kernel<2 * NP, 1><<<blocks, 256, 0, ctx->stream>>>(N, 1, vw, ctx->e_w16, (uint16_t *)ctx->d_wt_split16);
  GF2_CK_LAUNCH(ctx, "split_w_kernel");
  if (vorth) {
    GF2_CK(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(vorth);
    cudaFree(vfold);
  }
  ctx->split_terms = TMAX;
  ctx->tc_planes_stale = false;
  return GF2_OK;
}

static gf2_status tc_workspace(gf2_ctx *ctx) {
  if (ctx->d_tc_ws) return GF2_OK;
  TcState *s = new (std::nothrow) TcState();
  if (!s) return gf2_fail(ctx, GF2_ERR_NOMEM, "tc state");
  s->C = std::max(2, std::min(ctx->tc_chunk_max, ((ctx->n_tau + 1) / 2) * 2));
  const int C = s->C;
  // slots of the whole grid, rounded up to whole chunks
  const int B = ctx->tc_pack;
  s->S = ((((ctx->n_tau + B - 1) / B) + C - 1) / C) * C;
  const int S = s->S;
  const size_t gbytes = (size_t)2 * TMAX * S * NP * NP * sizeof(uint16_t);
  const size_t ibytes = (size_t)C * kPlane4 * sizeof(float);
  cudaError_t e = cudaMalloc(&s->Gs, gbytes);
  if (e == cudaSuccess) e = cudaMalloc(&s->gexp, kExpSets * S * sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(s->gexp, 0, kExpSets * S * sizeof(int), ctx->stream);
  if (e == cudaSuccess) e = cudaMalloc(&s->T2, ibytes);
  if (e == cudaSuccess) e = cudaMalloc(&s->T3, ibytes);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->T2, 0, ibytes, ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->T3, 0, ibytes, ctx->stream);
  if (e != cudaSuccess) {
    if (s->Gs) cudaFree(s->Gs);
    if (s->gexp) cudaFree(s->gexp);
    if (s->T2) cudaFree(s->T2);
    if (s->T3) cudaFree(s->T3);
    delete s;
    return gf2_cuda_fail(ctx, e, "tc workspace");
  }
  bool ok = true;
  {  // v: dims (k, m, q, i, t), box (64, 64, 2, 1, 1) -> rows (q, m) of 64 k
    uint64_t dims[5] = {NP, NP, NP, NP, TMAX};
    uint64_t str[4] = {NP * 2, NP * NP * 2, (uint64_t)NP * NP * NP * 2, kPlane4 * 2};
    uint32_t box[5] = {64, 64, 2, 1, 1};
    ok &= make_map(&s->map_v, ctx->d_v_split, 5, dims, str, box);
    ok &= make_map(&s->map_v16, ctx->d_v_split16, 5, dims, str, box);
  }
  {  // G sets of every slot: dims (64, 64, 2*TMAX*S), box (64, 64, 1)
    uint64_t dims[3] = {NP, NP, (uint64_t)2 * TMAX * S};
    uint64_t str[2] = {NP * 2, NP * NP * 2};
    uint32_t box[3] = {64, 64, 1};
    ok &= make_map(&s->map_g, s->Gs, 3, dims, str, box);
  }
  {  // T2 (fp32): dims ((l,n) 4096, q 64, (c,i) C*64), box (128, 64, 1) -> F[q][128 (l,n)]
    uint64_t dims[3] = {NP * NP, NP, (uint64_t)C * NP};
    uint64_t str[2] = {NP * NP * 4, (uint64_t)NP * NP * NP * 4};
    uint32_t box[3] = {128, 64, 1};
    ok &= make_map(&s->map_t2, s->T2, 3, dims, str, box, true);
  }
  {  // T2 (fp32) as stored by stages 1+2: dims (n 64, (q,l) 4096, (c,i) C*64), box (32, 128, 1),
     // 128-byte swizzle: one half of the 64 n of 128 rows
    uint64_t dims[3] = {NP, NP * NP, (uint64_t)C * NP};
    uint64_t str[2] = {NP * 4, (uint64_t)NP * NP * NP * 4};
    uint32_t box[3] = {32, 128, 1};
    ok &= make_map(&s->map_t2s, s->T2, 3, dims, str, box, true, true);
  }
  {  // T3 (fp32): dims (K = NP^3, rows (c,i) C*64, 1), box (32, 128, 1), 128-byte swizzle:
     // F[row][32 k] per half of a 64-wide K step
    uint64_t dims[3] = {(uint64_t)NP * NP * NP, (uint64_t)C * NP, 1};
    uint64_t str[2] = {(uint64_t)NP * NP * NP * 4, (uint64_t)C * kPlane4 * 4};
    uint32_t box[3] = {32, 128, 1};
    ok &= make_map(&s->map_t3, s->T3, 3, dims, str, box, true, true);
  }
  {  // T3 (fp32) as stored by stage 3: dims (p 64, (l,n) 4096, (c,i) C*64), box (32, 128, 1),
     // 128-byte swizzle: one half of the 64 p of 128 rows
    uint64_t dims[3] = {NP, NP * NP, (uint64_t)C * NP};
    uint64_t str[2] = {NP * 4, (uint64_t)NP * NP * NP * 4};
    uint32_t box[3] = {32, 128, 1};
    ok &= make_map(&s->map_t3s, s->T3, 3, dims, str, box, true, true);
  }
  {  // W: dims (K = NP^3, j 64, t), box (64, 64, 1)
    uint64_t dims[3] = {(uint64_t)NP * NP * NP, NP, TMAX};
    uint64_t str[2] = {(uint64_t)NP * NP * NP * 2, kPlane4 * 2};
    uint32_t box[3] = {64, 64, 1};
    ok &= make_map(&s->map_w, ctx->d_wt_split, 3, dims, str, box);
    ok &= make_map(&s->map_w16, ctx->d_wt_split16, 3, dims, str, box);
  }
  if (!ok) {
    cudaFree(s->Gs);
    cudaFree(s->gexp);
    cudaFree(s->T2);
    cudaFree(s->T3);
    delete s;
    return gf2_fail(ctx, GF2_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  }
  ctx->d_tc_ws = s;
  ctx->tc_chunk = C;
  return GF2_OK;
}

void gf2_tc_release(gf2_ctx *ctx) {
  gf2_tc128_release(ctx);
  TcState *s = tc_state(ctx);
  if (!s) return;
  cudaFree(s->Gs);
  cudaFree(s->gexp);
  cudaFree(s->T2);
  cudaFree(s->T3);
  delete s;
  ctx->d_tc_ws = nullptr;
}

gf2_status gf2_sigma_tc(gf2_ctx *ctx, const double *d_G, int k0, int count, double *d_out, int prec) {
  if (ctx->N > 2 * NP) return gf2_fail(ctx, GF2_ERR_UNSUPPORTED, "tensor-core path needs N <= 128");
  gf2_status st;
  if (ctx->N > NP && ctx->tc_planes_stale && (st = gf2_tc_build_planes(ctx, 2 * NP)) != GF2_OK) return st;
  if (!ctx->d_v_split) return gf2_fail(ctx, GF2_ERR_UNSUPPORTED, "tensor-core path needs gf2_set_integrals");
  st = ctx->N > NP ? gf2_tc128_workspace(ctx) : tc_workspace(ctx);
  if (st != GF2_OK) return st;
  GF2_CK(ctx, cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
  TcState *s = tc_state(ctx);
  // in the orthonormal basis: G' = S^{1/2} G S^{1/2} in; the kernels write
  // Sigma' S^{1/2} (the right factor is folded into W), the left factor follows
  const double *G_use = d_G;
  double *out_use = d_out;
  if (ctx->d_Shalf) {
    double *Go = nullptr;
    if ((st = gf2_orth_transform_g(ctx, d_G, k0, count, &Go)) != GF2_OK) return st;
    G_use = Go;
    out_use = ctx->d_orth_ws + 2 * (size_t)ctx->n_tau * ctx->N * ctx->N;
  }
  if (ctx->N > NP) {
    st = gf2_tc128_run(ctx, G_use, k0, count, out_use, prec);
  } else {
    switch (prec) {
      case GF2_PREC_BF16X3: st = run_chunks<2, 0>(ctx, s, G_use, k0, count, out_use); break;
      case GF2_PREC_BF16X6: st = run_chunks<3, 0>(ctx, s, G_use, k0, count, out_use); break;
      case GF2_PREC_FP16X3: st = run_chunks<2, 1>(ctx, s, G_use, k0, count, out_use); break;
      default: st = run_chunks<3, 1>(ctx, s, G_use, k0, count, out_use); break;
    }
  }
  if (st != GF2_OK) return st;
  if (ctx->d_Shalf) {  // the row index: Sigma[b] = S^1/2 X[b]
    const long long N2 = (long long)ctx->N * ctx->N;
    for (int b0 = 0; b0 < count; b0 += 65535) {
      const int nb = std::min(65535, count - b0);
      Dgemm g{};
      g.M = ctx->N; g.N = ctx->N; g.K = ctx->N;
      g.A = ctx->d_Shalf; g.a_rs = ctx->N; g.a_cs = 1; g.a_b0 = 0;
      g.B = out_use + b0 * N2; g.b_rs = ctx->N; g.b_cs = 1; g.b_b0 = N2;
      g.C = d_out + b0 * N2; g.c_rs = ctx->N; g.c_cs = 1; g.c_b0 = N2;
      g.nb0 = nb; g.nb1 = 1; g.alpha = 1.0; g.beta_c = 0.0; g.split_k = 1;
      if ((st = gf2_dgemm(ctx, g)) != GF2_OK) return st;
    }
  }
  // Eq. Sigma is symmetric; the two triangles carry independent rounding of the
  // split arithmetic, and their average is the better estimate
  if ((st = gf2_symmetrize(ctx, d_out, count)) != GF2_OK) return st;
  if (ctx->defer_error_check) return GF2_OK;  // the batch reads d_err after the graph ran
  int flag = 0;
  GF2_CK(ctx, cudaMemcpyAsync(&flag, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  GF2_CK(ctx, cudaStreamSynchronize(ctx->stream));
  if (flag) return gf2_fail(ctx, GF2_ERR_TIMEOUT, "tensor-core Sigma: a pipeline wait timed out");
  return GF2_OK;
}

// test hook: one 128x64x64 BF16 tile through TMA, tcgen05.mma and tcgen05.ld
extern "C" gf2_status gf2_test_umma_tile(int a_mn_major, const void *d_A, const void *d_B, float *d_D,
                                         int *d_err, void *stream) {
  if (!d_A || !d_B || !d_D || !d_err || a_mn_major < 0 || a_mn_major > 2) return GF2_ERR_ARG;
  if (!encode_fn()) return GF2_ERR_UNSUPPORTED;
  CUtensorMap ma, mb;
  bool ok;
  if (a_mn_major == 2) {  // A [M=128][K=64] bf16 through TMEM
    uint64_t dims[3] = {64, 64, 1};
    uint64_t str[2] = {64 * 2, 64 * 64 * 2};
    uint32_t box[3] = {64, 64, 1};
    if (!make_map(&mb, d_B, 3, dims, str, box)) return GF2_ERR_CUDA;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t smem = 1024 + TILE64 + 256;
    if (cudaFuncSetAttribute(umma_tile_ts_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return GF2_ERR_CUDA;
    umma_tile_ts_kernel<<<1, 128, smem, st>>>(reinterpret_cast<const __nv_bfloat16 *>(d_A), mb, d_D, d_err);
    if (cudaGetLastError() != cudaSuccess) return GF2_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return GF2_ERR_CUDA;
    return GF2_OK;
  }
  if (a_mn_major) {  // A stored [K=64][M=128]: dims (128, 64, 1), box (64, 64, 1)
    uint64_t dims[3] = {128, 64, 1};
    uint64_t str[2] = {128 * 2, 128 * 64 * 2};
    uint32_t box[3] = {64, 64, 1};
    ok = make_map(&ma, d_A, 3, dims, str, box);
  } else {  // A stored [M=128][K=64]: dims (64, 128, 1), box (64, 128, 1)
    uint64_t dims[3] = {64, 128, 1};
    uint64_t str[2] = {64 * 2, 64 * 128 * 2};
    uint32_t box[3] = {64, 128, 1};
    ok = make_map(&ma, d_A, 3, dims, str, box);
  }
  uint64_t dims[3] = {64, 64, 1};
  uint64_t str[2] = {64 * 2, 64 * 64 * 2};
  uint32_t box[3] = {64, 64, 1};
  ok = ok && make_map(&mb, d_B, 3, dims, str, box);
  if (!ok) return GF2_ERR_CUDA;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t smem = 1024 + TILE128 + TILE64 + 256;
  if (cudaFuncSetAttribute(umma_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return GF2_ERR_CUDA;
  umma_tile_kernel<<<1, 128, smem, st>>>(ma, mb, a_mn_major, d_D, d_err);
  if (cudaGetLastError() != cudaSuccess) return GF2_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return GF2_ERR_CUDA;
  return GF2_OK;
}

// test hook: a pipeline wait that runs out (failure detection without a fault)
extern "C" gf2_status gf2_test_wait_timeout(int *d_err, void *stream) {
  if (!d_err) return GF2_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  wait_timeout_kernel<<<1, 32, 0, st>>>(d_err);
  if (cudaGetLastError() != cudaSuccess) return GF2_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return GF2_ERR_CUDA;
  return GF2_OK;
}
