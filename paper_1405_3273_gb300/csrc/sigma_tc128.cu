// Eq. Sigma on the tcgen05 tensor cores for bases of 65..128 functions, padded
// to P = 128: the same split arithmetic as the 64-wide pipeline (T 16-bit
// terms of every operand, the products a + b < T, FP32 accumulation, FP16
// operands with power-of-two scales), with tiles that are 128 wide in every
// index.  Per chunk of C time points three kernels run back to back:
//
//  sandwich128  stages 1+2 fused.  Unit (c, i, q), one time point.
//               MMA1 (transposed): D1t[l, m] = sum_k GT[l][k] V[m][k],
//               A = G(tau)^T, B = the v tile v[i][m][q][k], both from shared
//               memory (K = 128 in two 64-wide blocks), D1t in TMEM.  Four
//               warps read D1t row l (one TMEM lane each), split it into T
//               terms and write them back to TMEM as the A operand of MMA2
//               (lane l, m packed two per column), so no shared memory holds
//               the intermediate.
//               MMA2: D2[l, n] = sum_m A2[l, m] GT[n][m] (A from TMEM, B = the
//               same G(tau)^T tiles), written into the TMEM buffer that D1t
//               of the same unit occupied.  Four warps stage D2 as FP32 and
//               store T2[c][i][q][l][n] with TMA.  When v has the pair
//               symmetry (im|qk) = (qk|im), T2[c][i][q][l][n] =
//               T2[c][q][i][n][l]: only the units with q >= i run (8256 of
//               16384 per time point) and each tile with q > i is also
//               written transposed, as tile (q, i), by plain coalesced stores.
//  xform128     stage 3.  Unit (c, i, l): D3[n, p] = sum_q T2[c][i][q][l][n]
//               Gbar[p][q]; FP32 T2 tiles by TMA, split by eight converter
//               warps (one per TMEM lane and K block) into TMEM, A from TMEM,
//               B = the Gbar planes; T3[c][i][l][n][p] stored by TMA.
//  contract128  stage 4.  Rows (c, i) of one time point, K = (l, n, p) in
//               64-wide steps; unit (c, l) covers the 16384 values of K of one
//               l.  A CTA takes a contiguous block of units and keeps its
//               compensated FP32 sums (TwoSum of the group sums of two K steps)
//               while the time point stays the same, then adds them into the
//               FP64 output with atomics.
//
// Padding: rows and columns N..127 of G, Gbar, v and W are zero, so the padded
// indices contribute nothing; the output keeps rows and columns < N.
// Every wait is bounded (a timeout raises the context error word and the
// kernel drains and returns).
#include <algorithm>
#include <cstring>
#include <new>

#include "gf2_internal.cuh"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int P = 128;
constexpr uint32_t kTile = 128 * 64 * 2;        // 16 KB: 128 rows x 64 bf16 (one K block)
constexpr uint32_t kOperand = 2 * kTile;        // 32 KB: 128 rows x 128 K, one term
constexpr uint32_t kBox = 128 * 32 * 4;         // 16 KB: 128 rows x 32 fp32, 128-byte swizzle
constexpr uint32_t kF32Half = 2 * kBox;         // 32 KB: 128 rows x 64 fp32
constexpr size_t kPlane4 = (size_t)P * P * P * P;

// stage a row of 64 FP32 values (row `row` of a [2 boxes][128 rows][32] tile,
// 16-byte chunk j of a box row at chunk j ^ (row % 8)) for a TMA store
__device__ __forceinline__ void stage_row64(uint8_t *tile, int row, const float *v) {
  uint8_t *orow = tile + row * 128;
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int j = 0; j < 8; ++j)
      *reinterpret_cast<float4 *>(orow + h * kBox + ((j ^ (row & 7)) << 4)) =
          make_float4(v[32 * h + 4 * j], v[32 * h + 4 * j + 1], v[32 * h + 4 * j + 2], v[32 * h + 4 * j + 3]);
}

// ---------------------------------------------------------------------------
// stages 1+2.  320 threads: warp 0 TMA, warp 1 MMA, warps 2-5 the first
// epilogue (D1t -> A2 in TMEM), warps 6-9 the second epilogue.  Only one warp
// per TMEM lane quarter ever writes TMEM.
// TMEM: X buffers at columns 0 and 128 (D1t, then D2 of the same unit),
// A2 stages from column 256, [K block][term] x 32 columns each.
// ---------------------------------------------------------------------------
constexpr int kSym128Units = P * (P + 1) / 2;  // (i, q) with i <= q

// unit u of a launch -> (time point c, i, q); with the pair symmetry the units
// of a time point are the upper triangle i <= q, row by row
__device__ __forceinline__ void sandwich128_unit(int u, int sym, int &c, int &i, int &q) {
  if (!sym) {
    c = u / (P * P);
    i = (u / P) % P;
    q = u % P;
    return;
  }
  c = u / kSym128Units;
  const int r = u - c * kSym128Units;
  // rows before row i hold i P - i (i - 1) / 2 units
  const double b = 2.0 * P + 1.0;
  int ii = (int)((b - sqrt(b * b - 8.0 * r)) * 0.5);
  ii = max(0, min(P - 1, ii));
  while (ii > 0 && ii * P - ii * (ii - 1) / 2 > r) --ii;
  while (ii < P - 1 && (ii + 1) * P - (ii + 1) * ii / 2 <= r) ++ii;
  i = ii;
  q = ii + (r - (ii * P - ii * (ii - 1) / 2));
}

template <int T>
constexpr int sw128_vstages() { return T == 2 ? 2 : 1; }
template <int T>
constexpr int sw128_a2stages() { return T == 2 ? 2 : 1; }

template <int T, int F>
__global__ void __launch_bounds__(320, 1)
    sandwich128_kernel(const __grid_constant__ CUtensorMap map_v, const __grid_constant__ CUtensorMap map_g,
                       const __grid_constant__ CUtensorMap map_t2s, int S, int sl0, int n_units,
                       int *__restrict__ ex, int *err, int sym, float *__restrict__ t2) {
  constexpr int VS = sw128_vstages<T>(), A2S = sw128_a2stages<T>();
  constexpr uint32_t G_SET = T * kOperand, V_STAGE = T * kOperand, A2_COLS = 2 * T * 32;
  constexpr uint32_t kIdesc = idesc_fmt(F, 128, 128, 0, 0);
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = align1024(smem_raw);
  uint8_t *sG = smem;                 // [t][kb][128 l][64 k]
  uint8_t *sV = sG + G_SET;           // VS x [t][kb][128 m][64 k]
  uint8_t *sO = sV + VS * V_STAGE;    // staging: [2 boxes][128 rows][32 n] fp32
  uint64_t *bar = reinterpret_cast<uint64_t *>(sO + kF32Half);
  uint64_t *g_full = bar, *g_empty = bar + 1, *v_full = bar + 2, *v_empty = bar + 4;
  uint64_t *d1_full = bar + 6, *a2_full = bar + 8, *a2_empty = bar + 10, *d2_full = bar + 12;
  uint64_t *x_empty = bar + 14, *o_full = bar + 16, *o_empty = bar + 17;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 18);
  __shared__ int s_abort;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    tc::mbar_init(g_full, 1);
    tc::mbar_init(g_empty, 1);
    tc::mbar_init(o_full, 4);
    tc::mbar_init(o_empty, 1);
    for (int s = 0; s < 2; ++s) {
      tc::mbar_init(&v_full[s], 1);
      tc::mbar_init(&v_empty[s], 1);
      tc::mbar_init(&d1_full[s], 1);
      tc::mbar_init(&a2_full[s], 4);
      tc::mbar_init(&a2_empty[s], 1);
      tc::mbar_init(&d2_full[s], 1);
      tc::mbar_init(&x_empty[s], 4);
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
    int it = 0, cur_c = -1, gcount = 0;
    for (int u = u_begin; u < u_end; ++u, ++it) {
      int c, i, q;
      sandwich128_unit(u, sym, c, i, q);
      if (c != cur_c) {
        if (gcount >= 1 && !tc::mbar_wait(g_empty, (gcount - 1) & 1, abort)) { raise_abort(abort, err); break; }
        tc::mbar_arrive_expect_tx(g_full, G_SET);
        for (int t = 0; t < T; ++t)
          for (int kb = 0; kb < 2; ++kb)
            tc::tma_load_3d(sG + (t * 2 + kb) * kTile, &map_g, g_full, 64 * kb, 0, t * S + sl0 + c);
        cur_c = c;
        ++gcount;
      }
      const int st = it % VS;
      if (it >= VS && !tc::mbar_wait(&v_empty[st], ((it / VS) - 1) & 1, abort)) { raise_abort(abort, err); break; }
      tc::mbar_arrive_expect_tx(&v_full[st], V_STAGE);
      for (int t = 0; t < T; ++t)
        for (int kb = 0; kb < 2; ++kb)
          tc::tma_load_5d_hint(sV + st * V_STAGE + (t * 2 + kb) * kTile, &map_v, &v_full[st], 64 * kb, 0, q, i, t,
                               keep_pol);
    }
  } else if (warp == 1 && lane == 0) {
    int it = 0, cur_c = -1, gcount = 0;
    const int per_c = sym ? kSym128Units : P * P;
    for (int u = u_begin; u < u_end; ++u, ++it) {
      const int c = u / per_c;
      if (c != cur_c) {
        if (cur_c >= 0) tc::mma_commit(g_empty);
        if (!tc::mbar_wait(g_full, gcount & 1, abort)) { raise_abort(abort, err); break; }
        cur_c = c;
        ++gcount;
      }
      const int x = it & 1, st = it % VS, a2 = it % A2S;
      const uint32_t xcol = tmem + x * 128;
      // MMA1: D1t[l, m] = sum_k GT[l][k] V[m][k]
      if (!tc::mbar_wait(&v_full[st], (it / VS) & 1, abort)) { raise_abort(abort, err); break; }
      if (it >= 2 && !tc::mbar_wait(&x_empty[x], ((it >> 1) - 1) & 1, abort)) { raise_abort(abort, err); break; }
      tc::tc_fence_after();
      const uint32_t g0 = tc::smem_u32(sG), v0 = tc::smem_u32(sV + st * V_STAGE);
      for (int pr = 0; pr < Products<T>::n; ++pr) {
        const int ta = Products<T>::a(pr), tb = Products<T>::b(pr);
        for (int kb = 0; kb < 2; ++kb)
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t ad = tc::smem_desc(g0 + (ta * 2 + kb) * kTile + kk * 32, 16, 1024);
            const uint64_t bd = tc::smem_desc(v0 + (tb * 2 + kb) * kTile + kk * 32, 16, 1024);
            tc::mma_bf16(xcol, ad, bd, kIdesc, (pr | kb | kk) ? 1u : 0u);
          }
      }
      tc::mma_commit(&v_empty[st]);
      tc::mma_commit(&d1_full[x]);
      // MMA2: D2[l, n] = sum_m A2[l, m] GT[n][m], into the same X buffer
      if (!tc::mbar_wait(&a2_full[a2], (it / A2S) & 1, abort)) { raise_abort(abort, err); break; }
      tc::tc_fence_after();
      const uint32_t a0 = tmem + 256 + a2 * A2_COLS;
      for (int pr = 0; pr < Products<T>::n; ++pr) {
        const int ta = Products<T>::a(pr), tb = Products<T>::b(pr);
        for (int kb = 0; kb < 2; ++kb)
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t bd = tc::smem_desc(g0 + (tb * 2 + kb) * kTile + kk * 32, 16, 1024);
            tc::mma_bf16_ts(xcol, a0 + (kb * T + ta) * 32 + kk * 8, bd, kIdesc, (pr | kb | kk) ? 1u : 0u);
          }
      }
      tc::mma_commit(&a2_empty[a2]);
      tc::mma_commit(&d2_full[x]);
    }
  } else if (warp >= 2 && warp < 6) {
    // first epilogue: row l of D1t (TMEM lane) -> A2, K blocks 0 and 1 in turn
    // (one warp per TMEM lane quarter writes it)
    const int wq = warp & 3;
    const uint32_t lanes = (uint32_t)(wq * 32) << 16;
    int it = 0;
    bool ok = true;
    const int per_c = sym ? kSym128Units : P * P;
    for (int u = u_begin; u < u_end && ok; ++u, ++it) {
      const int c = u / per_c, x = it & 1, a2 = it % A2S;
      if (!tc::mbar_wait(&d1_full[x], (it >> 1) & 1, abort)) { raise_abort(abort, err); break; }
      __syncwarp();
      tc::tc_fence_after();
      const float scale = F == 0 ? 1.0f : exp2_scale(ex[kExpT1 * S + sl0 + c]);
      for (int kb = 0; kb < 2; ++kb) {
        float v[64];
        tc::tmem_ld_32x32b_x32(tmem + lanes + x * 128 + 64 * kb, v);
        tc::tmem_ld_32x32b_x32(tmem + lanes + x * 128 + 64 * kb + 32, v + 32);
        tc::tmem_ld_wait();
        if (kb == 0 && it >= A2S && !tc::mbar_wait(&a2_empty[a2], ((it / A2S) - 1) & 1, abort)) {
          raise_abort(abort, err);
          ok = false;
          break;
        }
        __syncwarp();
        tc::tc_fence_after();
        split_row_to_tmem<T, F>(v, tmem + lanes + 256 + a2 * A2_COLS + kb * T * 32, scale);
      }
      if (!ok) break;
      tc::tmem_st_wait();
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&a2_full[a2]);
    }
  } else if (warp >= 6 && warp < 10) {
    // second epilogue: row l of D2 -> T2[c][i][q][l][n], 64 n per staging pass
    const int wq = warp & 3, row = wq * 32 + lane;
    const uint32_t lanes = (uint32_t)(wq * 32) << 16;
    int it = 0, pass = 0, run_c = -1;
    float run_mx = 0.f;  // FP16: largest |T2| of time point run_c seen by this thread
    bool ok = true;
    for (int u = u_begin; u < u_end && ok; ++u, ++it) {
      int c, i, q;
      sandwich128_unit(u, sym, c, i, q);
      const int x = it & 1;
      // the mirrored tile (q, i): row l of this warp -> column l of T2[c][q][i][n][.]
      float *mirror = (sym && q > i) ? t2 + ((((size_t)c * P + q) * P + i) * P) * P + row : nullptr;
      if (F != 0 && c != run_c) {
        if (run_c >= 0) warp_absmax_to(&ex[kMaxT2 * S + sl0 + run_c], run_mx);
        run_c = c;
        run_mx = 0.f;
      }
      if (!tc::mbar_wait(&d2_full[x], (it >> 1) & 1, abort)) { raise_abort(abort, err); break; }
      tc::tc_fence_after();
      const float un = F == 0 ? 1.0f : exp2_scale(-ex[kExpT1 * S + sl0 + c]);
      for (int hh = 0; hh < 2; ++hh, ++pass) {
        float v[64];
        tc::tmem_ld_32x32b_x32(tmem + lanes + x * 128 + 64 * hh, v);
        tc::tmem_ld_32x32b_x32(tmem + lanes + x * 128 + 64 * hh + 32, v + 32);
        tc::tmem_ld_wait();
        if (hh == 1) {  // the X buffer may take the next unit's D1t
          tc::tc_fence_before();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&x_empty[x]);
        }
        if constexpr (F != 0) {
#pragma unroll
          for (int k = 0; k < 64; ++k) {
            v[k] *= un;
            run_mx = fmaxf(run_mx, fabsf(v[k]));
          }
        }
        if (pass >= 1 && !tc::mbar_wait(o_empty, (pass - 1) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
        if (mirror) {  // T2[c][q][i][n][l] = D2[l][n]: 32 lanes write 128 consecutive bytes per n
#pragma unroll
          for (int k = 0; k < 64; ++k) mirror[(size_t)(64 * hh + k) * P] = v[k];
        }
        stage_row64(sO, row, v);
        tc::fence_proxy_async_smem();  // these writes are read by the TMA store
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(o_full);
        if (warp == 6) {  // the whole warp waits (uniform exit on a timeout); lane 0 issues
          if (!tc::mbar_wait(o_full, pass & 1, abort)) { raise_abort(abort, err); ok = false; break; }
          if (lane == 0) {
            for (int b = 0; b < 2; ++b) tc::tma_store_3d(&map_t2s, sO + b * kBox, 64 * hh + 32 * b, q * P, c * P + i);
            tc::tma_store_commit();
            tc::tma_store_wait_read();
            tc::mbar_arrive(o_empty);
          }
          __syncwarp();
        }
      }
    }
    if (F != 0 && run_c >= 0) warp_absmax_to(&ex[kMaxT2 * S + sl0 + run_c], run_mx);
    if (warp == 6 && lane == 0) tc::tma_store_wait_all();
  }
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------------------
// stage 3.  320 threads: warp 0 TMA, warp 1 MMA, warps 2-5 epilogue, warps
// 6-9 convert (one warp per TMEM lane quarter, both K blocks of each unit).
// TMEM: accumulators at columns 0 and 128, A stages (one K block each, T x 32
// columns) from column 256.
// ---------------------------------------------------------------------------
template <int T>
constexpr int xf128_fstages() { return T == 2 ? 4 : 3; }
template <int T>
constexpr int xf128_astages() { return T == 2 ? 4 : 2; }

template <int T, int F>
__global__ void __launch_bounds__(320, 1)
    xform128_kernel(const __grid_constant__ CUtensorMap map_t2, const __grid_constant__ CUtensorMap map_g,
                    const __grid_constant__ CUtensorMap map_t3s, int S, int sl0, int n_units, int *__restrict__ ex,
                    int *err) {
  constexpr int SF = xf128_fstages<T>(), SA = xf128_astages<T>();
  constexpr uint32_t B_SET = T * kOperand, A_COLS = T * 32, F_TILE = 64 * 128 * 4;  // [64 q][128 n] fp32
  constexpr uint32_t kIdesc = idesc_fmt(F, 128, 128, 0, 0);
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = align1024(smem_raw);
  uint8_t *sF = smem;
  uint8_t *sB = sF + SF * F_TILE;  // Gbar: [t][kb][128 p][64 q]
  uint8_t *sO = sB + B_SET;        // staging [2 boxes][128 rows][32 p]
  uint64_t *bar = reinterpret_cast<uint64_t *>(sO + kF32Half);
  uint64_t *f_full = bar, *f_empty = bar + SF, *a_full = bar + 2 * SF, *a_empty = a_full + SA;
  uint64_t *b_full = a_empty + SA, *b_empty = b_full + 1, *d_full = b_full + 2, *d_empty = b_full + 4;
  uint64_t *o_full = b_full + 6, *o_empty = b_full + 7;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(b_full + 8);
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
    tc::mbar_init(b_full, 1);
    tc::mbar_init(b_empty, 1);
    for (int s = 0; s < 2; ++s) {
      tc::mbar_init(&d_full[s], 1);
      tc::mbar_init(&d_empty[s], 4);
    }
    tc::mbar_init(o_full, 4);
    tc::mbar_init(o_empty, 1);
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
  const int u_begin = (int)((long long)blockIdx.x * n_units / gridDim.x);
  const int u_end = (int)((long long)(blockIdx.x + 1) * n_units / gridDim.x);

  if (warp == 0 && lane == 0) {
    const uint64_t stream_pol = tc::policy_evict_first();
    int f = 0, cur_c = -1, gcount = 0;
    bool ok = true;
    for (int u = u_begin; u < u_end && ok; ++u) {
      const int c = u / (P * P), i = (u / P) % P, l = u % P;
      if (c != cur_c) {
        if (gcount >= 1 && !tc::mbar_wait(b_empty, (gcount - 1) & 1, abort)) { raise_abort(abort, err); break; }
        tc::mbar_arrive_expect_tx(b_full, B_SET);
        for (int t = 0; t < T; ++t)
          for (int kb = 0; kb < 2; ++kb)
            tc::tma_load_3d(sB + (t * 2 + kb) * kTile, &map_g, b_full, 64 * kb, 0, (TMAX + t) * S + sl0 + c);
        cur_c = c;
        ++gcount;
      }
      for (int kb = 0; kb < 2; ++kb, ++f) {
        const int s = f % SF;
        if (f >= SF && !tc::mbar_wait(&f_empty[s], ((f / SF) - 1) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
        tc::mbar_arrive_expect_tx(&f_full[s], F_TILE);
        tc::tma_load_3d_hint(sF + s * F_TILE, &map_t2, &f_full[s], l * P, 64 * kb, c * P + i, stream_pol);
      }
    }
  } else if (warp == 1 && lane == 0) {
    int it = 0, f = 0, cur_c = -1, gcount = 0;
    bool ok = true;
    for (int u = u_begin; u < u_end && ok; ++u, ++it) {
      const int c = u / (P * P);
      if (c != cur_c) {
        if (cur_c >= 0) tc::mma_commit(b_empty);
        if (!tc::mbar_wait(b_full, gcount & 1, abort)) { raise_abort(abort, err); break; }
        cur_c = c;
        ++gcount;
      }
      const int d = it & 1;
      if (it >= 2 && !tc::mbar_wait(&d_empty[d], ((it >> 1) - 1) & 1, abort)) { raise_abort(abort, err); break; }
      for (int kb = 0; kb < 2; ++kb, ++f) {
        const int sa = f % SA;
        if (!tc::mbar_wait(&a_full[sa], (f / SA) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
        tc::tc_fence_after();
        const uint32_t a0 = tmem + 256 + sa * A_COLS, b0 = tc::smem_u32(sB);
        for (int pr = 0; pr < Products<T>::n; ++pr) {
          const int ta = Products<T>::a(pr), tb = Products<T>::b(pr);
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t bd = tc::smem_desc(b0 + (tb * 2 + kb) * kTile + kk * 32, 16, 1024);
            tc::mma_bf16_ts(tmem + d * 128, a0 + ta * 32 + kk * 8, bd, kIdesc, (pr | kb | kk) ? 1u : 0u);
          }
        }
        tc::mma_commit(&a_empty[sa]);
      }
      if (ok) tc::mma_commit(&d_full[d]);
    }
  } else if (warp >= 2 && warp < 6) {
    // epilogue: row n of D3 -> T3[c][i][l][n][p], 64 p per staging pass
    const int wq = warp & 3, row = wq * 32 + lane;
    const uint32_t lanes = (uint32_t)(wq * 32) << 16;
    int it = 0, pass = 0, run_c = -1;
    float run_mx = 0.f;
    bool ok = true;
    for (int u = u_begin; u < u_end && ok; ++u, ++it) {
      const int c = u / (P * P), i = (u / P) % P, l = u % P, d = it & 1;
      if (F != 0 && c != run_c) {
        if (run_c >= 0) warp_absmax_to(&ex[kMaxT3 * S + sl0 + run_c], run_mx);
        run_c = c;
        run_mx = 0.f;
      }
      if (!tc::mbar_wait(&d_full[d], (it >> 1) & 1, abort)) { raise_abort(abort, err); break; }
      tc::tc_fence_after();
      const float un = F == 0 ? 1.0f : exp2_scale(-fp16_exponent_bits(ex[kMaxT2 * S + sl0 + c]));
      for (int hh = 0; hh < 2; ++hh, ++pass) {
        float v[64];
        tc::tmem_ld_32x32b_x32(tmem + lanes + d * 128 + 64 * hh, v);
        tc::tmem_ld_32x32b_x32(tmem + lanes + d * 128 + 64 * hh + 32, v + 32);
        tc::tmem_ld_wait();
        if (hh == 1) {
          tc::tc_fence_before();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&d_empty[d]);
        }
        if constexpr (F != 0) {
#pragma unroll
          for (int k = 0; k < 64; ++k) {
            v[k] *= un;
            run_mx = fmaxf(run_mx, fabsf(v[k]));
          }
        }
        if (pass >= 1 && !tc::mbar_wait(o_empty, (pass - 1) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
        stage_row64(sO, row, v);
        tc::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(o_full);
        if (warp == 2) {
          if (!tc::mbar_wait(o_full, pass & 1, abort)) { raise_abort(abort, err); ok = false; break; }
          if (lane == 0) {
            for (int b = 0; b < 2; ++b) tc::tma_store_3d(&map_t3s, sO + b * kBox, 64 * hh + 32 * b, l * P, c * P + i);
            tc::tma_store_commit();
            tc::tma_store_wait_read();
            tc::mbar_arrive(o_empty);
          }
          __syncwarp();
        }
      }
    }
    if (F != 0 && run_c >= 0) warp_absmax_to(&ex[kMaxT3 * S + sl0 + run_c], run_mx);
    if (warp == 2 && lane == 0) tc::tma_store_wait_all();
  } else if (warp >= 6) {
    // converters: row n = TMEM lane; both K blocks of every unit in order, so
    // each F and A stage has exactly one consumer that takes its phases in turn
    const int wq = warp & 3, n = wq * 32 + lane;
    const uint32_t lanes = (uint32_t)(wq * 32) << 16;
    int f = 0;
    bool ok = true;
    for (int u = u_begin; u < u_end && ok; ++u) {
      const int c = u / (P * P);
      const float scale = F == 0 ? 1.0f : exp2_scale(fp16_exponent_bits(ex[kMaxT2 * S + sl0 + c]));
      for (int kb = 0; kb < 2; ++kb, ++f) {
        const int s = f % SF, sa = f % SA;
        if (!tc::mbar_wait(&f_full[s], (f / SF) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
        float x[64];
        const float *src = reinterpret_cast<const float *>(sF + s * F_TILE) + n;
#pragma unroll
        for (int q = 0; q < 64; ++q) x[q] = src[q * 128];
        tc::fence_proxy_async_smem();  // the next TMA write to this stage must follow these reads
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&f_empty[s]);
        if (f >= SA && !tc::mbar_wait(&a_empty[sa], ((f / SA) - 1) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
        __syncwarp();
        tc::tc_fence_after();
        split_row_to_tmem<T, F>(x, tmem + lanes + 256 + sa * A_COLS, scale);
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
// stage 4.  320 threads: warp 0 TMA, warp 1 MMA, warps 2-5 epilogue (lane
// quarter w % 4, all 128 columns), warps 6-9 converters: one warp per TMEM
// lane quarter writes TMEM in each role.
// TMEM: accumulators at columns 0 and 128, A stages from column 256.
// Every split product accumulates into the same FP32 group sum (two K steps).
// The epilogue adds each group sum into a running FP32 sum (hi, in registers)
// by TwoSum and writes the exact rounding error of that addition back into the
// accumulator, where the MMAs of the group after next (same buffer) add their
// products onto it: compensated summation with the error term carried in TMEM.
// A run of groups of one time point starts on fresh accumulators; at its end
// the last carry of each buffer goes to the output with the running sum.
// ---------------------------------------------------------------------------
constexpr int kCt128Group = 2;
constexpr int kCt128Steps = P * P / 64;  // K steps of one unit (one l)
template <int T>
constexpr int ct128_fstages() { return T == 2 ? 4 : 3; }
template <int T>
constexpr int ct128_wstages() { return T == 2 ? 3 : 2; }
template <int T>
constexpr int ct128_astages() { return T == 2 ? 4 : 2; }

template <int T, int F>
__global__ void __launch_bounds__(320, 1)
    contract128_kernel(const __grid_constant__ CUtensorMap map_t3, const __grid_constant__ CUtensorMap map_w,
                       double *__restrict__ out, int N, int count, int S, int sl0, int n_units,
                       const int *__restrict__ ex, int e_fixed, int *err) {
  constexpr int SF = ct128_fstages<T>(), SW = ct128_wstages<T>(), SA = ct128_astages<T>();
  constexpr uint32_t W_STAGE = T * kTile, A_COLS = T * 32;
  constexpr uint32_t kIdesc = idesc_fmt(F, 128, 128, 0, 0);
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = align1024(smem_raw);
  uint8_t *sF = smem;                 // [2 boxes][128 rows][32 k] fp32 per stage
  uint8_t *sW = sF + SF * kF32Half;   // [t][128 j][64 k] per stage
  uint64_t *bar = reinterpret_cast<uint64_t *>(sW + SW * W_STAGE);
  uint64_t *f_full = bar, *f_empty = bar + SF, *w_full = bar + 2 * SF, *w_empty = w_full + SW;
  uint64_t *a_full = w_empty + SW, *a_empty = a_full + SA, *d_full = a_empty + SA, *d_empty = d_full + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(d_empty + 2);
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
    for (int s = 0; s < 2; ++s) {
      tc::mbar_init(&d_full[s], 1);
      tc::mbar_init(&d_empty[s], 4);
    }
    tc::fence_barrier_init();
    s_abort = 0;
    tc::prefetch_tmap(&map_t3);
    tc::prefetch_tmap(&map_w);
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
    const uint64_t stream_pol = tc::policy_evict_first(), keep_pol = tc::policy_evict_last();
    int g = 0;
    bool ok = true;
    for (int u = u_begin; u < u_end && ok; ++u) {
      const int c = u / P, l = u % P;
      for (int ks = 0; ks < kCt128Steps; ++ks, ++g) {
        const int k0 = l * P * P + ks * 64;
        const int s = g % SF, sw = g % SW;
        if (g >= SF && !tc::mbar_wait(&f_empty[s], ((g / SF) - 1) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
        tc::mbar_arrive_expect_tx(&f_full[s], kF32Half);
        for (int h = 0; h < 2; ++h)
          tc::tma_load_3d_hint(sF + s * kF32Half + h * kBox, &map_t3, &f_full[s], k0 + 32 * h, c * P, 0, stream_pol);
        if (g >= SW && !tc::mbar_wait(&w_empty[sw], ((g / SW) - 1) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
        tc::mbar_arrive_expect_tx(&w_full[sw], W_STAGE);
        for (int t = 0; t < T; ++t)
          tc::tma_load_3d_hint(sW + sw * W_STAGE + t * kTile, &map_w, &w_full[sw], k0, 0, t, keep_pol);
      }
    }
  } else if (warp == 1 && lane == 0) {
    int g = 0, grp = 0, run = 0;  // run: group index within the run of one time point
    bool ok = true;
    for (int u = u_begin; u < u_end && ok; ++u) {
      if (u > u_begin && u / P != (u - 1) / P) run = 0;
      for (int gi = 0; gi < kCt128Steps / kCt128Group && ok; ++gi, ++grp, ++run) {
        const int db = grp & 1;
        const uint32_t carry = run >= 2 ? 1u : 0u;  // add onto the error left two groups ago
        if (grp >= 2 && !tc::mbar_wait(&d_empty[db], ((grp >> 1) - 1) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
        tc::tc_fence_after();
        for (int kq = 0; kq < kCt128Group; ++kq, ++g) {
          const int sa = g % SA, sw = g % SW;
          if (!tc::mbar_wait(&a_full[sa], (g / SA) & 1, abort) || !tc::mbar_wait(&w_full[sw], (g / SW) & 1, abort)) {
            raise_abort(abort, err);
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const uint32_t a0 = tmem + 256 + sa * A_COLS, b0 = tc::smem_u32(sW + sw * W_STAGE);
          for (int pr = 0; pr < Products<T>::n; ++pr) {
            const int ta = Products<T>::a(pr), tb = Products<T>::b(pr);
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t bd = tc::smem_desc(b0 + tb * kTile + kk * 32, 16, 1024);
              tc::mma_bf16_ts(tmem + db * 128, a0 + ta * 32 + kk * 8, bd, kIdesc, (carry | kq | pr | kk) ? 1u : 0u);
            }
          }
          tc::mma_commit(&a_empty[sa]);
          tc::mma_commit(&w_empty[sw]);
        }
        if (ok) tc::mma_commit(&d_full[db]);
      }
    }
  } else if (warp >= 2 && warp < 6) {
    const int wq = warp & 3, row = wq * 32 + lane;
    const uint32_t lanes = (uint32_t)(wq * 32) << 16;
    constexpr int NG = kCt128Steps / kCt128Group;
    float hi[128];
#pragma unroll
    for (int j = 0; j < 128; ++j) hi[j] = 0.f;
    int grp = 0;
    bool ok = true;
    for (int u = u_begin; u < u_end && ok; ++u) {
      const int c = u / P;
      const bool run_ends = u + 1 == u_end || (u + 1) / P != c;
      const bool valid = row < N && c < count;
      const double unscale =
          F == 0 ? 1.0
                 : ldexp(1.0, -(e_fixed + 2 * ex[kExpG * S + sl0 + c] + ex[kExpGbar * S + sl0 + c] +
                                fp16_exponent_bits(ex[kMaxT3 * S + sl0 + c])));
      double *o = out + ((long long)c * N + row) * N;
      for (int gi = 0; gi < NG; ++gi, ++grp) {
        const int db = grp & 1;
        // the last two groups of the run: their errors go to the output, not to TMEM
        const int tail = run_ends ? (gi == NG - 1 ? 2 : (gi == NG - 2 ? 1 : 0)) : 0;
        if (!tc::mbar_wait(&d_full[db], (grp >> 1) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
        __syncwarp();
        tc::tc_fence_after();
#pragma unroll
        for (int hh = 0; hh < 8; ++hh) {
          float v[16];
          tc::tmem_ld_32x32b_x16(tmem + lanes + db * 128 + 16 * hh, v);
          tc::tmem_ld_wait();
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const float a = hi[16 * hh + jj], x = v[jj];
            const float s = __fadd_rn(a, x);
            const float bp = __fsub_rn(s, a);
            v[jj] = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(x, bp));  // a + x = s + v exactly
            hi[16 * hh + jj] = s;
          }
          if (tail) {
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
              const int j = 16 * hh + jj;
              const double add = tail == 2 ? (double)hi[j] + (double)v[jj] : (double)v[jj];
              if (valid && j < N) atomicAdd(o + j, -add * unscale);
              v[jj] = 0.f;
              if (tail == 2) hi[j] = 0.f;
            }
          }
          uint32_t w[16];
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) w[jj] = __float_as_uint(v[jj]);
          tc::tmem_st_32x32b_x16(tmem + lanes + db * 128 + 16 * hh, w);
        }
        tc::tmem_st_wait();
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&d_empty[db]);
      }
    }
  } else if (warp >= 6) {
    // converters: row r = TMEM lane; half h of the FP32 tile holds k = 32 h .. +31
    // of all rows, 128 bytes a row, 16-byte chunk j of row r at chunk j ^ (r % 8)
    const int wq = warp & 3, r = wq * 32 + lane;
    const uint32_t lanes = (uint32_t)(wq * 32) << 16;
    int g = 0;
    bool ok = true;
    for (int u = u_begin; u < u_end && ok; ++u) {
      const int c = u / P;
      const float scale = F == 0 ? 1.0f : exp2_scale(fp16_exponent_bits(ex[kMaxT3 * S + sl0 + c]));
      for (int ks = 0; ks < kCt128Steps; ++ks, ++g) {
        const int s = g % SF, sa = g % SA;
        if (!tc::mbar_wait(&f_full[s], (g / SF) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
        float x[64];
        const uint8_t *row_base = sF + s * kF32Half + r * 128;
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int cch = 0; cch < 8; ++cch) {
            const float4 q = *reinterpret_cast<const float4 *>(row_base + h * kBox + ((cch ^ (r & 7)) << 4));
            x[32 * h + 4 * cch] = q.x;
            x[32 * h + 4 * cch + 1] = q.y;
            x[32 * h + 4 * cch + 2] = q.z;
            x[32 * h + 4 * cch + 3] = q.w;
          }
        tc::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&f_empty[s]);
        if (g >= SA && !tc::mbar_wait(&a_empty[sa], ((g / SA) - 1) & 1, abort)) { raise_abort(abort, err); ok = false; break; }
        tc::tc_fence_after();
        split_row_to_tmem<T, F>(x, tmem + lanes + 256 + sa * A_COLS, scale);
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
// host side
// ---------------------------------------------------------------------------
struct TcState128 {
  int C = 0;                           // time points per chunk
  int S = 0;                           // slots of the whole grid (a multiple of C)
  uint16_t *Gs = nullptr;              // [2][TMAX][S][128][128]: G(tau)^T and Gbar terms
  int *gexp = nullptr;                 // [kExpSets][S]
  float *T2 = nullptr, *T3 = nullptr;  // C * 128^4 each
  CUtensorMap map_v, map_v16, map_g, map_t2, map_t2s, map_t3, map_t3s, map_w, map_w16;
};

template <int T>
size_t smem_sw128() {
  return 1024 + (size_t)T * kOperand * (1 + sw128_vstages<T>()) + kF32Half + 256;
}
template <int T>
size_t smem_xf128() {
  return 1024 + (size_t)xf128_fstages<T>() * 64 * 128 * 4 + (size_t)T * kOperand + kF32Half + 256;
}
template <int T>
size_t smem_ct128() {
  return 1024 + (size_t)ct128_fstages<T>() * kF32Half + (size_t)ct128_wstages<T>() * T * kTile + 256;
}

TcState128 *state(gf2_ctx *ctx) { return reinterpret_cast<TcState128 *>(ctx->d_tc128_ws); }

void free_state(TcState128 *s) {
  if (!s) return;
  cudaFree(s->Gs);
  cudaFree(s->gexp);
  cudaFree(s->T2);
  cudaFree(s->T3);
  delete s;
}

template <int T, int F>
gf2_status run128(gf2_ctx *ctx, TcState128 *s, const double *d_G, int k0, int count, double *d_out) {
  const int N = ctx->N, C = s->C, S = s->S, sms = ctx->num_sms;
  const size_t ssw = smem_sw128<T>(), sxf = smem_xf128<T>(), sct = smem_ct128<T>();
  GF2_CK(ctx, cudaFuncSetAttribute(sandwich128_kernel<T, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssw));
  GF2_CK(ctx, cudaFuncSetAttribute(xform128_kernel<T, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sxf));
  GF2_CK(ctx, cudaFuncSetAttribute(contract128_kernel<T, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sct));
  const CUtensorMap &map_v = F == 0 ? s->map_v : s->map_v16, &map_w = F == 0 ? s->map_w : s->map_w16;
  const int e_fixed = F == 0 ? 0 : ctx->e_v16 + ctx->e_w16;
  if (count <= 0) return GF2_OK;
  const int n_chunks = (count + C - 1) / C;
  GF2_PROF(ctx, GF2_K_SPLIT, (split_g_kernel<P, F><<<dim3(n_chunks * C, 2), 256, 0, ctx->stream>>>(
                                 N, 1, ctx->n_tau - 1, k0, count, S, d_G, s->Gs, s->gexp, ctx->vmax16)));
  GF2_CK_LAUNCH(ctx, "split_g_kernel");
  GF2_CK(ctx, cudaMemsetAsync(d_out, 0, sizeof(double) * (size_t)count * N * N, ctx->stream));
  for (int c0 = 0, sl0 = 0; c0 < count; c0 += C, sl0 += C) {
    const int cnt = std::min(C, count - c0);
    double *out = d_out + (size_t)c0 * N * N;
    const int u12 = cnt * P * P, sym = ctx->tc_pair_sym ? 1 : 0;
    const int u12s = sym ? cnt * kSym128Units : u12;
    GF2_PROF(ctx, GF2_K_SANDWICH,
             (sandwich128_kernel<T, F><<<std::min(u12s, sms), 320, ssw, ctx->stream>>>(
                 map_v, s->map_g, s->map_t2s, S, sl0, u12s, s->gexp, ctx->d_err, sym, s->T2)));
    GF2_CK_LAUNCH(ctx, "sandwich128_kernel");
    GF2_PROF(ctx, GF2_K_XFORM,
             (xform128_kernel<T, F><<<std::min(u12, sms), 320, sxf, ctx->stream>>>(
                 s->map_t2, s->map_g, s->map_t3s, S, sl0, u12, s->gexp, ctx->d_err)));
    GF2_CK_LAUNCH(ctx, "xform128_kernel");
    const int u3 = cnt * P;
    GF2_PROF(ctx, GF2_K_CONTRACT,
             (contract128_kernel<T, F><<<std::min(u3, sms), 320, sct, ctx->stream>>>(
                 s->map_t3, map_w, out, N, cnt, S, sl0, u3, s->gexp, e_fixed, ctx->d_err)));
    GF2_CK_LAUNCH(ctx, "contract128_kernel");
  }
  return GF2_OK;
}

}  // namespace

gf2_status gf2_tc128_workspace(gf2_ctx *ctx) {
  if (ctx->d_tc128_ws) return GF2_OK;
  TcState128 *s = new (std::nothrow) TcState128();
  if (!s) return gf2_fail(ctx, GF2_ERR_NOMEM, "tc128 state");
  // chunk: up to 16 time points (2 x 16 GB of FP32 intermediates), fewer if
  // the device has less room
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = 0;
  const size_t per_slot = 2 * kPlane4 * sizeof(float);
  int C = std::min(ctx->tc_chunk_max / 2, ctx->n_tau);
  while (C > 1 && (size_t)C * per_slot + ((size_t)2 << 30) > free_b) C /= 2;
  C = std::max(1, C);
  s->C = C;
  s->S = ((ctx->n_tau + C - 1) / C) * C;
  const int S = s->S;
  const size_t gbytes = (size_t)2 * TMAX * S * P * P * sizeof(uint16_t);
  const size_t ibytes = (size_t)C * kPlane4 * sizeof(float);
  cudaError_t e = cudaMalloc(&s->Gs, gbytes);
  if (e == cudaSuccess) e = cudaMalloc(&s->gexp, kExpSets * S * sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(s->gexp, 0, kExpSets * S * sizeof(int), ctx->stream);
  if (e == cudaSuccess) e = cudaMalloc(&s->T2, ibytes);
  if (e == cudaSuccess) e = cudaMalloc(&s->T3, ibytes);
  if (e != cudaSuccess) {
    free_state(s);
    return gf2_cuda_fail(ctx, e, "tc128 workspace");
  }
  bool ok = true;
  {  // v: dims (k, m, q, i, t), box (64, 128, 1, 1, 1) -> [128 m][64 k] of one (i, q)
    uint64_t dims[5] = {P, P, P, P, TMAX};
    uint64_t str[4] = {P * 2, P * P * 2, (uint64_t)P * P * P * 2, kPlane4 * 2};
    uint32_t box[5] = {64, 128, 1, 1, 1};
    ok &= make_map(&s->map_v, ctx->d_v_split, 5, dims, str, box);
    ok &= make_map(&s->map_v16, ctx->d_v_split16, 5, dims, str, box);
  }
  {  // G sets of every slot: dims (128, 128, 2*TMAX*S), box (64, 128, 1)
    uint64_t dims[3] = {P, P, (uint64_t)2 * TMAX * S};
    uint64_t str[2] = {P * 2, P * P * 2};
    uint32_t box[3] = {64, 128, 1};
    ok &= make_map(&s->map_g, s->Gs, 3, dims, str, box);
  }
  {  // T2 (fp32) for stage 3: dims ((l,n) 16384, q 128, (c,i) C*128), box (128, 64, 1) -> [64 q][128 n]
    uint64_t dims[3] = {P * P, P, (uint64_t)C * P};
    uint64_t str[2] = {P * P * 4, (uint64_t)P * P * P * 4};
    uint32_t box[3] = {128, 64, 1};
    ok &= make_map(&s->map_t2, s->T2, 3, dims, str, box, true);
  }
  {  // T2 as stored by stages 1+2: dims (n 128, (q,l) 16384, (c,i) C*128), box (32, 128, 1), swizzled
    uint64_t dims[3] = {P, P * P, (uint64_t)C * P};
    uint64_t str[2] = {P * 4, (uint64_t)P * P * P * 4};
    uint32_t box[3] = {32, 128, 1};
    ok &= make_map(&s->map_t2s, s->T2, 3, dims, str, box, true, true);
  }
  {  // T3 for stage 4: dims (K = 128^3, rows (c,i) C*128, 1), box (32, 128, 1), swizzled
    uint64_t dims[3] = {(uint64_t)P * P * P, (uint64_t)C * P, 1};
    uint64_t str[2] = {(uint64_t)P * P * P * 4, (uint64_t)C * kPlane4 * 4};
    uint32_t box[3] = {32, 128, 1};
    ok &= make_map(&s->map_t3, s->T3, 3, dims, str, box, true, true);
  }
  {  // T3 as stored by stage 3: dims (p 128, (l,n) 16384, (c,i) C*128), box (32, 128, 1), swizzled
    uint64_t dims[3] = {P, P * P, (uint64_t)C * P};
    uint64_t str[2] = {P * 4, (uint64_t)P * P * P * 4};
    uint32_t box[3] = {32, 128, 1};
    ok &= make_map(&s->map_t3s, s->T3, 3, dims, str, box, true, true);
  }
  {  // W: dims (K = 128^3, j 128, t), box (64, 128, 1)
    uint64_t dims[3] = {(uint64_t)P * P * P, P, TMAX};
    uint64_t str[2] = {(uint64_t)P * P * P * 2, kPlane4 * 2};
    uint32_t box[3] = {64, 128, 1};
    ok &= make_map(&s->map_w, ctx->d_wt_split, 3, dims, str, box);
    ok &= make_map(&s->map_w16, ctx->d_wt_split16, 3, dims, str, box);
  }
  if (!ok) {
    free_state(s);
    return gf2_fail(ctx, GF2_ERR_CUDA, "cuTensorMapEncodeTiled failed (128-wide tiles)");
  }
  ctx->d_tc128_ws = s;
  ctx->tc_chunk = C;
  return GF2_OK;
}

void gf2_tc128_release(gf2_ctx *ctx) {
  free_state(state(ctx));
  ctx->d_tc128_ws = nullptr;
}

gf2_status gf2_tc128_run(gf2_ctx *ctx, const double *d_G, int k0, int count, double *d_out, int prec) {
  TcState128 *s = state(ctx);
  if (!s) return gf2_fail(ctx, GF2_ERR_ARG, "tc128: no workspace");
  switch (prec) {
    case GF2_PREC_BF16X3: return run128<2, 0>(ctx, s, d_G, k0, count, d_out);
    case GF2_PREC_BF16X6: return run128<3, 0>(ctx, s, d_G, k0, count, d_out);
    case GF2_PREC_FP16X3: return run128<2, 1>(ctx, s, d_G, k0, count, d_out);
    default: return run128<3, 1>(ctx, s, d_G, k0, count, d_out);
  }
}
