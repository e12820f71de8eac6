// Eq. GF (per-frequency Dyson inverse), the density matrix, the chemical
// potential search (step 2.a), Eq. FockMatrix (step 2.b), the tail moments of
// G and the Galitskii-Migdal energy, all in FP64.
//
// Tail moments.  With X = F - mu S the moments are polynomials in mu:
//   G1 = A0,  G2 = A1 - mu A0,  G3 = A2 - 2mu A1 + mu^2 A0 + B1,
//   G4 = A3 - 3mu A2 + 3mu^2 A1 - mu^3 A0 + B2 - 2mu B1 + B3,
// A0 = S^-1, A_{r+1} = S^-1 F A_r, B1 = S^-1 Sig1 S^-1,
// B2 = S^-1 F B1 + B1 F S^-1, B3 = S^-1 Sig2 S^-1,
// so one set of N^3 products per (F, Sig1, Sig2) serves every mu of a search.
//
// Dyson.  A(i w) = (i w + mu) S - F - Sigma(i w) is complex symmetric with
// Im A = w S - Im Sigma positive definite for w > 0 (Im Sigma(i w) <= 0 for a
// causal self-energy), so elimination without pivoting is stable; pivots are
// still checked and a tiny one is reported as GF2_ERR_NONFINITE.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "gf2_internal.cuh"

namespace {

enum { SL_SINV = GF2_SL_SINV, SL_A1 = GF2_SL_A1, SL_A2 = GF2_SL_A2, SL_A3 = GF2_SL_A3,
       SL_B1 = GF2_SL_B1, SL_B2 = GF2_SL_B2, SL_B3 = GF2_SL_B3, SL_T1 = GF2_SL_T1, SL_TMP = GF2_SL_TMP,
       SL_MOM = GF2_SL_MOM, SL_COEF = GF2_SL_COEF, SL_MISC = GF2_SL_MISC };

using MuState = gf2_mu_state;

__global__ void pole_coef_kernel(int N2, double a, const double *mom, double *coef) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N2) return;
  const double g1 = mom[e], g2 = mom[N2 + e], g3 = mom[2 * N2 + e], g4 = mom[3 * N2 + e];
  coef[e] = g1;
  coef[N2 + e] = g2 - a * g1;
  coef[2 * N2 + e] = g3 - 2.0 * a * g2 + a * a * g1;
  coef[3 * N2 + e] = g4 - 3.0 * a * g3 + 3.0 * a * a * g2 - a * a * a * g1;
}

__global__ void moments_kernel(int N2, double mu, const double *basis, double *mom, const MuState *st = nullptr) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N2) return;
  if (st) mu = st->mu;
  const double A0 = basis[SL_SINV * N2 + e], A1 = basis[SL_A1 * N2 + e];
  const double A2 = basis[SL_A2 * N2 + e], A3 = basis[SL_A3 * N2 + e];
  const double B1 = basis[SL_B1 * N2 + e], B2 = basis[SL_B2 * N2 + e], B3 = basis[SL_B3 * N2 + e];
  mom[e] = A0;
  mom[N2 + e] = A1 - mu * A0;
  mom[2 * N2 + e] = A2 - 2.0 * mu * A1 + mu * mu * A0 + B1;
  mom[3 * N2 + e] = A3 - 3.0 * mu * A2 + 3.0 * mu * mu * A1 - mu * mu * mu * A0 + B2 - 2.0 * mu * B1 + B3;
}

// Inverse of the complex symmetric A(i w_n) by symmetric sweeps (Gauss-Jordan
// without pivoting, which keeps A symmetric at every step): sweeping pivot k
// maps a_kk -> -1/a_kk, a_ik -> a_ik/a_kk and a_ij -> a_ij - a_ik a_kj / a_kk;
// after all N pivots the matrix holds -A^-1.  Only the upper triangle is
// updated (N^3/2 complex multiply-adds instead of N^3); it is loaded as the
// symmetric part (A_ij + A_ji)/2, so inputs whose triangles differ by
// rounding (a split-precision Sigma) enter through their symmetric part.  Each thread keeps its
// share of the triangle in registers; the pivot column is published through
// shared memory once per step.  One CTA per frequency.
constexpr int kDysonThreads = 512;
constexpr int kDysonMaxPerThread = (GF2_MAX_N * (GF2_MAX_N + 1) / 2 + kDysonThreads - 1) / kDysonThreads;

// MINB = 2 (at most 64 registers) for the narrow layouts, so that two CTAs
// share an SM and one's barrier waits overlap the other's sweep.
template <int PER, int MINB>
__global__ void __launch_bounds__(kDysonThreads, MINB)
    dyson_kernel(int N, double beta, double mu, const double *__restrict__ S, const double *__restrict__ F,
                 const double2 *__restrict__ Sig, double2 *__restrict__ G, int *flag,
                 const MuState *st = nullptr) {
  if (st) {  // the device-resident search: mu and the frequency count come from its state
    if ((int)blockIdx.x >= st->nf) return;
    mu = st->mu;
  }
  __shared__ double2 v[GF2_MAX_N];  // pivot column a_ik
  __shared__ double2 w[GF2_MAX_N];  // a_ik / a_kk
  __shared__ double2 pinv;
  __shared__ int bad;
  const int N2 = N * N;
  const long long n = blockIdx.x;
  const double om = (2.0 * n + 1.0) * M_PI / beta;
  const int ntri = N * (N + 1) / 2;
  double2 a[PER];
  int ij[PER];  // (i << 8) | j, or -1
  if (threadIdx.x == 0) bad = 0;
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int e = threadIdx.x + r * kDysonThreads;
    ij[r] = -1;
    a[r] = make_double2(0.0, 0.0);
    if (e < ntri) {
      // row-major upper triangle: row i holds N - i elements
      int i = 0, rem = e;
      while (rem >= N - i) {
        rem -= N - i;
        ++i;
      }
      const int j = i + rem;
      ij[r] = (i << 8) | j;
      // the symmetric part of A (S, F and Sigma are symmetric up to rounding)
      const int idx = i * N + j, idt = j * N + i;
      const double sv = 0.5 * (S[idx] + S[idt]);
      double2 x = make_double2(mu * sv - 0.5 * (F[idx] + F[idt]), om * sv);
      if (Sig) x = csub(x, cscale(cadd(Sig[n * N2 + idx], Sig[n * N2 + idt]), 0.5));
      a[r] = x;
    }
  }
  for (int k = 0; k < N; ++k) {
    // 1. publish the pivot column v_i = a_ik (= a_ki) and 1/a_kk
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      if (ij[r] < 0) continue;
      const int i = ij[r] >> 8, j = ij[r] & 255;
      if (j == k) {
        v[i] = a[r];
        if (i == k) {
          if (!(fabs(a[r].x) + fabs(a[r].y) > 1e-280)) bad = 1;
          pinv = crecip(a[r]);
        }
      } else if (i == k) {
        v[j] = a[r];
      }
    }
    __syncthreads();
    // 2. scaled pivot column w_i = a_ik / a_kk
    const double2 p = pinv;
    for (int i = threadIdx.x; i < N; i += blockDim.x) w[i] = cmul(v[i], p);
    __syncthreads();
    // 3. rank-1 update of the upper triangle, a_ij -= w_i a_kj (four FP64 FMAs)
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      if (ij[r] < 0) continue;
      const int i = ij[r] >> 8, j = ij[r] & 255;
      if (i == k || j == k) {
        if (i == j) a[r] = make_double2(-p.x, -p.y);
        else a[r] = w[i == k ? j : i];
      } else {
        const double2 wi = w[i], vj = v[j];
        double2 x = a[r];
        x.x = fma(-wi.x, vj.x, x.x);
        x.x = fma(wi.y, vj.y, x.x);
        x.y = fma(-wi.x, vj.y, x.y);
        x.y = fma(-wi.y, vj.x, x.y);
        a[r] = x;
      }
    }
    __syncthreads();
  }
  if (bad && threadIdx.x == 0) atomicExch(flag, 1);
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    if (ij[r] < 0) continue;
    const int i = ij[r] >> 8, j = ij[r] & 255;
    const double2 g = make_double2(-a[r].x, -a[r].y);
    G[n * N2 + (size_t)i * N + j] = g;
    if (i != j) G[n * N2 + (size_t)j * N + i] = g;
  }
}

// partial[chunk][e] = sum_{n in chunk} Re G_e(n)
__global__ void density_partial_kernel(int N2, int n_iw, int chunk, const double2 *__restrict__ G,
                                       double *__restrict__ partial, const MuState *st = nullptr) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N2) return;
  const int c = blockIdx.y;
  if (st) {
    n_iw = st->nf;
    if (c * chunk >= n_iw) return;
  }
  const int n0 = c * chunk, n1 = min(n_iw, n0 + chunk);
  double acc = 0.0;
  for (int n = n0; n < n1; ++n) acc += G[(size_t)n * N2 + e].x;
  partial[(size_t)c * N2 + e] = acc;
}

// P_e = (4/beta) [sum_n Re G_e - sum_r c_r R_r] - 2 sum_r c_r g_r(beta)
__global__ void density_final_kernel(int N2, int nchunks, double beta, const double *partial,
                                     const double *coef, const double *pole_resum,
                                     const double *tau_pole_beta, double *P, const MuState *st = nullptr,
                                     const double *pole_resum_coarse = nullptr) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N2) return;
  if (st) {  // chunks of 256 frequencies over the evaluation's range, its tail sums
    nchunks = (st->nf + 255) / 256;
    if (st->stage == 0) pole_resum = pole_resum_coarse;
  }
  double s = 0.0;
  for (int c = 0; c < nchunks; ++c) s += partial[(size_t)c * N2 + e];
  double tail_sum = 0.0, tail_beta = 0.0;
  for (int r = 0; r < 4; ++r) {
    const double cr = coef[(size_t)r * N2 + e];
    tail_sum += cr * pole_resum[r];
    tail_beta += cr * tau_pole_beta[r];
  }
  P[e] = (4.0 / beta) * (s - tail_sum) - 2.0 * tail_beta;
}

// out[0] = sum_ij P_ij S_ji (single CTA, fixed order)
__global__ void trace_kernel(int N, const double *P, const double *S, double *out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int i = e / N, j = e - i * N;
    acc += P[e] * S[j * N + i];
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

// ---------------------------------------------------------------------------
// Device-resident chemical-potential search.  One evaluation of the count
// N(mu) - n_elec (moments, pole coefficients, Dyson, density, trace) is the
// body of a CUDA-graph WHILE loop; after it, mu_control_kernel (one thread)
// takes the decision the host would take -- bracket outward from the start,
// then Brent's method (inverse quadratic interpolation or secant steps with
// bisection safeguards, Brent 1973, "Algorithms for Minimization without
// Derivatives", ch. 4), first on the count over the lowest n_iw/8 frequencies
// and then on the full count -- writes the next mu into the state, and ends
// the loop when the tolerance is met, the evaluation cap is reached or a count
// is not finite.  The host reads the state once, after the graph.
// ---------------------------------------------------------------------------
__device__ void mu_solve_begin(MuState *s, double mu0, double slope_hint, double tol_f, int cap, int nf) {
  s->phase = 0;
  s->n = 0;
  s->have_prev = 0;
  s->slope_hint = slope_hint;
  s->tol_f = tol_f;
  s->cap = cap;
  s->nf = nf;
  s->mu = mu0;
}

// the end of one solve (coarse or full): the last point, found or not
__device__ void mu_solve_end(MuState *s, bool found) {
  const double slope =
      (s->have_prev && s->last_mu != s->prev_mu) ? (s->last_f - s->prev_f) / (s->last_mu - s->prev_mu) : 0.0;
  if (s->stage == 0) {  // coarse: the full search starts at its root, with its slope
    const double mu_start = (found && isfinite(s->last_mu)) ? s->last_mu : s->mu_out;
    s->stage = 1;
    mu_solve_begin(s, mu_start, found ? slope : 0.0, s->tol, s->max_iter, s->n_iw);
  } else {
    s->mu_out = s->last_mu;
    s->status = found ? 1 : 2;
    s->stage = 2;
  }
}

// one Brent step on the bracket [b, c]: sets the next point, or ends the solve
__device__ void mu_brent_next(MuState *s) {
  if (s->n >= s->cap) {
    mu_solve_end(s, false);
    return;
  }
  if ((s->fb > 0.0) == (s->fc > 0.0)) {
    s->c = s->a;
    s->fc = s->fa;
    s->d = s->e = s->b - s->a;
  }
  if (fabs(s->fc) < fabs(s->fb)) {
    s->a = s->b; s->b = s->c; s->c = s->a;
    s->fa = s->fb; s->fb = s->fc; s->fc = s->fa;
  }
  const double tol1 = 2.0 * 2.2e-16 * fabs(s->b) + 1e-16;
  const double xm = 0.5 * (s->c - s->b);
  if (fabs(xm) <= tol1) {  // bracket collapsed without reaching the tolerance
    mu_solve_end(s, false);
    return;
  }
  if (fabs(s->e) >= tol1 && fabs(s->fa) > fabs(s->fb)) {
    const double sq = s->fb / s->fa;
    double p, q;
    if (s->a == s->c) {
      p = 2.0 * xm * sq;
      q = 1.0 - sq;
    } else {
      const double qq = s->fa / s->fc, r = s->fb / s->fc;
      p = sq * (2.0 * xm * qq * (qq - r) - (s->b - s->a) * (r - 1.0));
      q = (qq - 1.0) * (r - 1.0) * (sq - 1.0);
    }
    if (p > 0.0) q = -q;
    p = fabs(p);
    if (2.0 * p < fmin(3.0 * xm * q - fabs(tol1 * q), fabs(s->e * q))) {
      s->e = s->d;
      s->d = p / q;
    } else {
      s->d = xm;
      s->e = s->d;
    }
  } else {
    s->d = xm;
    s->e = s->d;
  }
  s->a = s->b;
  s->fa = s->fb;
  s->b += (fabs(s->d) > tol1) ? s->d : (xm > 0.0 ? tol1 : -tol1);
  s->mu = s->b;
}

// enter Brent's method on the bracket [lo, hi] (f(lo) < 0 < f(hi))
__device__ void mu_brent_start(MuState *s) {
  s->phase = 3;
  s->a = s->lo; s->fa = s->flo; s->b = s->hi; s->fb = s->fhi;
  if (fabs(s->fa) < fabs(s->fb)) {
    double t = s->a; s->a = s->b; s->b = t;
    t = s->fa; s->fa = s->fb; s->fb = t;
  }
  s->c = s->a;
  s->fc = s->fa;
  s->d = s->b - s->a;
  s->e = s->d;
  mu_brent_next(s);
}

__device__ void mu_init(MuState *s, double mu0, double n_elec, double tol, int max_iter, int n_iw, int n_coarse) {
  s->n_elec = n_elec;
  s->tol = tol;
  s->tol_coarse = fmax(tol, 1e-9);
  s->max_iter = max_iter;
  s->cap_coarse = 60;
  s->n_iw = n_iw;
  s->n_coarse = n_coarse;
  s->status = 0;
  s->evals = 0;
  s->mu_out = mu0;
  s->stage = n_coarse > 0 ? 0 : 1;
  if (n_coarse > 0) mu_solve_begin(s, mu0, 0.0, s->tol_coarse, s->cap_coarse, n_coarse);
  else mu_solve_begin(s, mu0, 0.0, tol, max_iter, n_iw);
}

__global__ void mu_init_kernel(MuState *s, double mu0, double n_elec, double tol, int max_iter, int n_iw,
                               int n_coarse, int *flag) {
  if (threadIdx.x != 0) return;
  mu_init(s, mu0, n_elec, tol, max_iter, n_iw, n_coarse);
  *flag = 0;
}

// the same inside a graph: the start value and the search parameters come from
// device memory, prm = {mu0, n_elec, tol, max_iter}, and the loop that follows
// is armed (a WHILE node nested in another loop's body keeps the value its
// last run left)
__global__ void mu_start_kernel(MuState *s, const double *prm, int n_iw, int n_coarse, int *flag,
                                cudaGraphConditionalHandle loop) {
  if (threadIdx.x != 0) return;
  mu_init(s, prm[0], prm[1], prm[2], (int)prm[3], n_iw, n_coarse);
  *flag = 0;
  cudaGraphSetConditional(loop, 1u);
}

// after an evaluation at s->mu: record it and choose the next point
__global__ void mu_control_kernel(MuState *s, const double *count, const int *flag,
                                  cudaGraphConditionalHandle loop) {
  if (threadIdx.x != 0) return;
  const double f = count[0] - s->n_elec;
  ++s->evals;
  if (*flag) {
    s->status = 4;
    s->stage = 2;
  } else if (!isfinite(f)) {
    s->status = 3;
    s->stage = 2;
  } else {
    ++s->n;
    if (s->n > 1) {
      s->prev_mu = s->last_mu;
      s->prev_f = s->last_f;
      s->have_prev = 1;
    }
    s->last_mu = s->mu;
    s->last_f = f;
    if (fabs(f) <= s->tol_f) {
      mu_solve_end(s, true);
    } else if (s->phase == 0) {
      // N(mu) increases with mu; with a slope hint the first probe is the Newton step
      const double h = s->slope_hint;
      s->step = (h > 0.0 && isfinite(h)) ? fmin(0.05, fmax(1e-12, fabs(f) / h)) : 0.05;
      if (f < 0.0) {
        s->lo = s->mu; s->flo = f; s->hi = s->mu + s->step; s->phase = 1; s->mu = s->hi;
      } else {
        s->hi = s->mu; s->fhi = f; s->lo = s->mu - s->step; s->phase = 2; s->mu = s->lo;
      }
      if (s->n >= s->cap) mu_solve_end(s, false);
    } else if (s->phase == 1) {
      s->fhi = f;
      if (f > 0.0) {
        mu_brent_start(s);
      } else {
        s->lo = s->hi; s->flo = f; s->step *= 2.0; s->hi += s->step; s->mu = s->hi;
        if (s->n >= s->cap) mu_solve_end(s, false);
      }
    } else if (s->phase == 2) {
      s->flo = f;
      if (f < 0.0) {
        mu_brent_start(s);
      } else {
        s->hi = s->lo; s->fhi = f; s->step *= 2.0; s->lo -= s->step; s->mu = s->lo;
        if (s->n >= s->cap) mu_solve_end(s, false);
      }
    } else {
      s->fb = f;
      mu_brent_next(s);
    }
  }
  cudaGraphSetConditional(loop, s->stage == 2 ? 0u : 1u);
}

// Eq. FockMatrix, F = h + J - K/2 with J_ij = sum_kl P_kl v_ijlk and
// K_ij = sum_kl P_kl v_iklj, in one pass over v (HBM-bound: N^4 doubles read
// once).  Element v[a,b,c,d] adds v P[d,c] to J[a,b] and P[b,c] v to K[a,d].
// CTA (a, block of b rows): warp w takes rows c = w, w + 8, ... of v[a,b],
// lane l the columns d = l + 32 q (q < 4, N <= 128), four rows in flight per
// warp.  P^T sits in shared memory, so the column read P[d,c] is conflict-free.
// F holds h on entry (copied before the launch); each CTA adds its J entries
// and its partial K row by FP64 atomics.
constexpr int kFockThreads = 256, kFockWarps = kFockThreads / 32, kFockQ = 4, kFockUnroll = 4;
static_assert(GF2_MAX_N <= 32 * kFockQ, "fock_kernel covers N <= 32 kFockQ columns");

__global__ void __launch_bounds__(kFockThreads)
    fock_kernel(int N, int b_per_cta, const double *__restrict__ v, const double *__restrict__ P,
                double *__restrict__ F) {
  extern __shared__ double fock_sm[];
  double *Pt = fock_sm;                          // [N][N]: Pt[c N + d] = P[d N + c]
  double *jred = Pt + N * N;                     // [warps][b_per_cta]
  double *kred = jred + kFockWarps * b_per_cta;  // [warps][N]
  const int a = blockIdx.x, b0 = blockIdx.y * b_per_cta, b1 = min(N, b0 + b_per_cta);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (int e = threadIdx.x; e < N * N; e += kFockThreads) {
    const int d = e / N, c = e - d * N;
    Pt[c * N + d] = P[e];
  }
  __syncthreads();
  double kacc[kFockQ] = {};
  for (int b = b0; b < b1; ++b) {
    const double *vb = v + ((size_t)a * N + b) * N * N;  // v[a, b, :, :]
    double jpart = 0.0;
    for (int c0 = warp; c0 < N; c0 += kFockWarps * kFockUnroll) {
      double x[kFockUnroll][kFockQ];
#pragma unroll
      for (int u = 0; u < kFockUnroll; ++u) {
        const int c = c0 + u * kFockWarps;
#pragma unroll
        for (int q = 0; q < kFockQ; ++q) {
          const int d = lane + 32 * q;
          x[u][q] = (c < N && d < N) ? vb[(size_t)c * N + d] : 0.0;
        }
      }
#pragma unroll
      for (int u = 0; u < kFockUnroll; ++u) {
        const int c = c0 + u * kFockWarps;
        if (c >= N) break;
        const double pbc = Pt[c * N + b];  // P[b, c]
#pragma unroll
        for (int q = 0; q < kFockQ; ++q) {
          const int d = lane + 32 * q;
          if (d < N) {
            jpart = fma(x[u][q], Pt[c * N + d], jpart);  // v[a,b,c,d] P[d,c]
            kacc[q] = fma(pbc, x[u][q], kacc[q]);        // P[b,c] v[a,b,c,d]
          }
        }
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) jpart += __shfl_xor_sync(0xffffffffu, jpart, off);
    if (lane == 0) jred[warp * b_per_cta + (b - b0)] = jpart;
  }
#pragma unroll
  for (int q = 0; q < kFockQ; ++q) {
    const int d = lane + 32 * q;
    if (d < N) kred[warp * N + d] = kacc[q];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < N; t += kFockThreads) {
    double k = 0.0;
    for (int w = 0; w < kFockWarps; ++w) k += kred[w * N + t];
    atomicAdd(&F[(size_t)a * N + t], -0.5 * k);
  }
  for (int t = threadIdx.x; t < b1 - b0; t += kFockThreads) {
    double j = 0.0;
    for (int w = 0; w < kFockWarps; ++w) j += jred[w * b_per_cta + t];
    atomicAdd(&F[(size_t)a * N + b0 + t], j);
  }
}

// partial[n] = sum_ij Re(G_ij Sigma_ji) at frequency n (32x32 tiles through smem)
__global__ void energy_partial_kernel(int N, const double2 *__restrict__ G, const double2 *__restrict__ Sig,
                                      double *__restrict__ partial) {
  __shared__ double2 st[32][33];
  __shared__ double red[256];
  const long long n = blockIdx.x;
  const size_t base = (size_t)n * N * N;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 32 x 8
  double acc = 0.0;
  for (int ib = 0; ib < N; ib += 32)
    for (int jb = 0; jb < N; jb += 32) {
      // stage Sigma[jb + r][ib + c] into st[r][c]
      for (int r = ty; r < 32; r += 8) {
        const int jj = jb + r, ii = ib + tx;
        st[r][tx] = (jj < N && ii < N) ? Sig[base + (size_t)jj * N + ii] : make_double2(0.0, 0.0);
      }
      __syncthreads();
      for (int r = ty; r < 32; r += 8) {
        const int ii = ib + r, jj = jb + tx;
        if (ii < N && jj < N) {
          const double2 g = G[base + (size_t)ii * N + jj];
          const double2 s = st[tx][r];  // Sigma[jj][ii]
          acc += g.x * s.x - g.y * s.y;
        }
      }
      __syncthreads();
    }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[n] = red[0];
}

// Trigamma psi_1(x) for x > 0 by the standard method of Abramowitz & Stegun
// (Handbook of Mathematical Functions, 6.4.6 and 6.4.12): the recurrence
// psi_1(x) = psi_1(x + 1) + 1/x^2 raises the argument to x >= 20, where the
// asymptotic series 1/x + 1/(2x^2) + sum_k B_2k / x^(2k+1) (Bernoulli numbers
// B_2..B_10 = 1/6, -1/30, 1/42, -1/30, 5/66) is accurate to rounding.
__device__ double trigamma(double x) {
  double acc = 0.0;
  while (x < 20.0) {
    acc += 1.0 / (x * x);
    x += 1.0;
  }
  const double ix = 1.0 / x, ix2 = ix * ix;
  return acc + ix + 0.5 * ix2 +
         ix * ix2 * (1.0 / 6.0 - ix2 * (1.0 / 30.0 - ix2 * (1.0 / 42.0 - ix2 * (1.0 / 30.0 - ix2 * (5.0 / 66.0)))));
}

// out[0] = E1 = 1/2 Tr[P(h+F)], out[1] = E2 incl. tail
__global__ void energy_final_kernel(int N, int n_iw, double beta, const double *partial, const double *P,
                                    const double *h, const double *F, const double *Sinv,
                                    const double *sig1, double *out) {
  __shared__ double r1[256], r2[256], r3[256];
  double a1 = 0.0, a2 = 0.0, a3 = 0.0;
  for (int n = threadIdx.x; n < n_iw; n += blockDim.x) a2 += partial[n];
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int i = e / N, j = e - i * N;
    a1 += P[e] * (h[j * N + i] + F[j * N + i]);
    if (sig1) a3 += Sinv[e] * sig1[j * N + i];
  }
  r1[threadIdx.x] = a1;
  r2[threadIdx.x] = a2;
  r3[threadIdx.x] = a3;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      r1[threadIdx.x] += r1[threadIdx.x + s];
      r2[threadIdx.x] += r2[threadIdx.x + s];
      r3[threadIdx.x] += r3[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = 0.5 * r1[0];
    double e2 = (2.0 / beta) * r2[0];
    if (sig1) e2 -= beta / (2.0 * M_PI * M_PI) * trigamma(n_iw + 0.5) * r3[0];
    out[1] = e2;
  }
}

// ---------------- host helpers ----------------

double *slot(gf2_ctx *ctx, int s) { return ctx->d_small + (size_t)s * ctx->N * ctx->N; }

Dgemm square_gemm(int N, const double *A, const double *B, double *C, double alpha, double beta_c,
                  bool transB = false) {
  Dgemm g{};
  g.M = N; g.N = N; g.K = N;
  g.A = A; g.a_rs = N; g.a_cs = 1;
  g.B = B; g.b_rs = transB ? 1 : N; g.b_cs = transB ? N : 1;
  g.C = C; g.c_rs = N; g.c_cs = 1;
  g.nb0 = 1; g.nb1 = 1; g.alpha = alpha; g.beta_c = beta_c; g.split_k = 1;
  return g;
}

// moment basis A0..A3, B1..B3 into the small slots (S^-1 kept from the last
// call when invert_S is false)
gf2_status build_moment_basis(gf2_ctx *ctx, const double *S, const double *F, const double *sig12,
                              bool invert_S = true) {
  const int N = ctx->N;
  const size_t N2 = (size_t)N * N;
  gf2_status st;
  if (invert_S && (st = gf2_inverse_spd(ctx, S, slot(ctx, SL_SINV))) != GF2_OK) return st;
  double *Sinv = slot(ctx, SL_SINV), *T1 = slot(ctx, SL_T1), *tmp = slot(ctx, SL_TMP);
  if ((st = gf2_dgemm(ctx, square_gemm(N, Sinv, F, T1, 1.0, 0.0))) != GF2_OK) return st;
  if ((st = gf2_dgemm(ctx, square_gemm(N, T1, Sinv, slot(ctx, SL_A1), 1.0, 0.0))) != GF2_OK) return st;
  if ((st = gf2_dgemm(ctx, square_gemm(N, T1, slot(ctx, SL_A1), slot(ctx, SL_A2), 1.0, 0.0))) != GF2_OK) return st;
  if ((st = gf2_dgemm(ctx, square_gemm(N, T1, slot(ctx, SL_A2), slot(ctx, SL_A3), 1.0, 0.0))) != GF2_OK) return st;
  if (!sig12) {
    GF2_CK(ctx, cudaMemsetAsync(slot(ctx, SL_B1), 0, 3 * N2 * sizeof(double), ctx->stream));
    return GF2_OK;
  }
  const double *sig1 = sig12, *sig2 = sig12 + N2;
  if ((st = gf2_dgemm(ctx, square_gemm(N, sig1, Sinv, tmp, 1.0, 0.0))) != GF2_OK) return st;
  if ((st = gf2_dgemm(ctx, square_gemm(N, Sinv, tmp, slot(ctx, SL_B1), 1.0, 0.0))) != GF2_OK) return st;
  if ((st = gf2_dgemm(ctx, square_gemm(N, T1, slot(ctx, SL_B1), slot(ctx, SL_B2), 1.0, 0.0))) != GF2_OK) return st;
  // B2 += B1 (S^-1 F)^T  (= B1 F S^-1 for symmetric S, F)
  if ((st = gf2_dgemm(ctx, square_gemm(N, slot(ctx, SL_B1), T1, slot(ctx, SL_B2), 1.0, 1.0, true))) != GF2_OK) return st;
  if ((st = gf2_dgemm(ctx, square_gemm(N, sig2, Sinv, tmp, 1.0, 0.0))) != GF2_OK) return st;
  if ((st = gf2_dgemm(ctx, square_gemm(N, Sinv, tmp, slot(ctx, SL_B3), 1.0, 0.0))) != GF2_OK) return st;
  return GF2_OK;
}

gf2_status launch_moments(gf2_ctx *ctx, double mu, double *mom) {
  const int N2 = ctx->N * ctx->N;
  moments_kernel<<<(N2 + 255) / 256, 256, 0, ctx->stream>>>(N2, mu, ctx->d_small, mom);
  GF2_CK_LAUNCH(ctx, "moments_kernel");
  return GF2_OK;
}

// Dyson at the lowest nb frequencies (all of them when nb = n_iw)
gf2_status launch_dyson(gf2_ctx *ctx, double mu, const double *S, const double *F, const double *Sig,
                        double *G, int nb) {
  const int N = ctx->N;
  const int per = (N * (N + 1) / 2 + kDysonThreads - 1) / kDysonThreads;
  GF2_CK(ctx, cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
  const double2 *sg = reinterpret_cast<const double2 *>(Sig);
  double2 *gg = reinterpret_cast<double2 *>(G);
  cudaStream_t st = ctx->stream;
  if (per <= 1) GF2_PROF(ctx, GF2_K_DYSON, (dyson_kernel<1, 2><<<nb, kDysonThreads, 0, st>>>(N, ctx->beta, mu, S, F, sg, gg, ctx->d_err)));
  else if (per <= 2) GF2_PROF(ctx, GF2_K_DYSON, (dyson_kernel<2, 2><<<nb, kDysonThreads, 0, st>>>(N, ctx->beta, mu, S, F, sg, gg, ctx->d_err)));
  else if (per <= 4) GF2_PROF(ctx, GF2_K_DYSON, (dyson_kernel<4, 2><<<nb, kDysonThreads, 0, st>>>(N, ctx->beta, mu, S, F, sg, gg, ctx->d_err)));
  else if (per <= 5) GF2_PROF(ctx, GF2_K_DYSON, (dyson_kernel<5, 2><<<nb, kDysonThreads, 0, st>>>(N, ctx->beta, mu, S, F, sg, gg, ctx->d_err)));
  else if (per <= 9) GF2_PROF(ctx, GF2_K_DYSON, (dyson_kernel<9, 1><<<nb, kDysonThreads, 0, st>>>(N, ctx->beta, mu, S, F, sg, gg, ctx->d_err)));
  else if (per <= 16) GF2_PROF(ctx, GF2_K_DYSON, (dyson_kernel<16, 1><<<nb, kDysonThreads, 0, st>>>(N, ctx->beta, mu, S, F, sg, gg, ctx->d_err)));
  else GF2_PROF(ctx, GF2_K_DYSON, (dyson_kernel<kDysonMaxPerThread, 1><<<nb, kDysonThreads, 0, st>>>(N, ctx->beta, mu, S, F, sg, gg, ctx->d_err)));
  GF2_CK_LAUNCH(ctx, "dyson_kernel");
  return GF2_OK;
}

// density from the lowest n_f frequencies; resum holds the tail sums over the same range
gf2_status launch_density(gf2_ctx *ctx, const double *G, const double *coef, double *P, int n_f,
                          const double *resum) {
  const int N2 = ctx->N * ctx->N;
  const int chunk = 256;
  const int nchunks = (n_f + chunk - 1) / chunk;
  dim3 grid((N2 + 127) / 128, nchunks);
  GF2_PROF(ctx, GF2_K_DENSITY,
           (density_partial_kernel<<<grid, 128, 0, ctx->stream>>>(N2, n_f, chunk,
                                                                  reinterpret_cast<const double2 *>(G), ctx->d_red)));
  GF2_CK_LAUNCH(ctx, "density_partial_kernel");
  density_final_kernel<<<(N2 + 255) / 256, 256, 0, ctx->stream>>>(
      N2, nchunks, ctx->beta, ctx->d_red, coef, resum, ctx->d_tau_pole + 4 * (size_t)(ctx->n_tau - 1), P);
  GF2_CK_LAUNCH(ctx, "density_final_kernel");
  return GF2_OK;
}

}  // namespace

gf2_status gf2_pole_coefficients(gf2_ctx *ctx, const double *d_moments, double *d_coef) {
  const int N2 = ctx->N * ctx->N;
  pole_coef_kernel<<<(N2 + 255) / 256, 256, 0, ctx->stream>>>(N2, GF2_TAIL_POLE, d_moments, d_coef);
  GF2_CK_LAUNCH(ctx, "pole_coef_kernel");
  return GF2_OK;
}

extern "C" gf2_status gf2_tail_moments(gf2_ctx *ctx, const double *d_S, const double *d_F, double mu,
                                       const double *d_sig12, double *d_moments) {
  if (!ctx) return GF2_ERR_ARG;
  if (!d_S || !d_F || !d_moments) return gf2_fail(ctx, GF2_ERR_ARG, "gf2_tail_moments: NULL pointer");
  gf2_status st = build_moment_basis(ctx, d_S, d_F, d_sig12);
  if (st != GF2_OK) return st;
  return launch_moments(ctx, mu, d_moments);
}

extern "C" gf2_status gf2_dyson(gf2_ctx *ctx, double mu, const double *d_S, const double *d_F,
                                const double *d_Sigma_iw, double *d_G_iw) {
  if (!ctx) return GF2_ERR_ARG;
  if (!d_S || !d_F || !d_G_iw) return gf2_fail(ctx, GF2_ERR_ARG, "gf2_dyson: NULL pointer");
  if (!std::isfinite(mu)) return gf2_fail(ctx, GF2_ERR_ARG, "gf2_dyson: mu not finite");
  return launch_dyson(ctx, mu, d_S, d_F, d_Sigma_iw, d_G_iw, ctx->n_iw);
}

extern "C" gf2_status gf2_density(gf2_ctx *ctx, const double *d_G_iw, const double *d_moments, double *d_P) {
  if (!ctx) return GF2_ERR_ARG;
  if (!d_G_iw || !d_moments || !d_P) return gf2_fail(ctx, GF2_ERR_ARG, "gf2_density: NULL pointer");
  double *coef = slot(ctx, SL_COEF);
  gf2_status st = gf2_pole_coefficients(ctx, d_moments, coef);
  if (st != GF2_OK) return st;
  return launch_density(ctx, d_G_iw, coef, d_P, ctx->n_iw, ctx->d_pole_resum);
}

// One count evaluation at the state's mu, then the controller: the body of the
// search's WHILE loop (seven kernels), launched on the capturing stream cs.
static void launch_mu_body(gf2_ctx *ctx, cudaStream_t cs, const double *S, const double *F, const double *Sig,
                    double *G, double *P, MuState *ms, cudaGraphConditionalHandle loop) {
  const int N = ctx->N, N2 = N * N, n_iw = ctx->n_iw;
  double *mom = slot(ctx, SL_MOM), *coef = slot(ctx, SL_COEF), *cnt = slot(ctx, SL_MISC);
  moments_kernel<<<(N2 + 255) / 256, 256, 0, cs>>>(N2, 0.0, ctx->d_small, mom, ms);
  pole_coef_kernel<<<(N2 + 255) / 256, 256, 0, cs>>>(N2, GF2_TAIL_POLE, mom, coef);
  const int per = (N * (N + 1) / 2 + kDysonThreads - 1) / kDysonThreads;
  const double2 *sg = reinterpret_cast<const double2 *>(Sig);
  double2 *gg = reinterpret_cast<double2 *>(G);
  const double b = ctx->beta;
  int *fl = ctx->d_err;
  if (per <= 1) dyson_kernel<1, 2><<<n_iw, kDysonThreads, 0, cs>>>(N, b, 0.0, S, F, sg, gg, fl, ms);
  else if (per <= 2) dyson_kernel<2, 2><<<n_iw, kDysonThreads, 0, cs>>>(N, b, 0.0, S, F, sg, gg, fl, ms);
  else if (per <= 4) dyson_kernel<4, 2><<<n_iw, kDysonThreads, 0, cs>>>(N, b, 0.0, S, F, sg, gg, fl, ms);
  else if (per <= 5) dyson_kernel<5, 2><<<n_iw, kDysonThreads, 0, cs>>>(N, b, 0.0, S, F, sg, gg, fl, ms);
  else if (per <= 9) dyson_kernel<9, 1><<<n_iw, kDysonThreads, 0, cs>>>(N, b, 0.0, S, F, sg, gg, fl, ms);
  else if (per <= 16) dyson_kernel<16, 1><<<n_iw, kDysonThreads, 0, cs>>>(N, b, 0.0, S, F, sg, gg, fl, ms);
  else dyson_kernel<kDysonMaxPerThread, 1><<<n_iw, kDysonThreads, 0, cs>>>(N, b, 0.0, S, F, sg, gg, fl, ms);
  const int chunk = 256, nchunks = (n_iw + chunk - 1) / chunk;
  density_partial_kernel<<<dim3((N2 + 127) / 128, nchunks), 128, 0, cs>>>(
      N2, n_iw, chunk, reinterpret_cast<const double2 *>(G), ctx->d_red, ms);
  density_final_kernel<<<(N2 + 255) / 256, 256, 0, cs>>>(N2, nchunks, ctx->beta, ctx->d_red, coef,
                                                          ctx->d_pole_resum, ctx->d_tau_pole + 4 * (size_t)(ctx->n_tau - 1),
                                                          P, ms, ctx->d_pole_resum + 4);
  trace_kernel<<<1, 256, 0, cs>>>(N, P, S, cnt);
  mu_control_kernel<<<1, 32, 0, cs>>>(ms, cnt, fl, loop);
}

// The WHILE graph of the device-resident search for one set of buffers (kept
// while the buffers stay the same): moments, pole coefficients, Dyson over the
// largest frequency range (blocks past the evaluation's range return), density,
// trace and the controller, captured on a private stream into the loop body.
static gf2_status mu_search_graph(gf2_ctx *ctx, const double *S, const double *F, const double *Sig,
                                  double *G, double *P) {
  const void *key[5] = {S, F, Sig, G, P};
  if (ctx->mu_graph_exec && std::equal(key, key + 5, ctx->mu_graph_key)) return GF2_OK;
  if (ctx->mu_graph_exec) cudaGraphExecDestroy(ctx->mu_graph_exec);
  if (ctx->mu_graph) cudaGraphDestroy(ctx->mu_graph);
  ctx->mu_graph_exec = nullptr;
  ctx->mu_graph = nullptr;
  if (!ctx->d_mu_state) GF2_CK(ctx, cudaMalloc(&ctx->d_mu_state, sizeof(MuState)));
  if (!ctx->capture_stream) GF2_CK(ctx, cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
  MuState *ms = static_cast<MuState *>(ctx->d_mu_state);
  cudaGraph_t graph = nullptr;
  GF2_CK(ctx, cudaGraphCreate(&graph, 0));
  ctx->mu_graph = graph;
  cudaGraphConditionalHandle loop;
  GF2_CK(ctx, cudaGraphConditionalHandleCreate(&loop, graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = loop;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  GF2_CK(ctx, cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  cudaStream_t cs = ctx->capture_stream;
  GF2_CK(ctx, cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  launch_mu_body(ctx, cs, S, F, Sig, G, P, ms, loop);
  const cudaError_t launch_err = cudaGetLastError();
  cudaGraph_t captured = nullptr;
  const cudaError_t end_err = cudaStreamEndCapture(cs, &captured);
  if (launch_err != cudaSuccess) return gf2_cuda_fail(ctx, launch_err, "mu search graph: kernel capture");
  if (end_err != cudaSuccess) return gf2_cuda_fail(ctx, end_err, "mu search graph: end of capture");
  GF2_CK(ctx, cudaGraphInstantiate(&ctx->mu_graph_exec, graph, 0));
  std::copy(key, key + 5, ctx->mu_graph_key);
  return GF2_OK;
}

gf2_status gf2_build_moment_basis(gf2_ctx *ctx, const double *S, const double *F, const double *sig12,
                                  bool invert_S) {
  return build_moment_basis(ctx, S, F, sig12, invert_S);
}

gf2_status gf2_capture_mu_search(gf2_ctx *ctx, cudaStream_t parent, cudaStream_t body_stream, const double *S,
                                 const double *F, const double *Sig, double *G, double *P, const double *prm) {
  if (!ctx->d_mu_state) GF2_CK(ctx, cudaMalloc(&ctx->d_mu_state, sizeof(MuState)));
  MuState *ms = static_cast<MuState *>(ctx->d_mu_state);
  cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  GF2_CK(ctx, cudaStreamGetCaptureInfo(parent, &cst, nullptr, &g));
  if (cst != cudaStreamCaptureStatusActive || !g)
    return gf2_fail(ctx, GF2_ERR_ARG, "gf2_capture_mu_search: parent stream is not capturing");
  cudaGraphConditionalHandle loop;
  GF2_CK(ctx, cudaGraphConditionalHandleCreate(&loop, g, 0, 0));  // armed by mu_start_kernel
  mu_start_kernel<<<1, 32, 0, parent>>>(ms, prm, ctx->n_iw, ctx->n_coarse, ctx->d_err, loop);
  GF2_CK(ctx, cudaGetLastError());
  const cudaGraphNode_t *deps = nullptr;
  size_t n_deps = 0;
  GF2_CK(ctx, cudaStreamGetCaptureInfo(parent, &cst, nullptr, &g, &deps, nullptr, &n_deps));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = loop;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  GF2_CK(ctx, cudaGraphAddNode(&node, g, deps, nullptr, n_deps, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  GF2_CK(ctx, cudaStreamBeginCaptureToGraph(body_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  launch_mu_body(ctx, body_stream, S, F, Sig, G, P, ms, loop);
  const cudaError_t launch_err = cudaGetLastError();
  cudaGraph_t captured = nullptr;
  const cudaError_t end_err = cudaStreamEndCapture(body_stream, &captured);
  if (launch_err != cudaSuccess) return gf2_cuda_fail(ctx, launch_err, "nested mu search: kernel capture");
  if (end_err != cudaSuccess) return gf2_cuda_fail(ctx, end_err, "nested mu search: end of capture");
  GF2_CK(ctx, cudaStreamUpdateCaptureDependencies(parent, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return GF2_OK;
}

extern "C" gf2_status gf2_mu_search(gf2_ctx *ctx, const double *d_S, const double *d_F,
                                    const double *d_Sigma_iw, const double *d_sig12, double n_elec,
                                    double tol, int max_iter, double *mu_inout, double *d_G_iw,
                                    double *d_P, int *n_eval) {
  if (!ctx) return GF2_ERR_ARG;
  if (!d_S || !d_F || !mu_inout || !d_G_iw || !d_P)
    return gf2_fail(ctx, GF2_ERR_ARG, "gf2_mu_search: NULL pointer");
  if (!(tol > 0.0) || max_iter < 1 || !std::isfinite(*mu_inout) || !(n_elec > 0.0) ||
      !(n_elec < 2.0 * ctx->N))
    return gf2_fail(ctx, GF2_ERR_ARG, "gf2_mu_search: bad tol, max_iter, mu or n_elec");
  gf2_status st = build_moment_basis(ctx, d_S, d_F, d_sig12);
  if (st != GF2_OK) return st;
  if ((st = mu_search_graph(ctx, d_S, d_F, d_Sigma_iw, d_G_iw, d_P)) != GF2_OK) return st;
  MuState *ms = static_cast<MuState *>(ctx->d_mu_state);
  mu_init_kernel<<<1, 32, 0, ctx->stream>>>(ms, *mu_inout, n_elec, tol, max_iter, ctx->n_iw, ctx->n_coarse,
                                           ctx->d_err);
  GF2_CK_LAUNCH(ctx, "mu_init_kernel");
  GF2_PROF(ctx, GF2_K_DYSON, GF2_CK(ctx, cudaGraphLaunch(ctx->mu_graph_exec, ctx->stream)));
  // the one host synchronization of the search: its result
  static_assert(sizeof(MuState) >= 3 * sizeof(double), "state");
  GF2_CK(ctx, cudaMemcpyAsync(ctx->h_pinned, &ms->mu_out, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  GF2_CK(ctx, cudaMemcpyAsync(ctx->h_pinned + 1, &ms->status, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  GF2_CK(ctx, cudaStreamSynchronize(ctx->stream));
  int st_ev[2];
  std::memcpy(st_ev, ctx->h_pinned + 1, sizeof(st_ev));
  const int status = st_ev[0], evals = st_ev[1];
  ctx->launches += 7LL * evals;  // the graph's kernels: seven per count evaluation
  if (n_eval) *n_eval = evals;
  if (status == 4) return gf2_fail(ctx, GF2_ERR_NONFINITE, "gf2_mu_search: vanishing Dyson pivot");
  if (status == 3) return gf2_fail(ctx, GF2_ERR_NONFINITE, "gf2_mu_search: non-finite count");
  *mu_inout = ctx->h_pinned[0];
  if (status != 1) return gf2_fail(ctx, GF2_ERR_NOT_CONVERGED, "gf2_mu_search: tolerance not reached");
  return GF2_OK;
}

extern "C" gf2_status gf2_fock(gf2_ctx *ctx, const double *d_h, const double *d_P, double *d_F) {
  if (!ctx) return GF2_ERR_ARG;
  if (!d_h || !d_P || !d_F) return gf2_fail(ctx, GF2_ERR_ARG, "gf2_fock: NULL pointer");
  if (!ctx->have_integrals) return gf2_fail(ctx, GF2_ERR_ARG, "gf2_fock: gf2_set_integrals not called");
  if (d_F == d_P) return gf2_fail(ctx, GF2_ERR_ARG, "gf2_fock: d_F must not alias d_P");
  const int N = ctx->N;
  // about four CTAs per SM: N rows a times ceil(N / b_per_cta) blocks of b
  const int want = std::min(N, std::max(1, (4 * ctx->num_sms + N - 1) / N));
  const int b_per_cta = (N + want - 1) / want;
  const dim3 grid(N, (N + b_per_cta - 1) / b_per_cta);
  const size_t smem = sizeof(double) * ((size_t)N * N + (size_t)kFockWarps * b_per_cta + (size_t)kFockWarps * N);
  GF2_CK(ctx, cudaFuncSetAttribute(fock_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (d_F != d_h)
    GF2_CK(ctx, cudaMemcpyAsync(d_F, d_h, sizeof(double) * N * N, cudaMemcpyDeviceToDevice, ctx->stream));
  GF2_PROF(ctx, GF2_K_FOCK,
           (fock_kernel<<<grid, kFockThreads, smem, ctx->stream>>>(N, b_per_cta, ctx->d_v, d_P, d_F)));
  GF2_CK_LAUNCH(ctx, "fock_kernel");
  return GF2_OK;
}

extern "C" gf2_status gf2_energy(gf2_ctx *ctx, const double *d_h, const double *d_F, const double *d_P,
                                 const double *d_S, const double *d_G_iw, const double *d_Sigma_iw,
                                 const double *d_sig12, double *e_one_body, double *e_two_body) {
  if (!ctx) return GF2_ERR_ARG;
  if (!d_h || !d_F || !d_P || !d_S || !d_G_iw || !d_Sigma_iw || !e_one_body || !e_two_body)
    return gf2_fail(ctx, GF2_ERR_ARG, "gf2_energy: NULL pointer");
  gf2_status st;
  if (d_sig12 && (st = gf2_inverse_spd(ctx, d_S, slot(ctx, SL_SINV))) != GF2_OK) return st;
  GF2_PROF(ctx, GF2_K_ENERGY,
           (energy_partial_kernel<<<ctx->n_iw, 256, 0, ctx->stream>>>(
               ctx->N, reinterpret_cast<const double2 *>(d_G_iw), reinterpret_cast<const double2 *>(d_Sigma_iw),
               ctx->d_red)));
  GF2_CK_LAUNCH(ctx, "energy_partial_kernel");
  double *out = slot(ctx, SL_MISC);
  energy_final_kernel<<<1, 256, 0, ctx->stream>>>(ctx->N, ctx->n_iw, ctx->beta, ctx->d_red, d_P, d_h, d_F,
                                                  slot(ctx, SL_SINV), d_sig12, out);
  GF2_CK_LAUNCH(ctx, "energy_final_kernel");
  GF2_CK(ctx, cudaMemcpyAsync(ctx->h_pinned, out, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  GF2_CK(ctx, cudaStreamSynchronize(ctx->stream));
  *e_one_body = ctx->h_pinned[0];
  *e_two_body = ctx->h_pinned[1];
  return GF2_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of gf2_energy.
//
// For callers that cannot allocate device memory -- a host that gives the
// library a fixed memory budget and forbids the device allocator, or code that
// must not meet an out-of-memory failure in the middle of a run -- this entry
// point needs no context and makes no cudaMalloc/cudaFree (nor any allocating
// library call).  Its scratch (one partial sum per frequency, S^-1 and the two
// results) lives in a file-scope __device__ array of fixed size, present on
// every device that loads the library until the process exits.  It copies the
// two results to the host and synchronizes the caller's stream.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr int kNoallocMaxN = GF2_MAX_N;                 // 128
constexpr int kNoallocMaxIw = 65536;
constexpr size_t kNoallocDoubles = (size_t)kNoallocMaxIw + (size_t)kNoallocMaxN * kNoallocMaxN + 8;

static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

std::mutex g_noalloc_mutex;
double *g_noalloc_addr[256] = {};

// device address of g_noalloc_scratch on the current device, looked up once per device
gf2_status noalloc_scratch(double **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return GF2_ERR_CUDA;
  if (dev < 0 || dev >= 256) return GF2_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GF2_ERR_CUDA;
    g_noalloc_addr[dev] = static_cast<double *>(p);
  }
  *out = g_noalloc_addr[dev];
  return GF2_OK;
}

// S^-1 by Gauss-Jordan in shared memory (S symmetric positive definite)
__global__ void noalloc_inverse_kernel(const double *A, double *Ainv, int n) {
  extern __shared__ double noalloc_sm[];
  double *a = noalloc_sm, *col = noalloc_sm + n * n, *row = col + n;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) a[e] = A[e];
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] = a[i * n + k];
    __syncthreads();
    const double p = 1.0 / col[k];
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const double r = (j == k) ? p : a[k * n + j] * p;
      row[j] = r;
      a[k * n + j] = r;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int i = e / n, j = e - i * n;
      if (i == k) continue;
      if (j == k) a[e] = -col[i] * p;
      else a[e] -= col[i] * row[j];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) Ainv[e] = a[e];
}

}  // namespace

extern "C" gf2_status gf2_energy_noalloc(int n_bf, int n_iw, double beta, const double *d_h, const double *d_F,
                                         const double *d_P, const double *d_S, const double *d_G_iw,
                                         const double *d_Sigma_iw, const double *d_sig12, double *e_one_body,
                                         double *e_two_body, void *stream) {
  if (!d_h || !d_F || !d_P || !d_S || !d_G_iw || !d_Sigma_iw || !e_one_body || !e_two_body) return GF2_ERR_ARG;
  if (n_bf < 1 || n_iw < 1 || !(beta > 0.0) || !std::isfinite(beta)) return GF2_ERR_ARG;
  if (n_bf > kNoallocMaxN || n_iw > kNoallocMaxIw) return GF2_ERR_UNSUPPORTED;
  double *scratch = nullptr;
  gf2_status st = noalloc_scratch(&scratch);
  if (st != GF2_OK) return st;
  double *partial = scratch;                            // [n_iw]
  double *sinv = scratch + kNoallocMaxIw;               // [N][N]
  double *res = sinv + (size_t)kNoallocMaxN * kNoallocMaxN;  // [2]
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  energy_partial_kernel<<<n_iw, 256, 0, s>>>(n_bf, reinterpret_cast<const double2 *>(d_G_iw),
                                             reinterpret_cast<const double2 *>(d_Sigma_iw), partial);
  if (cudaGetLastError() != cudaSuccess) return GF2_ERR_CUDA;
  if (d_sig12) {
    const size_t smem = sizeof(double) * ((size_t)n_bf * n_bf + 2 * (size_t)n_bf);
    if (cudaFuncSetAttribute(noalloc_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return GF2_ERR_CUDA;
    noalloc_inverse_kernel<<<1, 256, smem, s>>>(d_S, sinv, n_bf);
    if (cudaGetLastError() != cudaSuccess) return GF2_ERR_CUDA;
  }
  energy_final_kernel<<<1, 256, 0, s>>>(n_bf, n_iw, beta, partial, d_P, d_h, d_F, sinv, d_sig12, res);
  if (cudaGetLastError() != cudaSuccess) return GF2_ERR_CUDA;
  double host[2];
  if (cudaMemcpyAsync(host, res, sizeof host, cudaMemcpyDeviceToHost, s) != cudaSuccess) return GF2_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return GF2_ERR_CUDA;
  *e_one_body = host[0];
  *e_two_body = host[1];
  return GF2_OK;
}
