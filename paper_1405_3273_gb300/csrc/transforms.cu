// Matsubara <-> imaginary-time transforms (the FFT steps of the GF2 loop).
//
// Both directions run one M-point complex FFT per matrix element in shared
// memory (decimation in frequency in radix-4 passes, bit-reversed output read
// back through __brev), E adjacent elements per CTA so that every global access
// of a frequency or time row touches E*16 contiguous bytes.
//
// iw -> tau:  X(tau_k) = (2/beta) Re[e^{-i pi k/M} Z_k] + T(tau_k),
//             Z = FFT_M(Y),  Y_j = sum_{n = j mod M, n < n_iw} (X - T)(i w_n)
//             (the tail's folded sums per j are a table: Y_j = sum X - sum_r c_r Q_jr)
//             (w_n tau_k = pi (2n+1) k / M, so frequencies fold modulo M;
//             tau_M = beta uses e^{-i pi (2n+1)} = -1).
// tau -> iw:  the exact Fourier integral of the piecewise-cubic interpolant:
//             X(i w_n) = h W(theta_n) D_n + sum_{end nodes q} c_q(n) X_q,
//             D_n = sum_{k=0..M} e^{i w_n tau_k} X_k = IFFT_M(X_k e^{i pi k/M})(n mod M) - X_M,
//             theta = w h, W the attenuation factor of the interior scheme and
//             c_q the differences between the exact weights of the end nodes
//             0..3, M-3..M and the interior formula.
// The tables (twiddles, tail images, W, end corrections) depend only on the
// grid and are built once per context.
//
// Non-equidistant grid (points tau_k = idx_k beta / M, a subset of the uniform
// grid of M intervals, symmetric about beta / 2):
// iw -> tau:  the same FFT over the M-interval grid, written at the points only.
// tau -> iw:  the local cubics now pass through unequally spaced nodes.  On
//             uniform interval f inside grid interval a (d = f - idx_a steps
//             in, r = idx_a+1 - idx_a steps long) the cubic of a, in the local
//             variable y = (tau - f h) / h, h = beta / M, has coefficients
//             m'_fq = sum_{p >= q} m_ap binom(p, q) d^(p-q) / r^p (m_ap: its
//             coefficients in x = (tau - tau_a) / h_a), so
//             X(i w_n) = h sum_q mu_q(w_n h) D_q(n),
//             D_q(n) = sum_f m'_fq e^{i w_n f h} = FFT_M(m'_fq e^{i pi f / M})(n mod M),
//             two real sequences per complex FFT (q = 0,1 then q = 2,3),
//             separated by D(n) = [Z(n) +- conj Z(M-1-n)] / (2 or 2i).
#include <algorithm>
#include <cmath>
#include <vector>

#include "gf2_internal.cuh"

namespace {

// monomial coefficients (ascending powers of x in [0,1]) of the Lagrange
// basis polynomials of the three node patterns of the cubic interpolant:
// interior nodes at offsets -1,0,1,2; first interval 0,1,2,3; last -2,-1,0,1.
__constant__ double kLagInterior[4][4] = {
    {0.0, -1.0 / 3.0, 0.5, -1.0 / 6.0},
    {1.0, -0.5, -1.0, 0.5},
    {0.0, 1.0, 0.5, -0.5},
    {0.0, -1.0 / 6.0, 0.0, 1.0 / 6.0}};
__constant__ double kLagFirst[4][4] = {
    {1.0, -11.0 / 6.0, 1.0, -1.0 / 6.0},
    {0.0, 3.0, -2.5, 0.5},
    {0.0, -1.5, 2.0, -0.5},
    {0.0, 1.0 / 3.0, -0.5, 1.0 / 6.0}};
__constant__ double kLagLast[4][4] = {
    {0.0, 1.0 / 6.0, 0.0, -1.0 / 6.0},
    {0.0, -1.0, 0.5, 0.5},
    {1.0, 0.5, -1.0, -0.5},
    {0.0, 1.0 / 3.0, 0.5, 1.0 / 6.0}};

// mu_p(theta) = int_0^1 x^p e^{i theta x} dx, p = 0..3.
__device__ void monomial_moments(double theta, double2 mu[4]) {
  if (fabs(theta) < 1.0) {
    for (int p = 0; p < 4; ++p) mu[p] = make_double2(0.0, 0.0);
    double2 term = make_double2(1.0, 0.0);  // (i theta)^m / m!
    for (int m = 0; m < 28; ++m) {
      for (int p = 0; p < 4; ++p) mu[p] = cadd(mu[p], cscale(term, 1.0 / (p + m + 1)));
      term = cscale(cmul(term, make_double2(0.0, theta)), 1.0 / (m + 1));
    }
  } else {
    double s, c;
    sincos(theta, &s, &c);
    const double2 e = make_double2(c, s);
    const double2 inv_itheta = make_double2(0.0, -1.0 / theta);  // 1/(i theta)
    mu[0] = cmul(csub(e, make_double2(1.0, 0.0)), inv_itheta);
    for (int p = 1; p < 4; ++p) mu[p] = cmul(csub(e, cscale(mu[p - 1], (double)p)), inv_itheta);
  }
}

// e^{i pi (2n+1) a / M} with the angle reduced exactly (a may be negative)
__device__ double2 phase_na(long long n, long long a, int M) {
  long long t = ((2 * n + 1) * a) % (2LL * M);
  if (t < 0) t += 2LL * M;
  double s, c;
  sincospi((double)t / (double)M, &s, &c);
  return make_double2(c, s);
}

__device__ double2 interval_weight(const double (*lag)[4], int o_idx, const double2 mu[4]) {
  double2 r = make_double2(0.0, 0.0);
  for (int p = 0; p < 4; ++p) r = cadd(r, cscale(mu[p], lag[o_idx][p]));
  return r;
}

__global__ void tables_kernel(int M, int n_tau, int n_iw, double beta, double a, double2 *twiddle,
                              double2 *iw_pole, double *tau_pole, double2 *t2w_w,
                              double2 *t2w_corr, double2 *halfphase, const int *tau_index) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const double h = beta / M;
  if (tid < M / 2) {
    double s, c;
    sincospi(2.0 * (double)tid / (double)M, &s, &c);
    twiddle[tid] = make_double2(c, -s);
  }
  if (tid < M) {
    double s, c;
    sincospi((double)tid / (double)M, &s, &c);
    halfphase[tid] = make_double2(c, -s);  // e^{-i pi k / M}
  }
  if (tid < n_tau) {
    const double t = (tau_index ? tau_index[tid] : tid) * h;
    const double E = exp(-a * t), q = exp(-a * beta);
    const double u = 1.0 / (1.0 + q), v = u * (q / (1.0 + q));
    const double u1 = beta * v, u2 = beta * beta * v * (1.0 - 2.0 * u);
    const double u3 = beta * beta * beta * v * (1.0 - 6.0 * u + 6.0 * u * u);
    double *g = tau_pole + 4 * tid;
    g[0] = -E * u;
    g[1] = E * (t * u - u1);
    g[2] = E * (-t * t * u + 2.0 * t * u1 - u2) / 2.0;
    g[3] = E * (t * t * t * u - 3.0 * t * t * u1 + 3.0 * t * u2 - u3) / 6.0;
  }
  if (tid < n_iw) {
    const long long n = tid;
    const double w = (2.0 * n + 1.0) * M_PI / beta;
    const double2 inv = crecip(make_double2(-a, w));
    double2 pw = inv;
    for (int r = 0; r < 4; ++r) {
      iw_pole[4 * n + r] = pw;
      pw = cmul(pw, inv);
    }
    // tau -> iw weights
    const double theta = (2.0 * n + 1.0) * M_PI / (double)M;
    double2 mu[4];
    monomial_moments(theta, mu);
    double2 W = make_double2(0.0, 0.0);
    for (int o = -1; o <= 2; ++o) {
      double s, c;
      sincos(-theta * o, &s, &c);
      W = cadd(W, cmul(make_double2(c, s), interval_weight(kLagInterior, o + 1, mu)));
    }
    t2w_w[n] = cscale(W, h);
    const int nodes[8] = {0, 1, 2, 3, M - 3, M - 2, M - 1, M};
    for (int qi = 0; qi < 8; ++qi) {
      const int k = nodes[qi];
      double2 exact = make_double2(0.0, 0.0);
      if (k <= 3) {  // first interval (pattern 0..3, offset o = k)
        exact = cadd(exact, cmul(phase_na(n, 0, M), interval_weight(kLagFirst, k, mu)));
      }
      if (k >= M - 3) {  // last interval a = M-1 (pattern -2..1, offset o = k-(M-1))
        exact = cadd(exact, cmul(phase_na(n, M - 1, M), interval_weight(kLagLast, k - (M - 1) + 2, mu)));
      }
      for (int o = -1; o <= 2; ++o) {  // interior intervals a = k - o, 1 <= a <= M-2
        const int aa = k - o;
        if (aa >= 1 && aa <= M - 2)
          exact = cadd(exact, cmul(phase_na(n, aa, M), interval_weight(kLagInterior, o + 1, mu)));
      }
      double2 interior = make_double2(0.0, 0.0);
      for (int o = -1; o <= 2; ++o)
        interior = cadd(interior, cmul(phase_na(n, k - o, M), interval_weight(kLagInterior, o + 1, mu)));
      t2w_corr[8 * n + qi] = cscale(csub(exact, interior), h);
    }
  }
}

__global__ void pole_resum_kernel(int n_iw, const double2 *iw_pole, double *out) {
  __shared__ double red[4][256];
  double acc[4] = {0, 0, 0, 0};
  for (int n = threadIdx.x; n < n_iw; n += blockDim.x)
    for (int r = 0; r < 4; ++r) acc[r] += iw_pole[4 * n + r].x;
  for (int r = 0; r < 4; ++r) red[r][threadIdx.x] = acc[r];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int r = 0; r < 4; ++r) red[r][threadIdx.x] += red[r][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 4) out[threadIdx.x] = red[threadIdx.x][0];
}

// In-place DIF FFT of E sequences of length M in shared memory.
// sign = -1: X_k = sum_j x_j e^{-2 pi i jk/M};  sign = +1: e^{+...}.
// Output in bit-reversed order.  Each pass applies two radix-2 stages at once
// (groups of 2 half, quarters q = half/2): the four values x[b], x[b+q],
// x[b+half], x[b+half+q] go through the stage-`half` butterflies (twiddles of
// positions p and p+q) and then the stage-`q` butterflies (twiddle of position
// p at twice the stride), the same operations in the same order as two
// radix-2 stages, with half the barriers and shared-memory round trips.  When
// log2 M is odd a last radix-2 stage (half = 1) follows.
__device__ void fft_dif_smem(double2 *x, int E, int M, const double2 *tw, int sign) {
  const int quarterM = M >> 2;
  int half = M >> 1, tstride = 1;
  for (; half >= 2; half >>= 2, tstride <<= 2) {
    const int q = half >> 1;
    for (int idx = threadIdx.x; idx < E * quarterM; idx += blockDim.x) {
      const int e = idx / quarterM, j = idx - e * quarterM;
      const int grp = j / q, p = j - grp * q;
      const int b = grp * 2 * half + p;
      double2 wa0 = tw[p * tstride], wa1 = tw[(p + q) * tstride], wb = tw[2 * p * tstride];
      if (sign > 0) {
        wa0.y = -wa0.y;
        wa1.y = -wa1.y;
        wb.y = -wb.y;
      }
      double2 *xe = x + (size_t)e * M;
      const double2 x0 = xe[b], x1 = xe[b + q], x2 = xe[b + half], x3 = xe[b + half + q];
      const double2 y0 = cadd(x0, x2), y2 = cmul(csub(x0, x2), wa0);
      const double2 y1 = cadd(x1, x3), y3 = cmul(csub(x1, x3), wa1);
      xe[b] = cadd(y0, y1);
      xe[b + q] = cmul(csub(y0, y1), wb);
      xe[b + half] = cadd(y2, y3);
      xe[b + half + q] = cmul(csub(y2, y3), wb);
    }
    __syncthreads();
  }
  if (half == 1) {  // tstride = M / 2: every twiddle is tw[0]
    const int halfM = M >> 1;
    for (int idx = threadIdx.x; idx < E * halfM; idx += blockDim.x) {
      const int e = idx / halfM, j = idx - e * halfM;
      double2 w = tw[0];
      if (sign > 0) w.y = -w.y;
      double2 *xe = x + (size_t)e * M;
      const double2 a = xe[2 * j], b = xe[2 * j + 1];
      xe[2 * j] = cadd(a, b);
      xe[2 * j + 1] = cmul(csub(a, b), w);
    }
    __syncthreads();
  }
}

// the pole terms folded like the frequencies: Q[j][r] = sum_{n = j mod M, n < n_iw} (i w_n - a)^-(r+1)
__global__ void pole_fold_kernel(int M, int n_iw, const double2 *__restrict__ iw_pole, double2 *__restrict__ fold) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  double2 q[4] = {};
  for (int n = j; n < n_iw; n += M)
    for (int r = 0; r < 4; ++r) q[r] = cadd(q[r], iw_pole[4 * (size_t)n + r]);
  for (int r = 0; r < 4; ++r) fold[4 * (size_t)j + r] = q[r];
}

__global__ void __launch_bounds__(512, 3) iw_to_tau_kernel(int N2, int M, int log2M, int n_iw, int E, double beta,
                                 const double2 *__restrict__ X_iw, const double *__restrict__ coef,
                                 const double2 *__restrict__ pole_fold, const double *__restrict__ tau_pole,
                                 const double2 *__restrict__ tw, const double2 *__restrict__ halfphase,
                                 int n_tau, const int *__restrict__ tau_index, double *__restrict__ X_tau) {
  extern __shared__ double2 sm[];
  double2 *x = sm;                              // [E][M]
  double *c = reinterpret_cast<double *>(x + (size_t)E * M);  // [E][4]
  const int e0 = blockIdx.x * E;
  for (int i = threadIdx.x; i < 4 * E; i += blockDim.x) {
    const int e = i / 4, r = i % 4;
    c[i] = coef[(size_t)r * N2 + e0 + e];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < E * M; idx += blockDim.x) {
    const int j = idx / E, e = idx - j * E;
    const double *ce = c + 4 * e;
    double2 acc = make_double2(0.0, 0.0);
    for (int n = j; n < n_iw; n += M) acc = cadd(acc, X_iw[(size_t)n * N2 + e0 + e]);
    // minus the tail, folded the same way: sum_r c_r Q[j][r]
    const double2 *q = pole_fold + 4 * (size_t)j;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      acc.x = fma(-ce[r], q[r].x, acc.x);
      acc.y = fma(-ce[r], q[r].y, acc.y);
    }
    x[(size_t)e * M + j] = acc;
  }
  __syncthreads();
  fft_dif_smem(x, E, M, tw, -1);
  const double s2b = 2.0 / beta;
  for (int idx = threadIdx.x; idx < E * n_tau; idx += blockDim.x) {
    const int k = idx / E, e = idx - k * E;
    const int j = tau_index ? tau_index[k] : k;  // the point on the uniform grid
    const double *ce = c + 4 * e;
    double val;
    if (j < M) {
      const int br = (int)(__brev((unsigned)j) >> (32 - log2M));
      const double2 z = x[(size_t)e * M + br];
      const double2 ph = halfphase[j];
      val = s2b * (z.x * ph.x - z.y * ph.y);
    } else {
      val = -s2b * x[(size_t)e * M].x;
    }
    const double *g = tau_pole + 4 * (size_t)k;
    val += ce[0] * g[0] + ce[1] * g[1] + ce[2] * g[2] + ce[3] * g[3];
    X_tau[(size_t)k * N2 + e0 + e] = val;
  }
}

__global__ void __launch_bounds__(512, 3) tau_to_iw_kernel(int N2, int M, int log2M, int n_iw, int E,
                                 const double *__restrict__ X_tau, const double2 *__restrict__ tw,
                                 const double2 *__restrict__ halfphase, const double2 *__restrict__ t2w_w,
                                 const double2 *__restrict__ t2w_corr, double2 *__restrict__ X_iw) {
  extern __shared__ double2 sm[];
  double2 *x = sm;                                          // [E][M]
  double *ends = reinterpret_cast<double *>(x + (size_t)E * M);  // [E][8]
  const int e0 = blockIdx.x * E;
  for (int i = threadIdx.x; i < 8 * E; i += blockDim.x) {
    const int e = i / 8, q = i % 8;
    const int node = q < 4 ? q : M - 7 + q;
    ends[i] = X_tau[(size_t)node * N2 + e0 + e];
  }
  for (int idx = threadIdx.x; idx < E * M; idx += blockDim.x) {
    const int k = idx / E, e = idx - k * E;
    const double v = X_tau[(size_t)k * N2 + e0 + e];
    const double2 ph = halfphase[k];  // e^{-i pi k/M}; we need its conjugate
    x[(size_t)e * M + k] = make_double2(v * ph.x, -v * ph.y);
  }
  __syncthreads();
  fft_dif_smem(x, E, M, tw, +1);
  for (int idx = threadIdx.x; idx < E * n_iw; idx += blockDim.x) {
    const int n = idx / E, e = idx - n * E;
    const int j = n & (M - 1);
    const int br = (int)(__brev((unsigned)j) >> (32 - log2M));
    const double *en = ends + 8 * e;
    double2 d = x[(size_t)e * M + br];
    d.x -= en[7];  // - X_M
    double2 val = cmul(t2w_w[n], d);
    const double2 *cq = t2w_corr + 8 * (size_t)n;
#pragma unroll
    for (int q = 0; q < 8; ++q) val = cadd(val, cscale(cq[q], en[q]));
    X_iw[(size_t)n * N2 + e0 + e] = val;
  }
}

// Sig1 = -(X_0 + X_M), Sig2 = X~'(0+) + X~'(beta-) of the end cubics
__global__ void sigma_ends_kernel(int N2, int M, double h, const double *X, double *sig12) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N2) return;
  const double x0 = X[e], x1 = X[(size_t)N2 + e], x2 = X[2 * (size_t)N2 + e], x3 = X[3 * (size_t)N2 + e];
  const double y0 = X[(size_t)M * N2 + e], y1 = X[(size_t)(M - 1) * N2 + e];
  const double y2 = X[(size_t)(M - 2) * N2 + e], y3 = X[(size_t)(M - 3) * N2 + e];
  sig12[e] = -(x0 + y0);
  const double d0 = (-11.0 * x0 + 18.0 * x1 - 9.0 * x2 + 2.0 * x3) / (6.0 * h);
  const double dM = (11.0 * y0 - 18.0 * y1 + 9.0 * y2 - 2.0 * y3) / (6.0 * h);
  sig12[(size_t)N2 + e] = d0 + dM;
}

// [n_iw][4]: h mu_q(w_n h), h = beta / M (the uniform step)
__global__ void grid_mu_kernel(int n_iw, int M, double beta, double2 *out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_iw) return;
  const double h = beta / M;
  double2 mu[4];
  monomial_moments((2.0 * n + 1.0) * M_PI / (double)M, mu);  // w_n h
  for (int q = 0; q < 4; ++q) out[4 * (size_t)n + q] = cscale(mu[q], h);
}

// tau -> iw on a non-equidistant grid of K + 1 points, one matrix element per
// CTA: the node values, the cubic of every grid interval, then two passes of
// (expand onto the uniform intervals, FFT, accumulate X(i w_n)).
__global__ void tau_to_iw_grid_kernel(int N2, int M, int log2M, int K, int n_iw,
                                      const double *__restrict__ X_tau, const double2 *__restrict__ tw,
                                      const double2 *__restrict__ halfphase, const double *__restrict__ lag,
                                      const int *__restrict__ tau_index, const int *__restrict__ fine_a,
                                      const double2 *__restrict__ gmu, double2 *__restrict__ X_iw) {
  extern __shared__ double2 sm[];
  double2 *x = sm;                                           // [M]
  double *xs = reinterpret_cast<double *>(x + M);            // [K + 1] node values
  double *mc = xs + (K + 1);                                 // [K][4] cubic of each interval
  const int e = blockIdx.x;
  for (int k = threadIdx.x; k <= K; k += blockDim.x) xs[k] = X_tau[(size_t)k * N2 + e];
  __syncthreads();
  for (int i = threadIdx.x; i < 4 * K; i += blockDim.x) {
    const int a = i >> 2, p = i & 3;
    const int first = a == 0 ? 0 : (a == K - 1 ? K - 3 : a - 1);
    const double *c = lag + 16 * (size_t)a;  // [4 nodes][4 powers]
    mc[i] = c[p] * xs[first] + c[4 + p] * xs[first + 1] + c[8 + p] * xs[first + 2] + c[12 + p] * xs[first + 3];
  }
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
    for (int f = threadIdx.x; f < M; f += blockDim.x) {
      const int a = fine_a[f];
      const int i0 = tau_index[a];
      const double ir = 1.0 / (double)(tau_index[a + 1] - i0), d = (double)(f - i0);
      // the cubic of interval a in y = (tau - f h) / h: powers of (d + y) / r
      const double m1 = mc[4 * a + 1] * ir, m2 = mc[4 * a + 2] * ir * ir, m3 = mc[4 * a + 3] * ir * ir * ir;
      double lo, hi;
      if (pass == 0) {
        lo = mc[4 * a] + d * (m1 + d * (m2 + d * m3));
        hi = m1 + d * (2.0 * m2 + 3.0 * d * m3);
      } else {
        lo = m2 + 3.0 * d * m3;
        hi = m3;
      }
      const double2 ph = halfphase[f];  // e^{-i pi f / M}; the twist is its conjugate
      x[f] = make_double2(lo * ph.x + hi * ph.y, hi * ph.x - lo * ph.y);
    }
    __syncthreads();
    fft_dif_smem(x, 1, M, tw, +1);
    for (int n = threadIdx.x; n < n_iw; n += blockDim.x) {
      const int j = n & (M - 1), jm = M - 1 - j;
      const double2 z = x[__brev((unsigned)j) >> (32 - log2M)];
      const double2 zm = x[__brev((unsigned)jm) >> (32 - log2M)];
      const double2 A = make_double2(0.5 * (z.x + zm.x), 0.5 * (z.y - zm.y));   // (Z + conj Zm) / 2
      const double2 B = make_double2(0.5 * (z.y + zm.y), -0.5 * (z.x - zm.x));  // (Z - conj Zm) / 2i
      const double2 *mu = gmu + 4 * (size_t)n + 2 * pass;
      const double2 val = cadd(cmul(mu[0], A), cmul(mu[1], B));
      double2 *out = X_iw + (size_t)n * N2 + e;
      *out = pass == 0 ? val : cadd(*out, val);
    }
    __syncthreads();
  }
}

// Sig1 = -(X_0 + X_K), Sig2 = the slopes of the end cubics (weights w[0..7])
struct SlopeWeights {
  double w[8];
};
__global__ void sigma_ends_grid_kernel(int N2, int K, SlopeWeights sw, const double *X, double *sig12) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N2) return;
  double d = 0.0;
  for (int j = 0; j < 4; ++j)
    d += sw.w[j] * X[(size_t)j * N2 + e] + sw.w[4 + j] * X[(size_t)(K - 3 + j) * N2 + e];
  sig12[e] = -(X[e] + X[(size_t)K * N2 + e]);
  sig12[(size_t)N2 + e] = d;
}

// monomial coefficients c[j][p] (powers of x) of the Lagrange basis of the nodes s[0..3]
void lagrange_monomials(const double s[4], double c[4][4]) {
  for (int j = 0; j < 4; ++j) {
    double poly[4] = {1.0, 0.0, 0.0, 0.0}, denom = 1.0;
    for (int m = 0; m < 4; ++m) {
      if (m == j) continue;
      for (int p = 3; p >= 1; --p) poly[p] = poly[p - 1] - s[m] * poly[p];  // times (x - s_m)
      poly[0] = -s[m] * poly[0];
      denom *= s[j] - s[m];
    }
    for (int p = 0; p < 4; ++p) c[j][p] = poly[p] / denom;
  }
}

int pick_elems_per_cta(int N2, int M) {
  const size_t budget = 130 * 1024;
  for (int E = 4; E >= 1; E >>= 1)
    if (N2 % E == 0 && (size_t)E * M * sizeof(double2) + 64 * E <= budget) return E;
  return 1;
}

}  // namespace

size_t gf2_grid_smem_bytes(int M, int n_tau) {
  return sizeof(double2) * (size_t)M + sizeof(double) * (size_t)n_tau + sizeof(double) * 4 * (size_t)(n_tau - 1);
}

// the host-side tables of a non-equidistant grid: each interval's local cubic
// (nodes a-1..a+2, 0..3 first, K-3..K last, offsets in units of its length),
// the interval of every uniform step, and the end slopes of Sig2
static gf2_status grid_tables(gf2_ctx *ctx, const int *idx) {
  const int M = ctx->M, K = ctx->n_tau - 1;
  std::vector<double> lag(16 * (size_t)K);
  std::vector<int> fine_a(M);
  for (int a = 0; a < K; ++a) {
    const int first = a == 0 ? 0 : (a == K - 1 ? K - 3 : a - 1);
    const double r = (double)(idx[a + 1] - idx[a]);
    double s[4], c[4][4];
    for (int j = 0; j < 4; ++j) s[j] = (double)(idx[first + j] - idx[a]) / r;
    lagrange_monomials(s, c);
    for (int j = 0; j < 4; ++j)
      for (int p = 0; p < 4; ++p) lag[16 * (size_t)a + 4 * j + p] = c[j][p];
    for (int f = idx[a]; f < idx[a + 1]; ++f) fine_a[f] = a;
    const double h = r * ctx->beta / M;
    if (a == 0)
      for (int j = 0; j < 4; ++j) ctx->grid_dw[j] = c[j][1] / h;  // d/dtau at x = 0
    if (a == K - 1)
      for (int j = 0; j < 4; ++j) ctx->grid_dw[4 + j] = (c[j][1] + 2.0 * c[j][2] + 3.0 * c[j][3]) / h;  // at x = 1
  }
  GF2_CK(ctx, cudaMalloc(&ctx->d_grid_lag, sizeof(double) * lag.size()));
  GF2_CK(ctx, cudaMalloc(&ctx->d_fine_a, sizeof(int) * M));
  GF2_CK(ctx, cudaMalloc(&ctx->d_grid_mu, sizeof(double2) * 4 * (size_t)ctx->n_iw));
  GF2_CK(ctx, cudaMemcpy(ctx->d_grid_lag, lag.data(), sizeof(double) * lag.size(), cudaMemcpyHostToDevice));
  GF2_CK(ctx, cudaMemcpy(ctx->d_fine_a, fine_a.data(), sizeof(int) * M, cudaMemcpyHostToDevice));
  grid_mu_kernel<<<(ctx->n_iw + 127) / 128, 128, 0, ctx->stream>>>(ctx->n_iw, M, ctx->beta, ctx->d_grid_mu);
  GF2_CK_LAUNCH(ctx, "grid_mu_kernel");
  return GF2_OK;
}

gf2_status gf2_tables_build(gf2_ctx *ctx, const int *h_tau_index) {
  const int M = ctx->M, n_tau = ctx->n_tau, n_iw = ctx->n_iw;
  GF2_CK(ctx, cudaMalloc(&ctx->d_twiddle, sizeof(double2) * (M / 2 + M)));
  GF2_CK(ctx, cudaMalloc(&ctx->d_iw_pole, sizeof(double2) * 4 * (size_t)n_iw));
  GF2_CK(ctx, cudaMalloc(&ctx->d_tau_pole, sizeof(double) * 4 * (size_t)n_tau));
  GF2_CK(ctx, cudaMalloc(&ctx->d_pole_resum, sizeof(double) * 8));
  GF2_CK(ctx, cudaMalloc(&ctx->d_t2w_w, sizeof(double2) * (size_t)n_iw));
  GF2_CK(ctx, cudaMalloc(&ctx->d_t2w_corr, sizeof(double2) * 8 * (size_t)n_iw));
  const int total = std::max(std::max(M, n_tau), n_iw);
  tables_kernel<<<(total + 127) / 128, 128, 0, ctx->stream>>>(
      M, n_tau, n_iw, ctx->beta, GF2_TAIL_POLE, ctx->d_twiddle, ctx->d_iw_pole, ctx->d_tau_pole,
      ctx->d_t2w_w, ctx->d_t2w_corr, ctx->d_twiddle + M / 2, ctx->d_tau_index);
  GF2_CK_LAUNCH(ctx, "tables_kernel");
  if (h_tau_index) {
    gf2_status st = grid_tables(ctx, h_tau_index);
    if (st != GF2_OK) return st;
  }
  pole_resum_kernel<<<1, 256, 0, ctx->stream>>>(n_iw, ctx->d_iw_pole, ctx->d_pole_resum);
  GF2_CK_LAUNCH(ctx, "pole_resum_kernel");
  GF2_CK(ctx, cudaMalloc(&ctx->d_iw_pole_fold, sizeof(double2) * 4 * (size_t)M));
  pole_fold_kernel<<<(M + 127) / 128, 128, 0, ctx->stream>>>(M, n_iw, ctx->d_iw_pole, ctx->d_iw_pole_fold);
  GF2_CK_LAUNCH(ctx, "pole_fold_kernel");
  // the lowest n_iw / 8 frequencies serve the coarse counts of the mu search
  ctx->n_coarse = (n_iw >= 2048) ? n_iw / 8 : 0;
  if (ctx->n_coarse) {
    pole_resum_kernel<<<1, 256, 0, ctx->stream>>>(ctx->n_coarse, ctx->d_iw_pole, ctx->d_pole_resum + 4);
    GF2_CK_LAUNCH(ctx, "pole_resum_kernel");
  }
  return GF2_OK;
}

extern "C" gf2_status gf2_fft_iw_to_tau(gf2_ctx *ctx, const double *d_X_iw, const double *d_moments,
                                        double *d_X_tau) {
  if (!ctx) return GF2_ERR_ARG;
  if (!d_X_iw || !d_moments || !d_X_tau) return gf2_fail(ctx, GF2_ERR_ARG, "gf2_fft_iw_to_tau: NULL pointer");
  const int N2 = ctx->N * ctx->N, M = ctx->M;
  double *coef = ctx->d_small + GF2_SL_COEF * (size_t)N2;
  gf2_status st = gf2_pole_coefficients(ctx, d_moments, coef);
  if (st != GF2_OK) return st;
  const int E = pick_elems_per_cta(N2, M);
  const size_t smem = (size_t)E * M * sizeof(double2) + sizeof(double) * 4 * E;
  GF2_CK(ctx, cudaFuncSetAttribute(iw_to_tau_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  GF2_PROF(ctx, GF2_K_IW2TAU,
           (iw_to_tau_kernel<<<N2 / E, 512, smem, ctx->stream>>>(
               N2, M, ctx->log2M, ctx->n_iw, E, ctx->beta, reinterpret_cast<const double2 *>(d_X_iw), coef,
               ctx->d_iw_pole_fold, ctx->d_tau_pole, ctx->d_twiddle, ctx->d_twiddle + M / 2, ctx->n_tau,
               ctx->d_tau_index, d_X_tau)));
  GF2_CK_LAUNCH(ctx, "iw_to_tau_kernel");
  return GF2_OK;
}

extern "C" gf2_status gf2_fft_tau_to_iw(gf2_ctx *ctx, const double *d_X_tau, double *d_X_iw, double *d_sig12) {
  if (!ctx) return GF2_ERR_ARG;
  if (!d_X_tau || !d_X_iw) return gf2_fail(ctx, GF2_ERR_ARG, "gf2_fft_tau_to_iw: NULL pointer");
  const int N2 = ctx->N * ctx->N, M = ctx->M;
  if (ctx->d_tau_index) {  // non-equidistant grid
    const int K = ctx->n_tau - 1;
    const size_t smem = gf2_grid_smem_bytes(M, ctx->n_tau);
    GF2_CK(ctx, cudaFuncSetAttribute(tau_to_iw_grid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    GF2_PROF(ctx, GF2_K_TAU2IW,
             (tau_to_iw_grid_kernel<<<N2, 512, smem, ctx->stream>>>(
                 N2, M, ctx->log2M, K, ctx->n_iw, d_X_tau, ctx->d_twiddle, ctx->d_twiddle + M / 2, ctx->d_grid_lag,
                 ctx->d_tau_index, ctx->d_fine_a, ctx->d_grid_mu, reinterpret_cast<double2 *>(d_X_iw))));
    GF2_CK_LAUNCH(ctx, "tau_to_iw_grid_kernel");
    if (d_sig12) {
      SlopeWeights sw;
      for (int j = 0; j < 8; ++j) sw.w[j] = ctx->grid_dw[j];
      sigma_ends_grid_kernel<<<(N2 + 255) / 256, 256, 0, ctx->stream>>>(N2, K, sw, d_X_tau, d_sig12);
      GF2_CK_LAUNCH(ctx, "sigma_ends_grid_kernel");
    }
    return GF2_OK;
  }
  const int E = pick_elems_per_cta(N2, M);
  const size_t smem = (size_t)E * M * sizeof(double2) + sizeof(double) * 8 * E;
  GF2_CK(ctx, cudaFuncSetAttribute(tau_to_iw_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  GF2_PROF(ctx, GF2_K_TAU2IW,
           (tau_to_iw_kernel<<<N2 / E, 512, smem, ctx->stream>>>(
               N2, M, ctx->log2M, ctx->n_iw, E, d_X_tau, ctx->d_twiddle, ctx->d_twiddle + M / 2, ctx->d_t2w_w,
               ctx->d_t2w_corr, reinterpret_cast<double2 *>(d_X_iw))));
  GF2_CK_LAUNCH(ctx, "tau_to_iw_kernel");
  if (d_sig12) {
    sigma_ends_kernel<<<(N2 + 255) / 256, 256, 0, ctx->stream>>>(N2, M, ctx->beta / M, d_X_tau, d_sig12);
    GF2_CK_LAUNCH(ctx, "sigma_ends_kernel");
  }
  return GF2_OK;
}
