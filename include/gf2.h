/*
 * libgf2 -- GB300 (sm_103a) library for the hot path of one self-consistent
 * GF2 iteration (Phillips & Zgid, arXiv:1405.3273).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - N basis functions (real, non-orthogonal AO basis), closed shell.
 *  - Matrices are dense row-major [N][N] FP64.  Integrals are chemists'
 *    notation, v[i][j][k][l] = (ij|kl), dense [N][N][N][N] FP64 with the
 *    8-fold permutational symmetry of real orbitals.
 *  - Imaginary time: uniform grid tau_k = k*beta/M, k = 0..M, M = n_tau-1.
 *    Tau-dependent matrices are [n_tau][N][N] FP64, real symmetric.
 *  - Matsubara frequencies w_n = (2n+1)*pi/beta for n = 0..n_iw-1 (negative
 *    frequencies follow from X(-iw) = conj X(iw)).  Frequency-dependent
 *    matrices are [n_iw][N][N] complex128 stored as interleaved (re, im)
 *    FP64 pairs.
 *  - Transform conventions: X(iw) = int_0^beta e^{iw tau} X(tau) dtau and
 *    X(tau) = (1/beta) sum_n e^{-iw tau} X(iw).  G is the per-spin Green's
 *    function, P the spin-summed density (P = -2 G(beta^-)).
 *
 * Ownership and errors
 * --------------------
 *  - Every d_* argument is a DEVICE pointer owned by the caller; the library
 *    never frees or retains it beyond the call (except gf2_set_integrals,
 *    which copies).  Host scalars are returned through host pointers.
 *  - The context owns its workspace (intermediates, split copies of the
 *    integrals, grid tables) and allocates it at gf2_create /
 *    gf2_set_integrals.  All work is stream-ordered on the context stream;
 *    calls that return host scalars or check a device error word synchronize
 *    that stream (each says so below).
 *  - Every call returns a gf2_status.  Invalid sizes or NULL pointers give
 *    GF2_ERR_ARG before any launch; a CUDA failure gives GF2_ERR_CUDA; device
 *    loops that give up after their iteration limit report GF2_ERR_TIMEOUT.
 *    gf2_last_error() returns a message for the last failure on the context.
 *    No call aborts the process or throws across the ABI.
 */
#ifndef GF2_H
#define GF2_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GF2_OK = 0,
  GF2_ERR_ARG = 1,
  GF2_ERR_CUDA = 2,
  GF2_ERR_NOMEM = 3,
  GF2_ERR_NOT_CONVERGED = 4,
  GF2_ERR_TIMEOUT = 5,
  GF2_ERR_NONFINITE = 6,
  GF2_ERR_UNSUPPORTED = 7
} gf2_status;

/* Arithmetic of the self-energy contraction.
 *   GF2_PREC_FP64    FP64 everywhere (CUDA cores).
 *   GF2_PREC_BF16X3  every operand split x = x_hi + x_lo into two BF16 terms,
 *                    three products hi*hi + hi*lo + lo*hi per multiply, FP32
 *                    accumulation on the tcgen05 tensor cores, FP64 for the
 *                    final sum over each block of the last contraction.
 *   GF2_PREC_BF16X6  three BF16 terms, six products (i + j <= 2).
 *   GF2_PREC_FP16X3  two FP16 terms, three products.  FP16 has three more
 *                    significand bits than BF16 but a narrow exponent range, so
 *                    every FP16 operand carries a power-of-two scale that puts
 *                    its largest entry in [2^13, 2^14): one for v, one for W,
 *                    one per G(tau) and per G(-tau), and per time point for
 *                    each intermediate (from a bound for the first, from the
 *                    measured maximum for the other two); the scales are
 *                    removed exactly.
 *   GF2_PREC_FP16X6  three FP16 terms, six products, the same scaling. */
typedef enum {
  GF2_PREC_FP64 = 0,
  GF2_PREC_BF16X3 = 1,
  GF2_PREC_BF16X6 = 2,
  GF2_PREC_FP16X3 = 3,
  GF2_PREC_FP16X6 = 4
} gf2_prec;

typedef struct gf2_ctx gf2_ctx;

/* Create a context for N basis functions (1 <= N <= 128), n_tau time points
 * of the uniform grid tau_k = k beta / M (M = n_tau - 1 a power of two,
 * 8 <= M <= 8192), 1 <= n_iw <= 2^20 Matsubara frequencies and inverse
 * temperature beta > 0, bound to the CUDA stream `stream` (a cudaStream_t;
 * NULL = legacy default stream) on the current device.  *out receives the
 * context; GF2_ERR_ARG for sizes out of range (nothing is touched then). */
gf2_status gf2_create(gf2_ctx **out, int n_bf, int n_tau, int n_iw, double beta, void *stream);

/* The same on a non-equidistant time grid (the paper builds Sigma(tau) on a
 * non-equidistant grid of a few thousand points, Computational details): the
 * n_tau points tau_k = tau_index[k] beta / M, a subset of the uniform grid of
 * M intervals (M a power of two, 8 <= M <= 8192).  h_tau_index: host array
 * of n_tau ints (8 <= n_tau <= M + 1), strictly increasing from 0 to M and
 * symmetric, tau_index[k] + tau_index[n_tau-1-k] = M (so that G(-tau_k) =
 * -G(tau_{n_tau-1-k}) stays on the grid); copied, not kept.  The uniform
 * power mesh (p halvings, u steps per interval: M = 2^(p+1) u, 2 (p+1) u + 1
 * points) is the intended use.  On such a context gf2_fft_iw_to_tau writes
 * the n_tau grid points, gf2_fft_tau_to_iw integrates the local cubics
 * through the unequally spaced nodes (see there), and every other call works
 * on the n_tau points unchanged.  GF2_ERR_ARG for an invalid grid,
 * GF2_ERR_UNSUPPORTED when the transform's shared memory (16 M + 40 n_tau
 * bytes) exceeds 227 KB. */
gf2_status gf2_create_grid(gf2_ctx **out, int n_bf, int M, int n_tau, const int *h_tau_index, int n_iw,
                           double beta, void *stream);
gf2_status gf2_destroy(gf2_ctx *ctx);
gf2_status gf2_set_stream(gf2_ctx *ctx, void *stream);
const char *gf2_status_string(gf2_status s);
const char *gf2_last_error(const gf2_ctx *ctx);

/* Copy the two-electron integrals v [N^4] into the context and build the
 * exchange combination W_lpnj = 2 v_lpnj - v_nplj of Eq. Sigma plus its BF16
 * and FP16 split copies for the tensor-core path (for N <= 32 as floor(64/N)
 * diagonal blocks, so that several time points share one 64-wide tile; for
 * N > 64 the 128-wide copies are built by the first split-precision call). */
gf2_status gf2_set_integrals(gf2_ctx *ctx, const double *d_v);

/* Give the context the overlap S [N][N] (symmetric positive definite).  The
 * split-precision Sigma path then evaluates Eq. Sigma in the symmetrically
 * orthogonalised basis (G' = S^1/2 G S^1/2, v' = (S^-1/2)^{x4} v, returned as
 * Sigma = S^1/2 Sigma' S^1/2), where the entries of G' are bounded by one and
 * FP32 accumulation loses no digits to the cancellations that an ill-
 * conditioned S produces in the AO basis.  Mathematically the same Sigma (the
 * equation is covariant); the FP64 path is unaffected.  Optional; may be
 * called before or after gf2_set_integrals. */
gf2_status gf2_set_overlap(gf2_ctx *ctx, const double *d_S);

/* Eq. Sigma (the paper's second-order self-energy):
 *   Sigma_ij(tau) = - sum_klmnpq G_kl(tau) G_mn(tau) G_pq(-tau) v_imqk (2 v_lpnj - v_nplj)
 * with G(-tau_k) = -G(tau_{M-k}).  d_G_tau [n_tau][N][N] in, d_Sigma_tau
 * [n_tau][N][N] out.  Requires gf2_set_integrals first.  prec is a gf2_prec;
 * the split precisions run on 64-wide tiles for N <= 64 and on 128-wide tiles
 * for 64 < N <= 128 (whose term planes, about 6.4 GB, and FP32 intermediates,
 * up to 2 x 16 GB for chunks of 16 time points, are allocated by the first
 * split call), and synchronize the context stream to read the pipeline's
 * error word (GF2_ERR_TIMEOUT if a bounded wait gave up); FP64 is
 * stream-ordered.  When v has the pair symmetry (ij|kl) = (kl|ij) (checked at
 * gf2_set_integrals, to 1e-12 relative) the 64-wide path computes half of the
 * stage-2 intermediate and mirrors it. */
gf2_status gf2_sigma_tau(gf2_ctx *ctx, const double *d_G_tau, double *d_Sigma_tau, int prec);

/* The same for the `count` grid points k0 .. k0+count-1 only: d_G_tau is the
 * full [n_tau][N][N] grid (G(-tau) needs the mirrored points), d_Sigma_out
 * receives [count][N][N]. */
gf2_status gf2_sigma_tau_points(gf2_ctx *ctx, const double *d_G_tau, int k0, int count,
                                double *d_Sigma_out, int prec);

/* Density-fitted integrals (the O(n^3 m) route named in the paper's
 * computational details and conclusions, m auxiliary functions):
 *   v_ijkl = sum_Q B[Q][i][j] B[Q][k][l].
 * d_B: device [m][N][N] FP64, row-major, read during the call (the context
 * keeps a copy).  The fitted v replaces the context's integrals, with W and
 * the split copies rebuilt as by gf2_set_integrals, so gf2_sigma_tau, the
 * Fock build and the energy then use them too.  A later gf2_set_integrals
 * discards the factor.  GF2_ERR_ARG for a NULL pointer or m outside
 * 1..65535; GF2_ERR_NOMEM if the copy (m N^2 doubles) cannot be allocated. */
gf2_status gf2_set_df_integrals(gf2_ctx *ctx, const double *d_B, int m);

/* Eq. Sigma on the density-fitted integrals, in the factor order: with
 * C^Q = B^Q G(tau) and X^Q = G(-tau) C^Q,
 *   Sigma(tau) = - sum_Q C^Q U^Q,   U^Q_nj = sum_lp X^Q_pl (2 v_lpnj - v_nplj),
 * 2 m N^4 + 6 m N^3 flops per time point and 3 m N^2 doubles of workspace per
 * time point (chunks of up to 1 GB, allocated by the first call), no N^4
 * intermediate.  The same Sigma as gf2_sigma_tau after gf2_set_df_integrals,
 * to rounding.  Grid points k0 .. k0+count-1 of the full d_G_tau
 * [n_tau][N][N]; d_Sigma_out [count][N][N].  prec: GF2_PREC_FP64 (others give
 * GF2_ERR_UNSUPPORTED).  GF2_ERR_ARG without gf2_set_df_integrals, for a NULL
 * pointer or a range outside the grid.  Stream-ordered. */
gf2_status gf2_sigma_tau_df(gf2_ctx *ctx, const double *d_G_tau, int k0, int count, double *d_Sigma_out,
                            int prec);

/* High-frequency moments G1..G4 of G(z) = [(z + mu) S - F - Sigma(z)]^-1 for
 * Sigma(z) ~ Sig1/z + Sig2/z^2 (the analytic tail named in the paper's
 * section on the Fourier transforms):
 *   G1 = S^-1, G2 = S^-1 X S^-1, G3 = S^-1 (X S^-1 X + Sig1) S^-1,
 *   G4 = S^-1 (X S^-1 X S^-1 X + X S^-1 Sig1 + Sig1 S^-1 X + Sig2) S^-1,
 * X = F - mu S.  d_sig12 = [2][N][N] (Sig1, Sig2) or NULL for zero.
 * d_moments receives [4][N][N]. */
gf2_status gf2_tail_moments(gf2_ctx *ctx, const double *d_S, const double *d_F, double mu,
                            const double *d_sig12, double *d_moments);

/* Matsubara -> imaginary time (G(w) -> G(tau) of step 2.b):
 *   X(tau_k) = (2/beta) sum_{n<n_iw} Re[e^{-i w_n tau_k} (X - T)(i w_n)] + T(tau_k),
 * T = the moment series of d_moments [4][N][N] resummed about a real pole
 * a = 1 hartree, T(z) = sum_r c_r (z - a)^-r, whose tau image is closed form.
 * Evaluated by one M-point FFT per matrix element (n_iw may exceed M; the
 * frequencies are folded modulo M) and written at the context's n_tau grid
 * points.  d_X_iw [n_iw][N][N] c128 in, d_X_tau [n_tau][N][N] out. */
gf2_status gf2_fft_iw_to_tau(gf2_ctx *ctx, const double *d_X_iw, const double *d_moments,
                             double *d_X_tau);

/* Imaginary time -> Matsubara (Sigma(tau) -> Sigma(w) of step 3):
 *   X(i w_n) = int_0^beta e^{i w_n tau} X~(tau) dtau,
 * X~ = the piecewise-cubic interpolant of the samples (on [tau_a, tau_a+1]
 * the cubic through nodes a-1..a+2; nodes 0..3 and K-3..K at the ends,
 * K = n_tau - 1), integrated exactly.  Uniform grid: an M-point FFT times an
 * attenuation factor plus end-point corrections.  Non-equidistant grid
 * (gf2_create_grid): each grid interval's cubic re-expanded on the uniform
 * steps inside it, then two M-point FFTs of those coefficients (four real
 * sequences) weighted by the exact monomial integrals of one step.
 * d_X_tau [n_tau][N][N] in, d_X_iw [n_iw][N][N] c128 out.  If d_sig12 is not NULL it receives [2][N][N] = (Sig1, Sig2), the
 * 1/z and 1/z^2 coefficients of the result: Sig1 = -(X(0) + X(beta)),
 * Sig2 = X~'(0+) + X~'(beta-). */
gf2_status gf2_fft_tau_to_iw(gf2_ctx *ctx, const double *d_X_tau, double *d_X_iw, double *d_sig12);

/* Eq. GF: G(i w_n) = [(i w_n + mu) S - F - Sigma(i w_n)]^-1 for every n
 * (FP64 complex; d_Sigma_iw may be NULL for Sigma = 0). */
gf2_status gf2_dyson(gf2_ctx *ctx, double mu, const double *d_S, const double *d_F,
                     const double *d_Sigma_iw, double *d_G_iw);

/* Spin-summed density P = -2 G(beta^-) = (4/beta) sum_n Re (G - T)(i w_n) - 2 T(beta),
 * with T built from d_moments [4][N][N] as in gf2_fft_iw_to_tau. */
gf2_status gf2_density(gf2_ctx *ctx, const double *d_G_iw, const double *d_moments, double *d_P);

/* Step 2.a: find mu with Tr(P(mu) S) = n_elec to |error| <= tol, P(mu) from
 * Eq. GF and gf2_density.  Bracketing search started at *mu_inout (expanded
 * outward until it brackets), then Brent's method (inverse quadratic
 * interpolation with bisection safeguards).  When n_iw >= 2048 a coarse stage
 * runs first: the same search on the count from the lowest n_iw/8 frequencies
 * plus the analytic tail (Dyson at an eighth of the cost), which places mu
 * and the local slope dN/dmu; the full-frequency search then starts there
 * with the Newton step as its first probe.  Convergence is decided on the
 * full count only.  At most max_iter full evaluations (GF2_ERR_NOT_CONVERGED
 * beyond).  On success *mu_inout = mu, d_G_iw and d_P hold G(i w) and P at that
 * mu from a full evaluation, *n_eval (if not NULL) = number of Dyson
 * evaluations, coarse and full.  Synchronizes. */
gf2_status gf2_mu_search(gf2_ctx *ctx, const double *d_S, const double *d_F,
                         const double *d_Sigma_iw, const double *d_sig12, double n_elec,
                         double tol, int max_iter, double *mu_inout, double *d_G_iw,
                         double *d_P, int *n_eval);

/* Steps 2.a-2.b, the inner self-consistency loop at fixed Sigma: alternate
 * the mu search (as gf2_mu_search, tolerance mu_tol, at most 100 full
 * evaluations) and the Fock rebuild F_out = Fock(P) (as gf2_fock) until the
 * residual R = F_out - F has Frobenius norm below tol; then F = F_out and a
 * last mu search gives G(i w), P and mu at that F.  The next F while
 * |R| > diis_from (or diis = 0) is the damped step F + mix R, which also
 * empties the history; for |R| <= diis_from it is the Pulay (DIIS)
 * combination sum_k c_k F_out_k of the last diis (<= 8) rebuilt matrices,
 * c minimising |sum_k c_k R_k| under sum_k c_k = 1 (the bordered Gram system
 * solved by Gaussian elimination with partial pivoting; a singular system
 * drops the oldest entry).  The supplement damps P instead; the Fock-matrix
 * schedule is this library's convergence aid.
 * The whole loop runs as one CUDA graph whose decisions are taken on the
 * device (a WHILE node around one iteration, the mu search's WHILE node
 * nested in it); the host reads one block of scalars at the end.
 * d_S, d_h [N][N] in; d_F [N][N] in: the start, out: the converged F;
 * d_Sigma_iw [n_iw][N][N] c128 and d_sig12 [2][N][N] in (both may be NULL for
 * Sigma = 0); *mu_inout in: the first search's start, out: mu; d_G_iw, d_P
 * out (must not alias the inputs).  *n_iter = Fock rebuilds, *n_mu_eval =
 * Dyson evaluations of all searches (either may be NULL).  Errors:
 * GF2_ERR_NOT_CONVERGED after max_iter rebuilds or when a mu search misses
 * its tolerance (d_F then holds the last iterate), GF2_ERR_NONFINITE for a
 * vanishing Dyson pivot or a non-finite count or residual.  Synchronizes. */
gf2_status gf2_inner_loop(gf2_ctx *ctx, const double *d_S, const double *d_h, double *d_F,
                          const double *d_Sigma_iw, const double *d_sig12, double n_elec,
                          double *mu_inout, double *d_G_iw, double *d_P, double tol, int max_iter,
                          double mu_tol, int diis, double mix, double diis_from, int *n_iter,
                          int *n_mu_eval);

/* Eq. FockMatrix: F_ij = h_ij + sum_kl P_kl (v_ijlk - v_iklj / 2), with the
 * integrals given to gf2_set_integrals (no index symmetry of v is assumed).
 * d_h, d_P [N][N] in, d_F [N][N] out.  d_F may be d_h (F replaces h in
 * place) but must not be d_P (GF2_ERR_ARG).  The sums are accumulated with
 * FP64 atomics, so their rounding order varies from call to call. */
gf2_status gf2_fock(gf2_ctx *ctx, const double *d_h, const double *d_P, double *d_F);

/* Galitskii-Migdal energy (the paper reports energies but prints no formula):
 *   e_one_body = (1/2) Tr[P (h + F)]
 *   e_two_body = (2/beta) sum_{n<n_iw} Re Tr[G(i w_n) Sigma(i w_n)]
 *                - beta/(2 pi^2) psi_1(n_iw + 1/2) Tr[S^-1 Sig1]
 * (the second term completes the sum over n >= n_iw with G Sigma ~ G1 Sig1 / z^2).
 * d_sig12 may be NULL (no tail).  Synchronizes. */
gf2_status gf2_energy(gf2_ctx *ctx, const double *d_h, const double *d_F, const double *d_P,
                      const double *d_S, const double *d_G_iw, const double *d_Sigma_iw,
                      const double *d_sig12, double *e_one_body, double *e_two_body);

/* Convergence aids of the self-consistent loop.  The supplement damps P in
 * the inner loop and Sigma(tau) in the outer loop (amounts unstated); both
 * are linear combinations of device arrays.  The inner loop also uses Pulay
 * extrapolation of F (no counterpart in the paper), which needs the Gram
 * matrix of the residuals.
 *   gf2_combine: d_out[e] = sum_{k<n} coef[k] d_src[k][e], e < count
 *                (coef: host array of n doubles; d_src: host array of n device
 *                pointers; 1 <= n <= 16; d_out may alias one source).
 *   gf2_gram:    gram_out[a*n + b] = sum_e d_vecs[a][e] d_vecs[b][e]
 *                (gram_out: host array of n*n doubles).  Synchronizes. */
gf2_status gf2_combine(gf2_ctx *ctx, int n, const double *coef, const double *const *d_src,
                       long long count, double *d_out);
gf2_status gf2_gram(gf2_ctx *ctx, int n, const double *const *d_vecs, long long count, double *gram_out);

/* Natural occupation numbers (the observable of the paper's H32 lattice
 * results): d_occ[k] = k-th largest eigenvalue of S^1/2 P S^1/2, halved, i.e.
 * the occupation of the k-th natural spatial orbital (0..1 for a physical
 * closed-shell P; they sum to Tr(PS)/2).  d_P [N][N] spin-summed density in,
 * d_occ [N] out.  Needs gf2_set_overlap (for S^1/2); GF2_ERR_ARG otherwise.
 * Eigenvalues by cyclic Jacobi sweeps; GF2_ERR_NOT_CONVERGED after 60 sweeps.
 * Synchronizes the context stream. */
gf2_status gf2_natural_occupations(gf2_ctx *ctx, const double *d_P, double *d_occ);

/* ---- Batched Eq. Sigma over many systems of uneven size ----
 * The paper builds Sigma(tau) one system at a time; the batch runs the Sigma
 * builds of many independent systems (molecules, geometries) together on one
 * GPU.  Instance i has n_bf[i] basis functions (1..128) and n_tau[i] time
 * points (the gf2_create rules).  Every instance owns a context; the batch
 * also creates up to four worker streams that fork from and join back into
 * `stream` (a cudaStream_t, NULL = legacy default stream).
 *   gf2_batch_set_system: integrals v [N^4] of an instance (copied) and its
 *     overlap S [N][N] (may be NULL: no orthogonalisation, as gf2_set_overlap).
 *   gf2_batch_tune: autotuner.  For every instance it times each admissible
 *     path on a sample of d_G_tau[i] -- the FP64 staged contraction (32
 *     points), and for N <= 64 the split tensor-core pipeline in `prec` with
 *     32 or 16 time-point slots per launch (one chunk each) -- keeps the
 *     fastest (FP64 is always admissible, being more accurate), and
 *     spreads the instances over the worker streams, longest estimated time
 *     first.  d_G_tau: host array of n_inst device pointers [n_tau[i]][N][N].
 *   gf2_batch_plan: the tuner's choice for one instance: precision code it
 *     runs with, estimated ms of one full-grid build, worker stream index,
 *     time-point slots per launch of the split pipeline (32 or 16).  Any
 *     output pointer may be NULL.
 *   gf2_sigma_tau_batched: d_Sigma_tau[i] [n_tau[i]][N][N] <- Eq. Sigma of
 *     instance i from d_G_tau[i] (host arrays of device pointers).  Tunes first
 *     if `prec` differs from the last tuning.  The first call with a given set
 *     of buffers records every instance's launches into one CUDA graph; later
 *     calls with the same buffers (contents may change) replay it with one
 *     graph launch.  Synchronizes `stream`, then checks every instance's
 *     pipeline error word (GF2_ERR_TIMEOUT if a wait gave up).
 *   Errors: GF2_ERR_ARG for bad sizes, instances or NULL pointers; instance
 *   failures are reported with the instance index by gf2_batch_last_error. */
typedef struct gf2_batch gf2_batch;
gf2_status gf2_batch_create(gf2_batch **out, int n_inst, const int *n_bf, const int *n_tau, void *stream);
gf2_status gf2_batch_destroy(gf2_batch *b);
const char *gf2_batch_last_error(const gf2_batch *b);
gf2_status gf2_batch_set_system(gf2_batch *b, int inst, const double *d_v, const double *d_S);
gf2_status gf2_batch_tune(gf2_batch *b, const double *const *d_G_tau, int prec);
gf2_status gf2_batch_plan(const gf2_batch *b, int inst, int *path, double *est_ms, int *lane, int *chunk);
/* Shared tiles: with a BF16 split (GF2_PREC_BF16X3/X6) the tuner pairs every
 * split-path instance with 32 < N <= 64, which pays the whole 64-wide tile
 * set, with the largest other instance of the same n_tau (and both with or
 * both without an overlap) that fits beside it, N_a + N_b <= 64, and runs the
 * two as one block-diagonal system (its Sigma is block-diagonal with the two
 * Sigmas on its diagonal, Eq. Sigma never coupling the blocks); the smaller
 * one then reports est_ms = 0.  *partner = the other instance of inst's pair,
 * or -1.  GF2_ERR_ARG before gf2_batch_tune or for a bad instance. */
gf2_status gf2_batch_partner(const gf2_batch *b, int inst, int *partner);
gf2_status gf2_sigma_tau_batched(gf2_batch *b, const double *const *d_G_tau, double *const *d_Sigma_tau,
                                 int prec);

/* Allocation-free Galitskii-Migdal energy (no counterpart in the paper).
 * The same inputs and outputs as gf2_energy, and the same result to rounding
 * (S^-1 comes from its own Gauss-Jordan sweep), but without a context and
 * without allocating device memory.  It is meant for callers that cannot call
 * cudaMalloc: a host program that gives the library a fixed device-memory
 * budget and forbids the device allocator (an embedding whose own pool owns
 * every byte of the GPU), or code that must not fail on an out-of-memory
 * allocation in the middle of a run.  Its scratch (per-frequency partial sums,
 * S^-1, the two results) is a fixed __device__ array of 65536 + 128*128 + 8
 * doubles (about 655 KB) that every device loading the library keeps until
 * the process exits.
 *   Limits: n_bf <= 128 and n_iw <= 65536, else GF2_ERR_UNSUPPORTED before any
 *   launch; NULL pointers or bad sizes give GF2_ERR_ARG; CUDA failures
 *   GF2_ERR_CUDA.  d_sig12 may be NULL (no tail term).
 *   The first call on a device looks up the array's device address (once per
 *   device, with that device current).  Every call overwrites the shared
 *   array and fully rewrites what it reads, so consecutive calls are
 *   independent; calls that overlap on the GPU (other streams or threads at
 *   the same time) race on it.
 *   Runs on `stream` (a cudaStream_t; NULL = legacy default stream), copies the
 *   two results to the host and synchronizes that stream before returning. */
gf2_status gf2_energy_noalloc(int n_bf, int n_iw, double beta, const double *d_h, const double *d_F,
                              const double *d_P, const double *d_S, const double *d_G_iw,
                              const double *d_Sigma_iw, const double *d_sig12, double *e_one_body,
                              double *e_two_body, void *stream);

/* Tracing (no counterpart in the paper).  gf2_profile(ctx, 1) clears the
 * counters and starts timing every kernel launch of the context with CUDA
 * events on its stream (0 stops; launches are counted either way).
 * gf2_profile_report writes one line "name launches total_ms" per kernel kind
 * into buf (NUL-terminated; GF2_ERR_ARG if buflen is too small) and the
 * number of kernel launches since the last gf2_profile call into *launches
 * (may be NULL).  The report synchronizes on the recorded events. */
gf2_status gf2_profile(gf2_ctx *ctx, int enable);
gf2_status gf2_profile_report(gf2_ctx *ctx, char *buf, int buflen, long long *launches);

#ifdef __cplusplus
}
#endif
#endif /* GF2_H */
