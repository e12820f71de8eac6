"""Matsubara <-> imaginary-time transforms, written as direct sums.

Conventions (fermions, real AO basis, closed shell):
    X(i w_n) = int_0^beta e^{i w_n tau} X(tau) dtau,
    X(tau)   = (1/beta) sum_{n in Z} e^{-i w_n tau} X(i w_n),
    w_n = (2n+1) pi / beta,  X(-i w) = conj X(i w).

High-frequency tail (the paper's G ~ G1/w + G2/w^2 + G3/w^3 + ..., with the
moments written out here from the expansion of Eq. GF, four of them):
    G1 = S^-1,  G2 = S^-1 X S^-1,  G3 = S^-1 (X S^-1 X + Sig1) S^-1,
    G4 = S^-1 (X S^-1 X S^-1 X + X S^-1 Sig1 + Sig1 S^-1 X + Sig2) S^-1,
with X = F - mu S and Sigma(z) ~ Sig1/z + Sig2/z^2 + ...  The tail function
is this moment series resummed about a real pole a > 0,
    T(z) = sum_{r=1..4} c_r / (z - a)^r,   c_r = sum_j binom(r-1, j) (-a)^j G_{r-j},
which has the same expansion G1/z + ... + G4/z^4 + O(z^-5) but stays bounded
at low frequency (|T| <= sum |c_r| / a^r), so that subtracting it costs no
digits.  Its imaginary-time image on (0, beta) is
    1/(z-a)^r -> (1/(r-1)!) d^{r-1}/da^{r-1} [ -e^{-a tau} / (1 + e^{-a beta}) ].

iw -> tau:  X(tau_k) = (2/beta) sum_{n<n_iw} Re[e^{-i w_n tau_k} (X - T)(i w_n)] + T(tau_k).

tau -> iw:  the integral of e^{i w tau} times the piecewise-cubic interpolant of
the samples: on [tau_a, tau_{a+1}] the cubic through nodes a-1..a+2 (nodes
0..3 on the first interval, M-3..M on the last), integrated exactly.  The
same interpolant gives the expansion coefficients Sig1 = -(X(0)+X(beta)) and
Sig2 = X'(0+) + X'(beta-).

On a non-equidistant grid (``grids.power_mesh``) both directions keep these
definitions: iw -> tau is the same sum evaluated at the grid's points, and
tau -> iw integrates the same local cubics, now through unequally spaced
nodes (``grid_fourier_weights``, ``sigma_expansion_grid``).
"""

import numpy as np

from .grids import matsubara, tau_grid


def tail_moments(S, F, mu, sig1=None, sig2=None):
    """[4, N, N] moments G1..G4 of G(z) = [(z+mu)S - F - Sigma(z)]^-1."""
    n = S.shape[0]
    sig1 = np.zeros((n, n)) if sig1 is None else sig1
    sig2 = np.zeros((n, n)) if sig2 is None else sig2
    Si = np.linalg.inv(S)
    X = F - mu * S
    g1 = Si
    g2 = Si @ X @ Si
    g3 = Si @ (X @ Si @ X + sig1) @ Si
    g4 = Si @ (X @ Si @ X @ Si @ X + X @ Si @ sig1 + sig1 @ Si @ X + sig2) @ Si
    return np.array([g1, g2, g3, g4])


TAIL_POLE = 1.0   # a, in hartree


def pole_coefficients(moments, a=TAIL_POLE):
    """c_1..c_4 of T(z) = sum c_r (z-a)^-r matching G_1..G_4 to order z^-4."""
    g1, g2, g3, g4 = moments
    c1 = g1
    c2 = g2 - a * g1
    c3 = g3 - 2.0 * a * g2 + a * a * g1
    c4 = g4 - 3.0 * a * g3 + 3.0 * a * a * g2 - a ** 3 * g1
    return np.array([c1, c2, c3, c4])


def tail_iw(moments, w, a=TAIL_POLE):
    c = pole_coefficients(moments, a)
    d = 1j * np.asarray(w)[:, None, None] - a
    return sum(c[r][None] / d ** (r + 1) for r in range(4))


def tail_tau(moments, tau, beta, a=TAIL_POLE):
    """Imaginary-time image of ``tail_iw`` at the given 0 <= tau <= beta."""
    c = pole_coefficients(moments, a)
    t = np.asarray(tau, dtype=np.float64)[:, None, None]
    e = np.exp(-a * t)
    q = np.exp(-a * beta)
    u = 1.0 / (1.0 + q)                      # 1 - f(a)
    v = u * (q / (1.0 + q))                  # u (1 - u)
    u1 = beta * v                            # du/da
    u2 = beta ** 2 * v * (1.0 - 2.0 * u)     # d2u/da2
    u3 = beta ** 3 * v * (1.0 - 6.0 * u + 6.0 * u * u)
    g = [-e * u,
         e * (t * u - u1),
         e * (-t * t * u + 2.0 * t * u1 - u2) / 2.0,
         e * (t ** 3 * u - 3.0 * t * t * u1 + 3.0 * t * u2 - u3) / 6.0]
    return sum(g[r] * c[r][None] for r in range(4))


def _phase(n_idx, k_idx, M, sign):
    """exp(sign * i * w_n * tau_k) with w_n tau_k = pi (2n+1) k / M, reduced exactly."""
    num = np.mod(np.outer(k_idx, 2 * np.asarray(n_idx) + 1), 2 * M)
    return np.exp(sign * 1j * np.pi * num / M)


def iw_to_tau(X_iw, moments, beta, n_tau, chunk=512, taus=None):
    """[n_tau, N, N] real X(tau_k) from X(i w_n), n = 0..n_iw-1 (or only the
    grid indices listed in ``taus``, in that order)."""
    n_iw, n, _ = X_iw.shape
    M = n_tau - 1
    ks_all = np.arange(n_tau) if taus is None else np.asarray(taus, dtype=np.int64)
    w = matsubara(beta, n_iw)
    R = (X_iw - tail_iw(moments, w)).reshape(n_iw, n * n)
    out = np.empty((len(ks_all), n * n))
    for i0 in range(0, len(ks_all), chunk):
        ks = ks_all[i0:i0 + chunk]
        E = _phase(np.arange(n_iw), ks, M, -1.0)
        out[i0:i0 + len(ks)] = (2.0 / beta) * np.real(E @ R)
    return out.reshape(len(ks_all), n, n) + tail_tau(moments, tau_grid(beta, n_tau)[ks_all], beta)


def _monomial_moments(theta):
    """mu_p(theta) = int_0^1 x^p e^{i theta x} dx for p = 0..3 (array over theta)."""
    theta = np.asarray(theta, dtype=np.float64)
    out = np.empty((4,) + theta.shape, dtype=np.complex128)
    small = np.abs(theta) < 1.0
    ts = theta[small]
    for p in range(4):
        acc = np.zeros(ts.shape, dtype=np.complex128)
        term = np.ones(ts.shape, dtype=np.complex128)
        for m in range(30):
            acc += term / (p + m + 1)
            term = term * (1j * ts) / (m + 1)
        out[p][small] = acc
    tl = theta[~small]
    e = np.exp(1j * tl)
    prev = (e - 1.0) / (1j * tl)
    out[0][~small] = prev
    for p in range(1, 4):
        prev = (e - p * prev) / (1j * tl)
        out[p][~small] = prev
    return out


def _lagrange_monomials(offsets):
    """coef[j, p]: x^p coefficient of the Lagrange basis polynomial of node j."""
    coef = np.zeros((4, 4))
    for j, sj in enumerate(offsets):
        others = [s for r, s in enumerate(offsets) if r != j]
        denom = np.prod([sj - s for s in others])
        poly = np.poly(others)[::-1] / denom   # ascending powers
        coef[j] = poly
    return coef


def cubic_fourier_weights(beta, n_tau, n_iw):
    """[n_iw, n_tau] complex weights: X(i w_n) = sum_k Wt[n, k] X(tau_k)."""
    M = n_tau - 1
    h = beta / M
    w = matsubara(beta, n_iw)
    mu = _monomial_moments(w * h)                      # [4, n_iw]
    Wt = np.zeros((n_iw, n_tau), dtype=np.complex128)
    n_idx = np.arange(n_iw)
    patterns = {"first": (0, 1, 2, 3), "interior": (-1, 0, 1, 2), "last": (-2, -1, 0, 1)}
    coefs = {k: _lagrange_monomials(v) for k, v in patterns.items()}
    for a in range(M):
        kind = "first" if a == 0 else ("last" if a == M - 1 else "interior")
        offs = patterns[kind]
        ph = _phase(n_idx, [a], M, 1.0)[0]            # e^{i w_n tau_a}
        integ = coefs[kind] @ mu                       # [4 nodes, n_iw]
        for j, s in enumerate(offs):
            Wt[:, a + s] += h * ph * integ[j]
    return Wt


def tau_to_iw(X_tau, beta, n_iw, chunk=1024):
    """[n_iw, N, N] complex X(i w_n) from samples X(tau_k), k = 0..M."""
    n_tau, n, _ = X_tau.shape
    Wt = cubic_fourier_weights(beta, n_tau, n_iw)
    flat = X_tau.reshape(n_tau, n * n)
    out = np.empty((n_iw, n * n), dtype=np.complex128)
    for i0 in range(0, n_iw, chunk):
        out[i0:i0 + chunk] = Wt[i0:i0 + chunk] @ flat
    return out.reshape(n_iw, n, n)


def sigma_expansion(X_tau, beta):
    """(Sig1, Sig2): coefficients of 1/z and 1/z^2 in the transform of the interpolant."""
    M = X_tau.shape[0] - 1
    h = beta / M
    x = X_tau
    sig1 = -(x[0] + x[M])
    d0 = (-11.0 * x[0] + 18.0 * x[1] - 9.0 * x[2] + 2.0 * x[3]) / (6.0 * h)
    dM = (11.0 * x[M] - 18.0 * x[M - 1] + 9.0 * x[M - 2] - 2.0 * x[M - 3]) / (6.0 * h)
    return sig1, d0 + dM


def grid_fourier_weights(beta, M, index, n_iw):
    """[n_iw, n_tau] complex weights, X(i w_n) = sum_k Wt[n, k] X(tau_k), on the
    grid tau_k = index[k] beta / M: on [tau_a, tau_a+1] the cubic through the
    nodes a-1..a+2 (0..3 on the first interval, K-3..K on the last, K = n_tau - 1),
    integrated exactly against e^{i w tau}.  With index = 0..M this is
    ``cubic_fourier_weights``."""
    idx = np.asarray(index, dtype=np.int64)
    K = len(idx) - 1
    w = matsubara(beta, n_iw)
    n_idx = np.arange(n_iw)
    Wt = np.zeros((n_iw, K + 1), dtype=np.complex128)
    moments = {}
    for a in range(K):
        first = 0 if a == 0 else (K - 3 if a == K - 1 else a - 1)
        nodes = list(range(first, first + 4))
        r = int(idx[a + 1] - idx[a])                 # interval length in steps of beta / M
        h = r * beta / M
        offs = [(idx[j] - idx[a]) / r for j in nodes]
        if r not in moments:
            moments[r] = _monomial_moments(w * h)    # [4, n_iw]
        integ = _lagrange_monomials(offs) @ moments[r]
        ph = _phase(n_idx, [idx[a]], M, 1.0)[0]     # e^{i w_n tau_a}
        for j, node in enumerate(nodes):
            Wt[:, node] += h * ph * integ[j]
    return Wt


def tau_to_iw_grid(X_tau, beta, M, index, n_iw, chunk=1024):
    """[n_iw, N, N] complex X(i w_n) from the samples on a non-equidistant grid."""
    n_tau, n, _ = X_tau.shape
    Wt = grid_fourier_weights(beta, M, index, n_iw)
    flat = X_tau.reshape(n_tau, n * n)
    out = np.empty((n_iw, n * n), dtype=np.complex128)
    for i0 in range(0, n_iw, chunk):
        out[i0:i0 + chunk] = Wt[i0:i0 + chunk] @ flat
    return out.reshape(n_iw, n, n)


def _lagrange_derivative(nodes, at):
    """d/dtau of the Lagrange basis polynomials of ``nodes`` at ``at``."""
    out = []
    for j, tj in enumerate(nodes):
        acc = 0.0
        for m, tm in enumerate(nodes):
            if m == j:
                continue
            term = 1.0 / (tj - tm)
            for l, tl in enumerate(nodes):
                if l != j and l != m:
                    term *= (at - tl) / (tj - tl)
            acc += term
        out.append(acc)
    return np.array(out)


def sigma_expansion_grid(X_tau, beta, M, index):
    """(Sig1, Sig2) of the interpolant on a non-equidistant grid: -(X(0)+X(beta))
    and the slopes of the first and last cubics at tau = 0 and tau = beta."""
    t = np.asarray(index, dtype=np.float64) * (beta / M)
    K = len(t) - 1
    sig1 = -(X_tau[0] + X_tau[K])
    w0 = _lagrange_derivative(t[:4], t[0])
    wK = _lagrange_derivative(t[K - 3:], t[K])
    d0 = sum(w0[j] * X_tau[j] for j in range(4))
    dK = sum(wK[j] * X_tau[K - 3 + j] for j in range(4))
    return sig1, d0 + dK
