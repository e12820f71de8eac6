"""Eq. GF, the density matrix and the chemical-potential search.

    G(i w_n) = [(i w_n + mu) S - F - Sigma(i w_n)]^-1      (dense LU inverse)

Density (spin-summed): P = -2 G(beta^-), i.e. the tau -> beta^- end of the
Matsubara sum with the tail of ``transforms.tail_iw`` taken out and added back
in closed form:

    P = (4/beta) sum_{n<n_iw} Re (G - T)(i w_n) - 2 T(beta)

Chemical potential (step 2.a of the supplement: a mu giving the right particle
number): plain bisection on N(mu) = Tr(P(mu) S), stopping at the first
midpoint with |N(mu) - N_e| <= tol.
"""

import numpy as np
import scipy.linalg as sla

from .grids import matsubara
from .transforms import tail_iw, tail_moments, tail_tau


def dyson(mu, S, F, Sigma_iw, beta, n_iw=None):
    n_iw = Sigma_iw.shape[0] if Sigma_iw is not None else n_iw
    w = matsubara(beta, n_iw)
    A = (1j * w + mu)[:, None, None] * S[None] - F[None]
    if Sigma_iw is not None:
        A = A - Sigma_iw
    return np.linalg.inv(A)


def density(G_iw, moments, beta):
    w = matsubara(beta, G_iw.shape[0])
    R = np.real(G_iw - tail_iw(moments, w)).sum(axis=0)
    return (4.0 / beta) * R - 2.0 * tail_tau(moments, [beta], beta)[0]


def electron_count(P, S):
    return float(np.trace(P @ S))


def density_at(mu, S, F, Sigma_iw, sig1, sig2, beta, n_iw):
    G = dyson(mu, S, F, Sigma_iw, beta, n_iw)
    P = density(G, tail_moments(S, F, mu, sig1, sig2), beta)
    return G, P


def mu_search(S, F, Sigma_iw, sig1, sig2, n_elec, beta, n_iw, tol=1e-10, max_iter=200):
    """Bisection for mu; returns (mu, G_iw, P, n_evaluations)."""
    eps = sla.eigh(F, S, eigvals_only=True)
    lo, hi = eps.min() - 1.0, eps.max() + 1.0
    evals = 0

    def count(mu):
        nonlocal evals
        evals += 1
        G, P = density_at(mu, S, F, Sigma_iw, sig1, sig2, beta, n_iw)
        return electron_count(P, S), G, P

    for _ in range(60):
        if count(lo)[0] < n_elec:
            break
        lo -= 2.0 * (hi - lo)
    for _ in range(60):
        if count(hi)[0] > n_elec:
            break
        hi += 2.0 * (hi - lo)
    for _ in range(max_iter):
        mid = 0.5 * (lo + hi)
        n, G, P = count(mid)
        if abs(n - n_elec) <= tol:
            return mid, G, P, evals
        if n < n_elec:
            lo = mid
        else:
            hi = mid
    raise RuntimeError("chemical-potential bisection did not converge")
