"""Eq. Sigma on density-fitted integrals: the cost-reduction route that the
paper's computational details and conclusions name (O(n^3 m), m auxiliary
functions).  The paper gives no formula beyond that remark; this module takes
the integrals as the three-index factorisation

    v_ijkl = sum_Q B[Q,i,j] B[Q,k,l]

and evaluates Eq. Sigma with them.  TEST INFRASTRUCTURE ONLY: see the
package header.

``df_eri`` writes the fitted integrals out; ``sigma_df`` is Eq. Sigma on them
(the definition, through ``sigma.sigma_factored``).  ``sigma_df_factors`` is
the same quantity written in the factors alone, with no four-index tensor:
substituting the factorisation into Eq. Sigma and summing over k, l, m, n, p, q
in matrix products gives

    C^Q  = B^Q G,   X^Q = Gbar C^Q = Gbar B^Q G,   t_QR = Tr(X^Q B^R)
    Sigma = - sum_Q C^Q ( 2 sum_R t_QR B^R  -  sum_R B^R X^Q B^R )

The first (Coulomb-like) term costs O(m n^3 + m^2 n^2) per time point, which
is the paper's O(n^3 m); the second (exchange-like) term costs O(m^2 n^3), or
O(m n^4) when sum_R B^R X B^R is taken as the contraction of X with the
fitted four-index v.
"""

import numpy as np

from .sigma import exchange_combination, gbar_from_grid, sigma_factored


def df_eri(B):
    """v[i,j,k,l] = sum_Q B[Q,i,j] B[Q,k,l]."""
    m, n = B.shape[0], B.shape[1]
    Bf = B.reshape(m, n * n)
    return (Bf.T @ Bf).reshape(n, n, n, n)


def sigma_df(G, Gbar, B):
    """Eq. Sigma for one time point on the fitted integrals."""
    return sigma_factored(G, Gbar, df_eri(B))


def sigma_df_factors(G, Gbar, B):
    """The same from the factors: C^Q, X^Q, t_QR and the two terms above."""
    C = B @ G                                         # [Q, i, n] = (B^Q G)_in
    X = Gbar[None] @ C                                # [Q, p, l] = (Gbar B^Q G)_pl
    t = np.einsum("qpl,rlp->qr", X, B)                # Tr(X^Q B^R)
    coul = np.einsum("qr,rnj->qnj", t, B)             # sum_R t_QR B^R
    exch = np.array([np.matmul(B @ Xq, B).sum(0) for Xq in X])   # sum_R B^R X^Q B^R
    return -np.einsum("qin,qnj->ij", C, 2.0 * coul - exch)


def sigma_tau_df(G_tau, B, taus=None):
    """Sigma(tau_k) on the fitted integrals for every grid point (or ``taus``)."""
    v = df_eri(B)
    W = exchange_combination(v)
    idx = range(G_tau.shape[0]) if taus is None else taus
    return np.array([sigma_factored(G_tau[k], gbar_from_grid(G_tau, k), v, W) for k in idx])
