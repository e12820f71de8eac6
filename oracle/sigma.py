"""Second-order self-energy in the AO basis (Eq. Sigma of the paper).

    Sigma_ij(tau) = - sum_{klmnpq} G_kl(tau) G_mn(tau) G_pq(-tau)
                                   v_imqk (2 v_lpnj - v_nplj)

with v in chemists' notation, v[i,j,k,l] = (ij|kl), and G(-tau) = -G(beta-tau)
(antiperiodicity), so on the uniform grid G(-tau_k) = -G(tau_{M-k}).

``sigma_literal`` evaluates the eight-index sum exactly as written (N^8 per
point; small N only).  ``sigma_factored`` performs the same sum as four
successive single-index contractions, the O(n_tau N^5) route the paper quotes:

    T1[i,m,q,l] = sum_k v[i,m,q,k] G[k,l]
    T2[i,n,q,l] = sum_m G[m,n] T1[i,m,q,l]
    T3[i,n,p,l] = sum_q Gbar[p,q] T2[i,n,q,l]
    Sigma[i,j]  = - sum_{n,p,l} T3[i,n,p,l] W[l,p,n,j],  W = 2 v[l,p,n,j] - v[n,p,l,j]
"""

import numpy as np


def exchange_combination(v):
    """W[l,p,n,j] = 2 v[l,p,n,j] - v[n,p,l,j]."""
    return 2.0 * v - v.transpose(2, 1, 0, 3)


def sigma_literal(G, Gbar, v):
    """Eq. Sigma for one time point by the full eight-index sum (no factoring)."""
    W = exchange_combination(v)
    return -np.einsum("kl,mn,pq,imqk,lpnj->ij", G, G, Gbar, v, W, optimize=False)


def sigma_factored(G, Gbar, v, W=None):
    """Eq. Sigma for one time point by four N^5 contractions (matrix products)."""
    n = G.shape[0]
    if W is None:
        W = exchange_combination(v)
    t1 = (v.reshape(n ** 3, n) @ G).reshape(n, n, n, n)              # [i,m,q,l]
    t2 = np.matmul(G.T, t1.reshape(n, n, n * n)).reshape(n, n, n, n)  # [i,n,q,l]
    t3 = np.matmul(Gbar, t2)                                          # [i,n,p,l]
    w2 = W.transpose(2, 1, 0, 3).reshape(n ** 3, n)                   # [(n,p,l), j]
    return -(t3.reshape(n, n ** 3) @ w2)


def gbar_from_grid(G_tau, k):
    """G(-tau_k) = -G(tau_{M-k}) on the uniform grid."""
    M = G_tau.shape[0] - 1
    return -G_tau[M - k]


def sigma_tau(G_tau, v, taus=None, literal=False):
    """Sigma(tau_k) for every grid point (or the listed indices ``taus``)."""
    W = exchange_combination(v)
    idx = range(G_tau.shape[0]) if taus is None else taus
    out = []
    for k in idx:
        Gb = gbar_from_grid(G_tau, k)
        if literal:
            out.append(sigma_literal(G_tau[k], Gb, v))
        else:
            out.append(sigma_factored(G_tau[k], Gb, v, W))
    return np.array(out)
