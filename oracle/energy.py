"""Galitskii-Migdal energy of a closed-shell GF2 state.

The paper reports GF2 energies but does not print the expression; the standard
Galitskii-Migdal form for a spin-summed density P is used:

    E   = E_nuc + (1/2) Tr[P (h + F)] + E2
    E2  = (1/beta) sum_{n in Z} Tr[G(i w_n) Sigma(i w_n)]
        = (2/beta) sum_{n>=0} Re Tr[G Sigma](i w_n)
        = int_0^beta Tr[Sigma(tau) G(-tau)] dtau.

The Matsubara sum is cut at n_iw and completed with its leading tail,
G Sigma ~ G1 Sig1 / z^2, whose sum over n >= n_iw is
    (2/beta) (-Tr[S^-1 Sig1]) (beta/pi)^2 psi_1(n_iw + 1/2) / 4
(psi_1 = trigamma, taken from scipy).
"""

import numpy as np
from scipy.special import polygamma


def e_one_body(P, h, F):
    return 0.5 * float(np.sum(P * (h + F).T))


def e_two_body(G_iw, Sigma_iw, sig1, S, beta):
    n_iw = G_iw.shape[0]
    tr = np.einsum("wij,wji->w", G_iw, Sigma_iw)
    body = (2.0 / beta) * float(np.sum(tr.real))
    if sig1 is None:
        return body
    tail_sum = (beta / np.pi) ** 2 * float(polygamma(1, n_iw + 0.5)) / 4.0
    tail = (2.0 / beta) * (-float(np.trace(np.linalg.solve(S, sig1)))) * tail_sum
    return body + tail


def e_two_body_tau(Sigma_tau, G_tau, beta):
    """int_0^beta Tr[Sigma(tau) G(-tau)] dtau by Simpson's rule, G(-tau_k) = -G(tau_{M-k})."""
    M = G_tau.shape[0] - 1
    h = beta / M
    f = np.array([np.sum(Sigma_tau[k] * (-G_tau[M - k]).T) for k in range(M + 1)])
    w = np.ones(M + 1)
    w[1:M:2] = 4.0
    w[2:M:2] = 2.0
    return float(h / 3.0 * np.dot(w, f))
