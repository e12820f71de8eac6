"""Closed-form results that pin the oracle (independent of oracle/ code).

All formulas work in the molecular-orbital basis of a Fock matrix F with
overlap S (F C = S C eps, C^T S C = 1), where a Green's function with no
self-energy is diagonal: for xi = eps - mu and f = 1/(1+e^{beta xi}),
    G_a(i w)   = 1/(i w - xi_a)
    G_a(tau)   = -e^{-xi_a tau}/(1 + e^{-beta xi_a})      (0 < tau < beta)
    G_a(-tau)  =  e^{ xi_a tau}/(1 + e^{ beta xi_a})
    P          = 2 C diag(f) C^T
"""

import numpy as np
import scipy.linalg as sla
from scipy.special import expit


def mo_basis(F, S, mu, beta):
    eps, C = sla.eigh(F, S)
    xi = eps - mu
    return eps, C, xi, expit(-beta * xi)


def g_tau_ao(C, xi, beta, taus):
    """AO-basis G(tau) of a Sigma = 0 system, stable for large beta |xi|."""
    taus = np.asarray(taus)
    # -e^{-xi tau}/(1+e^{-beta xi}) written without overflow
    val = np.where(xi[None, :] >= 0,
                   -np.exp(-np.outer(taus, xi)) * expit(beta * xi)[None, :],
                   -np.exp(np.outer(beta - taus, xi)) * expit(-beta * xi)[None, :])
    return np.einsum("ia,ta,ja->tij", C, val, C)


def density_closed(C, f):
    return 2.0 * (C * f) @ C.T


def mo_integrals(C, eri):
    return np.einsum("pi,qj,rk,sl,pqrs->ijkl", C, C, C, C, eri, optimize=True)


def e2_first_order(vmo, xi, beta):
    """(1/beta) sum_n Tr[G0 Sigma[G0]] for the Sigma=0 Green's function G0.

    With A_impk = (im|pk)[2(im|pk) - (ik|pm)] and D = xi_k + xi_m - xi_p - xi_i:
        E2 = - sum A [(1-f_k)(1-f_m) f_p f_i - f_k f_m (1-f_p)(1-f_i)] / D
    (the D -> 0 limit is beta (1-f_k)(1-f_m) f_p f_i).  For beta -> infinity
    the two terms give equal contributions: E2 -> 2 E_MP2.
    """
    n = len(xi)
    f = expit(-beta * xi)
    g = expit(beta * xi)             # 1 - f
    A = vmo * (2.0 * vmo - vmo.transpose(0, 3, 2, 1))
    # A[i,m,p,k] = (im|pk)[2(im|pk) - (ik|pm)]
    i, m, p, k = np.meshgrid(*(np.arange(n),) * 4, indexing="ij")
    D = xi[k] + xi[m] - xi[p] - xi[i]
    a = g[k] * g[m] * f[p] * f[i]
    b = f[k] * f[m] * g[p] * g[i]
    with np.errstate(divide="ignore", invalid="ignore"):
        pos = a * (-np.expm1(-beta * D)) / D
        neg = b * np.expm1(beta * D) / D
    w = np.where(D > 0, pos, neg)
    w = np.where(np.abs(beta * D) < 1e-12, a * beta, w)
    return -float(np.sum(A * w))


def mp2_closed_shell(vmo, eps, nocc):
    """sum_{ijab} (ia|jb)[2(ia|jb) - (ib|ja)] / (e_i + e_j - e_a - e_b)."""
    o, v = slice(0, nocc), slice(nocc, len(eps))
    iajb = vmo[o, v, o, v]
    eo, ev = eps[o], eps[v]
    den = eo[:, None, None, None] - ev[None, :, None, None] + eo[None, None, :, None] - ev[None, None, None, :]
    return float(np.sum(iajb * (2.0 * iajb - iajb.transpose(0, 3, 2, 1)) / den))


def e_hf_finite_t(F, h, P, e_nuc):
    return e_nuc + 0.5 * float(np.sum(P * (h + F)))
