"""Auxiliary s-Gaussian bases and the three-index factor of density-fitted
two-electron integrals (Coulomb metric), for the density-fitted route to the
self-energy that the paper names as its cost reduction.

Density fitting expands every orbital product in m auxiliary functions
chi_P, with coefficients chosen to minimise the Coulomb self-repulsion of the
fitting error (Whitten 1973; Dunlap, Connolly & Sabin 1979; Vahtras, Almloef &
Feyereisen 1993):

    (ij|kl) ~ sum_PQ (ij|P) [J^-1]_PQ (Q|kl),   J_PQ = (P|Q).

Written with the symmetric square root, (ij|kl) ~ sum_Q B[Q,i,j] B[Q,k,l]
with B = J^-1/2 (P|ij).  J is diagonalised and directions with eigenvalues
below ``cutoff`` times the largest are dropped, so B has m' <= m rows.

The auxiliary functions are unnormalised s primitives exp(-g |r - C|^2) (the
fitted integrals do not depend on their normalisation).  The integrals are the
s-type repulsion formula of ``integrals`` with one primitive pair replaced by a
single Gaussian:

    (ab|P) = 2 pi^(5/2) / (p g sqrt(p + g)) K_ab F0(p g / (p + g) |P_ab - C|^2)
    (P|Q)  = 2 pi^(5/2) / (g d sqrt(g + d))      F0(g d / (g + d) |C - D|^2)

The library takes B as input; this module, like the rest of ``gf2_inputs``,
holds none of the self-energy arithmetic.
"""

import numpy as np

from .basis import basis_functions
from .integrals import _primitives, boys0

# even-tempered s exponents g_k = 0.3 * 2.6^k, k = 0..5, on every hydrogen: they
# span the primitive-pair exponents of 6-31G and STO-3G (0.32 .. 37.5)
EVEN_TEMPERED_H = 0.3 * 2.6 ** np.arange(6)


def aux_even_tempered(coords, exponents=EVEN_TEMPERED_H):
    """(centres [m,3], exponents [m]): the same s exponents on every atom."""
    coords = np.asarray(coords, dtype=np.float64)
    ex = np.asarray(exponents, dtype=np.float64)
    return np.repeat(coords, len(ex), axis=0), np.tile(ex, len(coords))


def aux_products(funcs):
    """(centres, exponents) of every primitive-pair product of the orbital basis:
    a product of two s Gaussians is one s Gaussian at the weighted centre with
    the summed exponent, so this auxiliary set spans every orbital product and
    the fit is exact."""
    a, c, _, _ = _primitives(funcs)
    iu, ju = np.triu_indices(len(a))
    p = a[iu] + a[ju]
    P = (a[iu, None] * c[iu] + a[ju, None] * c[ju]) / p[:, None]
    return P, p


def three_center(funcs, aux):
    """(P|ij) [m, N, N] for the contracted orbital basis ``funcs``."""
    a, c, w, own = _primitives(funcs)
    C, g = aux
    n, npr = len(funcs), len(a)
    p = a[:, None] + a[None, :]
    Pc = (a[:, None, None] * c[:, None, :] + a[None, :, None] * c[None, :, :]) / p[..., None]
    K = np.exp(-a[:, None] * a[None, :] / p * ((c[:, None, :] - c[None, :, :]) ** 2).sum(-1))
    K *= w[:, None] * w[None, :]
    O = np.zeros((n, npr))
    O[own, np.arange(npr)] = 1.0
    out = np.empty((len(g), n, n))
    for q in range(len(g)):
        d2 = ((Pc - C[q]) ** 2).sum(-1)
        val = 2.0 * np.pi ** 2.5 / (p * g[q] * np.sqrt(p + g[q])) * K * boys0(p * g[q] / (p + g[q]) * d2)
        out[q] = O @ val @ O.T
    return out


def two_center(aux):
    """J[P, Q] = (P|Q) [m, m]."""
    C, g = aux
    s = g[:, None] + g[None, :]
    d2 = ((C[:, None, :] - C[None, :, :]) ** 2).sum(-1)
    return 2.0 * np.pi ** 2.5 / (g[:, None] * g[None, :] * np.sqrt(s)) * boys0(g[:, None] * g[None, :] / s * d2)


def df_factor(three, J, cutoff=1e-12):
    """B [m', N, N] = J^-1/2 (P|ij) over the eigen-directions of J above ``cutoff``."""
    lam, U = np.linalg.eigh(J)
    keep = lam > cutoff * lam.max()
    T = U[:, keep].T / np.sqrt(lam[keep])[:, None]
    m, n = three.shape[0], three.shape[1]
    return (T @ three.reshape(m, n * n)).reshape(-1, n, n)


def build_df(coords, basis, aux="even-tempered", cutoff=1e-12):
    """Three-index factor B for the hydrogen geometry ``coords`` in ``basis``
    with the auxiliary set ``aux``: "even-tempered" (EVEN_TEMPERED_H on every
    atom), "products" (exact fit), or explicit (centres, exponents)."""
    funcs = basis_functions(coords, basis)
    if isinstance(aux, str):
        aux = aux_even_tempered(coords) if aux == "even-tempered" else aux_products(funcs)
    return df_factor(three_center(funcs, aux), two_center(aux), cutoff)
