"""Contracted s-type Gaussian basis sets for hydrogen.

Each contracted function is phi(r) = sum_p c_p * n(a_p) * exp(-a_p |r-A|^2),
with n(a) = (2a/pi)^(3/4) the primitive normalisation; the contraction is then
rescaled so that <phi|phi> = 1.
"""

import numpy as np

# STO-3G hydrogen 1s (the zeta=1.24 scaled set).
_STO3G_H = [
    ([3.42525091, 0.62391373, 0.16885540], [0.15432897, 0.53532814, 0.44463454]),
]

# 6-31G hydrogen: a 3-primitive inner shell and a 1-primitive outer shell.
_631G_H = [
    ([18.7311370, 2.8253937, 0.6401217], [0.03349460, 0.23472695, 0.81375733]),
    ([0.1612778], [1.0]),
]

BASIS_SETS = {"sto-3g": _STO3G_H, "6-31g": _631G_H}


def _contraction_norm(alphas, coefs):
    """Scale factor making a contraction of normalised s primitives unit-norm."""
    a = np.asarray(alphas, dtype=np.float64)
    c = np.asarray(coefs, dtype=np.float64)
    n = (2.0 * a / np.pi) ** 0.75
    # overlap of two normalised s primitives on the same centre
    s = (np.pi / (a[:, None] + a[None, :])) ** 1.5 * n[:, None] * n[None, :]
    return 1.0 / np.sqrt(c @ s @ c)


def basis_functions(coords, basis):
    """List of (centre[3], alphas[np], weights[np]) for every contracted function.

    ``weights`` already include the primitive normalisation and the contraction
    renormalisation, so phi = sum_p weights_p exp(-alphas_p |r - centre|^2).
    """
    shells = BASIS_SETS[basis.lower()]
    out = []
    for centre in np.asarray(coords, dtype=np.float64):
        for alphas, coefs in shells:
            a = np.asarray(alphas, dtype=np.float64)
            c = np.asarray(coefs, dtype=np.float64)
            w = c * (2.0 * a / np.pi) ** 0.75 * _contraction_norm(a, c)
            out.append((centre.copy(), a, w))
    return out
