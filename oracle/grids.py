"""Imaginary-time and Matsubara grids.

Matsubara frequencies omega_n = (2n+1) pi / beta (the paper's omega_n, with the
factor i kept separate), n = 0 .. n_iw-1; the negative ones follow from
G(-i omega) = conj G(i omega) for a real basis.  The time grid is uniform,
tau_k = k beta / M for k = 0 .. M with M = n_tau - 1.
"""

import numpy as np


def matsubara(beta, n_iw):
    return (2.0 * np.arange(n_iw) + 1.0) * np.pi / beta


def tau_grid(beta, n_tau):
    return np.arange(n_tau) * (beta / (n_tau - 1))
