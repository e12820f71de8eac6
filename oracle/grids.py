"""Imaginary-time and Matsubara grids.

Matsubara frequencies omega_n = (2n+1) pi / beta (the paper's omega_n, with the
factor i kept separate), n = 0 .. n_iw-1; the negative ones follow from
G(-i omega) = conj G(i omega) for a real basis.  The uniform time grid is
tau_k = k beta / M for k = 0 .. M with M = n_tau - 1.

The paper builds Sigma(tau) on a non-equidistant grid of a few thousand points
(Computational details) without listing the points.  The reading taken here is
the uniform power mesh of Ku and Eguiluz (Phys. Rev. Lett. 89, 126401 (2002)),
the grid of the ALPS codes the paper cites for it: the intervals
[beta/2^(j+1), beta/2^j], j = 1..p, and [0, beta/2^(p+1)] are each cut into u
equal steps, and the upper half of [0, beta] mirrors the lower.  Every point
is a point of the uniform grid with M = 2^(p+1) u intervals, so a grid is
given by M and the sorted indices of its points on that uniform grid.
"""

import numpy as np


def matsubara(beta, n_iw):
    return (2.0 * np.arange(n_iw) + 1.0) * np.pi / beta


def tau_grid(beta, n_tau):
    return np.arange(n_tau) * (beta / (n_tau - 1))


def power_mesh(p, u):
    """(M, index): the uniform power mesh with p halvings and u steps per
    interval, as indices into the uniform grid of M = 2^(p+1) u intervals
    (2 (p+1) u + 1 points, symmetric: index[k] + index[-1-k] = M)."""
    if p < 0 or u < 1:
        raise ValueError("power mesh needs p >= 0 and u >= 1")
    M = 2 ** (p + 1) * u
    lower = list(range(u + 1))                       # [0, beta/2^(p+1)], step beta/M
    for j in range(p, 0, -1):                        # [beta/2^(j+1), beta/2^j], step 2^(p-j) beta/M
        step = 2 ** (p - j)
        lower += [u * step + step * i for i in range(1, u + 1)]
    upper = [M - i for i in reversed(lower[:-1])]
    return M, np.array(lower + upper, dtype=np.int64)


def grid_points(beta, M, index):
    """tau_k = index[k] beta / M."""
    return np.asarray(index, dtype=np.float64) * (beta / M)
