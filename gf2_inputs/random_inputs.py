"""Seeded random tensors with the symmetries of the physical ones.

Used by unit tests that need inputs of arbitrary size: a real symmetric G(tau)
per grid point and an 8-fold symmetric integral tensor v[i,j,k,l] = (ij|kl).
"""

import numpy as np

SEED = 1405327


def random_symmetric_g(n, n_tau, seed=SEED, decay=4.0):
    """[n_tau, n, n] real symmetric matrices, entries ~U(-1,1) * exp(-|i-j|/decay)."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1.0, 1.0, size=(n_tau, n, n))
    d = np.abs(np.arange(n)[:, None] - np.arange(n)[None, :])
    a = a * np.exp(-d / decay)
    return 0.5 * (a + np.swapaxes(a, 1, 2))


def random_eri(n, seed=SEED + 1):
    """[n,n,n,n] tensor with (ij|kl) = (ji|kl) = (ij|lk) = (kl|ij)."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1.0, 1.0, size=(n, n, n, n))
    a = a + a.transpose(1, 0, 2, 3)
    a = a + a.transpose(0, 1, 3, 2)
    a = a + a.transpose(2, 3, 0, 1)
    return a / 8.0
