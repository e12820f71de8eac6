"""Natural occupation numbers, the observable the paper plots for the H32
lattices (results section): the eigenvalues of the spin-summed density in the
symmetrically orthogonalised basis, halved to give occupations per spatial
orbital,
    n_k = eig( S^1/2 P S^1/2 ) / 2,   sorted from largest to smallest.
S^1/2 comes from the eigendecomposition of S; eigenvalues from LAPACK's
symmetric solver.  TEST INFRASTRUCTURE ONLY (see the package docstring).
"""

import numpy as np


def s_half(S):
    w, U = np.linalg.eigh(S)
    return (U * np.sqrt(w)) @ U.T


def natural_occupations(P, S):
    Sh = s_half(S)
    X = Sh @ P @ Sh
    return np.sort(np.linalg.eigvalsh(0.5 * (X + X.T)))[::-1] / 2.0
