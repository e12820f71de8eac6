"""Closed-shell restricted Hartree-Fock (the reference a GF2 run starts from).

Roothaan equations F C = S C eps with the closed-shell density
P = 2 C_occ C_occ^T (spin-summed) and F = h + J(P) - K(P)/2, accelerated by
Pulay's DIIS on the commutator F P S - S P F.
"""

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla


@dataclass
class RHFResult:
    F: np.ndarray
    P: np.ndarray
    C: np.ndarray
    eps: np.ndarray
    e_elec: float
    e_total: float
    iterations: int
    comm_norm: float


def _fock(h, eri, P):
    n = h.shape[0]
    v2 = eri.reshape(n * n, n * n)
    J = (v2 @ P.reshape(-1)).reshape(n, n)
    K = np.einsum("ikjl,kl->ij", eri, P, optimize=True)
    return h + J - 0.5 * K


def rhf(system, max_iter=500, e_tol=1e-12, comm_tol=1e-10, diis_size=8):
    S, h, eri = system.S, system.h, system.eri
    nocc = system.n_elec // 2
    eps, C = sla.eigh(h, S)
    P = 2.0 * C[:, :nocc] @ C[:, :nocc].T
    e_old = None
    fs, es = [], []
    for it in range(1, max_iter + 1):
        F = _fock(h, eri, P)
        e_elec = 0.5 * np.sum(P * (h + F))
        err = F @ P @ S - S @ P @ F
        cn = np.abs(err).max()
        if e_old is not None and abs(e_elec - e_old) < e_tol and cn < comm_tol:
            eps, C = sla.eigh(F, S)
            return RHFResult(F=F, P=P, C=C, eps=eps, e_elec=e_elec,
                             e_total=e_elec + system.e_nuc, iterations=it, comm_norm=cn)
        e_old = e_elec
        fs.append(F)
        es.append(err)
        fs, es = fs[-diis_size:], es[-diis_size:]
        if len(fs) > 1:
            m = len(fs)
            B = -np.ones((m + 1, m + 1))
            B[m, m] = 0.0
            for a in range(m):
                for b in range(m):
                    B[a, b] = np.sum(es[a] * es[b])
            rhs = np.zeros(m + 1)
            rhs[m] = -1.0
            coef = np.linalg.lstsq(B, rhs, rcond=None)[0][:m]
            Fd = sum(cf * f for cf, f in zip(coef, fs))
        else:
            Fd = F
        eps, C = sla.eigh(Fd, S)
        P = 2.0 * C[:, :nocc] @ C[:, :nocc].T
    raise RuntimeError(f"RHF did not converge in {max_iter} iterations")
