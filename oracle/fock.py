"""Eq. FockMatrix:  F_ij = h_ij + sum_kl P_kl (v_ijlk - v_iklj / 2),  v[i,j,k,l] = (ij|kl)."""

import numpy as np


def fock(h, v, P):
    coul = np.einsum("kl,ijlk->ij", P, v)
    exch = np.einsum("kl,iklj->ij", P, v)
    return h + coul - 0.5 * exch
