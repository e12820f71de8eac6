"""Pins for the oracle's self-energy (Eq. Sigma)."""

import numpy as np
import pytest

import gf2_inputs as gi
from oracle import sigma as osg
from tests import closed_forms as cf


@pytest.mark.parametrize("n", [2, 3, 5, 6])
def test_factored_equals_literal_eight_index_sum(n):
    G = gi.random_symmetric_g(n, 4, seed=gi.SEED + n)
    v = gi.random_eri(n, seed=gi.SEED + 10 + n)
    for k in range(4):
        Gb = osg.gbar_from_grid(G, k)
        lit = osg.sigma_literal(G[k], Gb, v)
        fac = osg.sigma_factored(G[k], Gb, v)
        assert np.abs(lit - fac).max() <= 1e-12 * np.abs(lit).max()


def test_literal_sum_against_explicit_loops():
    """The einsum string is checked against hand-written loops over all eight indices."""
    n = 2
    G = gi.random_symmetric_g(n, 2, seed=7)
    v = gi.random_eri(n, seed=8)
    g, gb = G[0], -G[1]
    ref = np.zeros((n, n))
    rng = range(n)
    for i in rng:
        for j in rng:
            acc = 0.0
            for k in rng:
                for l in rng:
                    for m in rng:
                        for nn in rng:
                            for p in rng:
                                for q in rng:
                                    acc += (g[k, l] * g[m, nn] * gb[p, q] * v[i, m, q, k]
                                            * (2.0 * v[l, p, nn, j] - v[nn, p, l, j]))
            ref[i, j] = -acc
    assert np.abs(osg.sigma_literal(g, gb, v) - ref).max() < 1e-14


def test_sigma_is_symmetric():
    G = gi.random_symmetric_g(6, 3)
    v = gi.random_eri(6)
    S = osg.sigma_tau(G, v)
    assert np.abs(S - np.swapaxes(S, 1, 2)).max() < 1e-13 * np.abs(S).max()


def test_ao_sigma_equals_mo_closed_form_at_hf():
    """Sigma^AO(tau) = S C Sigma^MO(tau) C^T S for the Sigma = 0 Green's function."""
    s = gi.build_system("chain", coords=gi.h_chain(4, 1.7), basis="sto-3g", beta=20, n_tau=33, n_iw=64)
    r = gi.rhf(s)
    beta = 20.0
    eps = r.eps
    mu = 0.5 * (eps[1] + eps[2])
    _, C, xi, f = cf.mo_basis(r.F, s.S, mu, beta)
    taus = np.arange(33) * beta / 32
    Gao = cf.g_tau_ao(C, xi, beta, taus)
    vmo = cf.mo_integrals(C, s.eri)
    for k in [1, 7, 16, 30]:
        # MO closed form: Sigma_ij = -sum_{kmp} G_k G_m Gbar_p (im|pk)[2(kp|mj) - (mp|kj)]
        gk = -np.exp(-xi * taus[k]) / (1 + np.exp(-beta * xi))
        gbar = np.exp(xi * taus[k]) / (1 + np.exp(beta * xi))
        smo = -np.einsum("k,m,p,impk,kpmj->ij", gk, gk, gbar, vmo,
                         2.0 * vmo - vmo.transpose(2, 1, 0, 3), optimize=True)
        ref = s.S @ C @ smo @ C.T @ s.S
        got = osg.sigma_factored(Gao[k], -Gao[32 - k], s.eri)
        assert np.abs(got - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())
