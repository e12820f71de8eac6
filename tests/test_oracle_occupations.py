"""Pins of the natural-occupation oracle (oracle/occupations.py) against closed forms:
the idempotent RHF density has occupations exactly 1 (occupied) and 0; a finite-
temperature HF density 2 C f C^T has the Fermi-Dirac values f themselves; and the
occupations sum to half the electron count Tr(PS) for any density."""

import numpy as np
import pytest

import gf2_inputs as gi
from oracle.occupations import natural_occupations
from tests import closed_forms as cf


@pytest.fixture(scope="module")
def h10():
    s = gi.build_system("h10_chain_sto3g")
    return s, gi.rhf(s)


def test_rhf_density_is_idempotent_ones_and_zeros(h10):
    s, r = h10
    occ = natural_occupations(r.P, s.S)
    n_occ = s.n_elec // 2
    expect = np.r_[np.ones(n_occ), np.zeros(s.nbf - n_occ)]
    assert np.abs(occ - expect).max() < 1e-10


def test_finite_temperature_density_gives_fermi_dirac_values(h10):
    s, r = h10
    beta = 20.0   # low enough that several f are neither 0 nor 1
    mu = 0.5 * (r.eps[4] + r.eps[5])
    _, C, xi, f = cf.mo_basis(r.F, s.S, mu, beta)
    P = cf.density_closed(C, f)
    occ = natural_occupations(P, s.S)
    assert np.abs(occ - np.sort(f)[::-1]).max() < 1e-12
    assert 0.0 < f[5] < 1.0


def test_occupations_sum_to_half_the_electron_count(h10):
    s, r = h10
    rng = np.random.default_rng(7)
    E = rng.normal(size=(s.nbf, s.nbf)) * 1e-2
    P = r.P + E + E.T
    occ = natural_occupations(P, s.S)
    assert abs(occ.sum() - 0.5 * np.trace(P @ s.S)) < 1e-12
    assert np.all(np.diff(occ) <= 0)


def test_orthonormal_basis_reduces_to_eigenvalues_of_p(h10):
    s, _ = h10
    rng = np.random.default_rng(8)
    A = rng.normal(size=(6, 6))
    P = A @ A.T
    occ = natural_occupations(P, np.eye(6))
    assert np.allclose(occ, np.sort(np.linalg.eigvalsh(P))[::-1] / 2, atol=1e-13)
