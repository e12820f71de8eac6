"""Pins for the input generator (integrals, RHF) against textbook values."""

import json
import os

import numpy as np
import pytest

import gf2_inputs as gi
from gf2_inputs.integrals import boys0

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "h2_sto3g_textbook.json")


@pytest.fixture(scope="module")
def h2():
    s = gi.build_system("h2_sto3g")
    return s, gi.rhf(s)


def test_h2_integrals_match_textbook(h2):
    s, _ = h2
    ref = json.load(open(GOLDEN))
    tol = ref["print_tolerance"]
    assert abs(s.S[0, 1] - ref["S12"]) < tol
    assert abs(s.T[0, 0] - ref["T11"]) < tol
    assert abs(s.T[0, 1] - ref["T12"]) < tol
    assert abs(s.V[0, 0] - ref["V11_total"]) < tol
    assert abs(s.V[0, 1] - ref["V12_total"]) < tol
    e = s.eri
    assert abs(e[0, 0, 0, 0] - ref["eri_1111"]) < tol
    assert abs(e[0, 0, 1, 1] - ref["eri_1122"]) < tol
    assert abs(e[1, 0, 0, 0] - ref["eri_2111"]) < tol
    assert abs(e[1, 0, 1, 0] - ref["eri_2121"]) < tol


def test_h2_rhf_matches_textbook(h2):
    s, r = h2
    ref = json.load(open(GOLDEN))
    assert abs(r.e_elec - ref["E0_electronic"]) < ref["print_tolerance"]
    assert abs(r.e_total - ref["E_total_hf"]) < ref["print_tolerance"]
    assert abs(r.eps[0] - ref["eps_1"]) < 1e-3
    assert abs(r.eps[1] - ref["eps_2"]) < 1e-3


def test_eri_eightfold_symmetry_and_unit_overlap():
    s = gi.build_system("chain", coords=gi.h_chain(3, 1.6), basis="6-31g", beta=10, n_tau=9, n_iw=16)
    e = s.eri
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0)]:
        assert np.abs(e - e.transpose(perm)).max() < 1e-13
    assert np.abs(np.diag(s.S) - 1.0).max() < 1e-12
    # (ii|jj) >= 0 and Cauchy-Schwarz |(ij|kl)|^2 <= (ij|ij)(kl|kl)
    n = s.nbf
    d = np.einsum("ijij->ij", e)
    assert (d > 0).all()
    assert (e.reshape(n * n, n * n) ** 2 <= np.outer(d.ravel(), d.ravel()) * (1 + 1e-12)).all()


def test_boys_function_limits_and_quadrature():
    assert boys0(np.array([0.0]))[0] == 1.0
    x = np.linspace(0.0, 1.0, 200001)
    for t in [1e-9, 1e-3, 0.5, 3.0, 30.0]:
        quad = np.trapezoid(np.exp(-t * x * x), x)
        assert abs(boys0(np.array([t]))[0] - quad) < 1e-9


def test_overlap_closed_form_against_quadrature():
    from gf2_inputs.integrals import one_electron
    A = np.array([0.0, 0.0, 0.0])
    B = np.array([0.7, -0.3, 0.2])
    a, b = 0.9, 0.35
    funcs = [(A, np.array([a]), np.array([1.0])), (B, np.array([b]), np.array([1.0]))]
    S, _, _ = one_electron(funcs, np.array([A, B]))
    x = np.linspace(-12, 12, 48001)
    quad = 1.0
    for d in range(3):
        quad *= np.trapezoid(np.exp(-a * (x - A[d]) ** 2 - b * (x - B[d]) ** 2), x)
    assert abs(S[0, 1] - quad) < 1e-12
