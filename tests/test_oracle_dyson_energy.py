"""Pins for the oracle's Dyson solve, density, mu search, Fock build and energy."""

import json
import os

import numpy as np
import pytest

import gf2_inputs as gi
from oracle import dyson as od
from oracle import energy as oe
from oracle import gf2 as og
from oracle import sigma as osg
from oracle import transforms as ot
from oracle.fock import fock
from tests import closed_forms as cf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "h2_sto3g_textbook.json")


@pytest.fixture(scope="module")
def h4():
    s = gi.build_system("chain", coords=gi.h_chain(4, 1.7), basis="sto-3g", beta=100, n_tau=513, n_iw=1024)
    return s, gi.rhf(s)


@pytest.fixture(scope="module")
def h2():
    s = gi.build_system("h2_sto3g")
    return s, gi.rhf(s)


def test_dyson_residual_and_complex_symmetry(h4):
    s, r = h4
    beta, n_iw = 100.0, 256
    rng = np.random.default_rng(3)
    sig = rng.normal(size=(n_iw, s.nbf, s.nbf)) * 0.01 + 1j * rng.normal(size=(n_iw, s.nbf, s.nbf)) * 0.01
    sig = sig + np.swapaxes(sig, 1, 2)
    mu = -0.05
    G = od.dyson(mu, s.S, r.F, sig, beta)
    w = (2 * np.arange(n_iw) + 1) * np.pi / beta
    A = (1j * w + mu)[:, None, None] * s.S - r.F - sig
    assert np.abs(A @ G - np.eye(s.nbf)).max() < 1e-12
    assert np.abs(G - np.swapaxes(G, 1, 2)).max() < 1e-12 * np.abs(G).max()


def test_density_without_self_energy_is_fermi_dirac(h4):
    # after four tail moments the sum is cut with error ~ (4/beta) |X|^5 / (5 w_max^5 / (beta/2pi))
    s, r = h4
    beta, n_iw = 100.0, 2048
    for mu in (-0.2, 0.5 * (r.eps[1] + r.eps[2]), r.eps[1] + 1e-3):
        G = od.dyson(mu, s.S, r.F, None, beta, n_iw)
        P = od.density(G, ot.tail_moments(s.S, r.F, mu), beta)
        _, C, xi, f = cf.mo_basis(r.F, s.S, mu, beta)
        assert np.abs(P - cf.density_closed(C, f)).max() < 1e-10


def test_mu_search_hits_particle_number_and_is_monotone(h4):
    s, r = h4
    beta, n_iw = 100.0, 512
    counts = []
    for mu in np.linspace(r.eps[0] - 0.2, r.eps[-1] + 0.2, 9):
        _, P = od.density_at(mu, s.S, r.F, None, None, None, beta, n_iw)
        counts.append(od.electron_count(P, s.S))
    assert np.all(np.diff(counts) > 0)
    assert counts[0] < 1e-3 and abs(counts[-1] - 2 * s.nbf) < 1e-3
    mu, G, P, _ = od.mu_search(s.S, r.F, None, None, None, s.n_elec, beta, n_iw)
    assert abs(od.electron_count(P, s.S) - s.n_elec) <= 1e-10


def test_fock_matches_roothaan_reference(h4):
    s, r = h4
    F = fock(s.h, s.eri, r.P)
    assert np.abs(F - r.F).max() < 1e-10
    # Roothaan: F C = S C eps
    assert np.abs(F @ r.C - s.S @ r.C * r.eps).max() < 1e-9


def test_sigma_zero_energy_is_finite_temperature_hf(h2):
    s, r = h2
    beta, n_iw = 100.0, 1024
    F, mu, G, P = og.inner_loop(s, r.F, None, None, None, beta, n_iw)
    st = og.GF2State(F=F, mu=mu, P=P, G_iw=G)
    E, _, _ = og.energy(s, st, beta)
    _, C, xi, f = cf.mo_basis(F, s.S, mu, beta)
    assert abs(E - cf.e_hf_finite_t(F, s.h, cf.density_closed(C, f), s.e_nuc)) < 1e-9
    # gap 1.25 Eh at beta = 100: smearing ~ exp(-60), so this is the T = 0 RHF energy
    assert abs(E - r.e_total) < 1e-9


def _first_order(s, F0, beta, n_tau, n_iw, sigma_fn=None):
    F, mu, G, P = og.inner_loop(s, F0, None, None, None, beta, n_iw)
    st = og.GF2State(F=F, mu=mu, P=P, G_iw=G, sig1=np.zeros_like(F), sig2=np.zeros_like(F))
    G_tau, Sig_tau = og.self_energy_step(s, st, beta, n_tau, n_iw, sigma_fn)
    Sig_iw = ot.tau_to_iw(Sig_tau, beta, n_iw)
    sig1, _ = ot.sigma_expansion(Sig_tau, beta)
    e2 = oe.e_two_body(G, Sig_iw, sig1, s.S, beta)
    e2_tau = oe.e_two_body_tau(Sig_tau, G_tau, beta)
    return F, mu, e2, e2_tau


def test_first_iteration_energy_matches_finite_beta_closed_form(h4):
    """(1/beta) sum_n Tr[G0 Sigma[G0]] against its MO closed form; the gap shrinks with the grid."""
    s, r = h4
    beta = 100.0
    errs = []
    for n_tau, n_iw in ((1025, 2048), (2049, 4096)):
        F, mu, e2, e2_tau = _first_order(s, r.F, beta, n_tau, n_iw)
        eps, C, xi, f = cf.mo_basis(F, s.S, mu, beta)
        ref = cf.e2_first_order(cf.mo_integrals(C, s.eri), xi, beta)
        errs.append(abs(e2 - ref))
        # Simpson on the tau grid is an independent quadrature of the same integral
        assert abs(e2 - e2_tau) < 3e-5 * abs(ref)
    assert errs[-1] < 1e-7 and errs[-1] < errs[0] / 4.0


def test_first_iteration_is_twice_textbook_mp2(h2):
    s, r = h2
    ref = json.load(open(GOLDEN))
    beta = 100.0
    F, mu, e2, _ = _first_order(s, r.F, beta, 1025, 2048)
    eps, C, xi, f = cf.mo_basis(F, s.S, mu, beta)
    mp2 = cf.mp2_closed_shell(cf.mo_integrals(C, s.eri), eps, 1)
    assert abs(mp2 - ref["E_mp2"]) < ref["print_tolerance"]
    assert abs(e2 - 2.0 * mp2) < 1e-6


def test_alternative_index_string_fails_the_mp2_pin(h4):
    """v_imqk (2 v_lnpj - v_pnlj) (pairing j with the G(-tau) partner) is not MP2."""
    s, r = h4

    def sigma_alt(G_tau, v):
        M = G_tau.shape[0] - 1
        # W_alt[l,p,n,j] = 2 v[l,n,p,j] - v[p,n,l,j]
        W = 2.0 * np.einsum("lnpj->lpnj", v) - np.einsum("pnlj->lpnj", v)
        return np.array([osg.sigma_factored(G_tau[k], -G_tau[M - k], v, W) for k in range(M + 1)])

    beta = 100.0
    F, mu, e2, _ = _first_order(s, r.F, beta, 513, 1024)
    F2, mu2, e2_alt, _ = _first_order(s, r.F, beta, 513, 1024, sigma_fn=sigma_alt)
    eps, C, xi, f = cf.mo_basis(F, s.S, mu, beta)
    ref = cf.e2_first_order(cf.mo_integrals(C, s.eri), xi, beta)
    assert abs(e2 - ref) < 1e-5            # grid-limited at this coarse grid
    assert abs(e2_alt - ref) > 1e-3
