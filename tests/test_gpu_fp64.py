"""GPU parity of every C-ABI call (FP64 path) against the CPU oracle.

All inputs are seeded or come from ``gf2_inputs``; the expected values come
from ``oracle/`` only.  Sizes span several 64-wide GEMM tiles with ragged
tails (N = 5, 10, 33, 70), odd N (one matrix element per FFT CTA), frequency
counts below, equal to and not a multiple of the FFT length.
"""

import numpy as np
import pytest
import torch

import gf2_inputs as gi
from oracle import dyson as od
from oracle import energy as oe
from oracle import gf2 as og
from oracle import sigma as osg
from oracle import transforms as ot
from oracle.fock import fock as oracle_fock

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def library():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1405_3273_gb300 as g
    from paper_1405_3273_gb300 import build
    import os
    if not os.path.exists(g.LIB_PATH):
        build.build()
    g.lib()
    return g


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def h4():
    s = gi.build_system("chain", coords=gi.h_chain(4, 1.7), basis="sto-3g", beta=50.0, n_tau=257, n_iw=512)
    return s, gi.rhf(s)


@pytest.mark.parametrize("n,n_tau", [(5, 17), (10, 33), (33, 9)])
def test_sigma_fp64_matches_oracle(library, n, n_tau):
    g = library
    G = gi.random_symmetric_g(n, n_tau, seed=100 + n)
    v = gi.random_eri(n, seed=200 + n)
    ref = osg.sigma_tau(G, v)
    with g.Context(n, n_tau, 8, 10.0) as ctx:
        g.gf2_set_integrals(ctx.handle, dev(v))
        out = torch.zeros(n_tau, n, n, dtype=torch.float64, device="cuda")
        g.gf2_sigma_tau(ctx.handle, dev(G), out, g.GF2_PREC_FP64)
        got = host(out)
    assert np.abs(got - ref).max() <= 1e-10
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_sigma_fp64_points_ragged_tiles(library):
    """N = 70: two full 64-wide tiles plus a ragged one in every stage; two grid points."""
    g = library
    n, n_tau = 70, 9
    G = gi.random_symmetric_g(n, n_tau, seed=7)
    v = gi.random_eri(n, seed=8) * 0.1
    W = osg.exchange_combination(v)
    with g.Context(n, n_tau, 8, 10.0) as ctx:
        g.gf2_set_integrals(ctx.handle, dev(v))
        out = torch.zeros(2, n, n, dtype=torch.float64, device="cuda")
        g.gf2_sigma_tau_points(ctx.handle, dev(G), 3, 2, out, g.GF2_PREC_FP64)
        got = host(out)
    for j, k in enumerate((3, 4)):
        ref = osg.sigma_factored(G[k], -G[n_tau - 1 - k], v, W)
        assert np.abs(got[j] - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("n_iw", [5, 256, 389, 512])
def test_iw_to_tau_matches_oracle(library, h4, n_iw):
    g = library
    s, r = h4
    beta, n_tau = 50.0, 257
    mu = 0.5 * (r.eps[1] + r.eps[2])
    sig1 = 0.01 * np.diag(np.arange(1, s.nbf + 1.0))
    sig2 = 0.003 * np.ones((s.nbf, s.nbf))
    rng = np.random.default_rng(5)
    sig_iw = 0.01 * (rng.normal(size=(n_iw, s.nbf, s.nbf)) + 1j * rng.normal(size=(n_iw, s.nbf, s.nbf)))
    sig_iw = sig_iw + np.swapaxes(sig_iw, 1, 2)
    G_iw = od.dyson(mu, s.S, r.F, sig_iw, beta)
    mom = ot.tail_moments(s.S, r.F, mu, sig1, sig2)
    ref = ot.iw_to_tau(G_iw, mom, beta, n_tau)
    with g.Context(s.nbf, n_tau, n_iw, beta) as ctx:
        out = torch.zeros(n_tau, s.nbf, s.nbf, dtype=torch.float64, device="cuda")
        g.gf2_fft_iw_to_tau(ctx.handle, dev(G_iw), dev(mom), out)
        got = host(out)
    assert np.abs(got - ref).max() < 1e-11


@pytest.mark.parametrize("n,n_iw", [(4, 256), (5, 1000), (3, 7)])
def test_tau_to_iw_matches_oracle(library, n, n_iw):
    g = library
    beta, n_tau = 20.0, 129
    rng = np.random.default_rng(n)
    t = np.arange(n_tau) * beta / (n_tau - 1)
    A = rng.normal(size=(n, n))
    B = rng.normal(size=(n, n))
    X = -np.exp(-0.7 * t)[:, None, None] * (A + A.T) - np.exp(-1.3 * (beta - t))[:, None, None] * (B + B.T)
    ref = ot.tau_to_iw(X, beta, n_iw)
    s1, s2 = ot.sigma_expansion(X, beta)
    with g.Context(n, n_tau, n_iw, beta) as ctx:
        out = torch.zeros(n_iw, n, n, dtype=torch.complex128, device="cuda")
        sig12 = torch.zeros(2, n, n, dtype=torch.float64, device="cuda")
        g.gf2_fft_tau_to_iw(ctx.handle, dev(X), out, sig12)
        got = host(out)
        gs = host(sig12)
    assert np.abs(got - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())
    assert np.abs(gs[0] - s1).max() < 1e-12 and np.abs(gs[1] - s2).max() < 1e-9


def test_tail_moments_dyson_density_match_oracle(library, h4):
    g = library
    s, r = h4
    beta, n_tau, n_iw = 50.0, 257, 512
    mu = -0.07
    rng = np.random.default_rng(9)
    sig1 = 0.02 * rng.normal(size=(s.nbf, s.nbf))
    sig1 = sig1 + sig1.T
    sig2 = 0.01 * rng.normal(size=(s.nbf, s.nbf))
    sig2 = sig2 + sig2.T
    sig_iw = 0.01 * (rng.normal(size=(n_iw, s.nbf, s.nbf)) - 1j * np.abs(rng.normal(size=(n_iw, s.nbf, s.nbf))))
    sig_iw = sig_iw + np.swapaxes(sig_iw, 1, 2)
    mom_ref = ot.tail_moments(s.S, r.F, mu, sig1, sig2)
    G_ref = od.dyson(mu, s.S, r.F, sig_iw, beta)
    P_ref = od.density(G_ref, mom_ref, beta)
    with g.Context(s.nbf, n_tau, n_iw, beta) as ctx:
        mom = torch.zeros(4, s.nbf, s.nbf, dtype=torch.float64, device="cuda")
        g.gf2_tail_moments(ctx.handle, dev(s.S), dev(r.F), mu, dev(np.stack([sig1, sig2])), mom)
        G = torch.zeros(n_iw, s.nbf, s.nbf, dtype=torch.complex128, device="cuda")
        g.gf2_dyson(ctx.handle, mu, dev(s.S), dev(r.F), dev(sig_iw), G)
        P = torch.zeros(s.nbf, s.nbf, dtype=torch.float64, device="cuda")
        g.gf2_density(ctx.handle, G, mom, P)
        got_m, got_G, got_P = host(mom), host(G), host(P)
    assert np.abs(got_m - mom_ref).max() < 1e-11 * np.abs(mom_ref).max()
    assert np.abs(got_G - G_ref).max() < 1e-12
    assert np.abs(got_P - P_ref).max() < 1e-11


def test_mu_search_and_fock_match_oracle(library, h4):
    g = library
    s, r = h4
    beta, n_tau, n_iw = 50.0, 257, 512
    mu_ref, G_ref, P_ref, _ = od.mu_search(s.S, r.F, None, None, None, s.n_elec, beta, n_iw)
    with g.Context(s.nbf, n_tau, n_iw, beta) as ctx:
        g.gf2_set_integrals(ctx.handle, dev(s.eri))
        G = torch.zeros(n_iw, s.nbf, s.nbf, dtype=torch.complex128, device="cuda")
        P = torch.zeros(s.nbf, s.nbf, dtype=torch.float64, device="cuda")
        S = dev(s.S)
        mu, nev = g.gf2_mu_search(ctx.handle, S, dev(r.F), None, None, s.n_elec, 0.3, G, P)
        Pn = host(P)
        F = torch.zeros_like(P)
        g.gf2_fock(ctx.handle, dev(s.h), dev(P_ref), F)
        got_F = host(F)
    assert abs(np.trace(Pn @ s.S) - s.n_elec) <= 1e-10
    assert np.abs(Pn - P_ref).max() < 1e-8
    assert nev < 40
    assert np.abs(got_F - oracle_fock(s.h, s.eri, P_ref)).max() < 1e-12


@pytest.mark.parametrize("n", [4, 5, 33, 64])
def test_fock_matches_oracle_without_index_symmetry(library, n):
    """Eq. FockMatrix on a v and a P with no index symmetry (the build reads
    v_ijlk and v_iklj as given); F in place of h; F aliasing P is refused."""
    g = library
    rng = np.random.default_rng(40 + n)
    v = rng.normal(size=(n, n, n, n))
    P = rng.normal(size=(n, n))
    h = rng.normal(size=(n, n))
    ref = oracle_fock(h, v, P)
    with g.Context(n, 9, 8, 10.0) as ctx:
        g.gf2_set_integrals(ctx.handle, dev(v))
        F = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
        g.gf2_fock(ctx.handle, dev(h), dev(P), F)
        got = host(F)
        hd = dev(h)
        g.gf2_fock(ctx.handle, hd, dev(P), hd)
        in_place = host(hd)
        Pd = dev(P)
        with pytest.raises(g.GF2Error):
            g.gf2_fock(ctx.handle, dev(h), Pd, Pd)
    scale = max(1.0, np.abs(ref).max())
    assert np.abs(got - ref).max() <= 1e-12 * scale
    assert np.abs(in_place - ref).max() <= 1e-12 * scale


def test_mu_search_coarse_stage_matches_oracle(library, h4):
    """n_iw = 2048 switches on the coarse (n_iw/8 frequency) stage of the GPU
    search; with a correlated Sigma the converged count and P must still match
    the oracle's bisection on the full frequency sum."""
    g = library
    s, r = h4
    beta, n_tau, n_iw = 50.0, 129, 2048
    F, mu, G, P = og.inner_loop(s, r.F, None, None, None, beta, n_iw)
    st = og.GF2State(F=F, mu=mu, P=P, G_iw=G, sig1=np.zeros_like(F), sig2=np.zeros_like(F))
    _, Sig_tau = og.self_energy_step(s, st, beta, n_tau, n_iw)
    Sig_iw = ot.tau_to_iw(Sig_tau, beta, n_iw)
    sig1, sig2 = ot.sigma_expansion(Sig_tau, beta)
    mu_ref, G_ref, P_ref, _ = od.mu_search(s.S, F, Sig_iw, sig1, sig2, s.n_elec, beta, n_iw)
    with g.Context(s.nbf, n_tau, n_iw, beta) as ctx:
        Gd = torch.zeros(n_iw, s.nbf, s.nbf, dtype=torch.complex128, device="cuda")
        Pd = torch.zeros(s.nbf, s.nbf, dtype=torch.float64, device="cuda")
        for start in (mu_ref + 0.05, mu_ref - 0.2):
            got_mu, nev = g.gf2_mu_search(ctx.handle, dev(s.S), dev(F), dev(Sig_iw), dev(np.stack([sig1, sig2])),
                                          s.n_elec, start, Gd, Pd)
            Pn = host(Pd)
            assert abs(np.trace(Pn @ s.S) - s.n_elec) <= 1e-10
            assert np.abs(Pn - P_ref).max() < 1e-8
            assert nev < 60


def test_energy_matches_oracle(library, h4):
    g = library
    s, r = h4
    beta, n_tau, n_iw = 50.0, 257, 512
    F, mu, G, P = og.inner_loop(s, r.F, None, None, None, beta, n_iw)
    st = og.GF2State(F=F, mu=mu, P=P, G_iw=G, sig1=np.zeros_like(F), sig2=np.zeros_like(F))
    _, Sig_tau = og.self_energy_step(s, st, beta, n_tau, n_iw)
    Sig_iw = ot.tau_to_iw(Sig_tau, beta, n_iw)
    sig1, sig2 = ot.sigma_expansion(Sig_tau, beta)
    e1_ref = oe.e_one_body(P, s.h, F)
    e2_ref = oe.e_two_body(G, Sig_iw, sig1, s.S, beta)
    with g.Context(s.nbf, n_tau, n_iw, beta) as ctx:
        e1, e2 = g.gf2_energy(ctx.handle, dev(s.h), dev(F), dev(P), dev(s.S), dev(G), dev(Sig_iw),
                              dev(np.stack([sig1, sig2])))
    assert abs(e1 - e1_ref) < 1e-12
    assert abs(e2 - e2_ref) < 1e-12


def _gf2_both(system, beta, n_tau, n_iw, max_outer):
    from paper_1405_3273_gb300 import driver
    r = gi.rhf(system)
    ref = og.run(system, r.F, beta, n_tau, n_iw, max_outer=max_outer, e_tol=0.0)
    system.beta, system.n_tau, system.n_iw = beta, n_tau, n_iw
    mu0 = 0.5 * (r.eps[system.n_elec // 2 - 1] + r.eps[system.n_elec // 2])
    ds = driver.to_device(system, r.F, mu0)
    got = driver.run_gf2(ds, max_outer=max_outer, e_tol=0.0)
    return ref, got


def test_full_gf2_h4_matches_oracle_every_iteration(library):
    s = gi.build_system("chain", coords=gi.h_chain(4, 1.7), basis="sto-3g", beta=50.0, n_tau=257, n_iw=512)
    ref, got = _gf2_both(s, 50.0, 257, 512, 4)
    e_ref = np.array([e[0] for e in ref.energies])
    e_got = np.array([e[0] for e in got.energies])
    assert len(e_ref) == len(e_got)
    assert np.abs(e_ref - e_got).max() < 1e-9
    assert np.abs(host(got.P) - ref.P).max() < 1e-8
    # Sigma(tau) itself is not compared after a mu search: with mu inside the
    # HOMO-LUMO gap N(mu) is flat, both searches stop at different (equally
    # valid) mu, and G(tau) ~ e^{mu tau} shifts while P and E do not.


def test_h10_chain_sto3g_workload_first_iterations(library):
    """Linear H10, 1.8 bohr, STO-3G, beta = 100, n_tau = 2049, n_iw = 4096 (full size)."""
    s = gi.build_system("h10_chain_sto3g")
    ref, got = _gf2_both(s, 100.0, 2049, 4096, 2)
    e_ref = np.array([e[0] for e in ref.energies])
    e_got = np.array([e[0] for e in got.energies])
    assert np.abs(e_ref - e_got).max() < 1e-8
    assert np.abs(host(got.P) - ref.P).max() < 1e-8


@pytest.mark.parametrize("beta", [20.0, 100.0])
def test_natural_occupations_match_oracle_and_fermi_dirac(library, beta):
    """H32 2x4x4 lattice, 6-31G (N = 64): occupations of a finite-temperature HF
    density against the oracle and against the Fermi-Dirac values themselves."""
    from oracle.occupations import natural_occupations
    from tests import closed_forms as cf
    s = gi.build_system("h32_lattice_631g")
    r = gi.rhf(s)
    mu = 0.5 * (r.eps[15] + r.eps[16])
    _, C, _, f = cf.mo_basis(r.F, s.S, mu, beta)
    P = cf.density_closed(C, f)
    g = library
    with g.Context(s.nbf, 65, 8, beta) as ctx:
        g.gf2_set_overlap(ctx.handle, dev(s.S))
        occ = torch.empty(s.nbf, dtype=torch.float64, device="cuda")
        g.gf2_natural_occupations(ctx.handle, dev(P), occ)
        got = occ.cpu().numpy()
    assert np.abs(got - natural_occupations(P, s.S)).max() < 1e-10
    assert np.abs(got - np.sort(f)[::-1]).max() < 1e-10
    assert abs(got.sum() - 0.5 * np.trace(P @ s.S)) < 1e-10


def test_natural_occupations_need_the_overlap(library):
    g = library
    with g.Context(6, 65, 8, 10.0) as ctx:
        occ = torch.empty(6, dtype=torch.float64, device="cuda")
        with pytest.raises(g.GF2Error):
            g.gf2_natural_occupations(ctx.handle, torch.eye(6, dtype=torch.float64, device="cuda"), occ)
