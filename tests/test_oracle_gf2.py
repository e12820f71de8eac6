"""The oracle's full GF2 loop on H2/STO-3G (small grids)."""

import numpy as np
import pytest

import gf2_inputs as gi
from oracle import gf2 as og
from oracle import sigma as osg


@pytest.fixture(scope="module")
def h2():
    s = gi.build_system("h2_sto3g")
    return s, gi.rhf(s)


def test_gf2_converges_and_literal_sum_gives_the_same_run(h2):
    s, r = h2
    beta, n_tau, n_iw = 50.0, 257, 512
    fac = og.run(s, r.F, beta, n_tau, n_iw, max_outer=40, e_tol=1e-10)
    lit = og.run(s, r.F, beta, n_tau, n_iw, max_outer=40, e_tol=1e-10,
                 sigma_fn=lambda G, v: osg.sigma_tau(G, v, literal=True))
    e_fac = np.array([e[0] for e in fac.energies])
    e_lit = np.array([e[0] for e in lit.energies])
    assert len(e_fac) == len(e_lit)
    assert np.abs(e_fac - e_lit).max() < 1e-12
    # converged, correlated, and below HF
    assert abs(e_fac[-1] - e_fac[-2]) < 1e-10
    assert e_fac[-1] < r.e_total - 1e-3
    # particle number at convergence
    assert abs(np.trace(fac.P @ s.S) - 2.0) < 1e-9
    # Sigma(tau) real symmetric
    assert np.abs(fac.Sigma_tau - np.swapaxes(fac.Sigma_tau, 1, 2)).max() < 1e-14


def test_inner_loop_converges_on_the_h32_lattice():
    """H32 2x4x4 lattice (STO-3G, 2.0 bohr), beta = 100, no self-energy: the plain
    fixed-point map of steps 2.a-2.b has an unstable mode there (residual growth
    about 1.76 per step below 1e-9); the extrapolated loop converges."""
    s = gi.build_system("h32_lattice_sto3g")
    r = gi.rhf(s)
    F, mu, G, P = og.inner_loop(s, r.F, None, None, None, 100.0, 256, tol=1e-8)
    from oracle.fock import fock
    R = fock(s.h, s.eri, P) - F
    assert np.sqrt(np.sum(R * R)) < 1e-8
    assert abs(np.trace(P @ s.S) - 32.0) < 1e-9
