"""Pins of the oracle's non-equidistant time grid (the uniform power mesh) and
of the transforms on it, against closed forms and the uniform-grid scheme.

* the mesh itself: point count, symmetry, the doubling of the step per level;
* tau -> iw weights on the grid 0..M are those of the uniform scheme;
* a global cubic is reproduced by every local cubic, so its transform is the
  exact Fourier integral (closed form by parts) and Sig1, Sig2 its end values
  and slopes;
* single fermionic pole G(tau) = -e^{-eps tau} / (1 + e^{-beta eps}) with
  G(i w) = 1/(i w - eps): fourth-order convergence in the steps per level, and
  a far smaller error than a uniform grid of as many points;
* iw -> tau on the mesh points against the same closed form.
"""

import numpy as np
import pytest

from oracle import grids
from oracle import transforms as ot


def test_power_mesh_structure():
    for p, u in [(0, 4), (3, 4), (5, 16), (7, 32)]:
        M, idx = grids.power_mesh(p, u)
        assert M == 2 ** (p + 1) * u
        assert len(idx) == 2 * (p + 1) * u + 1
        assert idx[0] == 0 and idx[-1] == M and M // 2 in idx
        assert np.all(np.diff(idx) > 0)
        assert np.all(idx + idx[::-1] == M)
        steps = np.diff(idx[: len(idx) // 2 + 1])
        # u steps of 1 on [0, beta/2^(p+1)], then u steps of 2^(p-j) on [beta/2^(j+1), beta/2^j]
        expect = np.concatenate([np.ones(u)] + [np.full(u, 2 ** (p - j)) for j in range(p, 0, -1)])
        assert np.array_equal(steps, expect)
    with pytest.raises(ValueError):
        grids.power_mesh(-1, 4)


def test_grid_weights_reduce_to_the_uniform_scheme():
    for beta, M, n_iw in [(10.0, 64, 40), (50.0, 256, 700)]:
        W_grid = ot.grid_fourier_weights(beta, M, np.arange(M + 1), n_iw)
        W_uni = ot.cubic_fourier_weights(beta, M + 1, n_iw)
        assert np.abs(W_grid - W_uni).max() <= 1e-14 * np.abs(W_uni).max()


def _cubic_fourier_exact(c, beta, w):
    """int_0^beta e^{i w tau} sum_k c_k tau^k dtau for fermionic w (e^{i w beta} = -1),
    by parts: I_k = (-beta^k - 0^k) / (i w) - k I_{k-1} / (i w)."""
    iw = 1j * w
    I = [(-1.0 - 1.0) / iw]
    for k in range(1, 4):
        I.append(-(beta ** k) / iw - k * I[k - 1] / iw)
    return sum(c[k][None] * I[k][:, None, None] for k in range(4))


@pytest.mark.parametrize("p,u", [(3, 4), (5, 8)])
def test_global_cubic_is_transformed_exactly(p, u):
    beta, n_iw = 20.0, 300
    rng = np.random.default_rng(7)
    c = rng.standard_normal((4, 3, 3)) * np.array([1.0, 0.3, 0.02, 1e-3])[:, None, None]
    M, idx = grids.power_mesh(p, u)
    t = grids.grid_points(beta, M, idx)
    X = sum(c[k][None] * t[:, None, None] ** k for k in range(4))
    got = ot.tau_to_iw_grid(X, beta, M, idx, n_iw)
    exact = _cubic_fourier_exact(c, beta, grids.matsubara(beta, n_iw))
    assert np.abs(got - exact).max() <= 1e-12 * np.abs(exact).max()
    sig1, sig2 = ot.sigma_expansion_grid(X, beta, M, idx)
    X0, Xb = c[0], sum(c[k] * beta ** k for k in range(4))
    d0, db = c[1], sum(k * c[k] * beta ** (k - 1) for k in range(1, 4))
    assert np.abs(sig1 + X0 + Xb).max() <= 1e-12 * np.abs(Xb).max()
    assert np.abs(sig2 - (d0 + db)).max() <= 1e-10 * np.abs(db).max()


def _pole(eps, beta, t):
    return (-np.exp(-eps * t) / (1.0 + np.exp(-beta * eps)))[:, None, None]


@pytest.mark.parametrize("eps", [0.5, -0.3, 2.0])
def test_single_pole_converges_at_fourth_order_and_beats_the_uniform_grid(eps):
    beta, n_iw = 100.0, 2048
    w = grids.matsubara(beta, n_iw)
    exact = 1.0 / (1j * w - eps)
    errs = []
    for u in (8, 16, 32):
        M, idx = grids.power_mesh(5, u)
        got = ot.tau_to_iw_grid(_pole(eps, beta, grids.grid_points(beta, M, idx)), beta, M, idx, n_iw)[:, 0, 0]
        errs.append(np.abs(got - exact).max())
        n = len(idx)
        uni = ot.tau_to_iw(_pole(eps, beta, np.linspace(0.0, beta, n)), beta, n_iw)[:, 0, 0]
        assert errs[-1] < np.abs(uni - exact).max()
    # halving the step divides the error by ~16 (cubic interpolant)
    assert 10.0 < errs[0] / errs[1] < 22.0 and 10.0 < errs[1] / errs[2] < 22.0
    if eps == 2.0:  # a sharp pole: the mesh is orders of magnitude better
        assert errs[1] < 1e-2 * np.abs(ot.tau_to_iw(_pole(eps, beta, np.linspace(0.0, beta, 193)),
                                                   beta, n_iw)[:, 0, 0] - exact).max()


def test_iw_to_tau_on_mesh_points_matches_the_pole():
    beta, n_iw, eps = 40.0, 1024, 0.7
    M, idx = grids.power_mesh(4, 8)
    w = grids.matsubara(beta, n_iw)
    X_iw = (1.0 / (1j * w - eps))[:, None, None] * np.ones((1, 1, 1))
    moments = np.array([[[1.0]], [[eps]], [[eps ** 2]], [[eps ** 3]]])
    got = ot.iw_to_tau(X_iw, moments, beta, M + 1, taus=idx)
    exact = _pole(eps, beta, grids.grid_points(beta, M, idx))
    assert np.abs(got - exact).max() < 1e-9


def test_gf2_energy_on_the_mesh_matches_a_fine_uniform_grid():
    """H4 chain (STO-3G, 1.7 bohr), beta = 50, two GF2 iterations: the mesh of
    193 points reaches the energy of the 4097-point uniform grid to 1e-7 Eh,
    a uniform grid of 193 points misses it by more than 1e-5 Eh."""
    import gf2_inputs as gi
    from oracle import gf2 as og
    s = gi.build_system("chain", coords=gi.h_chain(4, 1.7), basis="sto-3g", beta=50.0, n_tau=257, n_iw=512)
    r = gi.rhf(s)
    ref = og.run(s, r.F, 50.0, 4097, 2048, max_outer=2, e_tol=0.0)
    M, idx = grids.power_mesh(5, 16)
    mesh = og.run(s, r.F, 50.0, None, 2048, max_outer=2, e_tol=0.0, grid=(M, idx))
    uni = og.run(s, r.F, 50.0, len(idx), 2048, max_outer=2, e_tol=0.0)
    d_mesh = abs(mesh.energies[-1][0] - ref.energies[-1][0])
    d_uni = abs(uni.energies[-1][0] - ref.energies[-1][0])
    assert d_mesh < 1e-7 and d_uni > 1e-5
