"""Pins for the oracle's Matsubara <-> imaginary-time transforms."""

import numpy as np
import pytest

import gf2_inputs as gi
from oracle import dyson as od
from oracle import transforms as ot
from oracle.grids import matsubara, tau_grid
from tests import closed_forms as cf


@pytest.fixture(scope="module")
def h4():
    s = gi.build_system("chain", coords=gi.h_chain(4, 1.7), basis="sto-3g", beta=100, n_tau=513, n_iw=1024)
    return s, gi.rhf(s)


def test_iw_to_tau_reproduces_single_pole_green_function(h4):
    s, r = h4
    beta, n_tau, n_iw = 100.0, 513, 2048
    mu = 0.5 * (r.eps[1] + r.eps[2])
    G_iw = od.dyson(mu, s.S, r.F, None, beta, n_iw)
    mom = ot.tail_moments(s.S, r.F, mu)
    G_tau = ot.iw_to_tau(G_iw, mom, beta, n_tau)
    _, C, xi, f = cf.mo_basis(r.F, s.S, mu, beta)
    ref = cf.g_tau_ao(C, xi, beta, tau_grid(beta, n_tau))
    # left over after four moments: Re[e^{-iwt} G5/(iw)^5] summed past n_iw,
    # about (2/beta) |G5| (beta/2pi) / (4 w_max^4) ~ 3e-10 |G5| here
    # (the floor near 1e-10 is rounding in the beta^3/48 G4 tail term)
    err = np.abs(G_tau - ref).max()
    assert err < 1e-9
    G_half = od.dyson(mu, s.S, r.F, None, beta, n_iw // 2)
    err_half = np.abs(ot.iw_to_tau(G_half, mom, beta, n_tau) - ref).max()
    assert err < err_half / 8.0


def test_tail_moments_are_the_high_frequency_expansion(h4):
    s, r = h4
    beta, mu = 100.0, -0.1
    sig1 = np.diag(np.linspace(-0.1, 0.2, s.nbf))
    sig2 = 0.05 * np.ones((s.nbf, s.nbf))
    mom = ot.tail_moments(s.S, r.F, mu, sig1, sig2)
    for w in [1e3, 3e3]:
        z = 1j * w
        G = np.linalg.inv((z + mu) * s.S - r.F - sig1 / z - sig2 / z ** 2)
        T = sum(mom[r_] / z ** (r_ + 1) for r_ in range(4))
        # the remainder is O(1/w^5)
        assert np.abs(G - T).max() < 50.0 / w ** 5


def test_tau_to_iw_is_exact_for_cubic_polynomials():
    beta, n_tau, n_iw = 5.0, 65, 300
    c = np.array([0.3, -1.1, 0.7, -0.2])
    t = tau_grid(beta, n_tau)
    X = (c[0] + c[1] * t + c[2] * t ** 2 + c[3] * t ** 3)[:, None, None]
    Xw = ot.tau_to_iw(X, beta, n_iw)[:, 0, 0]
    # repeated integration by parts (X'''' = 0, e^{i w beta} = -1):
    # int_0^beta e^{i w t} X = -s0/z + s1/z^2 - s2/z^3 + s3/z^4, s_r = X^(r)(0) + X^(r)(beta)
    d0 = [c[0], c[1], 2 * c[2], 6 * c[3]]
    db = [c[0] + c[1] * beta + c[2] * beta ** 2 + c[3] * beta ** 3,
          c[1] + 2 * c[2] * beta + 3 * c[3] * beta ** 2,
          2 * c[2] + 6 * c[3] * beta, 6 * c[3]]
    sr = [a + b for a, b in zip(d0, db)]
    z = 1j * matsubara(beta, n_iw)
    ref = -sr[0] / z + sr[1] / z ** 2 - sr[2] / z ** 3 + sr[3] / z ** 4
    assert np.abs(Xw - ref).max() < 1e-12 * np.abs(ref).max()
    sig1, sig2 = ot.sigma_expansion(X, beta)
    assert abs(sig1[0, 0] + sr[0]) < 1e-12 and abs(sig2[0, 0] - sr[1]) < 1e-10


def test_tau_to_iw_of_an_exponential_converges_at_fourth_order():
    beta, a, n_iw = 10.0, 1.3, 200
    errs = []
    for n_tau in (257, 513, 1025):
        t = tau_grid(beta, n_tau)
        X = np.exp(-a * t)[:, None, None]
        Xw = ot.tau_to_iw(X, beta, n_iw)[:, 0, 0]
        z = 1j * matsubara(beta, n_iw)
        ref = -(1.0 + np.exp(-a * beta)) / (z - a)
        errs.append(np.abs(Xw - ref).max())
    assert errs[-1] < 1e-9
    assert errs[0] / errs[1] > 12 and errs[1] / errs[2] > 12


def test_round_trip_tau_iw_tau(h4):
    """Sigma-like tau function -> i w -> tau (with its own tail) recovers the samples."""
    beta, n_tau, n_iw = 20.0, 257, 4096
    t = tau_grid(beta, n_tau)
    X = (-np.exp(-0.8 * t) - 0.5 * np.exp(-1.5 * (beta - t)))[:, None, None]
    Xw = ot.tau_to_iw(X, beta, n_iw)
    sig1, sig2 = ot.sigma_expansion(X, beta)
    zero = np.zeros((1, 1))
    # the expansion Sig1/z + Sig2/z^2 goes into the first two tail slots
    mom = np.array([sig1, sig2, zero, zero])
    back = ot.iw_to_tau(Xw, mom, beta, n_tau)
    assert np.abs(back[1:-1] - X[1:-1]).max() < 2e-5


def test_pole_tail_has_the_moment_expansion_and_its_tau_image():
    rng = np.random.default_rng(11)
    mom = rng.normal(size=(4, 3, 3))
    mom = mom + np.swapaxes(mom, 1, 2)
    # high frequency: T(z) - sum G_r z^-r = O(z^-5)
    for w in (3e2, 6e2):
        z = 1j * w
        T = ot.tail_iw(mom, [w])[0]
        poly = sum(mom[r] / z ** (r + 1) for r in range(4))
        assert np.abs(T - poly).max() < 40.0 * np.abs(mom).max() / w ** 5
    # tau image of 1/(z-a)^r equals the (r-1)-th a-derivative of the single pole / (r-1)!
    beta, a, h = 7.0, ot.TAIL_POLE, 1e-3
    taus = np.linspace(0.0, beta, 11)

    def g1(aa):
        return -np.exp(-aa * taus) / (1.0 + np.exp(-aa * beta))

    fd = [g1(a),
          (g1(a + h) - g1(a - h)) / (2 * h),
          (g1(a + h) - 2 * g1(a) + g1(a - h)) / h ** 2 / 2.0,
          (g1(a + 2 * h) - 2 * g1(a + h) + 2 * g1(a - h) - g1(a - 2 * h)) / (2 * h ** 3) / 6.0]
    for r in range(4):
        unit = np.zeros((4, 1, 1))
        # moments whose pole coefficients are the unit vector e_r
        c = np.zeros(4)
        c[r] = 1.0
        # invert c = L m (L lower triangular in powers of a)
        L = np.array([[1, 0, 0, 0], [-a, 1, 0, 0], [a * a, -2 * a, 1, 0], [-a ** 3, 3 * a * a, -3 * a, 1]])
        unit[:, 0, 0] = np.linalg.solve(L, c)
        got = ot.tail_tau(unit, taus, beta)[:, 0, 0]
        assert np.abs(got - fd[r]).max() < 2e-5


def test_iw_to_tau_on_selected_points_equals_the_full_grid_rows():
    """The subset option (used to time the oracle on a sample of time points)
    returns exactly the rows of the full transform."""
    rng = np.random.default_rng(11)
    n, beta, n_tau, n_iw = 3, 20.0, 33, 48
    X = rng.normal(size=(n_iw, n, n)) + 1j * rng.normal(size=(n_iw, n, n))
    mom = rng.normal(size=(4, n, n))
    full = ot.iw_to_tau(X, mom, beta, n_tau)
    taus = [5, 0, 32, 17]
    sub = ot.iw_to_tau(X, mom, beta, n_tau, taus=taus)
    assert np.abs(sub - full[taus]).max() <= 1e-14 * np.abs(full).max()
