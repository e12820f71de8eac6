"""The self-consistent GF2 loop of the paper's supplement (steps 1-3).

1. restricted HF reference (F_HF, P_HF, S) -- supplied by ``gf2_inputs``;
2. build G(i w) by Eq. GF (Sigma = 0 and F = F_HF at the start);
   2.a find mu giving the right particle number,
   2.b rebuild F(P) by Eq. FockMatrix and update G; repeat 2.a-2.b to
       self-consistency; transform G(i w) -> G(tau);
3. build Sigma(tau) by Eq. Sigma, transform Sigma(tau) -> Sigma(i w) and go
   back to 2 until the energy stops changing.

Optional damping (the supplement damps P in the inner loop and Sigma(tau) in
the outer loop without stating amounts): P <- a_P P_new + (1-a_P) P_old and
Sigma <- a_S Sigma_new + (1-a_S) Sigma_old, both 1 (no damping) by default.
The inner loop takes damped steps far from its fixed point and Pulay (DIIS)
extrapolation near it (see ``inner_loop``).
"""

from dataclasses import dataclass, field

import numpy as np

from . import dyson as dy
from . import energy as en
from .fock import fock
from .sigma import sigma_tau
from .transforms import (iw_to_tau, sigma_expansion, sigma_expansion_grid, tail_moments, tau_to_iw,
                         tau_to_iw_grid)


@dataclass
class GF2State:
    F: np.ndarray
    mu: float
    P: np.ndarray
    G_iw: np.ndarray
    Sigma_iw: np.ndarray = None
    Sigma_tau: np.ndarray = None
    sig1: np.ndarray = None
    sig2: np.ndarray = None
    energies: list = field(default_factory=list)


def _diis_coefficients(gram):
    """Pulay weights: minimise |sum c_a R_a| subject to sum c_a = 1."""
    m = gram.shape[0]
    B = np.zeros((m + 1, m + 1))
    B[:m, :m] = gram
    B[m, :m] = B[:m, m] = -1.0
    rhs = np.zeros(m + 1)
    rhs[m] = -1.0
    return np.linalg.lstsq(B, rhs, rcond=None)[0][:m]


def inner_loop(system, F, Sigma_iw, sig1, sig2, beta, n_iw, tol=1e-8, max_iter=300,
               p_damping=1.0, diis=8, mix=0.5, diis_from=1e-3):
    """Steps 2.a-2.b: alternate the mu search and the Fock rebuild to self-consistency.

    Converged when the Fock residual R = F(P(F)) - F has Frobenius norm below
    ``tol`` (the mu search stops anywhere within 1e-10 electrons, which leaves
    a noise floor near 1e-9 in R).  The schedule of the next F:
      * far from the fixed point, |R| > ``diis_from`` (or ``diis`` <= 0): the
        damped step F + ``mix`` R (``mix`` = 1 is the plain map F <- F(P(F)));
      * closer in: the Pulay (DIIS) extrapolation of the last ``diis``
        rebuilt matrices, the history restarting whenever a damped step is
        taken.
    (The plain map is unstable for some lattices at finite temperature, and
    from the HF state of a correlated lattice the fixed point can sit 20 mEh
    away in mu, where DIIS alone wanders.)  G, P and mu are then re-evaluated
    at the converged F.
    """
    S, h, v = system.S, system.h, system.eri
    P_old = None
    hist_F, hist_R = [], []
    for _ in range(max_iter):
        mu, G, P, _ = dy.mu_search(S, F, Sigma_iw, sig1, sig2, system.n_elec, beta, n_iw)
        if P_old is not None and p_damping < 1.0:
            P = p_damping * P + (1.0 - p_damping) * P_old
        P_old = P
        F_out = fock(h, v, P)
        R = F_out - F
        r_norm = np.sqrt(np.sum(R * R))
        if r_norm < tol:
            F = F_out
            mu, G, P, _ = dy.mu_search(S, F, Sigma_iw, sig1, sig2, system.n_elec, beta, n_iw)
            return F, mu, G, P
        if r_norm > diis_from or diis <= 0:
            hist_F, hist_R = [], []
            F = F + mix * R
            continue
        hist_F.append(F_out)
        hist_R.append(R)
        hist_F, hist_R = hist_F[-diis:], hist_R[-diis:]
        if len(hist_F) > 1:
            gram = np.array([[np.sum(a * b) for b in hist_R] for a in hist_R])
            c = _diis_coefficients(gram)
            F = sum(ci * fi for ci, fi in zip(c, hist_F))
        else:
            F = F_out
    raise RuntimeError("inner loop did not converge")


def energy(system, state, beta):
    e1 = en.e_one_body(state.P, system.h, state.F)
    e2 = 0.0
    if state.Sigma_iw is not None:
        e2 = en.e_two_body(state.G_iw, state.Sigma_iw, state.sig1, system.S, beta)
    return system.e_nuc + e1 + e2, e1, e2


def self_energy_step(system, state, beta, n_tau, n_iw, sigma_fn=None, grid=None):
    """G(i w) -> G(tau) -> Sigma(tau) for the current state, on the uniform grid
    of n_tau points or on grid = (M, index) (``grids.power_mesh``)."""
    mom = tail_moments(system.S, state.F, state.mu, state.sig1, state.sig2)
    if grid is None:
        G_tau = iw_to_tau(state.G_iw, mom, beta, n_tau)
    else:
        G_tau = iw_to_tau(state.G_iw, mom, beta, grid[0] + 1, taus=grid[1])
    Sig_tau = (sigma_fn or sigma_tau)(G_tau, system.eri)
    return G_tau, Sig_tau


def sigma_to_iw(Sig_tau, beta, n_iw, grid=None):
    """Sigma(i w), Sig1, Sig2 from Sigma(tau) on the uniform grid or on grid = (M, index)."""
    if grid is None:
        return (tau_to_iw(Sig_tau, beta, n_iw),) + tuple(sigma_expansion(Sig_tau, beta))
    M, index = grid
    return (tau_to_iw_grid(Sig_tau, beta, M, index, n_iw),) + tuple(sigma_expansion_grid(Sig_tau, beta, M, index))


def run(system, F_start, beta, n_tau, n_iw, max_outer=30, e_tol=1e-8, sigma_damping=1.0,
        p_damping=1.0, inner_tol=1e-8, sigma_fn=None, callback=None, diis=8, mix=0.5, diis_from=1e-3,
        grid=None):
    """Full GF2; returns the final GF2State (energies[] holds (E, E1, E2) per iteration).
    ``grid`` = (M, index) replaces the uniform time grid of n_tau points."""
    n = system.nbf
    F, mu, G, P = inner_loop(system, F_start, None, None, None, beta, n_iw, inner_tol,
                             p_damping=p_damping, diis=diis, mix=mix, diis_from=diis_from)
    state = GF2State(F=F, mu=mu, P=P, G_iw=G, sig1=np.zeros((n, n)), sig2=np.zeros((n, n)))
    state.energies.append(energy(system, state, beta))
    for _ in range(max_outer):
        _, Sig_tau = self_energy_step(system, state, beta, n_tau, n_iw, sigma_fn, grid)
        if state.Sigma_tau is not None and sigma_damping < 1.0:
            Sig_tau = sigma_damping * Sig_tau + (1.0 - sigma_damping) * state.Sigma_tau
        state.Sigma_tau = Sig_tau
        state.Sigma_iw, state.sig1, state.sig2 = sigma_to_iw(Sig_tau, beta, n_iw, grid)
        state.F, state.mu, state.G_iw, state.P = inner_loop(
            system, state.F, state.Sigma_iw, state.sig1, state.sig2, beta, n_iw, inner_tol,
            p_damping=p_damping, diis=diis, mix=mix, diis_from=diis_from)
        state.energies.append(energy(system, state, beta))
        if callback is not None:
            callback(state)
        if abs(state.energies[-1][0] - state.energies[-2][0]) < e_tol:
            break
    return state
