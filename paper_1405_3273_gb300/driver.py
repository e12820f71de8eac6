"""The self-consistent GF2 loop (steps 1-3 of the paper's supplement) driven
through the libgf2 C-ABI.  Every numerical step runs in the library's CUDA
kernels; this module only sequences calls and moves a few scalars.

State kept on the device per iteration: F, mu, G(i w), P, Sigma(tau),
Sigma(i w) and the tail coefficients (Sig1, Sig2).
"""

from dataclasses import dataclass, field

import torch

import numpy as np

from . import (GF2_PREC_BF16X3, GF2_PREC_FP64, Context, gf2_combine, gf2_energy, gf2_fft_iw_to_tau,
               gf2_fft_tau_to_iw, gf2_fock, gf2_gram, gf2_inner_loop, gf2_mu_search, gf2_set_integrals,
               gf2_set_df_integrals, gf2_set_overlap, gf2_sigma_tau, gf2_sigma_tau_df, gf2_tail_moments)


@dataclass
class DeviceSystem:
    S: torch.Tensor
    h: torch.Tensor
    v: torch.Tensor
    F0: torch.Tensor
    e_nuc: float
    n_elec: int
    beta: float
    n_tau: int
    n_iw: int
    mu0: float
    grid: tuple = None   # (M, tau_index): a non-equidistant time grid replacing the n_tau uniform points
    df_B: torch.Tensor = None  # [m, N, N]: density-fitted integrals v_ijkl = sum_Q B_Qij B_Qkl replace v

    @property
    def nbf(self):
        return self.S.shape[0]


def to_device(system, F_start, mu0, device="cuda", grid=None, df_B=None):
    f = lambda a: torch.as_tensor(a, dtype=torch.float64, device=device).contiguous()
    n_tau = int(system.n_tau) if grid is None else len(grid[1])
    return DeviceSystem(S=f(system.S), h=f(system.h), v=f(system.eri), F0=f(F_start),
                        e_nuc=float(system.e_nuc), n_elec=int(system.n_elec), beta=float(system.beta),
                        n_tau=n_tau, n_iw=int(system.n_iw), mu0=float(mu0), grid=grid,
                        df_B=None if df_B is None else f(df_B))


@dataclass
class GF2Run:
    ctx: Context
    sys: DeviceSystem
    prec: int = GF2_PREC_FP64
    F: torch.Tensor = None
    mu: float = 0.0
    P: torch.Tensor = None
    G_iw: torch.Tensor = None
    G_tau: torch.Tensor = None
    Sigma_tau: torch.Tensor = None
    Sigma_iw: torch.Tensor = None
    sig12: torch.Tensor = None
    moments: torch.Tensor = None
    energies: list = field(default_factory=list)
    mu_evals: list = field(default_factory=list)
    inner_iters: list = field(default_factory=list)
    device_inner: bool = True
    df_order: bool = False   # Sigma by gf2_sigma_tau_df (the factor order) instead of gf2_sigma_tau


def start(sys, prec=GF2_PREC_FP64, df_order=False):
    n, nt, nw = sys.nbf, sys.n_tau, sys.n_iw
    ctx = Context(n, nt, nw, sys.beta, grid=sys.grid)
    if sys.df_B is not None:
        gf2_set_df_integrals(ctx.handle, sys.df_B)
    else:
        if df_order:
            raise ValueError("the factor-order Sigma needs density-fitted integrals (DeviceSystem.df_B)")
        gf2_set_integrals(ctx.handle, sys.v)
    gf2_set_overlap(ctx.handle, sys.S)
    dev = sys.S.device
    run = GF2Run(ctx=ctx, sys=sys, prec=prec, df_order=df_order)
    run.F = sys.F0.clone()
    run.mu = sys.mu0
    run.P = torch.zeros(n, n, dtype=torch.float64, device=dev)
    run.G_iw = torch.zeros(nw, n, n, dtype=torch.complex128, device=dev)
    run.G_tau = torch.zeros(nt, n, n, dtype=torch.float64, device=dev)
    run.Sigma_tau = torch.zeros(nt, n, n, dtype=torch.float64, device=dev)
    run.Sigma_iw = torch.zeros(nw, n, n, dtype=torch.complex128, device=dev)
    run.sig12 = None
    run.moments = torch.zeros(4, n, n, dtype=torch.float64, device=dev)
    return run


def _diis_coefficients(gram):
    """Pulay weights: minimise |sum c_a R_a| subject to sum c_a = 1 (host, tiny)."""
    m = len(gram)
    B = np.zeros((m + 1, m + 1))
    B[:m, :m] = np.asarray(gram)
    B[m, :m] = B[:m, m] = -1.0
    rhs = np.zeros(m + 1)
    rhs[m] = -1.0
    return np.linalg.lstsq(B, rhs, rcond=None)[0][:m]


def inner_loop(run, tol=1e-8, max_iter=300, mu_tol=1e-10, diis=8, mix=0.5, diis_from=1e-3, device=None):
    """Steps 2.a-2.b: mu search and Fock rebuild until the Fock residual
    R = F(P(F)) - F has Frobenius norm below ``tol``.  Far from the fixed point
    (|R| > ``diis_from``) the next F is the damped step F + mix R; closer in it is
    the Pulay (DIIS) extrapolation of the last ``diis`` rebuilt matrices.  (From
    the HF state of a correlated lattice the fixed point can sit 20 mEh away in
    mu, where DIIS alone wanders.)  G, P and mu are re-evaluated at the converged F.

    ``device`` (default: ``run.device_inner``) runs the whole loop as one
    device-resident graph (gf2_inner_loop); otherwise the host sequences the
    same steps call by call (one synchronization per mu search and Gram matrix)."""
    s = run.sys
    h = run.ctx.handle
    if run.device_inner if device is None else device:
        run.mu, nit, nev = gf2_inner_loop(h, s.S, s.h, run.F, run.Sigma_iw, run.sig12, s.n_elec, run.mu,
                                          run.G_iw, run.P, tol=tol, max_iter=max_iter, mu_tol=mu_tol, diis=diis,
                                          mix=mix, diis_from=diis_from)
        run.mu_evals.append(nev)
        run.inner_iters.append(nit)
        return
    hist_F, hist_R = [], []
    for _ in range(max_iter):
        run.mu, nev = gf2_mu_search(h, s.S, run.F, run.Sigma_iw, run.sig12, s.n_elec, run.mu,
                                    run.G_iw, run.P, tol=mu_tol)
        run.mu_evals.append(nev)
        F_out = torch.empty_like(run.F)
        gf2_fock(h, s.h, run.P, F_out)
        R = torch.empty_like(run.F)
        gf2_combine(h, [1.0, -1.0], [F_out, run.F], R)
        r_norm = gf2_gram(h, [R])[0][0] ** 0.5
        if r_norm < tol:
            run.F = F_out
            run.mu, nev = gf2_mu_search(h, s.S, run.F, run.Sigma_iw, run.sig12, s.n_elec, run.mu,
                                        run.G_iw, run.P, tol=mu_tol)
            run.mu_evals.append(nev)
            return
        if r_norm > diis_from or diis <= 0:
            hist_F, hist_R = [], []
            F_next = torch.empty_like(run.F)
            gf2_combine(h, [1.0, mix], [run.F, R], F_next)
            run.F = F_next
            continue
        hist_F.append(F_out)
        hist_R.append(R)
        hist_F, hist_R = hist_F[-diis:], hist_R[-diis:]
        if len(hist_F) > 1:
            c = _diis_coefficients(gf2_gram(h, hist_R))
            F_next = torch.empty_like(run.F)
            gf2_combine(h, list(c), hist_F, F_next)
            run.F = F_next
        else:
            run.F = F_out
    raise RuntimeError("inner loop did not converge")


def energy(run):
    s = run.sys
    e1, e2 = gf2_energy(run.ctx.handle, s.h, run.F, run.P, s.S, run.G_iw, run.Sigma_iw, run.sig12)
    return s.e_nuc + e1 + e2, e1, e2


def self_energy_step(run, damping=1.0):
    """G(i w) -> G(tau) -> Sigma(tau) (optionally damped) -> Sigma(i w)."""
    s = run.sys
    gf2_tail_moments(run.ctx.handle, s.S, run.F, run.mu, run.sig12, run.moments)
    gf2_fft_iw_to_tau(run.ctx.handle, run.G_iw, run.moments, run.G_tau)
    def sigma(out):
        if run.df_order:
            gf2_sigma_tau_df(run.ctx.handle, run.G_tau, 0, s.n_tau, out, run.prec)
        else:
            gf2_sigma_tau(run.ctx.handle, run.G_tau, out, run.prec)

    if damping < 1.0 and run.sig12 is not None:
        new = torch.empty_like(run.Sigma_tau)
        sigma(new)
        gf2_combine(run.ctx.handle, [damping, 1.0 - damping], [new, run.Sigma_tau], run.Sigma_tau)
    else:
        sigma(run.Sigma_tau)
    if run.sig12 is None:
        run.sig12 = torch.empty(2, s.nbf, s.nbf, dtype=torch.float64, device=s.S.device)
    gf2_fft_tau_to_iw(run.ctx.handle, run.Sigma_tau, run.Sigma_iw, run.sig12)


def run_gf2(sys, prec=GF2_PREC_FP64, max_outer=30, e_tol=1e-8, damping=1.0, inner_tol=1e-8, callback=None,
            df_order=False):
    run = start(sys, prec, df_order)
    inner_loop(run, inner_tol)
    run.energies.append(energy(run))
    for _ in range(max_outer):
        self_energy_step(run, damping)
        inner_loop(run, inner_tol)
        run.energies.append(energy(run))
        if callback is not None:
            callback(run)
        if abs(run.energies[-1][0] - run.energies[-2][0]) < e_tol:
            break
    return run


__all__ = ["DeviceSystem", "to_device", "GF2Run", "start", "inner_loop", "energy", "self_energy_step",
           "run_gf2", "GF2_PREC_FP64", "GF2_PREC_BF16X3"]
