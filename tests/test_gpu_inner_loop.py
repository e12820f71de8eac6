"""The device-resident inner loop (gf2_inner_loop: steps 2.a-2.b as one CUDA
graph with the mu search nested in it) against the oracle's inner loop and
against the same steps sequenced call by call from the host.

Both sides take one schedule: damped Fock steps F + mix R while |R| exceeds
diis_from, Pulay (DIIS) steps below.  The loop stops at |R| < 1e-8, so the
converged F, P and mu agree to that level (mu only where the count is not
flat: inside a gap N(mu) barely moves and any mu in it is a root).
"""

import numpy as np
import pytest
import torch

import gf2_inputs as gi
from oracle import gf2 as og
from oracle import transforms as ot

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import os

    import paper_1405_3273_gb300 as g
    from paper_1405_3273_gb300 import build
    if not os.path.exists(g.LIB_PATH):
        build.build()
    g.lib()
    return g


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def _sigma_of_hf(s, F, beta, n_tau, n_iw):
    """A correlated Sigma(i w) (the oracle's second-order Sigma of the HF state)."""
    F1, mu, G, P = og.inner_loop(s, F, None, None, None, beta, n_iw)
    st = og.GF2State(F=F1, mu=mu, P=P, G_iw=G, sig1=np.zeros_like(F1), sig2=np.zeros_like(F1))
    _, Sig_tau = og.self_energy_step(s, st, beta, n_tau, n_iw)
    sig1, sig2 = ot.sigma_expansion(Sig_tau, beta)
    return ot.tau_to_iw(Sig_tau, beta, n_iw), sig1, sig2, mu


def _device_loop(g, ctx, s, F0, mu0, Sig_iw, sig1, sig2, n_iw, **kw):
    n = s.nbf
    F = dev(F0)
    G = torch.zeros(n_iw, n, n, dtype=torch.complex128, device="cuda")
    P = torch.zeros(n, n, dtype=torch.float64, device="cuda")
    sig12 = None if sig1 is None else dev(np.stack([sig1, sig2]))
    Sd = None if Sig_iw is None else dev(Sig_iw)
    mu, nit, nev = g.gf2_inner_loop(ctx.handle, dev(s.S), dev(s.h), F, Sd, sig12, s.n_elec, mu0, G, P, **kw)
    return host(F), mu, host(P), nit, nev


def _check(F, P, Fr, Pr, s):
    assert np.abs(F - Fr).max() < 1e-8
    assert np.abs(P - Pr).max() < 1e-8
    assert abs(np.trace(P @ s.S) - s.n_elec) < 1e-9


@pytest.mark.parametrize("schedule", [dict(), dict(diis=0), dict(diis_from=1e3), dict(diis=3, mix=0.3)])
def test_h4_with_sigma_matches_oracle(g, schedule):
    s = gi.build_system("chain", coords=gi.h_chain(4, 1.7), basis="sto-3g", beta=50.0, n_tau=257, n_iw=512)
    r = gi.rhf(s)
    beta, n_tau, n_iw = 50.0, 257, 512
    Sig_iw, sig1, sig2, mu_hf = _sigma_of_hf(s, r.F, beta, n_tau, n_iw)
    Fr, mur, Gr, Pr = og.inner_loop(s, r.F, Sig_iw, sig1, sig2, beta, n_iw, **schedule)
    with g.Context(s.nbf, n_tau, n_iw, beta) as ctx:
        g.gf2_set_integrals(ctx.handle, dev(s.eri))
        F, mu, P, nit, nev = _device_loop(g, ctx, s, r.F, mu_hf, Sig_iw, sig1, sig2, n_iw, **schedule)
    print(f"H4 {schedule}: {nit} rebuilds, {nev} Dyson evaluations, |dF| {np.abs(F - Fr).max():.2e}")
    _check(F, P, Fr, Pr, s)
    assert nit >= 2 and nev > nit


def test_device_and_host_sequencing_agree(g):
    """The graph and the host-sequenced loop of the driver: same rebuild count
    (within one: the mu searches stop at slightly different points) and the
    same fixed point."""
    from paper_1405_3273_gb300 import driver
    s = gi.build_system("chain", coords=gi.h_chain(6, 1.6), basis="sto-3g", beta=40.0, n_tau=129, n_iw=1024)
    r = gi.rhf(s)
    mu0 = 0.5 * (r.eps[s.n_elec // 2 - 1] + r.eps[s.n_elec // 2])
    out = {}
    for device in (True, False):
        ds = driver.to_device(s, r.F, mu0)
        run = driver.start(ds)
        driver.inner_loop(run, device=device)
        driver.self_energy_step(run)
        n_before = len(run.mu_evals)
        driver.inner_loop(run, device=device)
        out[device] = (host(run.F), host(run.P), run.mu, run.mu_evals[n_before:], run.inner_iters)
        run.ctx.close()
    Fd, Pd, _, _, iters = out[True]
    Fh, Ph, _, _, _ = out[False]
    assert np.abs(Fd - Fh).max() < 1e-8
    assert np.abs(Pd - Ph).max() < 1e-8
    assert len(iters) == 2 and all(i >= 1 for i in iters)


def test_h32_lattice_at_hf_matches_oracle(g):
    """H32 2x4x4 lattice, 6-31G (N = 64), Sigma = 0, beta = 100 on 256
    frequencies: the damped start far from the fixed point, then DIIS."""
    s = gi.build_system("h32_lattice_631g")
    r = gi.rhf(s)
    beta, n_iw = 100.0, 256
    mu0 = 0.5 * (r.eps[s.n_elec // 2 - 1] + r.eps[s.n_elec // 2])
    Fr, mur, Gr, Pr = og.inner_loop(s, r.F, None, None, None, beta, n_iw, tol=1e-8)
    with g.Context(s.nbf, 65, n_iw, beta) as ctx:
        g.gf2_set_integrals(ctx.handle, dev(s.eri))
        F, mu, P, nit, nev = _device_loop(g, ctx, s, r.F, mu0, None, None, None, n_iw)
    print(f"H32: {nit} rebuilds, {nev} Dyson evaluations")
    _check(F, P, Fr, Pr, s)


def test_iteration_cap_reports_and_context_stays_usable(g):
    s = gi.build_system("chain", coords=gi.h_chain(4, 1.7), basis="sto-3g", beta=50.0, n_tau=257, n_iw=512)
    r = gi.rhf(s)
    beta, n_tau, n_iw = 50.0, 257, 512
    Sig_iw, sig1, sig2, mu_hf = _sigma_of_hf(s, r.F, beta, n_tau, n_iw)
    Fr, _, _, Pr = og.inner_loop(s, r.F, Sig_iw, sig1, sig2, beta, n_iw)
    with g.Context(s.nbf, n_tau, n_iw, beta) as ctx:
        g.gf2_set_integrals(ctx.handle, dev(s.eri))
        with pytest.raises(g.GF2Error, match="cap"):
            _device_loop(g, ctx, s, r.F, mu_hf, Sig_iw, sig1, sig2, n_iw, max_iter=1)
        with pytest.raises(g.GF2Error):
            _device_loop(g, ctx, s, r.F, mu_hf, Sig_iw, sig1, sig2, n_iw, diis=9)
        F, mu, P, nit, _ = _device_loop(g, ctx, s, r.F, mu_hf, Sig_iw, sig1, sig2, n_iw)
    _check(F, P, Fr, Pr, s)
