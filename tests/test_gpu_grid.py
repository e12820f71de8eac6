"""The non-equidistant time grid (gf2_create_grid, the uniform power mesh) on
the GPU against the oracle.

* both transforms on random data, element by element, with n_iw below and
  above the uniform grid's M (frequencies folded modulo M), and Sig1/Sig2;
* a context built with the grid 0..M agrees with the uniform context;
* GF2 on the H4 chain on a 193-point mesh, every outer iteration, FP64 and a
  split precision, against the oracle run on the same mesh.
"""

import numpy as np
import pytest
import torch

import gf2_inputs as gi
from oracle import gf2 as og
from oracle import grids
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


def _sym(a):
    return 0.5 * (a + np.swapaxes(a, -1, -2))


@pytest.mark.parametrize("p,u,n_iw", [(4, 8, 200), (4, 8, 700), (6, 4, 300)])
def test_grid_transforms_match_oracle(g, p, u, n_iw):
    M, idx = grids.power_mesh(p, u)
    n, beta = 5, 30.0
    rng = np.random.default_rng(p * 100 + n_iw)
    X_iw = _sym(rng.standard_normal((n_iw, n, n)) + 1j * rng.standard_normal((n_iw, n, n)))
    X_iw /= (1.0 + np.arange(n_iw))[:, None, None]
    mom = _sym(rng.standard_normal((4, n, n)))
    X_tau = _sym(rng.standard_normal((len(idx), n, n)))
    ref_tau = ot.iw_to_tau(X_iw, mom, beta, M + 1, taus=idx)
    ref_iw = ot.tau_to_iw_grid(X_tau, beta, M, idx, n_iw)
    ref_s1, ref_s2 = ot.sigma_expansion_grid(X_tau, beta, M, idx)
    with g.Context(n, None, n_iw, beta, grid=(M, idx)) as ctx:
        assert ctx.n_tau == len(idx)
        out_tau = torch.empty(len(idx), n, n, dtype=torch.float64, device="cuda")
        g.gf2_fft_iw_to_tau(ctx.handle, dev(X_iw), dev(mom), out_tau)
        out_iw = torch.empty(n_iw, n, n, dtype=torch.complex128, device="cuda")
        sig12 = torch.empty(2, n, n, dtype=torch.float64, device="cuda")
        g.gf2_fft_tau_to_iw(ctx.handle, dev(X_tau), out_iw, sig12)
        got_tau, got_iw, got_s = host(out_tau), host(out_iw), host(sig12)
    assert np.abs(got_tau - ref_tau).max() <= 1e-12 * np.abs(ref_tau).max()
    assert np.abs(got_iw - ref_iw).max() <= 1e-12 * np.abs(ref_iw).max()
    assert np.abs(got_s[0] - ref_s1).max() <= 1e-13 * np.abs(ref_s1).max()
    assert np.abs(got_s[1] - ref_s2).max() <= 1e-12 * np.abs(ref_s2).max()


def test_full_index_grid_agrees_with_the_uniform_context(g):
    n, beta, M, n_iw = 4, 20.0, 64, 150
    rng = np.random.default_rng(3)
    X_tau = _sym(rng.standard_normal((M + 1, n, n)))
    outs = []
    for grid in (None, (M, np.arange(M + 1))):
        with g.Context(n, M + 1, n_iw, beta, grid=grid) as ctx:
            o = torch.empty(n_iw, n, n, dtype=torch.complex128, device="cuda")
            s = torch.empty(2, n, n, dtype=torch.float64, device="cuda")
            g.gf2_fft_tau_to_iw(ctx.handle, dev(X_tau), o, s)
            outs.append((host(o), host(s)))
    assert np.abs(outs[0][0] - outs[1][0]).max() <= 1e-12 * np.abs(outs[0][0]).max()
    assert np.abs(outs[0][1] - outs[1][1]).max() <= 1e-11 * np.abs(outs[0][1]).max()


@pytest.mark.parametrize("prec,tol_e", [(0, 1e-9), (2, 1e-7)])
def test_gf2_on_the_power_mesh_matches_oracle(g, prec, tol_e):
    from paper_1405_3273_gb300 import driver
    s = gi.build_system("chain", coords=gi.h_chain(4, 1.7), basis="sto-3g", beta=50.0, n_tau=257, n_iw=2048)
    r = gi.rhf(s)
    M, idx = grids.power_mesh(5, 16)
    ref = og.run(s, r.F, 50.0, None, 2048, max_outer=2, e_tol=0.0, grid=(M, idx))
    mu0 = 0.5 * (r.eps[s.n_elec // 2 - 1] + r.eps[s.n_elec // 2])
    ds = driver.to_device(s, r.F, mu0, grid=(M, idx))
    run = driver.run_gf2(ds, prec=prec, max_outer=2, e_tol=0.0)
    e_ref = np.array([e[0] for e in ref.energies])
    e_got = np.array([e[0] for e in run.energies])
    print(f"mesh GF2 prec {prec}: |dE| per iteration {np.abs(e_ref - e_got)}")
    assert len(e_ref) == len(e_got)
    assert np.abs(e_ref - e_got).max() < tol_e
    assert np.abs(host(run.P) - ref.P).max() < 100 * tol_e
    run.ctx.close()
