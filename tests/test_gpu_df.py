"""Eq. Sigma on density-fitted integrals on the GPU (gf2_set_df_integrals,
gf2_sigma_tau_df) against the oracle's density-fitted Sigma (oracle/df.py).

* the factor-order Sigma and the four-stage Sigma on the fitted integrals,
  random factors, N = 5 .. 70 (ragged 64-wide GEMM tiles) and m = 1 .. 192;
* N = 64 with m = 192 over 129 grid points: three chunks of the workspace,
  the last ragged, checked at every chunk boundary; N = 128 with m = 384;
* a context on the power mesh (the mirrored G(-tau) of a non-equidistant grid);
* the H32 lattice (6-31G, N = 64) with the even-tempered auxiliary set
  (m = 192) and a physical G(tau); the split-precision four-stage path on the
  same fitted integrals;
* GF2 on the H4 chain with fitted integrals, every outer iteration, against
  the oracle run on the same fitted integrals;
* argument errors.
"""

import dataclasses

import numpy as np
import pytest
import torch

import gf2_inputs as gi
from gf2_inputs import density_fitting as dfi
from oracle import df as odf
from oracle import gf2 as og
from oracle import sigma as osg
from tests import closed_forms as cf

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


def _factor(m, n, seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((m, n, n)) / np.sqrt(m * n)
    return 0.5 * (B + np.swapaxes(B, 1, 2))


def _run(g, n, n_tau, B, G, ranges, prec=0, beta=10.0, exact_too=False):
    out, exact = [], None
    with g.Context(n, n_tau, 8, beta) as ctx:
        g.gf2_set_df_integrals(ctx.handle, dev(B))
        Gd = dev(G)
        for k0, cnt in ranges:
            o = torch.full((max(cnt, 1), n, n), 7.0, dtype=torch.float64, device="cuda")
            g.gf2_sigma_tau_df(ctx.handle, Gd, k0, cnt, o, prec)
            out.append(host(o))
        if exact_too:
            o = torch.zeros(n_tau, n, n, dtype=torch.float64, device="cuda")
            g.gf2_sigma_tau(ctx.handle, Gd, o, 0)
            exact = host(o)
    return out, exact


@pytest.mark.parametrize("n,m,n_tau", [(5, 1, 9), (10, 7, 17), (33, 50, 9), (64, 192, 9), (70, 100, 9)])
def test_factor_order_sigma_matches_oracle(g, n, m, n_tau):
    G = gi.random_symmetric_g(n, n_tau, seed=300 + n)
    B = _factor(m, n, 400 + m)
    ref = odf.sigma_tau_df(G, B)
    (got,), exact = _run(g, n, n_tau, B, G, [(0, n_tau)], exact_too=True)
    scale = np.abs(ref).max()
    print(f"N={n} m={m}: factor order rel {np.abs(got - ref).max() / scale:.2e}, "
          f"four stages rel {np.abs(exact - ref).max() / scale:.2e}")
    assert np.abs(got - ref).max() <= 1e-12 * scale
    assert np.abs(exact - ref).max() <= 1e-12 * scale


def test_ragged_ranges_and_chunk_boundaries(g):
    """N = 64, m = 192: 1 GB of workspace holds 56 time points, so 129 points
    run as chunks of 56, 56 and 17; sub-ranges start anywhere; count 0 leaves
    the output untouched."""
    n, m, n_tau = 64, 192, 129
    G = gi.random_symmetric_g(n, n_tau, seed=64)
    B = _factor(m, n, 65)
    ranges = [(0, n_tau), (55, 3), (127, 2), (3, 0)]
    outs, _ = _run(g, n, n_tau, B, G, ranges)
    v = odf.df_eri(B)
    W = osg.exchange_combination(v)
    ref = {k: osg.sigma_factored(G[k], osg.gbar_from_grid(G, k), v, W) for k in (0, 55, 56, 57, 111, 112, 127, 128)}
    scale = max(np.abs(r).max() for r in ref.values())
    for k in ref:
        assert np.abs(outs[0][k] - ref[k]).max() <= 1e-12 * scale, k
    for j, k in enumerate((55, 56, 57)):
        assert np.abs(outs[1][j] - ref[k]).max() <= 1e-12 * scale
    for j, k in enumerate((127, 128)):
        assert np.abs(outs[2][j] - ref[k]).max() <= 1e-12 * scale
    assert np.all(outs[3] == 7.0)


def test_largest_basis_n128(g):
    n, m, n_tau = 128, 384, 9
    G = gi.random_symmetric_g(n, n_tau, seed=128) * 0.3
    B = _factor(m, n, 129)
    (got,), _ = _run(g, n, n_tau, B, G, [(7, 2)])
    v = odf.df_eri(B)
    W = osg.exchange_combination(v)
    for j, k in enumerate((7, 8)):
        ref = osg.sigma_factored(G[k], osg.gbar_from_grid(G, k), v, W)
        assert np.abs(got[j] - ref).max() <= 1e-12 * np.abs(ref).max(), k


def test_factor_order_on_the_power_mesh(g):
    """A context on the non-equidistant grid: G(-tau_k) = -G(tau_{n_tau-1-k})
    through the mesh's mirror symmetry, every mesh point against the oracle."""
    from oracle import grids
    M, idx = grids.power_mesh(4, 8)
    n, m = 12, 30
    n_tau = len(idx)
    G = gi.random_symmetric_g(n, n_tau, seed=12)
    B = _factor(m, n, 13)
    ref = odf.sigma_tau_df(G, B)
    with g.Context(n, None, 64, 20.0, grid=(M, idx)) as ctx:
        g.gf2_set_df_integrals(ctx.handle, dev(B))
        o = torch.zeros(n_tau, n, n, dtype=torch.float64, device="cuda")
        g.gf2_sigma_tau_df(ctx.handle, dev(G), 0, n_tau, o, 0)
        got = host(o)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_h32_lattice_with_the_even_tempered_fit(g):
    """H32 2x4x4 lattice, 6-31G (N = 64), six s exponents per atom (m = 192),
    HF G(tau) at beta = 100 on 65 points: the factor order and the split
    four-stage path on the fitted integrals against the oracle."""
    s = gi.build_system("h32_lattice_631g")
    r = gi.rhf(s)
    B = dfi.build_df(s.coords, s.basis)
    n, beta, n_tau = s.nbf, 100.0, 65
    assert B.shape == (192, 64, 64)
    mu = 0.5 * (r.eps[s.n_elec // 2 - 1] + r.eps[s.n_elec // 2])
    _, C, xi, _ = cf.mo_basis(r.F, s.S, mu, beta)
    G = cf.g_tau_ao(C, xi, beta, np.linspace(0.0, beta, n_tau))
    pts = (0, 1, 32, 64)
    v = odf.df_eri(B)
    W = osg.exchange_combination(v)
    ref = {k: osg.sigma_factored(G[k], osg.gbar_from_grid(G, k), v, W) for k in pts}
    exact = osg.sigma_factored(G[32], osg.gbar_from_grid(G, 32), s.eri)
    print(f"fit error of Sigma(beta/2): {np.abs(ref[32] - exact).max() / np.abs(exact).max():.2e} relative")
    with g.Context(n, n_tau, 8, beta) as ctx:
        g.gf2_set_df_integrals(ctx.handle, dev(B))
        g.gf2_set_overlap(ctx.handle, dev(s.S))
        Gd = dev(G)
        got = {}
        for prec in (0, 2, 3):
            o = torch.zeros(len(pts), n, n, dtype=torch.float64, device="cuda")
            for j, k in enumerate(pts):
                if prec == 0:
                    g.gf2_sigma_tau_df(ctx.handle, Gd, k, 1, o[j:j + 1], 0)
                else:
                    g.gf2_sigma_tau_points(ctx.handle, Gd, k, 1, o[j:j + 1], prec)
            got[prec] = host(o)
    for prec, rtol in ((0, 1e-12), (2, 5e-6), (3, 5e-6)):
        for j, k in enumerate(pts):
            rel = np.abs(got[prec][j] - ref[k]).max() / np.abs(ref[k]).max()
            print(f"H32 fitted prec={prec} tau index {k}: rel {rel:.2e}")
            assert rel <= rtol, (prec, k)


def test_gf2_on_fitted_integrals_matches_oracle(g):
    """H4 chain, 6-31G (N = 8), m = 24: two outer iterations with the factor-
    order Sigma inside the driver's loop against the oracle's GF2 on the same
    fitted integrals."""
    from paper_1405_3273_gb300 import driver
    coords = gi.h_chain(4, 1.7)
    s = gi.build_system("chain", coords=coords, basis="6-31g", beta=50.0, n_tau=257, n_iw=1024)
    B = dfi.build_df(coords, "6-31g")
    s_df = dataclasses.replace(s, eri=odf.df_eri(B))
    r = gi.rhf(s_df)
    ref = og.run(s_df, r.F, 50.0, 257, 1024, max_outer=2, e_tol=0.0)
    mu0 = 0.5 * (r.eps[s.n_elec // 2 - 1] + r.eps[s.n_elec // 2])
    ds = driver.to_device(s, r.F, mu0, df_B=B)
    run = driver.run_gf2(ds, max_outer=2, e_tol=0.0, df_order=True)
    e_ref = np.array([e[0] for e in ref.energies])
    e_got = np.array([e[0] for e in run.energies])
    print(f"fitted GF2: |dE| per iteration {np.abs(e_ref - e_got)}")
    assert len(e_ref) == len(e_got) == 3
    # both mu searches stop anywhere inside the 1e-10-electron window; on this
    # system that moves E by up to ~7e-10 Eh (measured), within the 1e-8 Eh FP64 bound
    assert np.abs(e_ref - e_got).max() < 2e-9
    assert np.abs(host(run.P) - ref.P).max() < 1e-8
    run.ctx.close()


def test_argument_errors(g):
    n, n_tau = 6, 9
    G = dev(gi.random_symmetric_g(n, n_tau, seed=1))
    out = torch.zeros(n_tau, n, n, dtype=torch.float64, device="cuda")
    with g.Context(n, n_tau, 8, 10.0) as ctx:
        with pytest.raises(g.GF2Error, match="gf2_set_df_integrals"):
            g.gf2_sigma_tau_df(ctx.handle, G, 0, n_tau, out)
        B = dev(_factor(3, n, 2))
        assert g.lib().gf2_set_df_integrals(ctx.handle, g._ptr(B), 0) == 1
        g.gf2_set_df_integrals(ctx.handle, B)
        with pytest.raises(g.GF2Error, match="range"):
            g.gf2_sigma_tau_df(ctx.handle, G, 5, 5, out)
        with pytest.raises(g.GF2Error) as e:
            g.gf2_sigma_tau_df(ctx.handle, G, 0, n_tau, out, g.GF2_PREC_BF16X6)
        assert e.value.status == 7
        g.gf2_sigma_tau_df(ctx.handle, G, 0, n_tau, out)
        g.gf2_set_integrals(ctx.handle, dev(odf.df_eri(host(B))))
        with pytest.raises(g.GF2Error, match="gf2_set_df_integrals"):
            g.gf2_sigma_tau_df(ctx.handle, G, 0, n_tau, out)
