"""The 128-wide tensor-core Sigma pipeline (64 < N <= 128) against the oracle.

* N = 80 (padded to 128 inside: ragged rows and columns in every tile), all
  four split precisions, every point of a 9-point grid.
* N = 128 (no padding), 17 time points: one full 16-point chunk plus a ragged
  one-point chunk, BF16x6 and FP16x3 against the oracle point by point.
* The H64 4x4x4 lattice in 6-31G (N = 128, the largest workload) with the
  physical finite-temperature HF Green's function in the orthonormal basis,
  the split path against the FP64 GPU path on sampled points near tau = 0 and
  mid-grid (the FP64 path is itself checked against the oracle at N = 128).
* These integrals have the pair symmetry (im|qk) = (qk|im), so the sandwich
  computes the upper triangle of (i, q) tiles and mirrors it; N = 80 with
  integrals that lack it runs every tile.

Tolerances as for N = 64 (``tests/test_gpu_tc.py``): three BF16 terms or two
FP16 terms keep ~22-24 significant bits per operand, two BF16 terms ~16.
"""

import os

import numpy as np
import pytest
import torch

import gf2_inputs as gi
from oracle import sigma as osg

pytestmark = pytest.mark.gpu
RTOL = {1: 6e-5, 2: 4e-6, 3: 4e-6, 4: 4e-6}


@pytest.fixture(scope="module")
def g():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1405_3273_gb300 as g
    from paper_1405_3273_gb300 import build
    if not os.path.exists(g.LIB_PATH):
        build.build()
    g.lib()
    return g


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def split_sigma(g, G, v, precs, S=None):
    n_tau, n = G.shape[0], G.shape[1]
    out = {}
    with g.Context(n, n_tau, 8, 10.0) as ctx:
        g.gf2_set_integrals(ctx.handle, dev(v))
        if S is not None:
            g.gf2_set_overlap(ctx.handle, dev(S))
        Gd = dev(G)
        for prec in precs:
            o = torch.zeros(n_tau, n, n, dtype=torch.float64, device="cuda")
            g.gf2_sigma_tau(ctx.handle, Gd, o, prec)
            torch.cuda.synchronize()
            out[prec] = o.cpu().numpy()
    return out


def test_split_sigma_n80_padded_every_point(g):
    n, n_tau = 80, 9
    G = gi.random_symmetric_g(n, n_tau, seed=81) * 0.3
    v = gi.random_eri(n, seed=82)
    ref = osg.sigma_tau(G, v)
    got = split_sigma(g, G, v, sorted(RTOL))
    for prec, rtol in RTOL.items():
        rel = np.abs(got[prec] - ref).max() / np.abs(ref).max()
        print(f"N=80 split Sigma prec={prec}: max rel error {rel:.3e}")
        assert rel <= rtol, prec


def test_split_sigma_n128_full_chunk_and_ragged_tail(g):
    n, n_tau = 128, 17
    G = gi.random_symmetric_g(n, n_tau, seed=128) * 0.3
    v = gi.random_eri(n, seed=129)
    got = split_sigma(g, G, v, (2, 3))
    W = osg.exchange_combination(v)
    scale = 0.0
    errs = {2: 0.0, 3: 0.0}
    for k in range(n_tau):
        ref = osg.sigma_factored(G[k], -G[n_tau - 1 - k], v, W)
        scale = max(scale, np.abs(ref).max())
        for prec in errs:
            errs[prec] = max(errs[prec], np.abs(got[prec][k] - ref).max())
    for prec, e in errs.items():
        print(f"N=128 split Sigma prec={prec}: max rel error {e / scale:.3e} over {n_tau} points")
        assert e <= RTOL[prec] * scale, prec


def test_split_sigma_h64_lattice_physical_g(g):
    """H64 4x4x4 lattice, 6-31G, beta = 200: finite-temperature HF G(tau) on a
    65-point grid (G(tau) from the analytic single-pole form in the MO basis),
    split Sigma in the orthonormal basis against the FP64 GPU path."""
    from tests import closed_forms as cf
    s = gi.build_system("h64_lattice_631g")
    r = gi.rhf(s)
    n, beta, n_tau = s.nbf, 200.0, 65
    assert n == 128
    mu = 0.5 * (r.eps[s.n_elec // 2 - 1] + r.eps[s.n_elec // 2])
    taus = np.linspace(0.0, beta, n_tau)
    _, C, xi, _ = cf.mo_basis(r.F, s.S, mu, beta)
    G = cf.g_tau_ao(C, xi, beta, taus)
    pts = (0, 1, 32, 63)
    with g.Context(n, n_tau, 8, beta) as ctx:
        g.gf2_set_integrals(ctx.handle, dev(s.eri))
        g.gf2_set_overlap(ctx.handle, dev(s.S))
        Gd = dev(G)
        out = {}
        for prec in (0, 2, 3):
            o = torch.zeros(len(pts), n, n, dtype=torch.float64, device="cuda")
            for j, k in enumerate(pts):
                g.gf2_sigma_tau_points(ctx.handle, Gd, k, 1, o[j:j + 1], prec)
            torch.cuda.synchronize()
            out[prec] = o.cpu().numpy()
    for prec in (2, 3):
        for j, k in enumerate(pts):
            ref = out[0][j]
            rel = np.abs(out[prec][j] - ref).max() / np.abs(ref).max()
            print(f"H64 lattice split Sigma prec={prec} tau index {k}: max rel error {rel:.3e}")
            assert rel <= 5e-6, (prec, k)


def test_split_sigma_n80_without_pair_symmetry(g):
    """Integrals without the pair symmetry (im|qk) = (qk|im): the 128-wide
    sandwich then computes every (i, q) tile instead of the upper triangle and
    its mirror; the symmetric part of Sigma is returned."""
    n, n_tau = 80, 9
    G = gi.random_symmetric_g(n, n_tau, seed=83) * 0.3
    rng = np.random.default_rng(84)
    v = gi.random_eri(n, seed=85) + 0.05 * rng.normal(size=(n, n, n, n))
    ref = osg.sigma_tau(G, v)
    ref = 0.5 * (ref + np.swapaxes(ref, 1, 2))
    got = split_sigma(g, G, v, (2, 3))
    for prec in (2, 3):
        rel = np.abs(got[prec] - ref).max() / np.abs(ref).max()
        print(f"N=80 split Sigma without pair symmetry prec={prec}: max rel error {rel:.3e}")
        assert rel <= RTOL[prec], prec
