"""GPU parity at the largest sizes the library accepts.

N = 128 (the H64 lattice in 6-31G) is the largest basis a context takes: the
Dyson kernel keeps its share of the N(N+1)/2 triangle in registers and the
natural-occupation sweep keeps the N x N matrix in shared memory.  N = 80, 112
and 128 run the three widest register layouts of the Dyson kernel (9, 16 and
17 triangle elements per thread), which the N <= 64 workloads never reach.
Inputs are seeded; the expected values come from ``oracle/``.

The per-frequency matrices are complex symmetric with a positive-definite
imaginary part (omega_n S - Im Sigma, Im Sigma <= 0), the class for which the
unpivoted symmetric sweeps of Eq. GF stay well defined.
"""

import numpy as np
import pytest
import torch

import gf2_inputs as gi
from oracle import dyson as od
from oracle import energy as oe
from oracle import sigma as osg
from oracle import transforms as ot
from oracle.fock import fock as oracle_fock
from oracle.occupations import natural_occupations

pytestmark = pytest.mark.gpu

N_MAX = 128


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


def one_body(n, seed):
    """Seeded S (SPD, eigenvalues in [1, 3]), symmetric F and h, Sigma moments."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1.0, 1.0, size=(n, n))
    S = np.eye(n) + 0.5 * X @ X.T / n
    Y = rng.uniform(-1.0, 1.0, size=(n, n))
    F = 0.25 * (Y + Y.T) - 0.3 * np.eye(n)
    Z = rng.uniform(-1.0, 1.0, size=(n, n))
    h = 0.5 * (Z + Z.T) - np.eye(n)
    s1 = 0.02 * rng.normal(size=(n, n))
    s2 = 0.01 * rng.normal(size=(n, n))
    return S, F, h, s1 + s1.T, s2 + s2.T


def sigma_iw(n, n_iw, seed, scale=0.005):
    """Complex symmetric Sigma(i w_n) with Im Sigma <= 0 elementwise."""
    rng = np.random.default_rng(seed)
    re = rng.normal(size=(n_iw, n, n))
    im = np.abs(rng.normal(size=(n_iw, n, n)))
    x = scale * (re - 1j * im)
    return x + np.swapaxes(x, 1, 2)


@pytest.mark.parametrize("n", [80, 112, N_MAX])
def test_tail_dyson_density_energy_at_largest_bases(g, n):
    beta, n_tau, n_iw, mu = 10.0, 9, 64, -0.05
    S, F, h, sig1, sig2 = one_body(n, seed=500 + n)
    Sig = sigma_iw(n, n_iw, seed=600 + n)
    mom_ref = ot.tail_moments(S, F, mu, sig1, sig2)
    G_ref = od.dyson(mu, S, F, Sig, beta)
    P_ref = od.density(G_ref, mom_ref, beta)
    e1_ref = oe.e_one_body(P_ref, h, F)
    e2_ref = oe.e_two_body(G_ref, Sig, sig1, S, beta)
    with g.Context(n, n_tau, n_iw, beta) as ctx:
        mom = torch.zeros(4, n, n, dtype=torch.float64, device="cuda")
        g.gf2_tail_moments(ctx.handle, dev(S), dev(F), mu, dev(np.stack([sig1, sig2])), mom)
        G = torch.zeros(n_iw, n, n, dtype=torch.complex128, device="cuda")
        g.gf2_dyson(ctx.handle, mu, dev(S), dev(F), dev(Sig), G)
        P = torch.zeros(n, n, dtype=torch.float64, device="cuda")
        g.gf2_density(ctx.handle, G, mom, P)
        e1, e2 = g.gf2_energy(ctx.handle, dev(h), dev(F), dev(P_ref), dev(S), dev(G_ref), dev(Sig),
                              dev(np.stack([sig1, sig2])))
        got_m, got_G, got_P = host(mom), host(G), host(P)
    assert np.abs(got_m - mom_ref).max() <= 1e-11 * np.abs(mom_ref).max()
    assert np.abs(got_G - G_ref).max() <= 1e-11 * np.abs(G_ref).max()
    assert np.abs(got_P - P_ref).max() <= 1e-10 * max(1.0, np.abs(P_ref).max())
    assert abs(e1 - e1_ref) <= 1e-11 * max(1.0, abs(e1_ref))
    assert abs(e2 - e2_ref) <= 1e-11 * max(1.0, abs(e2_ref))


@pytest.mark.parametrize("n", [112, N_MAX])
def test_sigma_fp64_and_fock_at_largest_basis(g, n):
    """One grid point of Eq. Sigma on the FP64 path (and on the 128-wide
    split tensor-core path) and Eq. FockMatrix at N = 128 (two full 64-wide
    GEMM tiles in every stage), and at N = 112 (a 48-wide ragged tile)."""
    n_tau, k = 9, 3
    v = gi.random_eri(n, seed=5) * 0.1
    G = gi.random_symmetric_g(n, n_tau, seed=6)
    ref = osg.sigma_factored(G[k], -G[n_tau - 1 - k], v)
    S, F, h, _, _ = one_body(n, seed=7)
    rng = np.random.default_rng(8)
    A = rng.uniform(-1.0, 1.0, size=(n, n))
    P = 0.1 * (A @ A.T) / n
    F_ref = oracle_fock(h, v, P)
    with g.Context(n, n_tau, 8, 10.0) as ctx:
        g.gf2_set_integrals(ctx.handle, dev(v))
        out = torch.zeros(1, n, n, dtype=torch.float64, device="cuda")
        g.gf2_sigma_tau_points(ctx.handle, dev(G), k, 1, out, g.GF2_PREC_FP64)
        Fd = torch.zeros(n, n, dtype=torch.float64, device="cuda")
        g.gf2_fock(ctx.handle, dev(h), dev(P), Fd)
        got, got_F = host(out)[0], host(Fd)
        # the 128-wide tensor-core pipeline on the same point and context
        out_tc = torch.zeros_like(out)
        g.gf2_sigma_tau_points(ctx.handle, dev(G), k, 1, out_tc, g.GF2_PREC_BF16X6)
        got_tc = host(out_tc)[0]
        # the FP64 path again after the split one: the context's state is intact
        out2 = torch.zeros_like(out)
        g.gf2_sigma_tau_points(ctx.handle, dev(G), k, 1, out2, g.GF2_PREC_FP64)
        again = host(out2)[0]
    assert np.abs(again - got).max() <= 1e-13 * np.abs(got).max()
    assert np.abs(got_tc - ref).max() <= 4e-6 * np.abs(ref).max()
    # FP64 sums of up to N^3 = 2.1e6 products per entry in another order than numpy's
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
    assert np.abs(got_F - F_ref).max() <= 1e-12 * max(1.0, np.abs(F_ref).max())


def test_natural_occupations_at_largest_basis(g):
    n = N_MAX
    S, _, _, _, _ = one_body(n, seed=9)
    rng = np.random.default_rng(10)
    # a density with occupations spread over (0, 2): P = C diag(2f) C^T, C^T S C = 1
    w, U = np.linalg.eigh(S)
    C = U @ np.diag(w ** -0.5) @ np.linalg.qr(rng.normal(size=(n, n)))[0]
    f = np.sort(rng.uniform(0.0, 1.0, size=n))[::-1]
    P = C @ np.diag(2.0 * f) @ C.T
    with g.Context(n, 9, 8, 10.0) as ctx:
        g.gf2_set_overlap(ctx.handle, dev(S))
        occ = torch.empty(n, dtype=torch.float64, device="cuda")
        g.gf2_natural_occupations(ctx.handle, dev(P), occ)
        got = host(occ)
    assert np.abs(got - natural_occupations(P, S)).max() < 1e-10
    assert np.abs(got - f).max() < 1e-10
