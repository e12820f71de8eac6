"""GPU checks of the tensor-core (tcgen05) split-precision Sigma path.

Layout check: one 128x64x64 BF16 tile through TMA + tcgen05.mma + tcgen05.ld
against the exact product of the same BF16 values.  Parity: split Sigma(tau)
against the oracle's FP64 Eq. Sigma (sampled points at N = 64, the full grid
at small N through the padded path), and full GF2 energies with the split
Sigma against the oracle.  Tolerances follow from the split arithmetic:
two BF16 terms (three products) keep ~16 significant bits per operand, three
terms (six products) ~24 bits, two FP16 terms ~22 bits (three FP16 terms are
then limited by the FP32 sums), and FP32 accumulation adds ~2^-24 per sum.
Precision codes: 1 BF16x3, 2 BF16x6, 3 FP16x3, 4 FP16x6.
"""

import ctypes
import os

import numpy as np
import pytest
import torch

import gf2_inputs as gi
from oracle import gf2 as og
from oracle import sigma as osg

pytestmark = pytest.mark.gpu


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


def bf16_round(x):
    return torch.as_tensor(x, dtype=torch.float32).to(torch.bfloat16)


@pytest.mark.parametrize("mn_major", [0, 1, 2])
def test_single_tile_operand_layouts(g, mn_major):
    """K-major and MN-major A from shared memory, and A resident in TMEM (mode 2)."""
    rng = np.random.default_rng(42 + mn_major)
    A = bf16_round(rng.normal(size=(128, 64)))   # M x K
    B = bf16_round(rng.normal(size=(64, 64)))    # N x K
    ref = A.double() @ B.double().T
    a_dev = (A.T.contiguous() if mn_major == 1 else A.contiguous()).cuda()
    b_dev = B.contiguous().cuda()
    D = torch.zeros(128, 64, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    L = g.lib()
    f = L.gf2_test_umma_tile
    f.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    st = f(mn_major, a_dev.data_ptr(), b_dev.data_ptr(), D.data_ptr(), err.data_ptr(),
           torch.cuda.current_stream().cuda_stream)
    assert st == 0
    assert int(err.item()) == 0
    got = D.double().cpu()
    assert (got - ref).abs().max().item() < 1e-4 * ref.abs().max().item()


def _split_sigma(g, G, v, prec, k0=0, count=None):
    n_tau, n = G.shape[0], G.shape[1]
    count = n_tau if count is None else count
    with g.Context(n, n_tau, 8, 10.0) as ctx:
        g.gf2_set_integrals(ctx.handle, dev(v))
        out = torch.zeros(count, n, n, dtype=torch.float64, device="cuda")
        g.gf2_sigma_tau_points(ctx.handle, dev(G), k0, count, out, prec)
        torch.cuda.synchronize()
        return out.cpu().numpy()


@pytest.mark.parametrize("prec,rtol", [(1, 3e-4), (2, 3e-6), (3, 3e-6), (4, 3e-6)])
def test_split_sigma_padded_small_basis_full_grid(g, prec, rtol):
    """N = 10 (padded to 64 inside), 9 time points, random symmetric G and 8-fold symmetric v."""
    n, n_tau = 10, 9
    G = gi.random_symmetric_g(n, n_tau, seed=31)
    v = gi.random_eri(n, seed=32)
    ref = osg.sigma_tau(G, v)
    got = _split_sigma(g, G, v, prec)
    assert np.abs(got - ref).max() <= rtol * np.abs(ref).max()


@pytest.mark.parametrize("prec,rtol", [(1, 3e-4), (2, 5e-5), (3, 5e-5), (4, 5e-5)])
def test_split_sigma_n64_sampled_points(g, prec, rtol):
    """N = 64 (no padding), 17 time points: an odd count exercises the half-empty last pair;
    the oracle evaluates three of them one by one."""
    s = gi.build_system("h32_lattice_631g_small", coords=gi.h_lattice(2, 4, 4, 2.0), basis="6-31g",
                        beta=100.0, n_tau=17, n_iw=32)
    n, n_tau = s.nbf, 17
    assert n == 64
    G = gi.random_symmetric_g(n, n_tau, seed=33) * 0.3
    got = _split_sigma(g, G, s.eri, prec)
    W = osg.exchange_combination(s.eri)
    for k in (0, 7, 16):
        ref = osg.sigma_factored(G[k], -G[n_tau - 1 - k], s.eri, W)
        rel = np.abs(got[k] - ref).max() / np.abs(ref).max()
        print(f"split Sigma N=64 prec={prec} tau index {k}: max rel error {rel:.3e}")
        assert rel <= rtol, k


@pytest.mark.parametrize("prec,rtol", [(2, 3e-6), (3, 3e-6)])
def test_split_sigma_without_pair_symmetry(g, prec, rtol):
    """Integrals that lack the pair symmetry (im|qk) = (qk|im) make the library
    compute every tile of the stage-2 intermediate (the symmetric run computes
    half and mirrors them, which would be wrong here).  Sigma is then not
    symmetric either, and the library returns its symmetric part."""
    n, n_tau = 64, 9
    G = gi.random_symmetric_g(n, n_tau, seed=41) * 0.3
    rng = np.random.default_rng(42)
    v = gi.random_eri(n, seed=43) + 0.05 * rng.normal(size=(n, n, n, n))
    ref = osg.sigma_tau(G, v)
    ref = 0.5 * (ref + np.swapaxes(ref, 1, 2))
    got = _split_sigma(g, G, v, prec)
    rel = np.abs(got - ref).max() / np.abs(ref).max()
    print(f"split Sigma without pair symmetry, prec={prec}: max rel error {rel:.3e}")
    assert rel <= rtol


@pytest.fixture(scope="module")
def n64_every_point_case():
    n, n_tau, count = 64, 65, 37
    G = gi.random_symmetric_g(n, n_tau, seed=36)
    v = gi.random_eri(n, seed=37)
    return G, v, count, osg.sigma_tau(G, v, taus=range(count))


@pytest.mark.parametrize("prec,rtol", [(2, 3e-6), (1, 5e-5), (3, 3e-6), (4, 3e-6)])
def test_split_sigma_n64_every_point_full_chunk_and_ragged_tail(g, n64_every_point_case, prec, rtol):
    """N = 64 with random symmetric G and v on a 65-point grid, the first 37 points
    in one call: one full chunk of 32 and a last chunk of 5 (padded to three pairs),
    every point against the oracle.  Each pipeline stage of the three kernels cycles
    hundreds of times per CTA in the full chunk, so a stale or early-overwritten
    buffer shows up as a bad point."""
    G, v, count, ref = n64_every_point_case
    got = _split_sigma(g, G, v, prec, count=count)
    rel = np.abs(got - ref).max(axis=(1, 2)) / np.abs(ref).max()
    print(f"split Sigma N=64 prec={prec}: worst point {int(rel.argmax())} at {rel.max():.2e}")
    assert rel.max() <= rtol


@pytest.mark.parametrize("n,n_tau,prec,rtol", [(16, 33, 3, 3e-6), (21, 17, 3, 3e-6), (32, 17, 3, 3e-6),
                                               (32, 17, 1, 3e-4), (13, 65, 2, 3e-6)])
def test_split_sigma_packed_time_points(g, n, n_tau, prec, rtol):
    """N <= 32: floor(64/N) time points share one tile as diagonal blocks (4, 3, 2, 2
    and 4 here); every point against the oracle, including partly filled slots."""
    G = gi.random_symmetric_g(n, n_tau, seed=40 + n)
    v = gi.random_eri(n, seed=50 + n)
    ref = osg.sigma_tau(G, v)
    got = _split_sigma(g, G, v, prec)
    rel = np.abs(got - ref).max(axis=(1, 2)) / np.abs(ref).max()
    print(f"packed N={n} n_tau={n_tau} prec={prec}: worst point {int(rel.argmax())} at {rel.max():.2e}")
    assert rel.max() <= rtol


def test_split_sigma_points_offset_matches_full_grid(g):
    n, n_tau = 12, 17
    G = gi.random_symmetric_g(n, n_tau, seed=34)
    v = gi.random_eri(n, seed=35)
    full = _split_sigma(g, G, v, 1)
    part = _split_sigma(g, G, v, 1, k0=5, count=7)
    assert np.array_equal(full[5:12], part)


@pytest.mark.parametrize("prec,e_tol,p_tol", [(2, 1e-6, 1e-6), (1, 1e-6, 1e-6), (3, 1e-6, 1e-6)])
def test_split_gf2_energy_h10(g, prec, e_tol, p_tol):
    """Linear H10 (STO-3G, 1.8 bohr), beta = 100, 1025 time points, three GF2 iterations
    with the tensor-core Sigma (orthonormal basis) against the FP64 oracle: every energy
    within 1e-6 Eh and the density within 1e-6 (measured: BF16x6 ~3e-8, BF16x3 ~3e-7)."""
    from paper_1405_3273_gb300 import driver
    s = gi.build_system("h10_chain_sto3g", n_tau=1025, n_iw=2048)
    r = gi.rhf(s)
    ref = og.run(s, r.F, 100.0, 1025, 2048, max_outer=3, e_tol=0.0)
    mu0 = 0.5 * (r.eps[4] + r.eps[5])
    ds = driver.to_device(s, r.F, mu0)
    got = driver.run_gf2(ds, prec=prec, max_outer=3, e_tol=0.0)
    e_ref = np.array([e[0] for e in ref.energies])
    e_got = np.array([e[0] for e in got.energies])
    dp = np.abs(got.P.cpu().numpy() - ref.P).max()
    print(f"H10 split prec={prec}: |dE| per iteration {np.abs(e_ref - e_got).tolist()}, max|dP| {dp:.3e}")
    assert np.abs(e_ref - e_got).max() < e_tol
    assert dp < p_tol


@pytest.mark.parametrize("prec,rtol", [(2, 5e-6), (3, 5e-6), (1, 1e-4)])
def test_split_sigma_physical_g_packed_sto3g_lattice(g, prec, rtol):
    """H32 2x4x4 STO-3G lattice at 3.0 bohr (N = 32: two time points per tile) with the
    overlap given (Loewdin basis): the HF Green's function at the first grid points and
    at the middle of the grid, every point against the oracle."""
    from tests import closed_forms as cf
    s = gi.build_system("h32_lattice_sto3g", spacing=3.0)
    r = gi.rhf(s)
    beta, n_tau = 100.0, 4097
    M = n_tau - 1
    mu = 0.5 * (r.eps[15] + r.eps[16])
    _, C, xi, f = cf.mo_basis(r.F, s.S, mu, beta)
    taus = np.arange(n_tau) * beta / M
    G = np.zeros((n_tau, s.nbf, s.nbf))
    W = osg.exchange_combination(s.eri)
    with g.Context(s.nbf, n_tau, 8, beta) as ctx:
        g.gf2_set_integrals(ctx.handle, dev(s.eri))
        g.gf2_set_overlap(ctx.handle, dev(s.S))
        for k0 in (1, M // 2 - 2):
            ks = list(range(k0, k0 + 5))
            for k in ks:
                G[k] = cf.g_tau_ao(C, xi, beta, taus[[k]])[0]
                G[M - k] = cf.g_tau_ao(C, xi, beta, taus[[M - k]])[0]
            out = torch.zeros(len(ks), s.nbf, s.nbf, dtype=torch.float64, device="cuda")
            g.gf2_sigma_tau_points(ctx.handle, dev(G), ks[0], len(ks), out, prec)
            got = out.cpu().numpy()
            for j, k in enumerate(ks):
                ref = osg.sigma_factored(G[k], -G[M - k], s.eri, W)
                rel = np.abs(got[j] - ref).max() / np.abs(ref).max()
                print(f"packed STO-3G lattice, prec={prec}, tau index {k}: rel err {rel:.3e}")
                assert rel <= rtol, k


@pytest.mark.parametrize("prec,rtol", [(2, 5e-6), (3, 5e-6), (4, 5e-6)])
def test_split_sigma_physical_g_mid_grid_small_magnitudes(g, prec, rtol):
    """The same lattice at the middle of the grid, where the HF Green's function has
    decayed to ~e^(-beta gap / 2): FP16 operands keep their bits only through the
    per-time-point scales, which the relative error checks."""
    from tests import closed_forms as cf
    s = gi.build_system("h32_lattice_631g")
    r = gi.rhf(s)
    beta, n_tau = 100.0, 4097
    M = n_tau - 1
    mu = 0.5 * (r.eps[15] + r.eps[16])
    _, C, xi, f = cf.mo_basis(r.F, s.S, mu, beta)
    taus = np.arange(n_tau) * beta / M
    ks = [M // 2 - 1, M // 2, M // 2 + 1]
    G = np.zeros((n_tau, s.nbf, s.nbf))
    for k in ks:
        G[k] = cf.g_tau_ao(C, xi, beta, taus[[k]])[0]
        G[M - k] = cf.g_tau_ao(C, xi, beta, taus[[M - k]])[0]
    W = osg.exchange_combination(s.eri)
    with g.Context(s.nbf, n_tau, 8, beta) as ctx:
        g.gf2_set_integrals(ctx.handle, dev(s.eri))
        g.gf2_set_overlap(ctx.handle, dev(s.S))
        out = torch.zeros(len(ks), s.nbf, s.nbf, dtype=torch.float64, device="cuda")
        g.gf2_sigma_tau_points(ctx.handle, dev(G), ks[0], len(ks), out, prec)
        got = out.cpu().numpy()
    for j, k in enumerate(ks):
        ref = osg.sigma_factored(G[k], -G[M - k], s.eri, W)
        rel = np.abs(got[j] - ref).max() / np.abs(ref).max()
        print(f"mid-grid G, N=64, prec={prec}, tau index {k}: max|G|={np.abs(G[k]).max():.2e} "
              f"max|Sigma|={np.abs(ref).max():.2e} rel err {rel:.3e}")
        assert rel <= rtol


@pytest.mark.parametrize("prec,rtol", [(2, 5e-6), (1, 1e-4), (3, 5e-6)])
def test_split_sigma_physical_g_ill_conditioned_overlap(g, prec, rtol):
    """H32 2x4x4 lattice, 6-31G (cond(S) ~ 2e4): the HF Green's function near tau = 0
    has entries ~200 in the AO basis.  With the overlap given to the context the split
    path runs in the orthonormal basis and keeps the FP64 oracle's Sigma to rtol."""
    from tests import closed_forms as cf
    s = gi.build_system("h32_lattice_631g")
    r = gi.rhf(s)
    beta, n_tau = 100.0, 4097
    M = n_tau - 1
    mu = 0.5 * (r.eps[15] + r.eps[16])
    _, C, xi, f = cf.mo_basis(r.F, s.S, mu, beta)
    taus = np.arange(n_tau) * beta / M
    ks = [1, 2, 3]
    G = np.zeros((n_tau, s.nbf, s.nbf))
    for k in ks:
        G[k] = cf.g_tau_ao(C, xi, beta, taus[[k]])[0]
        G[M - k] = cf.g_tau_ao(C, xi, beta, taus[[M - k]])[0]
    W = osg.exchange_combination(s.eri)
    with g.Context(s.nbf, n_tau, 8, beta) as ctx:
        g.gf2_set_integrals(ctx.handle, dev(s.eri))
        g.gf2_set_overlap(ctx.handle, dev(s.S))
        out = torch.zeros(len(ks), s.nbf, s.nbf, dtype=torch.float64, device="cuda")
        g.gf2_sigma_tau_points(ctx.handle, dev(G), ks[0], len(ks), out, prec)
        got = out.cpu().numpy()
    for j, k in enumerate(ks):
        ref = osg.sigma_factored(G[k], -G[M - k], s.eri, W)
        rel = np.abs(got[j] - ref).max() / np.abs(ref).max()
        print(f"physical G, N=64, prec={prec}, tau index {k}: max|G|={np.abs(G[k]).max():.1f} rel err {rel:.3e}")
        assert rel <= rtol
