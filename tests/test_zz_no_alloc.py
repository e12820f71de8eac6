"""The allocation-free energy entry point against the context-based one.

gf2_energy_noalloc serves callers that cannot allocate device memory -- a host
that gives the library a fixed memory budget and forbids the device allocator,
or code that must not meet an out-of-memory failure in the middle of a run: it
has no context and keeps its scratch in a fixed device array.  Here it is
called twice in a row through the C-ABI and must reproduce gf2_energy (and the
oracle's energy) on the same inputs each time, including the largest sizes its
scratch accepts (N = 128, which needs the largest shared-memory S^-1 sweep, and
n_iw = 65536, which fills the whole partial-sum region), without changing the
device's free memory.  This file is named so that pytest collects it last.
"""

import ctypes
import os

import numpy as np
import pytest
import torch

import gf2_inputs as gi
from oracle import dyson as od
from oracle import energy as oe
from oracle import transforms as ot

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _chain_inputs(n_atoms, beta, n_iw, seed):
    s = gi.build_system("chain", coords=gi.h_chain(n_atoms, 1.7), basis="sto-3g", beta=beta, n_tau=17, n_iw=n_iw)
    r = gi.rhf(s)
    rng = np.random.default_rng(seed)
    sig = 0.02 * (rng.normal(size=(n_iw, s.nbf, s.nbf)) - 1j * np.abs(rng.normal(size=(n_iw, s.nbf, s.nbf))))
    sig = sig + np.swapaxes(sig, 1, 2)
    mu = 0.5 * (r.eps[n_atoms // 2 - 1] + r.eps[n_atoms // 2])
    G = od.dyson(mu, s.S, r.F, sig, beta)
    sig1 = 0.01 * rng.normal(size=(s.nbf, s.nbf))
    sig12 = np.stack([sig1 + sig1.T, np.zeros((s.nbf, s.nbf))])
    P = od.density(G, ot.tail_moments(s.S, r.F, mu), beta)
    return s.nbf, beta, s.h, r.F, P, s.S, G, sig, sig12


def _random_inputs(n, beta, n_iw, seed):
    """A random well-conditioned system of n basis functions (S = 1 + small
    symmetric part), its Green's function from Eq. GF with a random Sigma."""
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(n, n)) / np.sqrt(n)
    S = np.eye(n) + 0.1 * (a + a.T)
    h = rng.normal(size=(n, n))
    h = 0.5 * (h + h.T) - 2.0 * np.eye(n)
    F = h + 0.1 * np.eye(n)
    sig = 0.01 * (rng.normal(size=(n_iw, n, n)) - 1j * np.abs(rng.normal(size=(n_iw, n, n))))
    sig = sig + np.swapaxes(sig, 1, 2)
    G = od.dyson(0.0, S, F, sig, beta)
    b = rng.normal(size=(n, n))
    P = 0.1 * (b + b.T)
    sig1 = 0.01 * rng.normal(size=(n, n))
    sig12 = np.stack([sig1 + sig1.T, np.zeros((n, n))])
    return n, beta, h, F, P, S, G, sig, sig12


CASES = {
    "h4_512": lambda: _chain_inputs(4, 50.0, 512, 1),
    "h6_1000": lambda: _chain_inputs(6, 80.0, 1000, 2),
    "n128_max_basis": lambda: _random_inputs(128, 20.0, 48, 3),
    "n4_iw65536_max_frequencies": lambda: _random_inputs(4, 200.0, 65536, 4),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_noalloc_energy_matches_context_energy_on_two_calls(name):
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1405_3273_gb300 as g
    from paper_1405_3273_gb300 import build
    if not os.path.exists(g.LIB_PATH):
        build.build()
    n, beta, h, F, P, S, G, sig, sig12 = CASES[name]()
    n_iw = G.shape[0]
    e1_or = oe.e_one_body(P, h, F)
    e2_or = oe.e_two_body(G, sig, sig12[0], S, beta)
    args = [_dev(x) for x in (h, F, P, S, G, sig, sig12)]
    with g.Context(n, 17, n_iw, beta) as ctx:
        e1_ref, e2_ref = g.gf2_energy(ctx.handle, *args)
    assert abs(e1_ref - e1_or) <= 1e-11 * max(1.0, abs(e1_or))
    assert abs(e2_ref - e2_or) <= 1e-11 * max(1.0, abs(e2_or))
    g.gf2_energy_noalloc(n, n_iw, beta, *args)  # first call on the device: address look-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(2):
        e1, e2 = g.gf2_energy_noalloc(n, n_iw, beta, *args)
        # the same result as the context path, to rounding (S^-1 is computed differently)
        assert abs(e1 - e1_ref) <= 1e-12 * max(1.0, abs(e1_ref))
        assert abs(e2 - e2_ref) <= 1e-11 * max(1.0, abs(e2_ref))
        assert abs(e2 - e2_or) <= 1e-11 * max(1.0, abs(e2_or))
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0


def test_noalloc_energy_rejects_sizes_beyond_its_scratch():
    import paper_1405_3273_gb300 as g
    L = g.lib()
    f = L.gf2_energy_noalloc
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(x.data_ptr())
    e1, e2 = ctypes.c_double(), ctypes.c_double()
    # n_iw above 65536 and N above 128 are refused before any launch (GF2_ERR_UNSUPPORTED = 7)
    assert f(2, 65537, 10.0, p, p, p, p, p, p, None, ctypes.byref(e1), ctypes.byref(e2), None) == 7
    assert f(129, 8, 10.0, p, p, p, p, p, p, None, ctypes.byref(e1), ctypes.byref(e2), None) == 7
    assert f(2, 8, 10.0, None, p, p, p, p, p, None, ctypes.byref(e1), ctypes.byref(e2), None) == 1
