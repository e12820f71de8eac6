"""The allocation-free energy entry point against the context-based one.

gf2_energy_noalloc serves callers that must not allocate device memory (for
example code running under CUDA graph capture, or a host that hands the
library a fixed memory budget): it has no context and keeps its scratch in a
fixed device array.  Here it is called twice in a row through the C-ABI and
must reproduce gf2_energy on the same inputs each time.  This file is named so
that pytest collects it last.
"""

import ctypes
import os

import numpy as np
import pytest
import torch

import gf2_inputs as gi
from oracle import dyson as od
from oracle import transforms as ot

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _inputs(n_atoms, beta, n_iw, seed):
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
    return s, r, G, sig, sig12, P


def test_noalloc_energy_matches_context_energy_on_two_calls():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1405_3273_gb300 as g
    from paper_1405_3273_gb300 import build
    if not os.path.exists(g.LIB_PATH):
        build.build()
    cases = [_inputs(4, 50.0, 512, 1), _inputs(6, 80.0, 1000, 2)]
    for s, r, G, sig, sig12, P in cases:
        args = [_dev(x) for x in (s.h, r.F, P, s.S, G, sig, sig12)]
        with g.Context(s.nbf, 17, G.shape[0], s.beta) as ctx:
            e1_ref, e2_ref = g.gf2_energy(ctx.handle, *args)
        for _ in range(2):
            e1, e2 = g.gf2_energy_noalloc(s.nbf, G.shape[0], s.beta, *args)
            assert abs(e1 - e1_ref) <= 1e-12 * max(1.0, abs(e1_ref))
            assert abs(e2 - e2_ref) <= 1e-12 * max(1.0, abs(e2_ref))


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
