"""Failure detection on the GPU without a fault: a pipeline wait that nothing
satisfies gives up after its time limit, raises the error word, and the kernel
returns; the CUDA context stays usable afterwards."""

import ctypes
import os
import time

import numpy as np
import pytest
import torch

import gf2_inputs as gi
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


def test_bounded_wait_gives_up_and_leaves_the_context_usable(g):
    f = g.lib().gf2_test_wait_timeout
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    st = f(err.data_ptr(), torch.cuda.current_stream().cuda_stream)
    dt = time.perf_counter() - t0
    assert st == 0
    assert int(err.item()) == 1          # the timeout code
    assert 1.5 < dt < 60.0               # the 2 s wall-time limit, not an immediate return
    # the same context still runs the split Sigma pipeline correctly
    n, n_tau = 10, 9
    G = gi.random_symmetric_g(n, n_tau, seed=61)
    v = gi.random_eri(n, seed=62)
    with g.Context(n, n_tau, 8, 10.0) as ctx:
        g.gf2_set_integrals(ctx.handle, torch.as_tensor(v, device="cuda"))
        out = torch.zeros(n_tau, n, n, dtype=torch.float64, device="cuda")
        g.gf2_sigma_tau(ctx.handle, torch.as_tensor(G, device="cuda"), out, g.GF2_PREC_FP16X3)
        got = out.cpu().numpy()
    ref = osg.sigma_tau(G, v)
    assert np.abs(got - ref).max() <= 3e-6 * np.abs(ref).max()


def test_timeout_hook_rejects_a_null_error_word(g):
    f = g.lib().gf2_test_wait_timeout
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    assert f(None, None) == 1
