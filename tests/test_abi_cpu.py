"""Host-side checks of the C-ABI library (no GPU needed, no compute calls)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gf2.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:gf2_status|const char \*)\s*(gf2_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def library():
    from paper_1405_3273_gb300 import LIB_PATH, build
    if not os.path.exists(LIB_PATH):
        build.build()
    return ctypes.CDLL(LIB_PATH)


def test_header_declares_the_hot_path_calls():
    names = declared_functions()
    for required in ["gf2_sigma_tau", "gf2_fft_tau_to_iw", "gf2_fft_iw_to_tau", "gf2_dyson",
                     "gf2_mu_search", "gf2_inner_loop", "gf2_fock", "gf2_energy", "gf2_create", "gf2_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(library):
    for name in declared_functions():
        assert hasattr(library, name), name


def test_library_exports_the_test_hooks(library):
    text = open(os.path.join(ROOT, "include", "gf2_testing.h")).read()
    hooks = re.findall(r"^\s*gf2_status\s*(gf2_test_\w+)\s*\(", text, re.M)
    assert sorted(hooks) == ["gf2_test_umma_tile", "gf2_test_wait_timeout"]
    for name in hooks:
        assert hasattr(library, name), name


def test_binding_covers_every_declared_symbol():
    import paper_1405_3273_gb300 as g
    assert sorted(g.exported_symbols()) == declared_functions()
    for name in declared_functions():
        assert callable(getattr(g, name, None)) or name in ("gf2_status_string", "gf2_last_error")


def test_status_strings_without_gpu(library):
    library.gf2_status_string.restype = ctypes.c_char_p
    library.gf2_status_string.argtypes = [ctypes.c_int]
    assert library.gf2_status_string(0) == b"ok"
    assert library.gf2_status_string(1) == b"invalid argument"


def test_create_rejects_bad_sizes_before_touching_the_device(library):
    f = library.gf2_create
    f.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                  ctypes.c_double, ctypes.c_void_p]
    f.restype = ctypes.c_int
    h = ctypes.c_void_p()
    assert f(ctypes.byref(h), 10, 100, 64, 10.0, None) == 1       # M = 99 not a power of two
    assert f(ctypes.byref(h), 0, 129, 64, 10.0, None) == 1        # N = 0
    assert f(ctypes.byref(h), 10, 129, 64, -1.0, None) == 1       # beta < 0
    assert f(None, 10, 129, 64, 10.0, None) == 1                  # NULL out
    assert h.value is None


def test_batch_create_rejects_bad_sizes_before_touching_the_device(library):
    f = library.gf2_batch_create
    f.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                  ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]
    f.restype = ctypes.c_int
    h = ctypes.c_void_p()
    ints = lambda *x: (ctypes.c_int * len(x))(*x)
    assert f(ctypes.byref(h), 0, ints(10), ints(33), None) == 1              # no instances
    assert f(ctypes.byref(h), 1, None, ints(33), None) == 1                  # NULL sizes
    assert f(ctypes.byref(h), 2, ints(10, 0), ints(33, 33), None) == 1       # N = 0 in the second instance
    assert f(None, 1, ints(10), ints(33), None) == 1                         # NULL out
    assert h.value is None
    assert f(ctypes.byref(h), 1, ints(10), ints(100), None) == 1             # M = 99 not a power of two
    assert h.value is None


def test_create_grid_rejects_bad_grids_before_touching_the_device(library):
    f = library.gf2_create_grid
    f.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                  ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_double, ctypes.c_void_p]
    f.restype = ctypes.c_int
    h = ctypes.c_void_p()

    def call(M, idx, n_bf=4, n_iw=64, beta=10.0):
        arr = (ctypes.c_int * len(idx))(*idx) if idx is not None else None
        return f(ctypes.byref(h), n_bf, M, len(idx) if idx is not None else 9, arr, n_iw, beta, None)

    good = [0, 1, 2, 4, 8, 12, 14, 15, 16]
    assert call(16, good[:-1] + [15]) == 1                  # does not end at M
    assert call(16, [1] + good[1:]) == 1                    # does not start at 0
    assert call(16, [0, 1, 2, 4, 8, 13, 14, 15, 16]) == 1   # not symmetric about beta / 2
    assert call(16, [0, 1, 2, 8, 4, 12, 14, 15, 16]) == 1   # not increasing
    assert call(12, [0, 1, 2, 3, 6, 9, 10, 11, 12]) == 1    # M not a power of two
    assert call(16, [0, 2, 8, 14, 16]) == 1                 # fewer than 8 points
    assert call(16, None) == 1                              # NULL index
    assert call(16, good, n_bf=0) == 1
    assert call(16, good, beta=0.0) == 1
    assert h.value is None


def test_binding_power_mesh_matches_the_oracle_mesh():
    """The binding's power mesh (host logic, no GPU) and the oracle's, written
    separately, give the same grid."""
    import numpy as np
    import paper_1405_3273_gb300 as g
    from oracle import grids
    for p, u in [(0, 1), (0, 4), (2, 1), (3, 4), (5, 16), (7, 32), (6, 64)]:
        M, idx = g.power_mesh(p, u)
        M2, idx2 = grids.power_mesh(p, u)
        assert M == M2 and np.array_equal(np.asarray(idx), idx2), (p, u)
