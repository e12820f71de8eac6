"""Python binding of libgf2, the GB300 library for the hot path of one
self-consistent GF2 iteration (second-order self-energy, Matsubara/tau
transforms, Dyson solve, chemical-potential search, Fock build and energy).

Argument marshalling only: every function forwards to the C entry point of
the same name in ``libgf2.so`` (declared in ``include/gf2.h``) with device
pointers taken from CUDA torch tensors and the current torch stream.  There is
no CPU fallback: importing works without a GPU, but calling any function needs
the built library and a CUDA device, and fails loudly otherwise.
"""

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgf2.so")

GF2_OK = 0
GF2_PREC_FP64 = 0
GF2_PREC_BF16X3 = 1
GF2_PREC_BF16X6 = 2
GF2_PREC_FP16X3 = 3
GF2_PREC_FP16X6 = 4
STATUS_NAMES = {0: "GF2_OK", 1: "GF2_ERR_ARG", 2: "GF2_ERR_CUDA", 3: "GF2_ERR_NOMEM",
                4: "GF2_ERR_NOT_CONVERGED", 5: "GF2_ERR_TIMEOUT", 6: "GF2_ERR_NONFINITE",
                7: "GF2_ERR_UNSUPPORTED"}

_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SIGS = {
    "gf2_create": [ctypes.POINTER(_P), _I, _I, _I, _D, _P],
    "gf2_create_grid": [ctypes.POINTER(_P), _I, _I, _I, ctypes.POINTER(_I), _I, _D, _P],
    "gf2_destroy": [_P],
    "gf2_set_stream": [_P, _P],
    "gf2_status_string": [_I],
    "gf2_last_error": [_P],
    "gf2_set_integrals": [_P, _P],
    "gf2_set_overlap": [_P, _P],
    "gf2_sigma_tau": [_P, _P, _P, _I],
    "gf2_sigma_tau_points": [_P, _P, _I, _I, _P, _I],
    "gf2_set_df_integrals": [_P, _P, _I],
    "gf2_sigma_tau_df": [_P, _P, _I, _I, _P, _I],
    "gf2_tail_moments": [_P, _P, _P, _D, _P, _P],
    "gf2_fft_iw_to_tau": [_P, _P, _P, _P],
    "gf2_fft_tau_to_iw": [_P, _P, _P, _P],
    "gf2_dyson": [_P, _D, _P, _P, _P, _P],
    "gf2_density": [_P, _P, _P, _P],
    "gf2_mu_search": [_P, _P, _P, _P, _P, _D, _D, _I, ctypes.POINTER(_D), _P, _P, ctypes.POINTER(_I)],
    "gf2_inner_loop": [_P, _P, _P, _P, _P, _P, _D, ctypes.POINTER(_D), _P, _P, _D, _I, _D, _I, _D, _D,
                       ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "gf2_fock": [_P, _P, _P, _P],
    "gf2_energy": [_P, _P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(_D), ctypes.POINTER(_D)],
    "gf2_combine": [_P, _I, ctypes.POINTER(_D), ctypes.POINTER(_P), ctypes.c_longlong, _P],
    "gf2_gram": [_P, _I, ctypes.POINTER(_P), ctypes.c_longlong, ctypes.POINTER(_D)],
    "gf2_energy_noalloc": [_I, _I, _D, _P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(_D), ctypes.POINTER(_D), _P],
    "gf2_natural_occupations": [_P, _P, _P],
    "gf2_batch_create": [ctypes.POINTER(_P), _I, ctypes.POINTER(_I), ctypes.POINTER(_I), _P],
    "gf2_batch_destroy": [_P],
    "gf2_batch_last_error": [_P],
    "gf2_batch_set_system": [_P, _I, _P, _P],
    "gf2_batch_tune": [_P, ctypes.POINTER(_P), _I],
    "gf2_batch_plan": [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_D), ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "gf2_batch_partner": [_P, _I, ctypes.POINTER(_I)],
    "gf2_sigma_tau_batched": [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _I],
    "gf2_profile": [_P, _I],
    "gf2_profile_report": [_P, ctypes.c_char_p, _I, ctypes.POINTER(ctypes.c_longlong)],
}


class GF2Error(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def lib():
    """The loaded libgf2 (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgf2.so not built at {LIB_PATH}; run paper_1405_3273_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_char_p if name in ("gf2_status_string", "gf2_last_error",
                                                    "gf2_batch_last_error") else _I
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _ptr(t, dtype=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA torch tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(status, ctx):
    if status != GF2_OK:
        msg = lib().gf2_last_error(ctx).decode() if ctx else lib().gf2_status_string(status).decode()
        raise GF2Error(status, msg)


_F64 = torch.float64
_C128 = torch.complex128


def gf2_create(n_bf, n_tau, n_iw, beta):
    h = ctypes.c_void_p()
    st = lib().gf2_create(ctypes.byref(h), int(n_bf), int(n_tau), int(n_iw), float(beta), _stream())
    if st != GF2_OK:
        raise GF2Error(st, "gf2_create rejected the sizes or could not allocate")
    return h


def gf2_create_grid(n_bf, M, tau_index, n_iw, beta):
    """Context on the non-equidistant grid tau_k = tau_index[k] beta / M (host ints)."""
    idx = [int(i) for i in tau_index]
    arr = (ctypes.c_int * len(idx))(*idx)
    h = ctypes.c_void_p()
    st = lib().gf2_create_grid(ctypes.byref(h), int(n_bf), int(M), len(idx), arr, int(n_iw), float(beta), _stream())
    if st != GF2_OK:
        raise GF2Error(st, "gf2_create_grid rejected the grid or the sizes, or could not allocate")
    return h


def power_mesh(p, u):
    """(M, tau_index) of the uniform power mesh: [0, beta/2^(p+1)] and each
    [beta/2^(j+1), beta/2^j], j = 1..p, cut into u equal steps, the upper half of
    [0, beta] the mirror image; indices into the uniform grid of M = 2^(p+1) u
    intervals (2 (p+1) u + 1 points)."""
    if p < 0 or u < 1:
        raise ValueError("power mesh needs p >= 0 and u >= 1")
    M = (1 << (p + 1)) * u
    lower, pos = [0], 0
    for level in range(p + 1):                 # step 1 on the two innermost intervals, then 2, 4, ...
        step = 1 << max(0, level - 1)
        for _ in range(u):
            pos += step
            lower.append(pos)
    return M, lower + [M - i for i in reversed(lower[:-1])]


def gf2_destroy(ctx):
    _check(lib().gf2_destroy(ctx), None)


def gf2_set_stream(ctx):
    _check(lib().gf2_set_stream(ctx, _stream()), ctx)


def gf2_set_integrals(ctx, v):
    _check(lib().gf2_set_integrals(ctx, _ptr(v, _F64)), ctx)


def gf2_set_overlap(ctx, S):
    _check(lib().gf2_set_overlap(ctx, _ptr(S, _F64)), ctx)


def gf2_sigma_tau(ctx, G_tau, Sigma_tau, prec=GF2_PREC_FP64):
    _check(lib().gf2_sigma_tau(ctx, _ptr(G_tau, _F64), _ptr(Sigma_tau, _F64), int(prec)), ctx)


def gf2_sigma_tau_points(ctx, G_tau, k0, count, Sigma_out, prec=GF2_PREC_FP64):
    _check(lib().gf2_sigma_tau_points(ctx, _ptr(G_tau, _F64), int(k0), int(count),
                                      _ptr(Sigma_out, _F64), int(prec)), ctx)


def gf2_set_df_integrals(ctx, B):
    """B: [m, N, N] float64 CUDA tensor, v_ijkl = sum_Q B[Q,i,j] B[Q,k,l]."""
    _check(lib().gf2_set_df_integrals(ctx, _ptr(B, _F64), int(B.shape[0])), ctx)


def gf2_sigma_tau_df(ctx, G_tau, k0, count, Sigma_out, prec=GF2_PREC_FP64):
    _check(lib().gf2_sigma_tau_df(ctx, _ptr(G_tau, _F64), int(k0), int(count),
                                  _ptr(Sigma_out, _F64), int(prec)), ctx)


def gf2_tail_moments(ctx, S, F, mu, sig12, moments):
    _check(lib().gf2_tail_moments(ctx, _ptr(S, _F64), _ptr(F, _F64), float(mu), _ptr(sig12, _F64),
                                  _ptr(moments, _F64)), ctx)


def gf2_fft_iw_to_tau(ctx, X_iw, moments, X_tau):
    _check(lib().gf2_fft_iw_to_tau(ctx, _ptr(X_iw, _C128), _ptr(moments, _F64), _ptr(X_tau, _F64)), ctx)


def gf2_fft_tau_to_iw(ctx, X_tau, X_iw, sig12=None):
    _check(lib().gf2_fft_tau_to_iw(ctx, _ptr(X_tau, _F64), _ptr(X_iw, _C128), _ptr(sig12, _F64)), ctx)


def gf2_dyson(ctx, mu, S, F, Sigma_iw, G_iw):
    _check(lib().gf2_dyson(ctx, float(mu), _ptr(S, _F64), _ptr(F, _F64), _ptr(Sigma_iw, _C128),
                           _ptr(G_iw, _C128)), ctx)


def gf2_density(ctx, G_iw, moments, P):
    _check(lib().gf2_density(ctx, _ptr(G_iw, _C128), _ptr(moments, _F64), _ptr(P, _F64)), ctx)


def gf2_mu_search(ctx, S, F, Sigma_iw, sig12, n_elec, mu0, G_iw, P, tol=1e-10, max_iter=100):
    mu = ctypes.c_double(float(mu0))
    nev = ctypes.c_int(0)
    _check(lib().gf2_mu_search(ctx, _ptr(S, _F64), _ptr(F, _F64), _ptr(Sigma_iw, _C128),
                               _ptr(sig12, _F64), float(n_elec), float(tol), int(max_iter),
                               ctypes.byref(mu), _ptr(G_iw, _C128), _ptr(P, _F64),
                               ctypes.byref(nev)), ctx)
    return mu.value, nev.value


def gf2_inner_loop(ctx, S, h, F, Sigma_iw, sig12, n_elec, mu0, G_iw, P, tol=1e-8, max_iter=300,
                   mu_tol=1e-10, diis=8, mix=0.5, diis_from=1e-3):
    """Device-resident inner loop; F is updated in place.  Returns (mu, iterations, mu evaluations)."""
    mu = ctypes.c_double(float(mu0))
    nit, nev = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().gf2_inner_loop(ctx, _ptr(S, _F64), _ptr(h, _F64), _ptr(F, _F64), _ptr(Sigma_iw, _C128),
                                _ptr(sig12, _F64), float(n_elec), ctypes.byref(mu), _ptr(G_iw, _C128),
                                _ptr(P, _F64), float(tol), int(max_iter), float(mu_tol), int(diis), float(mix),
                                float(diis_from), ctypes.byref(nit), ctypes.byref(nev)), ctx)
    return mu.value, nit.value, nev.value


def gf2_fock(ctx, h, P, F):
    _check(lib().gf2_fock(ctx, _ptr(h, _F64), _ptr(P, _F64), _ptr(F, _F64)), ctx)


def gf2_energy(ctx, h, F, P, S, G_iw, Sigma_iw, sig12):
    e1, e2 = ctypes.c_double(), ctypes.c_double()
    _check(lib().gf2_energy(ctx, _ptr(h, _F64), _ptr(F, _F64), _ptr(P, _F64), _ptr(S, _F64),
                            _ptr(G_iw, _C128), _ptr(Sigma_iw, _C128), _ptr(sig12, _F64),
                            ctypes.byref(e1), ctypes.byref(e2)), ctx)
    return e1.value, e2.value


def gf2_energy_noalloc(n_bf, n_iw, beta, h, F, P, S, G_iw, Sigma_iw, sig12):
    """Allocation-free gf2_energy (no context); see include/gf2.h."""
    e1, e2 = ctypes.c_double(), ctypes.c_double()
    st = lib().gf2_energy_noalloc(int(n_bf), int(n_iw), float(beta), _ptr(h, _F64), _ptr(F, _F64),
                                  _ptr(P, _F64), _ptr(S, _F64), _ptr(G_iw, _C128), _ptr(Sigma_iw, _C128),
                                  _ptr(sig12, _F64), ctypes.byref(e1), ctypes.byref(e2), _stream())
    _check(st, None)
    return e1.value, e2.value


def gf2_combine(ctx, coefs, srcs, out):
    n = len(coefs)
    c = (ctypes.c_double * n)(*[float(x) for x in coefs])
    p = (ctypes.c_void_p * n)(*[_ptr(t, _F64) for t in srcs])
    _check(lib().gf2_combine(ctx, n, c, p, out.numel(), _ptr(out, _F64)), ctx)


def gf2_gram(ctx, vecs):
    n = len(vecs)
    p = (ctypes.c_void_p * n)(*[_ptr(t, _F64) for t in vecs])
    out = (ctypes.c_double * (n * n))()
    _check(lib().gf2_gram(ctx, n, p, vecs[0].numel(), out), ctx)
    return [[out[a * n + b] for b in range(n)] for a in range(n)]


def gf2_profile(ctx, enable=True):
    _check(lib().gf2_profile(ctx, 1 if enable else 0), ctx)


def gf2_profile_report(ctx):
    """{kernel: (launches, total_ms)} since the last gf2_profile call, and the launch count."""
    buf = ctypes.create_string_buffer(1 << 14)
    n = ctypes.c_longlong(0)
    _check(lib().gf2_profile_report(ctx, buf, len(buf), ctypes.byref(n)), ctx)
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms = line.split()
        out[name] = (int(cnt), float(ms))
    return out, n.value


def _ptr_array(ts):
    return (ctypes.c_void_p * len(ts))(*[_ptr(t, _F64).value for t in ts])


def _check_batch(status, b):
    if status != GF2_OK:
        raise GF2Error(status, lib().gf2_batch_last_error(b).decode() if b else "")


def gf2_natural_occupations(ctx, P, occ):
    _check(lib().gf2_natural_occupations(ctx, _ptr(P, _F64), _ptr(occ, _F64)), ctx)


def gf2_batch_last_error(b):
    return lib().gf2_batch_last_error(b).decode()


def gf2_batch_create(n_bf, n_tau):
    n = len(n_bf)
    h = ctypes.c_void_p()
    st = lib().gf2_batch_create(ctypes.byref(h), n, (ctypes.c_int * n)(*map(int, n_bf)),
                                (ctypes.c_int * n)(*map(int, n_tau)), _stream())
    if st != GF2_OK:
        raise GF2Error(st, "gf2_batch_create rejected the sizes or could not allocate")
    return h


def gf2_batch_destroy(b):
    _check(lib().gf2_batch_destroy(b), None)


def gf2_batch_set_system(b, inst, v, S=None):
    _check_batch(lib().gf2_batch_set_system(b, int(inst), _ptr(v, _F64), _ptr(S, _F64)), b)


def gf2_batch_tune(b, G_taus, prec):
    _check_batch(lib().gf2_batch_tune(b, _ptr_array(G_taus), int(prec)), b)


def gf2_batch_plan(b, inst):
    """(precision code, estimated ms per full-grid build, worker stream, slots per
    split-pipeline launch) chosen for an instance."""
    p, ms, lane, chunk = ctypes.c_int(), ctypes.c_double(), ctypes.c_int(), ctypes.c_int()
    _check_batch(lib().gf2_batch_plan(b, int(inst), ctypes.byref(p), ctypes.byref(ms), ctypes.byref(lane),
                                      ctypes.byref(chunk)), b)
    return p.value, ms.value, lane.value, chunk.value


def gf2_batch_partner(b, inst):
    """The instance sharing inst's block-diagonal system (BF16 splits), or -1."""
    q = ctypes.c_int(-1)
    _check_batch(lib().gf2_batch_partner(b, int(inst), ctypes.byref(q)), b)
    return q.value


def gf2_sigma_tau_batched(b, G_taus, Sigma_taus, prec):
    _check_batch(lib().gf2_sigma_tau_batched(b, _ptr_array(G_taus), _ptr_array(Sigma_taus), int(prec)), b)


class Batch:
    """Owning handle around a gf2_batch (destroyed on close / garbage collection)."""

    def __init__(self, n_bf, n_tau):
        self.n_bf, self.n_tau = list(n_bf), list(n_tau)
        self.handle = gf2_batch_create(self.n_bf, self.n_tau)

    def close(self):
        if getattr(self, "handle", None) is not None:
            gf2_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Context:
    """Owning handle around a gf2_ctx (destroyed on close / garbage collection)."""

    def __init__(self, n_bf, n_tau, n_iw, beta, grid=None):
        """grid = (M, tau_index): a non-equidistant time grid (n_tau is then len(tau_index))."""
        self.n_bf, self.n_iw, self.beta = int(n_bf), int(n_iw), float(beta)
        if grid is None:
            self.n_tau = int(n_tau)
            self.handle = gf2_create(n_bf, n_tau, n_iw, beta)
        else:
            self.n_tau = len(grid[1])
            self.handle = gf2_create_grid(n_bf, grid[0], grid[1], n_iw, beta)

    def close(self):
        if getattr(self, "handle", None) is not None:
            gf2_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
