"""Closed-form integrals over s-type Gaussians (textbook formulas).

For unnormalised s primitives exp(-a|r-A|^2), exp(-b|r-B|^2), with p = a+b,
P = (aA+bB)/p and K = exp(-ab/p |A-B|^2):

  overlap        (pi/p)^(3/2) K
  kinetic        ab/p (3 - 2ab/p |A-B|^2) * overlap
  nuclear        -Z 2pi/p K F0(p |P-C|^2)
  repulsion      2 pi^(5/2) / (p q sqrt(p+q)) K_ab K_cd F0(pq/(p+q) |P-Q|^2)

with the Boys function F0(t) = (1/2) sqrt(pi/t) erf(sqrt t).  The two-electron
integrals are returned in chemists' notation, v[i,j,k,l] = (ij|kl).
"""

from dataclasses import dataclass

import numpy as np
from scipy.special import erf

from .basis import basis_functions
from .geometry import workload_geometry


def boys0(t):
    t = np.asarray(t, dtype=np.float64)
    out = np.empty_like(t)
    small = t < 1e-7
    ts = t[small]
    out[small] = 1.0 - ts / 3.0 + ts * ts / 10.0
    tl = t[~small]
    rt = np.sqrt(tl)
    out[~small] = 0.5 * np.sqrt(np.pi) * erf(rt) / rt
    return out


def _primitives(funcs):
    alpha, centre, weight, owner = [], [], [], []
    for f, (c, a, w) in enumerate(funcs):
        for ap, wp in zip(a, w):
            alpha.append(ap)
            centre.append(c)
            weight.append(wp)
            owner.append(f)
    return (np.array(alpha), np.array(centre), np.array(weight), np.array(owner))


def nuclear_repulsion(coords, charges=None):
    coords = np.asarray(coords, dtype=np.float64)
    z = np.ones(len(coords)) if charges is None else np.asarray(charges, dtype=np.float64)
    e = 0.0
    for a in range(len(coords)):
        for b in range(a):
            e += z[a] * z[b] / np.linalg.norm(coords[a] - coords[b])
    return e


def one_electron(funcs, coords, charges=None):
    """(S, T, V) contracted one-electron matrices."""
    coords = np.asarray(coords, dtype=np.float64)
    z = np.ones(len(coords)) if charges is None else np.asarray(charges, dtype=np.float64)
    a, c, w, own = _primitives(funcs)
    n = len(funcs)
    p = a[:, None] + a[None, :]
    mu = a[:, None] * a[None, :] / p
    d2 = ((c[:, None, :] - c[None, :, :]) ** 2).sum(-1)
    K = np.exp(-mu * d2)
    s = (np.pi / p) ** 1.5 * K
    t = mu * (3.0 - 2.0 * mu * d2) * s
    P = (a[:, None, None] * c[:, None, :] + a[None, :, None] * c[None, :, :]) / p[..., None]
    v = np.zeros_like(s)
    for zc, cc in zip(z, coords):
        pc2 = ((P - cc) ** 2).sum(-1)
        v += -zc * 2.0 * np.pi / p * K * boys0(p * pc2)
    ww = w[:, None] * w[None, :]
    O = np.zeros((n, len(a)))
    O[own, np.arange(len(a))] = 1.0
    return tuple(O @ (m * ww) @ O.T for m in (s, t, v))


def two_electron(funcs, block=2048):
    """Dense (ij|kl) tensor [N,N,N,N], built from the i<=j pair list."""
    a, c, w, own = _primitives(funcs)
    n = len(funcs)
    npr = len(a)
    # primitive pairs (x,y) whose owners satisfy owner[x] <= owner[y]
    xs, ys = np.meshgrid(np.arange(npr), np.arange(npr), indexing="ij")
    xs, ys = xs.ravel(), ys.ravel()
    keep = own[xs] <= own[ys]
    xs, ys = xs[keep], ys[keep]
    pair_of = np.full((n, n), -1, dtype=np.int64)
    iu, ju = np.triu_indices(n)
    pair_of[iu, ju] = np.arange(len(iu))
    owner_pair = pair_of[own[xs], own[ys]]
    order = np.argsort(owner_pair, kind="stable")
    xs, ys, owner_pair = xs[order], ys[order], owner_pair[order]
    starts = np.flatnonzero(np.r_[True, owner_pair[1:] != owner_pair[:-1]])

    pa, pb = a[xs], a[ys]
    pp = pa + pb
    PP = (pa[:, None] * c[xs] + pb[:, None] * c[ys]) / pp[:, None]
    KK = np.exp(-pa * pb / pp * ((c[xs] - c[ys]) ** 2).sum(-1)) * w[xs] * w[ys]

    npair = len(iu)
    # accumulate contracted rows in blocks of primitive pairs
    acc = np.zeros((npair, npair))
    m = len(pp)
    for r0 in range(0, m, block):
        r1 = min(m, r0 + block)
        p1 = pp[r0:r1, None]
        q1 = pp[None, :]
        d2 = ((PP[r0:r1, None, :] - PP[None, :, :]) ** 2).sum(-1)
        val = (2.0 * np.pi ** 2.5 / (p1 * q1 * np.sqrt(p1 + q1))
               * KK[r0:r1, None] * KK[None, :] * boys0(p1 * q1 / (p1 + q1) * d2))
        colsum = np.add.reduceat(val, starts, axis=1)
        np.add.at(acc, owner_pair[r0:r1], colsum)
    idx = pair_of.copy()
    idx[ju, iu] = idx[iu, ju]
    return acc[idx[:, :, None, None], idx[None, None, :, :]]


@dataclass
class System:
    name: str
    coords: np.ndarray
    basis: str
    S: np.ndarray
    T: np.ndarray
    V: np.ndarray
    h: np.ndarray
    eri: np.ndarray
    e_nuc: float
    n_elec: int
    beta: float
    n_tau: int
    n_iw: int

    @property
    def nbf(self):
        return self.S.shape[0]


def build_system(name, spacing=None, coords=None, basis=None, beta=None, n_tau=None, n_iw=None):
    """Integrals and grid sizes of a named workload (or of explicit coordinates)."""
    if coords is None:
        coords, basis0, beta0, n_tau0, n_iw0 = workload_geometry(name, spacing)
        basis = basis or basis0
        beta = beta or beta0
        n_tau = n_tau or n_tau0
        n_iw = n_iw or n_iw0
    funcs = basis_functions(coords, basis)
    S, T, V = one_electron(funcs, coords)
    eri = two_electron(funcs)
    return System(name=name, coords=np.asarray(coords), basis=basis, S=S, T=T, V=V, h=T + V,
                  eri=eri, e_nuc=nuclear_repulsion(coords), n_elec=len(coords),
                  beta=float(beta), n_tau=int(n_tau), n_iw=int(n_iw))
