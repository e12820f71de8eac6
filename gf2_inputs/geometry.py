"""Hydrogen chain and lattice geometries of the benchmark workloads (bohr)."""

import numpy as np


def h_chain(n_atoms, spacing):
    """Linear H_n chain along x with uniform spacing."""
    x = np.arange(n_atoms, dtype=np.float64) * spacing
    return np.stack([x, np.zeros_like(x), np.zeros_like(x)], axis=1)


def h_lattice(nx, ny, nz, spacing):
    """Simple-cubic nx*ny*nz hydrogen lattice with one spacing on every axis."""
    g = np.array([(i, j, k) for i in range(nx) for j in range(ny) for k in range(nz)],
                 dtype=np.float64)
    return g * spacing


# name -> (geometry builder, basis, beta, n_tau, n_iw)
#   n_iw = 2 (n_tau - 1) wherever the workload leaves it unstated.
WORKLOADS = {
    "h2_sto3g": (lambda a=1.4: h_chain(2, a), "sto-3g", 100.0, 513, 1024),
    "h10_chain_sto3g": (lambda a=1.8: h_chain(10, a), "sto-3g", 100.0, 2049, 4096),
    "h32_lattice_sto3g": (lambda a=2.0: h_lattice(2, 4, 4, a), "sto-3g", 100.0, 4097, 8192),
    "h32_lattice_631g": (lambda a=2.0: h_lattice(2, 4, 4, a), "6-31g", 100.0, 4097, 8192),
    "h64_lattice_631g": (lambda a=2.0: h_lattice(4, 4, 4, a), "6-31g", 200.0, 8193, 16384),
}


def workload_geometry(name, spacing=None):
    """(coords, basis, beta, n_tau, n_iw) of a named workload."""
    build, basis, beta, n_tau, n_iw = WORKLOADS[name]
    coords = build() if spacing is None else build(spacing)
    return coords, basis, beta, n_tau, n_iw
