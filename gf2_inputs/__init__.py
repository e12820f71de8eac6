"""Synthetic inputs shared by the CPU oracle and the GPU library.

This package stands in for the quantum-chemistry program that supplies the
starting point of a GF2 calculation (step 1 of the GF2 algorithm in the
paper's supplement: a restricted Hartree-Fock reference, plus the AO
integrals).  It holds the hydrogen geometries and s-Gaussian basis sets of the
benchmark workloads, the closed-form s-type integrals, an RHF solver, seeded
random tensors for unit tests, and (``density_fitting``) auxiliary s bases with
the three-index factor of density-fitted integrals.  It contains none of the GF2 hot-path
arithmetic (self-energy, Fourier transforms, Dyson solve, chemical-potential
search, energy) and it imports neither ``oracle`` nor the GPU package.
"""

from .basis import BASIS_SETS, basis_functions
from .geometry import h_chain, h_lattice, WORKLOADS, workload_geometry
from .integrals import one_electron, two_electron, nuclear_repulsion, System, build_system
from .rhf import rhf, RHFResult
from .random_inputs import random_symmetric_g, random_eri, SEED
from . import density_fitting  # noqa: F401

__all__ = [
    "BASIS_SETS", "basis_functions", "h_chain", "h_lattice", "WORKLOADS",
    "workload_geometry", "one_electron", "two_electron", "nuclear_repulsion",
    "System", "build_system", "rhf", "RHFResult", "random_symmetric_g",
    "random_eri", "SEED",
]
