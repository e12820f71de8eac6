"""Plain, slow FP64 CPU oracle for the GF2 hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package.
The GPU library never calls it and shares no code with it; both sides take
their inputs from ``gf2_inputs``.

Every routine follows the paper's definitions directly:
  * ``sigma``      -- second-order self-energy (Eq. Sigma), as the literal
                      six-index sum and as four successive N^5 contractions;
  * ``transforms`` -- Matsubara <-> imaginary-time transforms as direct sums
                      with the analytic high-frequency tail;
  * ``dyson``      -- Eq. GF by dense LU inversion, density matrix,
                      chemical-potential bisection;
  * ``fock``       -- Eq. FockMatrix;
  * ``energy``     -- Galitskii-Migdal energy;
  * ``occupations`` -- natural occupation numbers eig(S^1/2 P S^1/2)/2;
  * ``df``         -- Eq. Sigma on density-fitted integrals, written out and
                      in the three-index factors alone;
  * ``gf2``        -- the self-consistent loop of the supplement (steps 1-3).
"""

from . import grids, sigma, transforms, dyson, fock, energy, gf2, occupations, df  # noqa: F401
