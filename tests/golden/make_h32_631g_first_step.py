"""Writes the oracle's first GF2 self-energy step on the H32 2x4x4 lattice
(2.0 bohr, 6-31G, N = 64, 32 electrons, beta = 100) into a JSON fixture; with
--system h64 the same step on the H64 4x4x4 lattice (2.0 bohr, 6-31G, N = 128,
64 electrons, beta = 200, 16384 frequencies).

The step is the one ``bench.py`` times, done here by the plain FP64 CPU oracle
only (``oracle/``; no GPU code is imported):

  1. finite-temperature HF state: F = F_HF (RHF Fock matrix), mu_0 from the
     chemical-potential bisection with Sigma = 0 (step 2.a), G(i w) at mu_0
     (Eq. GF);
  2. tail moments at (F_HF, mu_0), G(i w) -> G(tau) (direct sums);
  3. Sigma(tau) by Eq. Sigma (four factored contractions per time point);
  4. Sigma(tau) -> Sigma(i w) (cubic-interpolant Fourier integral) and its
     1/z, 1/z^2 coefficients;
  5. mu search at F = F_HF with that Sigma (step 2.a), P and G(i w);
  6. Galitskii-Migdal energy E = E_nuc + 1/2 Tr[P (h + F_HF)] + E2.

Usage:  python tests/golden/make_h32_631g_first_step.py [--n-tau 4097 --n-iw 8192]
                                                        [--mesh P U]
The full grid takes about 20 minutes on 8 cores (Sigma at 4097 time points
dominates).  Output: tests/golden/h32_631g_first_step_t{n_tau}_w{n_iw}.json,
or with --mesh the same step on the uniform power mesh with P halvings and U
steps per interval (``oracle.grids.power_mesh``; iw -> tau at the mesh
points, the local-cubic integral through its unequal nodes):
tests/golden/h32_631g_first_step_pm{P}x{U}_w{n_iw}.json (h64_... for --system h64;
    python tests/golden/make_h32_631g_first_step.py --system h64 --n-iw 16384 --mesh 7 32
takes about half an hour on 8 cores).
"""

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import gf2_inputs as gi  # noqa: E402
from oracle import dyson as od  # noqa: E402
from oracle import grids as og  # noqa: E402
from oracle import energy as oe  # noqa: E402
from oracle import sigma as osg  # noqa: E402
from oracle import transforms as ot  # noqa: E402


SYSTEMS = {"h32": ("h32_lattice_631g", 100.0, "H32 2x4x4 lattice at 2.0 bohr, 6-31G (N=64), beta=100"),
           "h64": ("h64_lattice_631g", 200.0, "H64 4x4x4 lattice at 2.0 bohr, 6-31G (N=128), beta=200")}


def fixture_path(n_tau, n_iw, mesh=None, system="h32"):
    if mesh is not None:
        return os.path.join(HERE, f"{system}_631g_first_step_pm{mesh[0]}x{mesh[1]}_w{n_iw}.json")
    return os.path.join(HERE, f"{system}_631g_first_step_t{n_tau}_w{n_iw}.json")


def first_step(n_tau, n_iw, beta=None, spacing=2.0, mesh=None, system="h32"):
    t0 = time.time()
    name, beta0, label = SYSTEMS[system]
    beta = beta0 if beta is None else beta
    s = gi.build_system(name, spacing=spacing)
    r = gi.rhf(s)
    F = r.F
    mu0, G0, P0, nev0 = od.mu_search(s.S, F, None, None, None, s.n_elec, beta, n_iw)
    e_hf = s.e_nuc + oe.e_one_body(P0, s.h, F)
    mom = ot.tail_moments(s.S, F, mu0)
    if mesh is None:
        G_tau = ot.iw_to_tau(G0, mom, beta, n_tau)
    else:
        M, index = og.power_mesh(*mesh)
        n_tau = len(index)
        G_tau = ot.iw_to_tau(G0, mom, beta, M + 1, taus=index)
    Sig_tau = osg.sigma_tau(G_tau, s.eri)
    if mesh is None:
        Sig_iw = ot.tau_to_iw(Sig_tau, beta, n_iw)
        sig1, sig2 = ot.sigma_expansion(Sig_tau, beta)
    else:
        Sig_iw = ot.tau_to_iw_grid(Sig_tau, beta, M, index, n_iw)
        sig1, sig2 = ot.sigma_expansion_grid(Sig_tau, beta, M, index)
    mu, G, P, nev = od.mu_search(s.S, F, Sig_iw, sig1, sig2, s.n_elec, beta, n_iw)
    e1 = oe.e_one_body(P, s.h, F)
    e2 = oe.e_two_body(G, Sig_iw, sig1, s.S, beta)
    ks = sorted({0, 1, (n_tau - 1) // 4, (n_tau - 1) // 2, n_tau - 2, n_tau - 1})
    return {
        "what": ("oracle first GF2 self-energy step from the finite-temperature HF state, "
                 f"{label}; F held at F_HF"),
        "written_by": "tests/golden/make_h32_631g_first_step.py (calls oracle/ and gf2_inputs only)",
        "n_bf": int(s.nbf), "n_elec": int(s.n_elec), "beta": beta, "n_tau": n_tau, "n_iw": n_iw,
        "mesh": None if mesh is None else {"p": mesh[0], "u": mesh[1], "M": int(M)},
        "spacing_bohr": spacing,
        "mu_hf": mu0, "E_hf": e_hf, "P_hf_trace_PS": float(np.trace(P0 @ s.S)),
        "mu": mu, "E": s.e_nuc + e1 + e2, "E_one_body": e1, "E_two_body": e2, "E_nuc": s.e_nuc,
        "trace_PS": float(np.trace(P @ s.S)),
        "P": P.tolist(),
        "sigma_tau_samples": {str(k): {"trace": float(np.trace(Sig_tau[k])),
                                       "frobenius": float(np.linalg.norm(Sig_tau[k])),
                                       "max_abs": float(np.abs(Sig_tau[k]).max())} for k in ks},
        "sig1_trace": float(np.trace(sig1)),
        "oracle_seconds": time.time() - t0,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-tau", type=int, default=4097)
    ap.add_argument("--n-iw", type=int, default=8192)
    ap.add_argument("--mesh", type=int, nargs=2, default=None, metavar=("P", "U"))
    ap.add_argument("--system", default="h32", choices=sorted(SYSTEMS))
    a = ap.parse_args()
    mesh = tuple(a.mesh) if a.mesh else None
    d = first_step(a.n_tau, a.n_iw, mesh=mesh, system=a.system)
    with open(fixture_path(a.n_tau, a.n_iw, mesh, a.system), "w") as f:
        json.dump(d, f, indent=0)
    print(json.dumps({k: v for k, v in d.items() if k not in ("P", "sigma_tau_samples")}))


if __name__ == "__main__":
    main()
