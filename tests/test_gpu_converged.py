"""Self-consistent GF2 to convergence on the linear H10 chain (STO-3G, 1.8 bohr,
beta = 100, n_tau = 2049, n_iw = 4096): the converged GPU energy against the
converged oracle energy, for the FP64 path (<= 1e-8 Eh) and the FP16x3 split
path (<= 1e-6 Eh, density <= 1e-6).  Both sides stop when the energy changes by
less than 1e-9 Eh between outer iterations."""

import numpy as np
import pytest
import torch

import gf2_inputs as gi
from oracle import gf2 as og

pytestmark = pytest.mark.gpu
E_TOL = 1e-9


@pytest.fixture(scope="module")
def converged_oracle():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    s = gi.build_system("h10_chain_sto3g")
    r = gi.rhf(s)
    ref = og.run(s, r.F, 100.0, 2049, 4096, max_outer=40, e_tol=E_TOL)
    assert abs(ref.energies[-1][0] - ref.energies[-2][0]) < E_TOL, "oracle did not converge"
    return s, r, ref


@pytest.mark.parametrize("prec,e_tol,p_tol", [(0, 1e-8, 1e-8), (3, 1e-6, 1e-6)])
def test_converged_h10_energy_matches_oracle(converged_oracle, prec, e_tol, p_tol):
    import os
    import paper_1405_3273_gb300 as g
    from paper_1405_3273_gb300 import build, driver
    if not os.path.exists(g.LIB_PATH):
        build.build()
    s, r, ref = converged_oracle
    mu0 = 0.5 * (r.eps[s.n_elec // 2 - 1] + r.eps[s.n_elec // 2])
    got = driver.run_gf2(driver.to_device(s, r.F, mu0), prec=prec, max_outer=40, e_tol=E_TOL)
    e_ref, e_got = ref.energies[-1][0], got.energies[-1][0]
    dp = np.abs(got.P.cpu().numpy() - ref.P).max()
    print(f"H10 converged, prec {prec}: oracle {e_ref:.10f} ({len(ref.energies) - 1} outer), "
          f"GPU {e_got:.10f} ({len(got.energies) - 1} outer), |dE| {abs(e_ref - e_got):.2e}, max|dP| {dp:.2e}")
    assert abs(e_got - e_ref) <= e_tol
    assert dp <= p_tol
    got.ctx.close()
