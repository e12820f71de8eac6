"""Sigma damping (the supplement's remark on damping the self-energy between
outer iterations) and the linear-algebra helpers of the convergence loop on
the GPU, against the oracle.

* ``gf2_combine`` and ``gf2_gram`` element by element against numpy, on
  ragged lengths (not multiples of the 256-thread blocks) and up to the
  16-term limit, with the output aliasing a source.
* GF2 with Sigma damping alpha < 1: every outer iteration's energy and
  density against ``oracle.gf2.run(..., sigma_damping=alpha)`` (the two loops
  use the same inner schedule: damped F steps while |R| > 1e-3, DIIS below),
  and every iteration's damped Sigma(tau) against
  alpha * Sigma_oracle[G(tau)] + (1 - alpha) * Sigma_previous on the GPU's own
  G(tau) (after a mu search the two sides may stop at different, equally valid
  mu inside the HOMO-LUMO gap, which moves G(tau) ~ e^{mu tau} but neither E
  nor P).
"""

import numpy as np
import pytest
import torch

import gf2_inputs as gi
from oracle import gf2 as og
from oracle import sigma as osg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def library():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import os
    import paper_1405_3273_gb300 as g
    from paper_1405_3273_gb300 import build
    if not os.path.exists(g.LIB_PATH):
        build.build()
    g.lib()
    return g


@pytest.mark.parametrize("count", [1, 7, 255, 257, 100003])
@pytest.mark.parametrize("n_terms", [1, 3, 16])
def test_combine_and_gram_match_numpy(library, count, n_terms):
    g = library
    rng = np.random.default_rng(1000 * n_terms + count)
    xs = [rng.normal(size=count) * (1.0 + k) for k in range(n_terms)]
    coef = list(rng.normal(size=n_terms))
    with g.Context(4, 9, 256, 10.0) as ctx:  # room for the 16 x 16 Gram matrix
        d = [torch.as_tensor(x, device="cuda") for x in xs]
        out = torch.empty(count, dtype=torch.float64, device="cuda")
        g.gf2_combine(ctx.handle, coef, d, out)
        ref = sum(c * x for c, x in zip(coef, xs))
        scale = sum(abs(c) * np.abs(x) for c, x in zip(coef, xs)).max()
        assert np.abs(out.cpu().numpy() - ref).max() <= 4e-16 * n_terms * scale
        # the output may alias a source (damping writes over the old Sigma)
        g.gf2_combine(ctx.handle, coef, d, d[0])
        assert np.abs(d[0].cpu().numpy() - ref).max() <= 4e-16 * n_terms * scale
        d[0].copy_(torch.as_tensor(xs[0]))
        gram = np.array(g.gf2_gram(ctx.handle, d))
        ref_g = np.array([[np.dot(a, b) for b in xs] for a in xs])
        norms = np.array([np.linalg.norm(x) for x in xs])
        assert gram.shape == (n_terms, n_terms)
        assert np.abs(gram - ref_g).max() <= 1e-14 * np.sqrt(count) * np.outer(norms, norms).max()
        assert np.array_equal(gram, gram.T)


def _damped_run(system, beta, n_tau, n_iw, alpha, max_outer):
    from paper_1405_3273_gb300 import driver
    r = gi.rhf(system)
    system.beta, system.n_tau, system.n_iw = beta, n_tau, n_iw
    ref_P = []
    ref = og.run(system, r.F, beta, n_tau, n_iw, max_outer=max_outer, e_tol=0.0, sigma_damping=alpha,
                 callback=lambda st: ref_P.append(st.P.copy()))
    mu0 = 0.5 * (r.eps[system.n_elec // 2 - 1] + r.eps[system.n_elec // 2])
    ds = driver.to_device(system, r.F, mu0)
    W = osg.exchange_combination(system.eri)
    seen = {"P": [], "sigma_err": [], "prev": None}

    def check(run):
        G_tau = run.G_tau.cpu().numpy()
        M = n_tau - 1
        exp = np.array([osg.sigma_factored(G_tau[k], -G_tau[M - k], system.eri, W) for k in range(n_tau)])
        if seen["prev"] is not None:
            exp = alpha * exp + (1.0 - alpha) * seen["prev"]
        got = run.Sigma_tau.cpu().numpy()
        seen["sigma_err"].append(np.abs(got - exp).max() / max(1.0, np.abs(exp).max()))
        seen["prev"] = got.copy()
        seen["P"].append(run.P.cpu().numpy())

    got = driver.run_gf2(ds, max_outer=max_outer, e_tol=0.0, damping=alpha, callback=check)
    got.ctx.close()
    return ref, ref_P, got, seen


@pytest.mark.parametrize("alpha", [0.5, 0.3])
def test_sigma_damping_h4_every_iteration(library, alpha):
    s = gi.build_system("chain", coords=gi.h_chain(4, 1.7), basis="sto-3g", beta=50.0, n_tau=257, n_iw=512)
    ref, ref_P, got, seen = _damped_run(s, 50.0, 257, 512, alpha, 4)
    e_ref = np.array([e[0] for e in ref.energies])
    e_got = np.array([e[0] for e in got.energies])
    assert len(e_ref) == len(e_got) == 5
    assert np.abs(e_ref - e_got).max() < 1e-9
    assert len(seen["P"]) == len(ref_P) == 4
    for a, b in zip(seen["P"], ref_P):
        assert np.abs(a - b).max() < 1e-8
    assert max(seen["sigma_err"]) <= 1e-12
    # damping changes the iterates: the undamped run takes other values
    und, _, _, _ = _damped_run(s, 50.0, 257, 512, 1.0, 2)
    assert abs(und.energies[2][0] - ref.energies[2][0]) > 1e-6


def test_sigma_damping_h10_every_iteration(library):
    s = gi.build_system("h10_chain_sto3g")
    ref, ref_P, got, seen = _damped_run(s, 100.0, 513, 1024, 0.5, 3)
    e_ref = np.array([e[0] for e in ref.energies])
    e_got = np.array([e[0] for e in got.energies])
    assert np.abs(e_ref - e_got).max() < 1e-8
    for a, b in zip(seen["P"], ref_P):
        assert np.abs(a - b).max() < 1e-8
    assert max(seen["sigma_err"]) <= 1e-12
