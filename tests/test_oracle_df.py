"""Pins of the density-fitted self-energy (oracle/df.py) and of the auxiliary
integrals that feed it (gf2_inputs/density_fitting.py).

* the factor form (no four-index tensor) equals Eq. Sigma's literal eight-
  index sum on the fitted integrals, for random factors: it was derived by
  hand from the equation, so a dropped term, a swapped index or a wrong
  factor of two fails here;
* an auxiliary set that spans every orbital product fits the exact
  repulsion integrals of ``integrals`` (an independent closed form) to
  rounding, and so reproduces the exact Sigma;
* the Coulomb-metric fit is variational: the error supermatrix is a Gram
  matrix of the fitting residuals (positive semidefinite) and never grows
  when the auxiliary span grows;
* Sigma is unchanged by an orthogonal rotation of the auxiliary index;
* GF2's first correlation energy with the factor-form Sigma approaches the
  finite-beta MO closed form on the fitted integrals as the grid grows.
"""

import numpy as np
import pytest

import gf2_inputs as gi
from gf2_inputs import density_fitting as dfi
from oracle import df as odf
from oracle import sigma as osg


def _random_factor(m, n, seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((m, n, n))
    return 0.5 * (B + np.swapaxes(B, 1, 2))


def test_fitted_integrals_by_explicit_loops():
    B = _random_factor(3, 2, 1)
    v = odf.df_eri(B)
    for i, j, k, l in np.ndindex(2, 2, 2, 2):
        assert abs(v[i, j, k, l] - sum(B[q, i, j] * B[q, k, l] for q in range(3))) < 1e-15


@pytest.mark.parametrize("m,n", [(1, 3), (3, 3), (5, 4), (9, 2)])
def test_factor_form_equals_the_literal_eight_index_sum(m, n):
    G = gi.random_symmetric_g(n, 3, seed=gi.SEED + 3 * m + n)
    B = _random_factor(m, n, 10 + m)
    v = odf.df_eri(B)
    for k in range(3):
        Gb = osg.gbar_from_grid(G, k)
        lit = osg.sigma_literal(G[k], Gb, v)
        scale = np.abs(lit).max()
        assert np.abs(odf.sigma_df_factors(G[k], Gb, B) - lit).max() <= 1e-12 * scale
        assert np.abs(odf.sigma_df(G[k], Gb, B) - lit).max() <= 1e-12 * scale


def test_factor_form_with_a_non_symmetric_green_function():
    """No symmetry of G or Gbar is assumed by the factor form."""
    rng = np.random.default_rng(5)
    G, Gb = rng.standard_normal((2, 3, 3))
    B = _random_factor(4, 3, 6)
    lit = osg.sigma_literal(G, Gb, odf.df_eri(B))
    assert np.abs(odf.sigma_df_factors(G, Gb, B) - lit).max() <= 1e-12 * np.abs(lit).max()


@pytest.mark.parametrize("basis", ["sto-3g", "6-31g"])
def test_product_auxiliary_set_fits_exactly(basis):
    coords = gi.h_chain(4, 1.7)
    s = gi.build_system("chain", coords=coords, basis=basis, beta=20.0, n_tau=9, n_iw=16)
    B = dfi.build_df(coords, basis, "products")
    v = odf.df_eri(B)
    assert np.abs(v - s.eri).max() < 1e-10 * np.abs(s.eri).max()
    G = gi.random_symmetric_g(s.nbf, 9, seed=11)
    exact = osg.sigma_tau(G, s.eri, taus=[0, 3, 8])
    fitted = odf.sigma_tau_df(G, B, taus=[0, 3, 8])
    assert np.abs(fitted - exact).max() < 1e-9 * np.abs(exact).max()


def test_coulomb_fit_error_is_a_gram_matrix_that_shrinks_with_the_span():
    coords = gi.h_chain(4, 1.7)
    s = gi.build_system("chain", coords=coords, basis="6-31g", beta=20.0, n_tau=9, n_iw=16)
    funcs = gi.basis_functions(coords, "6-31g")
    n2 = s.nbf ** 2
    prev = None
    for k in range(2, 7):   # nested even-tempered sets: the first k exponents on every atom
        aux = dfi.aux_even_tempered(coords, dfi.EVEN_TEMPERED_H[:k])
        B = dfi.df_factor(dfi.three_center(funcs, aux), dfi.two_center(aux))
        E = (s.eri - odf.df_eri(B)).reshape(n2, n2)
        assert np.abs(E - E.T).max() < 1e-12
        assert np.linalg.eigvalsh(E).min() > -1e-12
        d = np.diag(E)
        if prev is not None:
            assert np.all(d <= prev + 1e-12)
        prev = d
    assert prev.max() < 2e-2


def test_sigma_is_invariant_under_rotation_of_the_auxiliary_index():
    n, m = 4, 6
    G = gi.random_symmetric_g(n, 2, seed=21)
    B = _random_factor(m, n, 22)
    O, _ = np.linalg.qr(np.random.default_rng(23).standard_normal((m, m)))
    Gb = osg.gbar_from_grid(G, 0)
    a = odf.sigma_df_factors(G[0], Gb, B)
    b = odf.sigma_df_factors(G[0], Gb, np.einsum("qr,rij->qij", O, B))
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()


def test_first_iteration_energy_with_the_factor_form_matches_the_closed_form():
    """GF2's first correlation energy (1/beta) sum_n Tr[G0 Sigma[G0]] with Sigma
    taken in the factor form on fitted integrals, against the finite-beta MO
    closed form evaluated on the same fitted integrals (H4 chain, 6-31G,
    m = 24): the factor form inside the whole transform and energy path."""
    import dataclasses

    from oracle import energy as oe
    from oracle import gf2 as og
    from oracle import transforms as ot
    from tests import closed_forms as cf
    coords = gi.h_chain(4, 1.7)
    s = gi.build_system("chain", coords=coords, basis="6-31g", beta=100.0, n_tau=9, n_iw=16)
    B = dfi.build_df(coords, "6-31g")
    s_df = dataclasses.replace(s, eri=odf.df_eri(B))
    r = gi.rhf(s_df)
    beta = 100.0

    def sigma_factor_form(G_tau, _eri):
        return np.array([odf.sigma_df_factors(G_tau[k], osg.gbar_from_grid(G_tau, k), B)
                         for k in range(G_tau.shape[0])])

    errs = []
    for n_tau, n_iw in ((1025, 2048), (2049, 4096)):
        F, mu, G, P = og.inner_loop(s_df, r.F, None, None, None, beta, n_iw)
        st = og.GF2State(F=F, mu=mu, P=P, G_iw=G, sig1=np.zeros_like(F), sig2=np.zeros_like(F))
        _, Sig_tau = og.self_energy_step(s_df, st, beta, n_tau, n_iw, sigma_factor_form)
        sig1, _ = ot.sigma_expansion(Sig_tau, beta)
        e2 = oe.e_two_body(G, ot.tau_to_iw(Sig_tau, beta, n_iw), sig1, s.S, beta)
        _, C, xi, _ = cf.mo_basis(F, s.S, mu, beta)
        errs.append(abs(e2 - cf.e2_first_order(cf.mo_integrals(C, s_df.eri), xi, beta)))
    # grid-limited (8.0e-7 and 8.7e-8 Eh measured): the gap closes with the grid
    assert errs[-1] < 1.5e-7 and errs[-1] < errs[0] / 4.0
