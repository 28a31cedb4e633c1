"""Pins of the oracle's multigrid warm start (appendix "Multigrid
preconditioners"): exact conditioning on coarse FVM observations (nested
volumes, Eq. subdomain-partition), then IterGP with CG actions."""
import numpy as np
import pytest

import gpfvm_workloads as W
import oracle as O

SMALL = [
    lambda: W.heat_2d(4, 4, 6, n_ic=(4, 3), n_bc=(2, 3), pred=(3, 2, 4), ell=(0.4, 0.3, 0.35)),
    lambda: W.heat_1d(8, 12, n_ic=6, n_bc=4, pred=6),
    lambda: W.wave_2d(4, 6, 4, n_ic=(3, 4), n_bc=(2, 2), pred=(2, 3, 3), ell=(0.3, 0.3, 0.3)),
]


def coarse_problem(p, factor):
    """The same IBVP discretised on the coarse cells: edges every `factor`-th
    fine edge, the noise of a sum of factor^d fine observations, the coarse
    right-hand side W^T y."""
    import copy
    c = copy.deepcopy(p)
    c.edges = [e[::factor] for e in p.edges]
    c.jitter = p.jitter * factor ** p.ndim
    if p.rhs is not None:
        c.rhs = O.restriction(p.n_cells, factor).T @ np.ravel(p.rhs)
    return c


@pytest.mark.parametrize("mk", SMALL)
def test_coarse_actions_are_the_coarse_fvm_posterior(mk):
    """No CG step: conditioning on W^T y exactly is the posterior of the coarse
    discretisation (independently assembled from coarse 1D factors)."""
    p = mk()
    K = O.KronIBVP(p)
    x, down, it, Wm, dirs = O.multigrid_itergp(K, 2, 0)
    mean, var = O.posterior_from(K, x, down)
    mc, vc = O.dense_posterior(coarse_problem(p, 2))
    np.testing.assert_allclose(mean, mc, rtol=1e-7, atol=1e-9 * np.abs(mc).max())
    np.testing.assert_allclose(var, vc, rtol=0, atol=1e-8 * p.outputscale)


@pytest.mark.parametrize("mk", SMALL)
def test_multigrid_equals_itergp_with_the_same_actions(mk):
    p = mk()
    K = O.KronIBVP(p)
    x, down, it, Wm, dirs = O.multigrid_itergp(K, 2, 6)
    mean, var = O.posterior_from(K, x, down)
    S = np.column_stack([Wm] + [d for d, _ in dirs])
    m_ref, v_ref = O.itergp_actions(K, S)
    np.testing.assert_allclose(var, v_ref, rtol=0, atol=1e-9 * p.outputscale)
    np.testing.assert_allclose(mean, m_ref, rtol=1e-7, atol=1e-9 * np.abs(m_ref).max())


@pytest.mark.parametrize("mk", SMALL)
def test_multigrid_converges_to_the_dense_posterior(mk):
    p = mk()
    K = O.KronIBVP(p)
    x, down, it, Wm, dirs = O.multigrid_itergp(K, 2, 10 * p.N, rtol=1e-12)
    mean, var = O.posterior_from(K, x, down)
    m, v = O.dense_posterior(p)
    np.testing.assert_allclose(mean, m, rtol=1e-6, atol=1e-8 * np.abs(m).max())
    assert np.all(var >= v - 1e-9)
