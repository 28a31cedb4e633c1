"""Pins of the oracle's targeted uncertainty reduction (appendix "Targeted
uncertainty reduction"): the adjoint cross-covariance products, the deflated
cross-covariance against entrywise dense blocks, the targeted IterGP update
against the general IterGP posterior for the same actions, a closed form for a
single action, and convergence to the exact variance at a target point."""
import numpy as np
import pytest
import scipy.linalg as sla

import gpfvm_workloads as W
import oracle as O

SMALL = [
    lambda: W.heat_1d(5, 7, n_ic=6, n_bc=4, pred=6),
    lambda: W.heat_2d(3, 4, 5, n_ic=(4, 3), n_bc=(2, 3), pred=(3, 2, 4), ell=(0.4, 0.3, 0.35)),
    lambda: W.wave_2d(4, 3, 5, n_ic=(3, 4), n_bc=(2, 2), pred=(2, 3, 3), ell=(0.3, 0.3, 0.3)),
]


def _targets(p, k, seed=0):
    """k Dir(1, ..., 1) weight vectors over the points of the last time slice
    of the prediction grid (zero elsewhere)."""
    shape = tuple(len(g) for g in p.pred)
    mask = np.zeros(shape, bool)
    mask[-1] = True
    idx = np.flatnonzero(mask.ravel())
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(k):
        b = np.zeros(int(np.prod(shape)))
        b[idx] = rng.dirichlet(np.ones(idx.size))
        out.append(b)
    return out


@pytest.mark.parametrize("mk", SMALL)
def test_adjoint_cross_covariance_products(mk):
    p = mk()
    K = O.KronIBVP(p)
    rng = np.random.default_rng(3)
    x, w, beta = rng.normal(size=p.N), rng.normal(size=p.M), rng.normal(size=K.pred.size)
    assert abs(K.KPx(x) @ beta - x @ K.KPxT(beta)) <= 1e-12 * np.linalg.norm(K.KPx(x)) * np.linalg.norm(beta)
    assert abs(K.KBx(w) @ beta - w @ K.KBxT(beta)) <= 1e-12 * np.linalg.norm(K.KBx(w)) * np.linalg.norm(beta)


@pytest.mark.parametrize("mk", SMALL)
def test_lhat_k_equals_dense_blocks(mk):
    """Lhat k(X*) beta against L_PDE k(X*) - G_PB G_BB^-1 L_B k(X*) assembled
    entry by entry from the 1D closed forms (block_cov), not by Kronecker products."""
    p = mk()
    K = O.KronIBVP(p)
    G = O.dense_gram(p)
    M = p.M
    KP = O.block_cov(O.pde_block(p), O.pred_block(p), p.lengthscale, p.outputscale)
    KB = K.KB_dense()
    Lhat = KP - G[M:, :M] @ np.linalg.solve(G[:M, :M], KB)
    beta = np.random.default_rng(4).normal(size=K.pred.size)
    ref = Lhat @ beta
    np.testing.assert_allclose(K.Lhat_k(beta), ref, rtol=1e-9, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("mk", SMALL[1:])
def test_targeted_equals_itergp_with_the_same_actions(mk):
    """After CG, the targeted actions give the IterGP posterior of the action
    matrix [CG directions | targeted actions] (C = S (S^T G^ S)^-1 S^T)."""
    p = mk()
    K = O.KronIBVP(p)
    betas = _targets(p, 5)
    x, down, acts, dirs = O.targeted_itergp(K, 8, 0.0, betas)
    mean, var = O.posterior_from(K, x, down)
    S = np.column_stack([d for d, _ in dirs] + acts)
    m_ref, v_ref = O.itergp_actions(K, S)
    np.testing.assert_allclose(var, v_ref, atol=1e-9 * p.outputscale)
    np.testing.assert_allclose(mean, m_ref, rtol=1e-7, atol=1e-9 * np.abs(m_ref).max())
    # the targeted actions lower the variance (never below the exact one)
    m_ex, v_ex = O.dense_posterior(p)
    _, v_cg = O.posterior_from(K, *O.cg_itergp(K, 8, 0.0, True, True)[:2])
    assert np.all(var <= v_cg + 1e-12) and np.all(var >= v_ex - 1e-9)


def test_single_action_closed_form():
    """No CG directions and one action on one point x~: the action is
    t = Lhat k(x~) itself, and the variance at x~ drops by (t.t)^2 / (t.G^ t)."""
    p = SMALL[1]()
    K = O.KronIBVP(p)
    m = 5
    beta = np.zeros(K.pred.size)
    beta[m] = 1.0
    x, down, acts, dirs = O.targeted_itergp(K, 0, 0.0, [beta])
    t = K.Lhat_k(beta)
    np.testing.assert_allclose(acts[0], t, rtol=1e-14)
    np.testing.assert_allclose(down[m], (t @ t) ** 2 / (t @ K.Ghat(t)), rtol=1e-12)


def test_repeated_actions_reach_the_exact_variance_at_the_target():
    """Actions on one target point are CG on G^ z = Lhat k(x~): once it has
    converged the variance there is the exact (dense Cholesky) one."""
    p = W.heat_2d(3, 3, 4, n_ic=(3, 3), n_bc=(2, 2), pred=(2, 3, 3), ell=(0.5, 0.4, 0.4), jitter=1e-4)
    K = O.KronIBVP(p)
    m = K.pred.size - 2
    beta = np.zeros(K.pred.size)
    beta[m] = 1.0
    m_ex, v_ex = O.dense_posterior(p)
    x, down, acts, dirs = O.targeted_itergp(K, 0, 0.0, [beta] * 20)
    _, var = O.posterior_from(K, x, down)
    assert abs(var[m] - v_ex[m]) <= 1e-9 * p.outputscale
    # and each action lowered the variance at x~
    x1, d1, _, _ = O.targeted_itergp(K, 0, 0.0, [beta] * 3)
    assert O.posterior_from(K, x1, d1)[1][m] >= var[m] - 1e-12
