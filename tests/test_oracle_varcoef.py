"""Pins of the oracle's variable coefficients (App. C.4 "Variable
bathymetry": a piecewise-constant coefficient per cell makes every Kronecker
term of the Gram matrix a Hadamard product with a rank-one matrix)."""
import numpy as np
import pytest

import gpfvm_workloads as W
import oracle as O

SMALL = [
    lambda: W.heat_1d_varcoef(4, 6, pred=5),
    lambda: W.heat_2d_varcoef(3, 4, 5, n_ic=(4, 3), n_bc=(2, 3), pred=(3, 2, 4), ell=(0.4, 0.3, 0.35)),
]


@pytest.mark.parametrize("mk", SMALL)
def test_kronecker_with_diagonals_equals_dense_blocks(mk):
    p = mk()
    K = O.KronIBVP(p)
    G = O.dense_gram(p)
    M, N = p.M, p.N
    rng = np.random.default_rng(2)
    v, w = rng.normal(size=N), rng.normal(size=M)
    scale = np.abs(G).max()
    np.testing.assert_allclose(K.Gpp(v), G[M:, M:] @ v, rtol=1e-12, atol=1e-13 * scale * np.abs(v).sum())
    np.testing.assert_allclose(K.Gbp(v), G[:M, M:] @ v, rtol=1e-12, atol=1e-13 * scale * np.abs(v).sum())
    np.testing.assert_allclose(K.Gpb(w), G[M:, :M] @ w, rtol=1e-12, atol=1e-13 * scale * np.abs(w).sum())
    KP = O.block_cov(O.pde_block(p), O.pred_block(p), p.lengthscale, p.outputscale)
    beta = rng.normal(size=KP.shape[1])
    np.testing.assert_allclose(K.KPx(v), KP.T @ v, rtol=1e-12, atol=1e-13 * np.abs(KP).max() * np.abs(v).sum())
    np.testing.assert_allclose(K.KPxT(beta), KP @ beta, rtol=1e-12,
                               atol=1e-13 * np.abs(KP).max() * np.abs(beta).sum())
    # the Gram block is the Hadamard product of each Kronecker term with c_a c_b^T
    Gpp = np.zeros((N, N))
    for (ca, Fa) in O.pde_block(p).terms:
        for (cb, Fb) in O.pde_block(p).terms:
            kr = np.ones((1, 1))
            for i in range(p.ndim):
                kr = np.kron(kr, O.cov_1d(Fa[i], Fb[i], p.lengthscale[i]))
            Gpp += np.outer(np.broadcast_to(ca, (N,)), np.broadcast_to(cb, (N,))) * kr
    np.testing.assert_allclose(p.outputscale * Gpp + p.jitter * np.eye(N), G[M:, M:], rtol=1e-12,
                               atol=1e-13 * scale)


def test_constant_field_equals_scalar_coefficient():
    a = W.heat_2d(3, 4, 5, n_ic=(4, 3), n_bc=(2, 3), pred=(3, 2, 4), ell=(0.4, 0.3, 0.35), nu=0.05)
    b = W.heat_2d(3, 4, 5, n_ic=(4, 3), n_bc=(2, 3), pred=(3, 2, 4), ell=(0.4, 0.3, 0.35), nu=0.05)
    b.terms = [((1, 0, 0), 1.0), ((0, 2, 0), -1.0), ((0, 0, 2), -1.0)]
    f = np.full(b.N, 0.05)
    b.fields = [None, f, f]
    np.testing.assert_allclose(O.dense_gram(b), O.dense_gram(a), rtol=1e-14, atol=1e-15)


def test_manufactured_variable_coefficient_heat_solution():
    """u_t = nu(x) u_xx with piecewise-constant nu and a right-hand side built
    from u* = exp(-t) sin(pi x): the posterior mean approaches u* under refinement."""
    errs = []
    for nt, nx in ((4, 8), (8, 16), (16, 32)):
        p = W.heat_1d_varcoef(nt, nx)
        m, _ = O.dense_posterior(p)
        T, X = np.meshgrid(p.pred[0], p.pred[1], indexing="ij")
        errs.append(np.abs(m - (np.exp(-T) * np.sin(np.pi * X)).ravel()).max())
    assert errs[0] > errs[1] > errs[2] and errs[2] < 5e-3


@pytest.mark.parametrize("mk", SMALL)
def test_varcoef_deflated_cg_equals_cholesky(mk):
    p = mk()
    m, v = O.dense_posterior(p)
    r = O.kron_posterior(p, max_iter=10 * p.N, rtol=1e-13)
    np.testing.assert_allclose(r["mean"], m, rtol=1e-6, atol=1e-8 * np.abs(m).max())
    assert np.all(r["var"] >= v - 1e-9)
