"""Pins of the oracle's Gram assembly, Kronecker operator and posterior against
brute-force quadrature, analytic PDE solutions and exact invariants."""
import math

import numpy as np
import pytest

import gpfvm_workloads as W
import oracle as O


# ---------------------------------------------------------------------------
# brute-force multi-dimensional quadrature of Gram entries (Eq. LkL by Fubini-free integration)
# ---------------------------------------------------------------------------
def _kder_full(r, ell, n):
    """d^n/dr^n of the 1D Matern-5/2 up to n = 4, written out for this test."""
    s = math.sqrt(5.0) / ell
    z = s * np.abs(r)
    e = np.exp(-z)
    sg = np.sign(r)
    return [
        (1 + z + z * z / 3) * e,
        -sg * s * z * (1 + z) / 3 * e,
        -s * s * (1 + z - z * z) / 3 * e,
        sg * s ** 3 * z * (3 - z) / 3 * e,
        s ** 4 * (z * z - 5 * z + 3) / 3 * e,
    ][n]


def test_kder_full_by_finite_differences():
    ell, h = 0.3, 1e-5
    for r in (-0.4, -0.1, 0.07, 0.5):
        for n in (3, 4):
            fd = (_kder_full(r + h, ell, n - 1) - _kder_full(r - h, ell, n - 1)) / (2 * h)
            assert _kder_full(r, ell, n) == pytest.approx(fd, rel=1e-6)


def _gauss_box(lo, hi, n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (hi - lo) * x + 0.5 * (hi + lo), 0.5 * (hi - lo) * w


def _brute_pde_pde(prob, cell1, cell2, n=8):
    """int_{V1} int_{V2} D_x D_x' k dx dx' by tensor Gauss-Legendre in 2d dims."""
    d = prob.ndim
    total = 0.0
    for a, ca in prob.terms:
        for b, cb in prob.terms:
            prod = ca * cb
            for i in range(d):
                e = prob.edges[i]
                x1, w1 = _gauss_box(e[cell1[i]], e[cell1[i] + 1], n)
                x2, w2 = _gauss_box(e[cell2[i]], e[cell2[i] + 1], n)
                R = x1[:, None] - x2[None, :]
                val = (-1.0) ** b[i] * _kder_full(R, prob.lengthscale[i], a[i] + b[i])
                prod *= float(w1 @ val @ w2)
            total += prod
    return prob.outputscale * total


def _brute_pde_point(prob, cell, ps, idx, n=12):
    d = prob.ndim
    total = 0.0
    for a, ca in prob.terms:
        prod = ca
        for i in range(d):
            e = prob.edges[i]
            lo, hi = e[cell[i]], e[cell[i] + 1]
            x2 = ps.coords[i][idx[i]]
            if lo < x2 < hi:  # split the rule at the kink of k at r = 0
                xa, wa = _gauss_box(lo, x2, n)
                xb, wb = _gauss_box(x2, hi, n)
                x1, w1 = np.concatenate([xa, xb]), np.concatenate([wa, wb])
            else:
                x1, w1 = _gauss_box(lo, hi, n)
            m = ps.order[i]
            val = (-1.0) ** m * _kder_full(x1 - x2, prob.lengthscale[i], a[i] + m)
            prod *= float(w1 @ val)
        total += prod
    return prob.outputscale * total


@pytest.mark.parametrize("which", ["heat", "wave"])
def test_gram_entries_by_brute_force_quadrature(which):
    if which == "heat":
        p = W.heat_2d(3, 3, 3, nu=0.07, n_ic=(3, 3), n_bc=(2, 2), pred=(2, 2, 2), ell=(0.9, 0.7, 0.8))
    else:
        p = W.wave_2d(3, 3, 3, c=0.8, n_ic=(3, 3), n_bc=(2, 2), pred=(2, 2, 2), ell=(0.9, 0.7, 0.8))
    pde = O.pde_block(p)
    G = O.block_cov(pde, pde, p.lengthscale, p.outputscale)
    shape = p.n_cells
    # separated cells: smooth integrand, Gauss-Legendre converges fast
    for c1, c2 in [((0, 0, 0), (2, 2, 2)), ((0, 2, 0), (2, 0, 2)), ((2, 0, 1), (0, 2, 1))]:
        if c1[2] == c2[2]:
            continue
        i1, i2 = np.ravel_multi_index(c1, shape), np.ravel_multi_index(c2, shape)
        bf = _brute_pde_pde(p, c1, c2)
        assert G[i1, i2] == pytest.approx(bf, rel=1e-8, abs=1e-14), (c1, c2)
    # volume x point functionals (IC value / velocity / Neumann)
    for ps in p.sets:
        B = O.block_cov(pde, O.point_block(ps), p.lengthscale, p.outputscale)
        for cell in [(1, 1, 1), (2, 0, 1)]:
            for idx in [(0, 0, 0), tuple(n - 1 for n in ps.shape)]:
                bf = _brute_pde_point(p, cell, ps, idx)
                j = np.ravel_multi_index(idx, ps.shape)
                i = np.ravel_multi_index(cell, shape)
                assert B[i, j] == pytest.approx(bf, rel=1e-8, abs=1e-13), (ps.name, cell, idx)


def test_dense_gram_symmetric_positive_definite():
    for p in [W.heat_1d(4, 6, n_ic=5, n_bc=3, pred=4),
              W.wave_2d(3, 4, 2, n_ic=(3, 3), n_bc=(2, 2), pred=(2, 2, 2), ell=(0.3, 0.3, 0.3))]:
        G = O.dense_gram(p)
        np.testing.assert_allclose(G, G.T, rtol=1e-13, atol=1e-13 * np.abs(G).max())
        assert np.linalg.eigvalsh(G).min() > 0


# ---------------------------------------------------------------------------
# posterior against analytic solutions
# ---------------------------------------------------------------------------
def test_heat_1d_converges_to_analytic_solution():
    """u_t = 0.1 u_xx, u(0,x) = sin(pi x), zero Dirichlet: u = exp(-0.1 pi^2 t) sin(pi x)."""
    errs = []
    for nt, nx in [(4, 8), (8, 16), (16, 32)]:
        p = W.heat_1d(nt, nx, n_ic=nx, n_bc=nt, pred=33)
        m, v = O.dense_posterior(p)
        T, X = np.meshgrid(p.pred[0], p.pred[1], indexing="ij")
        ex = np.exp(-0.1 * np.pi ** 2 * T) * np.sin(np.pi * X)
        errs.append(np.sqrt(np.mean((m - ex.ravel()) ** 2)))
        assert v.min() > -1e-12
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 2e-3


def test_fig2_toy_recovers_sine():
    """Fig. 2: du/dx = cos x on [0, 2 pi], u(0) = u(2 pi) = 0 -> u = sin x."""
    errs = []
    for n in (4, 8, 16, 32):
        p = W.toy_cos(n, ell=1.0)
        m, v = O.dense_posterior(p)
        errs.append(np.abs(m - np.sin(p.pred[0])).max())
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[3] < 2e-3


def test_wave_benchmark_separation_of_variables():
    """App. C.3 wave benchmark: u = sum C_ij sin(i pi x) sin(j pi y) cos(c pi sqrt(i^2+j^2) t)."""
    errs = []
    for n in (2, 4, 6):
        p = W.wave_2d_sine(n, n, n, n_ic=8, n_bc=(8, 4), pred=(7, 7, 7), ell=(0.5, 0.3, 0.3))
        m, v = O.dense_posterior(p)
        C = p.meta["C"]
        T, X, Y = np.meshgrid(*p.pred, indexing="ij")
        ex = np.zeros_like(T)
        for i in range(2):
            for j in range(2):
                ex += (C[i, j] * np.sin((i + 1) * np.pi * X) * np.sin((j + 1) * np.pi * Y) *
                       np.cos(np.pi * math.sqrt((i + 1) ** 2 + (j + 1) ** 2) * T))
        errs.append(np.sqrt(np.mean((m - ex.ravel()) ** 2)))
    assert errs[0] > errs[1] > errs[2]


def test_posterior_satisfies_observations():
    """Sec. 2.2/3: posterior paths satisfy the observations, so L[m*] = y - Sigma G^-1 y."""
    p = W.heat_1d(6, 8, n_ic=8, n_bc=6, pred=5)
    G = O.dense_gram(p)
    y = O.observations(p)
    alpha = np.linalg.solve(G, y)
    Lm = (G - np.diag(O.noise_diag(p))) @ alpha
    np.testing.assert_allclose(Lm, y - O.noise_diag(p) * alpha, atol=1e-10)
    assert np.abs(Lm - y).max() < 1e-5
    # the posterior mean at the IC points interpolates the data
    pp = W.heat_1d(6, 8, n_ic=8, n_bc=6, pred=5)
    pp.pred = [np.array([0.0]), p.sets[0].coords[1]]
    m, v = O.dense_posterior(pp)
    np.testing.assert_allclose(m, p.sets[0].values, atol=1e-5)
    assert np.abs(v).max() < 1e-6


# ---------------------------------------------------------------------------
# Kronecker operator, deflation and IterGP against the dense path
# ---------------------------------------------------------------------------
SMALL = [
    lambda: W.heat_1d(5, 7, n_ic=6, n_bc=4, pred=6),
    lambda: W.heat_2d(3, 4, 5, n_ic=(4, 3), n_bc=(2, 3), pred=(3, 2, 4), ell=(0.4, 0.3, 0.35)),
    lambda: W.wave_2d(4, 3, 5, n_ic=(3, 4), n_bc=(2, 2), pred=(2, 3, 3), ell=(0.3, 0.3, 0.3)),
    lambda: W.toy_cos(9),
]


@pytest.mark.parametrize("mk", SMALL)
def test_kron_blocks_equal_dense_blocks(mk):
    p = mk()
    K = O.KronIBVP(p)
    G = O.dense_gram(p)
    M, N = p.M, p.N
    rng = np.random.default_rng(1)
    v = rng.normal(size=N)
    w = rng.normal(size=M)
    scale = np.abs(G).max()
    np.testing.assert_allclose(K.Gpp(v), G[M:, M:] @ v, rtol=1e-12, atol=1e-13 * scale * np.abs(v).sum())
    np.testing.assert_allclose(K.Gbp(v), G[:M, M:] @ v, rtol=1e-12, atol=1e-13 * scale * np.abs(v).sum())
    np.testing.assert_allclose(K.Gpb(w), G[M:, :M] @ w, rtol=1e-12, atol=1e-13 * scale * np.abs(w).sum())
    np.testing.assert_allclose(K.Gbb, G[:M, :M], rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("mk", SMALL)
def test_deflated_cg_mean_equals_cholesky(mk):
    """Cholesky (IC/BC) deflation + CG gives the dense Cholesky posterior mean
    (Sec. 4.2: the block elimination is exact), and its IterGP variance is an
    upper bound of the exact variance."""
    p = mk()
    m, v = O.dense_posterior(p)
    # stop at convergence (rtol 1e-13): past it the directions are rounding noise
    r = O.kron_posterior(p, max_iter=10 * p.N, rtol=1e-13)
    np.testing.assert_allclose(r["mean"], m, rtol=1e-7, atol=1e-8 * np.abs(m).max())
    assert np.all(r["var"] >= v - 1e-9)


@pytest.mark.parametrize("mk", SMALL)
def test_itergp_unit_actions_equal_cholesky(mk):
    """IterGP with unit-vector actions is the Cholesky posterior (Sec. 4.2),
    mean and variance, on the deflated system."""
    p = mk()
    m, v = O.dense_posterior(p)
    K = O.KronIBVP(p)
    mean, var = O.itergp_actions(K, np.eye(p.N))
    np.testing.assert_allclose(mean, m, rtol=1e-7, atol=1e-8 * np.abs(m).max())
    np.testing.assert_allclose(var, v, atol=1e-8 * p.outputscale)


@pytest.mark.parametrize("mk", SMALL[1:3])
def test_cg_downdate_equals_general_itergp_with_cg_actions(mk):
    """With (reorthogonalised) CG directions as actions, the general IterGP
    downdate S (S^T G S)^-1 S^T equals sum_j p_j p_j^T / eta_j."""
    p = mk()
    K = O.KronIBVP(p)
    dirs = []
    x, down, it, hist = O.cg_itergp(K, 12, 0.0, True, True, dirs)
    S = np.column_stack([d for d, _ in dirs])
    mean, var = O.itergp_actions(K, S)
    r = O.kron_posterior(p, max_iter=12, rtol=0.0, K=K)
    np.testing.assert_allclose(r["var"], var, atol=1e-9)
    np.testing.assert_allclose(r["mean"], mean, rtol=1e-6, atol=1e-8)


def test_itergp_variance_bounds_and_monotone():
    """Combined posterior variance >= exact variance and non-increasing in iterations."""
    p = W.heat_2d(4, 5, 4, n_ic=(4, 4), n_bc=(2, 2), pred=(3, 3, 3), ell=(0.4, 0.3, 0.3))
    m, v = O.dense_posterior(p)
    prev = None
    for it in (1, 5, 20, 60, p.N):
        r = O.kron_posterior(p, max_iter=it, rtol=1e-13)
        assert np.all(r["var"] >= v - 1e-9)
        if prev is not None:
            assert np.all(r["var"] <= prev + 1e-12)
        prev = r["var"]


def test_no_reorth_variance_breaks_down():
    """Without reorthogonalisation the sum over directions overshoots (the
    reason for the paper's stabilisation, Sec. 7); with it the bound holds."""
    p = W.heat_1d()
    m, v = O.dense_posterior(p)
    bad = O.kron_posterior(p, max_iter=300, rtol=0.0, reorth=False)
    good = O.kron_posterior(p, max_iter=300, rtol=0.0, reorth=True)
    assert (bad["var"] - v).min() < -1e-3
    assert (good["var"] - v).min() > -1e-9
