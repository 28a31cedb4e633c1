"""Pins of the collocation observations (Sec. 3: the collocation operator
L_x[u] = D[u](x), compared with FVM in Fig. 2 and App. C.3): the third and
fourth kernel derivatives, order-2 point covariances, and collocation
posteriors that converge to analytic PDE solutions."""
import math

import numpy as np
import pytest
import scipy.integrate as si

import gpfvm_workloads as W
import oracle as O


@pytest.mark.parametrize("ell", [0.1, 0.4, 1.3])
def test_third_and_fourth_derivatives_by_finite_differences(ell):
    r = np.concatenate([np.linspace(-3 * ell, -0.02 * ell, 40), np.linspace(0.02 * ell, 3 * ell, 40)])
    h = 1e-5 * ell
    for order in (3, 4):
        fd = (O.kderiv(r + h, ell, order - 1) - O.kderiv(r - h, ell, order - 1)) / (2 * h)
        ref = O.kderiv(r, ell, order)
        scale = np.abs(ref).max()
        np.testing.assert_allclose(ref, fd, rtol=0, atol=1e-6 * scale)
    # continuity at 0: k''' is odd and vanishes, k'''' is even
    eps = 1e-9 * ell
    assert abs(O.kderiv(eps, ell, 3)) < 1e-6 * (math.sqrt(5) / ell) ** 3
    assert abs(O.kderiv(eps, ell, 4) - O.kderiv(-eps, ell, 4)) < 1e-9 * (math.sqrt(5) / ell) ** 4


@pytest.mark.parametrize("ell", [0.2, 1.0])
def test_fourth_spectral_moment(ell):
    """k''''(0) = int w^4 S(w) dw / int S(w) dw for the Matern-5/2 spectral
    density S(w) ~ (5/ell^2 + w^2)^-3 (Var u'' of the prior)."""
    a2 = 5.0 / ell ** 2
    S = lambda w, p: w ** p * (a2 + w * w) ** -3
    m0 = si.quad(S, -np.inf, np.inf, args=(0,))[0]
    m4 = si.quad(S, -np.inf, np.inf, args=(4,))[0]
    assert abs(O.kderiv(0.0, ell, 4) - m4 / m0) <= 1e-8 * m4 / m0


def test_order2_point_covariance_by_finite_differences():
    """cov(u''(x), u''(x')) = d^2/dx^2 d^2/dx'^2 k(x - x'), by central differences
    of the kernel in both arguments."""
    ell = 0.5
    x = np.array([0.1, 0.35, 0.8])
    xp = np.array([0.2, 0.5])
    C = O.cov_1d(O.point_family(x, 2), O.point_family(xp, 2), ell)

    def fd(h):
        st = [(1.0, -h), (-2.0, 0.0), (1.0, h)]
        acc = np.zeros((x.size, xp.size))
        for wa, da in st:
            for wb, db in st:
                acc += wa * wb * O.kderiv((x[:, None] + da) - (xp[None, :] + db), ell, 0)
        return acc / h ** 4
    rich = (4.0 * fd(2e-3) - fd(4e-3)) / 3.0  # Richardson: O(h^4) truncation
    np.testing.assert_allclose(C, rich, rtol=2e-5)
    # mixed order (u'' with u') has the sign (-1)^n of the second argument's order
    C21 = O.cov_1d(O.point_family(x, 2), O.point_family(xp, 1), ell)
    np.testing.assert_allclose(C21, -O.kderiv(x[:, None] - xp[None, :], ell, 3), rtol=1e-14)


def test_fig2_toy_by_collocation_recovers_sine():
    """du/dx = cos x, u(0) = u(2 pi) = 0 observed at cell centres: the
    posterior mean approaches sin x as the points are refined (Fig. 2)."""
    errs = []
    for n in (6, 12, 24):
        p = W.toy_cos(n, observe="collocation")
        m, v = O.dense_posterior(p)
        errs.append(np.abs(m - np.sin(p.pred[0])).max())
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-2
    # and FVM does better at equal counts (the paper's comparison, Fig. 2 / Sec. 6.1)
    q = W.toy_cos(24)
    m_fvm, _ = O.dense_posterior(q)
    assert np.abs(m_fvm - np.sin(q.pred[0])).max() < errs[2]


def _problem_1d(n, terms, rhs_fn, sets, ell=0.3):
    e = np.linspace(0, 1, n + 1)
    mid = 0.5 * (e[1:] + e[:-1])
    return W.Problem([e], (ell,), 1.0, terms, 1e-10, sets, [np.linspace(0, 1, 21)],
                     rhs=None if rhs_fn is None else rhs_fn(mid), observe="collocation")


def test_ode_by_collocation_converges():
    """u' + u = 0, u(0) = 1 observed at cell centres: the mean approaches e^-t."""
    ic = W.PointSet((0,), [np.array([0.0])], np.ones(1), 1e-10, "ic")
    errs = []
    for n in (8, 16, 32):
        p = _problem_1d(n, [((1,), 1.0), ((0,), 1.0)], None, [ic])
        m, _ = O.dense_posterior(p)
        errs.append(np.abs(m - np.exp(-p.pred[0])).max())
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-3


def test_poisson_by_collocation_converges():
    """u'' = -pi^2 sin(pi x), u(0) = u(1) = 0 at cell centres (second
    derivatives of the Matern-5/2 prior, the fourth kernel derivative): the
    error to sin(pi x) falls under refinement."""
    bc = W.PointSet((0,), [np.array([0.0, 1.0])], np.zeros(2), 1e-10, "bc")
    errs = []
    for n in (8, 16, 32, 64):
        p = _problem_1d(n, [((2,), 1.0)], lambda x: -np.pi ** 2 * np.sin(np.pi * x), [bc])
        m, _ = O.dense_posterior(p)
        errs.append(np.abs(m - np.sin(np.pi * p.pred[0])).max())
    assert all(a > b for a, b in zip(errs, errs[1:])) and errs[-1] < 0.1


def test_heat_collocation_gram_entries_by_finite_differences():
    """cov(D u(p), D u(p')) for D = d_t - nu d_xx of the 2D product kernel,
    by central differences of k_t(t - t') k_x(x - x') in all four variables,
    against the collocation Gram block.  Off-diagonal entries only: at r = 0
    the fifth derivative of Matern-5/2 jumps, so a difference quotient across
    it is first-order accurate; the fourth derivative at 0 is pinned by the
    spectral moment instead."""
    p = W.collocation(W.heat_1d(3, 4, n_ic=3, n_bc=2, pred=3, ell=(0.5, 0.4)))
    nu = 0.1
    G = O.block_cov(O.pde_block(p), O.pde_block(p), p.lengthscale, p.outputscale)
    tc = 0.5 * (p.edges[0][1:] + p.edges[0][:-1])
    xc = 0.5 * (p.edges[1][1:] + p.edges[1][:-1])
    lt, lx = p.lengthscale

    def k(t, x, tp, xp):
        return O.kderiv(t - tp, lt, 0) * O.kderiv(x - xp, lx, 0)

    def D(f, h=1e-3):  # D acting on the first point
        return lambda t, x, tp, xp: ((f(t + h, x, tp, xp) - f(t - h, x, tp, xp)) / (2 * h)
                                     - nu * (f(t, x + h, tp, xp) - 2 * f(t, x, tp, xp) + f(t, x - h, tp, xp)) / h ** 2)

    def Dp(f, h=1e-3):  # the same on the second point
        return lambda t, x, tp, xp: ((f(t, x, tp + h, xp) - f(t, x, tp - h, xp)) / (2 * h)
                                     - nu * (f(t, x, tp, xp + h) - 2 * f(t, x, tp, xp) + f(t, x, tp, xp - h)) / h ** 2)
    DD = Dp(D(k))
    idx = [(0, 1), (2, 3), (1, 0)]
    for a in idx:
        for b in idx:
            if a == b:
                continue
            i = a[0] * xc.size + a[1]
            j = b[0] * xc.size + b[1]
            ref = DD(tc[a[0]], xc[a[1]], tc[b[0]], xc[b[1]])
            assert abs(G[i, j] - ref) <= 2e-4 * max(abs(G).max(), 1.0), (a, b, G[i, j], ref)


COLLOC = [
    lambda: W.collocation(W.heat_1d(5, 7, n_ic=6, n_bc=4, pred=6)),
    lambda: W.collocation(W.heat_2d(3, 4, 5, n_ic=(4, 3), n_bc=(2, 3), pred=(3, 2, 4), ell=(0.4, 0.3, 0.35))),
    lambda: W.collocation(W.wave_2d(4, 3, 5, n_ic=(3, 4), n_bc=(2, 2), pred=(2, 3, 3), ell=(0.3, 0.3, 0.3))),
    lambda: W.toy_cos(9, observe="collocation"),
]


@pytest.mark.parametrize("mk", COLLOC)
def test_collocation_kron_blocks_equal_dense_blocks(mk):
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
    # the deflated CG reaches the dense Cholesky posterior
    m, var = O.dense_posterior(p)
    r = O.kron_posterior(p, max_iter=10 * p.N, rtol=1e-13)
    np.testing.assert_allclose(r["mean"], m, rtol=1e-6, atol=1e-8 * np.abs(m).max())
