"""Pins of the oracle's multi-output posterior (Sec. 3.3, multi-dimensional
codomains: independent priors per output, operators summing derivatives of
several components), against things other than itself:

* a system of two decoupled equations is the pair of one-output posteriors;
* an output that no observation touches keeps its prior;
* the first-order form of the 1D wave equation (u_t + v_x = 0, v_t + u_x = 0)
  converges to its analytic solution under refinement, which fails if a term
  acts on the wrong component."""
from dataclasses import replace

import numpy as np
import pytest

import gpfvm_workloads as W
import oracle as O


def _system_of(a, b):
    """The two one-output problems a, b (same cells, kernel, grid) as one
    two-output system: equation 0 = a's PDE on u_0, equation 1 = b's on u_1."""
    sets = [replace(s, out=0) for s in a.sets] + [replace(s, out=1) for s in b.sets]
    terms = list(a.terms) + list(b.terms)
    eq = [0] * len(a.terms) + [1] * len(b.terms)
    return replace(a, terms=terms, sets=sets, n_out=2, term_eq=eq, term_out=list(eq), name="pair")


def test_decoupled_system_is_the_pair_of_single_posteriors():
    a = W.heat_1d(5, 6, nu=0.05, n_ic=5, n_bc=3, pred=5)
    b = W.heat_1d(5, 6, nu=0.2, n_ic=5, n_bc=3, pred=5)
    b = replace(b, sets=[replace(s, values=np.cos(np.arange(s.size))) for s in b.sets])
    ma, va = O.dense_posterior(a)
    mb, vb = O.dense_posterior(b)
    sysp = _system_of(a, b)
    assert sysp.N == a.N + b.N and sysp.P == a.P + b.P
    m, v = O.dense_posterior(sysp)
    P = a.P
    np.testing.assert_allclose(m[:P], ma, rtol=0, atol=1e-10 * max(1.0, np.abs(ma).max()))
    np.testing.assert_allclose(m[P:], mb, rtol=0, atol=1e-10 * max(1.0, np.abs(mb).max()))
    np.testing.assert_allclose(v[:P], va, rtol=0, atol=1e-10)
    np.testing.assert_allclose(v[P:], vb, rtol=0, atol=1e-10)


def test_unobserved_output_keeps_its_prior():
    a = W.heat_1d(5, 6, nu=0.1, n_ic=5, n_bc=3, pred=5)
    sysp = replace(a, n_out=2, term_eq=[0] * len(a.terms), term_out=[0] * len(a.terms))
    m, v = O.dense_posterior(sysp)
    ma, va = O.dense_posterior(a)
    P = a.P
    np.testing.assert_allclose(m[:P], ma, rtol=0, atol=1e-12)
    np.testing.assert_allclose(v[:P], va, rtol=0, atol=1e-12)
    assert np.all(m[P:] == 0.0)
    np.testing.assert_allclose(v[P:], a.outputscale, rtol=0, atol=1e-14)


@pytest.mark.parametrize("swap", [False, True])
def test_first_order_wave_system_converges_to_the_analytic_solution(swap):
    """u = sin(pi x) cos(pi t), v = -cos(pi x) sin(pi t).  With the components of
    equation 1 swapped (a plausible indexing mistake) the posterior does not
    approach that solution."""
    errs = []
    for n in (4, 8, 16):
        p = W.wave_1d_system(n, n, pred=(9, 9), ell=(0.5, 0.3))
        if swap:
            p = replace(p, term_out=[0, 1, 0, 1])
        m, _ = O.dense_posterior(p)
        T, X = np.meshgrid(p.pred[0], p.pred[1], indexing="ij")
        u = np.sin(np.pi * X) * np.cos(np.pi * T)
        v = -np.cos(np.pi * X) * np.sin(np.pi * T)
        P = T.size
        errs.append(max(np.abs(m[:P] - u.ravel()).max(), np.abs(m[P:] - v.ravel()).max()))
    if swap:
        assert errs[-1] > 0.1
    else:
        assert errs[0] > errs[1] > errs[2]
        assert errs[2] < 1e-3


def test_multi_output_blocks_zero_across_components():
    """Cross-covariances between observations of different outputs vanish
    (Eq. multioutput-cov-def); within one output they are the one-output ones."""
    p = W.wave_1d_system(4, 5)
    ic_u, ic_v = (O.point_block(s) for s in p.sets[:2])
    assert np.all(O.block_cov(ic_u, ic_v, p.lengthscale, p.outputscale) == 0.0)
    K = O.block_cov(ic_u, ic_u, p.lengthscale, p.outputscale)
    K1 = O.block_cov(O.point_block(replace(p.sets[0], out=1)), ic_v, p.lengthscale, p.outputscale)
    np.testing.assert_array_equal(K, K1)
    eq0, eq1 = O.pde_blocks(p)
    assert eq0.outs == [0, 1] and eq1.outs == [1, 0]


@pytest.mark.parametrize("swap", [False, True])
def test_shallow_water_standing_wave(swap):
    """Three outputs, three equations (linearised shallow water, f = k = 0):
    the posterior approaches h = cos(pi x) cos(w t), u = sqrt(g/H) sin(pi x)
    sin(w t), v = 0 (w = pi sqrt(g H)) under refinement; with the pressure
    term g h_x made to act on v instead of h it does not."""
    H, g = 1.0, 1.0
    errs = []
    for n in (4, 6, 8):
        p = W.shallow_water_2d(n, n, n, H=H, g=g, f=0.0, k=0.0, n_ic=(n + 1, n + 1), n_bc=(n, n), pred=(5, 5, 3),
                               ell=(0.4, 0.3, 0.5), jitter=1e-10, standing=True)
        if swap:
            outs = list(p.term_out)
            k = next(i for i, (a, c) in enumerate(p.terms) if a == (0, 1, 0) and p.term_eq[i] == 1)
            assert outs[k] == 0  # g h_x in the u equation
            outs[k] = 2
            p = replace(p, term_out=outs)
        m, _ = O.dense_posterior(p)
        T, X, Y = np.meshgrid(*p.pred, indexing="ij")
        w = np.pi * np.sqrt(g * H)
        exact = np.concatenate([(np.cos(np.pi * X) * np.cos(w * T)).ravel(),
                                (np.sqrt(g / H) * np.sin(np.pi * X) * np.sin(w * T)).ravel(), np.zeros(T.size)])
        errs.append(np.abs(m - exact).max())
    if swap:
        assert errs[-1] > 0.05
    else:
        assert errs[0] > errs[1] > errs[2]
        assert errs[2] < 1e-2


@pytest.mark.parametrize("make", [lambda: W.wave_1d_system(5, 6, pred=(4, 5)),
                                  lambda: W.shallow_water_2d(3, 4, 5, n_ic=(3, 4), n_bc=(2, 2), pred=(2, 3, 3)),
                                  lambda: W.collocation(W.wave_1d_system(4, 5, pred=(3, 4)))])
def test_kron_operator_of_systems_equals_dense_blocks(make):
    p = make()
    K = O.KronIBVP(p)
    cov = lambda X, Y: O.block_cov(X, Y, p.lengthscale, p.outputscale)  # noqa: E731
    eqs = O.pde_blocks(p)
    sets = [O.point_block(s) for s in p.sets]
    preds = O.pred_blocks(p)
    Gpp = np.vstack([np.hstack([cov(X, Y) for Y in eqs]) for X in eqs])
    Gbp = np.vstack([np.hstack([cov(S, Y) for Y in eqs]) for S in sets])
    Kp = np.vstack([np.hstack([cov(X, Q) for Q in preds]) for X in eqs])
    Kb = np.vstack([np.hstack([cov(S, Q) for Q in preds]) for S in sets])
    rng = np.random.default_rng(3)
    v, w, b = rng.normal(size=p.N), rng.normal(size=p.M), rng.normal(size=p.P)
    close = lambda a, ref: np.testing.assert_allclose(a, ref, rtol=0, atol=1e-12 * np.abs(ref).max())  # noqa: E731
    close(K.Gpp(v), Gpp @ v + p.jitter * v)
    close(K.Gbp(v), Gbp @ v)
    close(K.Gpb(w), Gbp.T @ w)
    close(K.KPx(v), Kp.T @ v)
    close(K.KBx(w), Kb.T @ w)
    close(K.KPxT(b), Kp @ b)
    close(K.KBxT(b), Kb @ b)
    close(K.KB_dense(), Kb)


def test_kron_posterior_of_a_system_equals_the_dense_posterior():
    p = W.shallow_water_2d(3, 4, 5, n_ic=(3, 4), n_bc=(2, 2), pred=(2, 3, 3))
    m, v = O.dense_posterior(p)
    r = O.kron_posterior(p, rtol=1e-13)
    assert np.linalg.norm(r["mean"] - m) / np.linalg.norm(m) < 1e-9
    assert np.all(r["var"] >= v - 1e-9)


def test_system_with_a_constant_depth_field_equals_constant_depth():
    """App. C.4's bathymetry enters the h equation as a per-cell field on its two
    velocity terms; a field equal to H everywhere gives the constant-depth system
    (dense and Kronecker oracles), a varying one a different posterior."""
    kw = dict(n_ic=(3, 4), n_bc=(2, 2), pred=(2, 3, 3), H=0.8)
    p = W.shallow_water_2d(3, 4, 5, **kw)
    q = W.shallow_water_2d(3, 4, 5, depth=np.full((4, 5), 0.8), **kw)
    assert sum(f is not None for f in q.fields) == 2
    m, v = O.dense_posterior(p)
    mq, vq = O.dense_posterior(q)
    np.testing.assert_allclose(mq, m, rtol=0, atol=1e-12 * np.abs(m).max())
    np.testing.assert_allclose(vq, v, rtol=0, atol=1e-12)
    K, Kq = O.KronIBVP(p), O.KronIBVP(q)
    x = np.random.default_rng(1).normal(size=p.N)
    np.testing.assert_allclose(Kq.Ghat(x), K.Ghat(x), rtol=0, atol=1e-12 * np.abs(K.Ghat(x)).max())
    X, Y = np.meshgrid(np.linspace(0, 1, 4), np.linspace(0, 1, 5), indexing="ij")
    r = W.shallow_water_2d(3, 4, 5, depth=0.5 + 0.5 * X * Y, **kw)
    mr, _ = O.dense_posterior(r)
    assert np.abs(mr - m).max() > 1e-4
    # Kronecker-with-diagonals == entrywise dense blocks for the varying field too
    Kr = O.KronIBVP(r)
    eqs = O.pde_blocks(r)
    Gpp = np.vstack([np.hstack([O.block_cov(A, B, r.lengthscale, r.outputscale) for B in eqs]) for A in eqs])
    np.testing.assert_allclose(Kr.Gpp(x), Gpp @ x + r.jitter * x, rtol=0, atol=1e-12 * np.abs(Gpp @ x).max())
