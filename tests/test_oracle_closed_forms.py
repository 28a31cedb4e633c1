"""Pins of the oracle's 1D Matern-5/2 closed forms and 1D functional covariances
against quadrature, finite differences and known integrals (Sec. 3.1)."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O
from oracle import gpfvm_oracle as OO

ELLS = [0.05, 0.2, 1.3]


def k0(r, ell):
    """Unit-scale Matern-5/2 straight from its definition (Sec. 3.1, q = 2)."""
    z = math.sqrt(5.0) * abs(r) / ell
    return (1.0 + z + z * z / 3.0) * math.exp(-z)


@pytest.mark.parametrize("ell", ELLS)
def test_k_matches_definition(ell):
    r = np.linspace(-3 * ell, 3 * ell, 41)
    np.testing.assert_allclose(O.kderiv(r, ell, 0), [k0(v, ell) for v in r], rtol=1e-15, atol=0)


@pytest.mark.parametrize("ell", ELLS)
def test_derivatives_by_finite_differences(ell):
    h = 1e-4 * ell
    for r in np.linspace(-2.7 * ell, 2.7 * ell, 17):
        if abs(r) < 3 * h:
            continue
        fd1 = (k0(r + h, ell) - k0(r - h, ell)) / (2 * h)
        fd2 = (k0(r + h, ell) - 2 * k0(r, ell) + k0(r - h, ell)) / (h * h)
        assert O.kderiv(r, ell, 1) == pytest.approx(fd1, rel=1e-7, abs=1e-9 / ell)
        assert O.kderiv(r, ell, 2) == pytest.approx(fd2, rel=1e-5, abs=1e-5 / ell ** 2)


@pytest.mark.parametrize("ell", ELLS)
def test_antiderivatives_by_quadrature(ell):
    for r in [-4.1 * ell, -1.0 * ell, -0.3 * ell, 0.02 * ell, 0.4472 * ell, 0.9 * ell, 2.5 * ell, 7 * ell]:
        K1q, _ = integrate.quad(lambda u: k0(u, ell), 0.0, r, epsabs=1e-300, epsrel=1e-13)
        assert O.kderiv(r, ell, -1) == pytest.approx(K1q, rel=1e-12, abs=1e-15 * ell)
        K2q, _ = integrate.quad(lambda u: float(O.kderiv(u, ell, -1)), 0.0, r, epsabs=1e-300, epsrel=1e-13)
        assert O.kderiv(r, ell, -2) == pytest.approx(K2q, rel=1e-11, abs=1e-15 * ell * ell)


@pytest.mark.parametrize("ell", ELLS)
def test_known_integrals_and_limits(ell):
    # int_R k = 16 ell / (3 sqrt 5): K1 tends to half of it
    assert O.kderiv(60 * ell, ell, -1) == pytest.approx(8 * ell / (3 * math.sqrt(5)), rel=1e-14)
    # Var u'(x) = -k''(0) = 5 / (3 ell^2)
    assert -O.kderiv(0.0, ell, 2) == pytest.approx(5 / (3 * ell * ell), rel=1e-15)
    # K2(r) ~ r^2/2 (k(0) = 1)
    r = 1e-4 * ell
    assert O.kderiv(r, ell, -2) == pytest.approx(r * r / 2, rel=1e-7)
    # odd / even symmetry
    r = 0.37 * ell
    assert O.kderiv(-r, ell, -1) == -O.kderiv(r, ell, -1)
    assert O.kderiv(-r, ell, -2) == O.kderiv(r, ell, -2)


def test_series_closed_form_switch_is_continuous():
    z = np.array([1.0 - 1e-12, 1.0 + 1e-12, 0.999, 1.001])
    closed1 = 8 / 3 - (8 / 3 + 5 * z / 3 + z * z / 3) * np.exp(-z)
    closed2 = 8 * z / 3 - 5 + (5 + 7 * z / 3 + z * z / 3) * np.exp(-z)
    np.testing.assert_allclose(O.g1(z), closed1, rtol=1e-14)
    np.testing.assert_allclose(O.f2(z), closed2, rtol=1e-13)
    # the series equals the closed form at mid range too
    zz = np.linspace(0.3, 0.99, 7)
    np.testing.assert_allclose(OO._poly(OO._F2, zz), 8 * zz / 3 - 5 + (5 + 7 * zz / 3 + zz ** 2 / 3) * np.exp(-zz),
                               rtol=1e-12)




@pytest.mark.parametrize("ell", [0.1, 0.5])
def test_cell_cell_integral_by_quadrature(ell):
    cells = [(0.0, 0.1), (0.1, 0.25), (0.05, 0.3), (0.7, 0.8), (2.0, 2.3)]
    a = np.array([c[0] for c in cells])
    b = np.array([c[1] for c in cells])
    C = O.cov_1d(O.cell_family(a, b, 0), O.cell_family(a, b, 0), ell)
    for i, (a1, b1) in enumerate(cells):
        for j, (a2, b2) in enumerate(cells):
            # split the inner integral at x' = x where k is not smooth
            def inner(x):
                lo, hi = a2, b2
                if lo < x < hi:
                    return (integrate.quad(lambda u: k0(x - u, ell), lo, x, epsabs=1e-300, epsrel=1e-13)[0] +
                            integrate.quad(lambda u: k0(x - u, ell), x, hi, epsabs=1e-300, epsrel=1e-13)[0])
                return integrate.quad(lambda u: k0(x - u, ell), lo, hi, epsabs=1e-300, epsrel=1e-13)[0]
            q = integrate.quad(inner, a1, b1, epsabs=1e-300, epsrel=1e-12, limit=200)[0]
            assert C[i, j] == pytest.approx(q, rel=1e-9, abs=1e-16), (i, j)


def test_far_cells_match_high_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    ell = 0.05
    a1, b1, a2, b2 = 0.0, 0.01, 0.9, 0.91  # z ~ 40: exponentially small entry

    def k_mp(r):
        z = mp.sqrt(5) * abs(r) / ell
        return (1 + z + z * z / 3) * mp.e ** (-z)

    exact = mp.quad(lambda x: mp.quad(lambda u: k_mp(x - u), [a2, b2]), [a1, b1])
    C = O.cov_1d(O.cell_family(np.array([a1]), np.array([b1]), 0),
                 O.cell_family(np.array([a2]), np.array([b2]), 0), ell)
    assert C[0, 0] == pytest.approx(float(exact), rel=1e-12)


@pytest.mark.parametrize("ell", [0.15, 0.6])
def test_mixed_functionals_by_quadrature_and_fd(ell):
    """Cell functionals of derivative order 1 and 2 against points of order 0/1,
    checked against integrals of finite-difference derivatives of k."""
    h = 1e-4
    a, b = np.array([0.2, 0.5]), np.array([0.35, 0.62])
    xs = np.array([0.0, 0.3, 0.9])

    def d_x(fun, x, xp):   # derivative in the first argument
        return (fun(x + h, xp) - fun(x - h, xp)) / (2 * h)

    kk = lambda x, xp: k0(x - xp, ell)
    for alpha in (0, 1, 2):
        for m in (0, 1):
            C = O.cov_1d(O.cell_family(a, b, alpha), O.point_family(xs, m), ell)
            for i in range(len(a)):
                for j in range(len(xs)):
                    # cov(int_a^b u^(alpha), d^m u(x')) = int_a^b d^alpha_x d^m_x' k dx
                    def integrand(x):
                        f = lambda X, XP: kk(X, XP)
                        if m == 1:
                            f0 = f
                            f = lambda X, XP, f0=f0: (f0(X, XP + h) - f0(X, XP - h)) / (2 * h)
                        if alpha >= 1:
                            g = f
                            f = lambda X, XP, g=g: d_x(g, X, XP)
                        if alpha == 2:
                            g2 = f
                            f = lambda X, XP, g2=g2: d_x(g2, X, XP)
                        return f(x, xs[j])
                    pts = [xs[j]] if a[i] < xs[j] < b[i] else None
                    if alpha == 0:
                        q = integrate.quad(integrand, a[i], b[i], points=pts, epsabs=1e-12, epsrel=1e-10)[0]
                    else:
                        # FTC: the integral of the alpha-th derivative is a difference (Eq. linop-simplified);
                        # here checked by quadrature of the FD derivative on a coarse rule
                        q = integrate.quad(integrand, a[i], b[i], points=pts, epsabs=1e-8, epsrel=1e-6, limit=200)[0]
                    tol = (1e-9 if m == 0 else 1e-6) if alpha == 0 else 2e-4  # FD step h = 1e-4
                    assert C[i, j] == pytest.approx(q, rel=tol, abs=tol * 1e-2), (alpha, m, i, j)


def test_symmetry_toeplitz_and_subcell_additivity():
    ell = 0.1
    e = np.linspace(0, 1, 17)
    for p in (0, 1, 2):
        for q in (0, 1, 2):
            A = O.cov_1d(O.cell_family(e[:-1], e[1:], p), O.cell_family(e[:-1], e[1:], q), ell)
            B = O.cov_1d(O.cell_family(e[:-1], e[1:], q), O.cell_family(e[:-1], e[1:], p), ell)
            np.testing.assert_allclose(A, B.T, rtol=1e-13, atol=1e-13 * np.abs(A).max())
            # Toeplitz on a uniform grid
            for d in range(-5, 6):
                dg = np.diag(A, d)
                np.testing.assert_allclose(dg, dg[0], rtol=1e-10, atol=1e-12 * np.abs(A).max())
    # sub-volume additivity (App. G): the integral over a cell is the sum over its halves
    mid = 0.5 * (e[:-1] + e[1:])
    pts = O.point_family(np.array([0.05, 0.33, 0.8]), 1)
    whole = O.cov_1d(O.cell_family(e[:-1], e[1:], 0), pts, ell)
    halves = O.cov_1d(O.cell_family(e[:-1], mid, 0), pts, ell) + O.cov_1d(O.cell_family(mid, e[1:], 0), pts, ell)
    np.testing.assert_allclose(whole, halves, rtol=1e-12, atol=1e-16)
    fam = O.cell_family(e[:-1], e[1:], 2)
    whole = O.cov_1d(O.cell_family(e[:-1], e[1:], 0), fam, ell)
    halves = O.cov_1d(O.cell_family(e[:-1], mid, 0), fam, ell) + O.cov_1d(O.cell_family(mid, e[1:], 0), fam, ell)
    np.testing.assert_allclose(whole, halves, rtol=1e-11, atol=1e-14)


def test_rejects_unsupported_orders():
    with pytest.raises(ValueError):
        O.cell_family(np.zeros(1), np.ones(1), 3)
    with pytest.raises(ValueError):
        O.point_family(np.zeros(1), 3)
    with pytest.raises(ValueError):
        O.kderiv(0.5, 1.0, 5)
