"""Seeded synthetic IBVP workloads for GP-FVM.

This module only *states problems*: cell grids, PDE operator terms, kernel
hyperparameters, initial/boundary point sets with their values, and the
prediction grid.  It contains none of the method's arithmetic (no covariance,
no Gram matrix, no solve), so that both the FP64 CPU oracle and the GPU library
can consume the same inputs without sharing any computation.

Problem statement (Sec. 2.2, Sec. 3.2 "Multi-dimensional domains", Sec. 4.1
"factorized box scheme"):
  * domain [lo, hi]^d, axis 0 is time for IBVPs;
  * a factorized box scheme: per-axis cell edges, every cell of the tensor
    grid is one finite-volume (PDE) observation  int_V D[u] = int_V f;
  * D = sum_alpha c_alpha d^alpha  (multi-indices alpha, entries 0..2);
  * tensor-product Matern-5/2 prior with per-axis lengthscales and one
    output scale (Eq. tensorproduct-cov-def);
  * initial/boundary data as tensor grids of point functionals
    d^m u(x) with a per-axis derivative order m in {0,1} and a noise variance.

Volume observations are ordered row-major over (t, x, y); a point set's values
are ordered row-major over its per-axis coordinate lists.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "PointSet", "Problem", "heat_1d", "heat_2d", "wave_2d", "wave_2d_sine",
    "toy_cos", "batch_heat", "serving_wave_stream", "uniform_edges",
    "gaussian_bumps", "wave_1d_system", "shallow_water_2d",
]


@dataclass
class PointSet:
    """A tensor grid of point functionals  d^order u (x)  (one per grid point);
    with several outputs, of the component u_out."""
    order: Tuple[int, ...]
    coords: List[np.ndarray]
    values: np.ndarray
    noise_var: float
    name: str = ""
    out: int = 0

    @property
    def shape(self) -> Tuple[int, ...]:
        return tuple(len(c) for c in self.coords)

    @property
    def size(self) -> int:
        return int(np.prod(self.shape))


@dataclass
class Problem:
    """A linear IBVP discretised by a factorized box FVM scheme."""
    edges: List[np.ndarray]
    lengthscale: Tuple[float, ...]
    outputscale: float
    terms: List[Tuple[Tuple[int, ...], float]]
    jitter: float
    sets: List[PointSet]
    pred: List[np.ndarray]
    rhs: Optional[np.ndarray] = None
    name: str = ""
    meta: dict = field(default_factory=dict)
    # "fvm": one volume integral of the PDE per cell; "collocation": the PDE
    # evaluated at each cell centre (rhs then holds point values of the forcing)
    observe: str = "fvm"
    # per term: None (constant coefficient) or one value per cell (row-major
    # over n_cells) multiplying the term's coefficient -- a piecewise-constant
    # variable coefficient such as a bathymetry-dependent wave speed
    fields: Optional[List[Optional[np.ndarray]]] = None
    # several outputs (Sec. 3.3, multi-dimensional codomains): u = (u_0 .. u_{n_out-1})
    # with independent tensor-product priors of the same hyperparameters; term k
    # belongs to equation term_eq[k] and differentiates component term_out[k]
    # (None: one equation, one output).  Every cell yields one observation per
    # equation; PDE observations are ordered equation-major, predictions
    # output-major.
    n_out: int = 1
    term_eq: Optional[List[int]] = None
    term_out: Optional[List[int]] = None

    @property
    def ndim(self) -> int:
        return len(self.edges)

    @property
    def n_cells(self) -> Tuple[int, ...]:
        return tuple(len(e) - 1 for e in self.edges)

    @property
    def n_eq(self) -> int:
        return 1 if self.term_eq is None else int(max(self.term_eq)) + 1

    @property
    def N(self) -> int:
        """PDE observations: one per cell and equation."""
        return self.n_eq * int(np.prod(self.n_cells))

    @property
    def M(self) -> int:
        return int(sum(s.size for s in self.sets))

    @property
    def P(self) -> int:
        """Prediction points: the grid for every output."""
        return self.n_out * int(np.prod([len(p) for p in self.pred]))


def uniform_edges(lo: float, hi: float, n: int) -> np.ndarray:
    return np.linspace(lo, hi, n + 1)


def _mid(lo: float, hi: float, n: int) -> np.ndarray:
    h = (hi - lo) / n
    return lo + h * (np.arange(n) + 0.5)


def gaussian_bumps(rng: np.random.Generator, n_bumps: int, amp=(0.5, 1.0),
                   width=(0.05, 0.15), centre=(0.2, 0.8)):
    """Draw bump parameters (amplitude, width, centre_x, centre_y)."""
    A = rng.uniform(amp[0], amp[1], n_bumps)
    w = rng.uniform(width[0], width[1], n_bumps)
    cx = rng.uniform(centre[0], centre[1], n_bumps)
    cy = rng.uniform(centre[0], centre[1], n_bumps)
    return A, w, cx, cy


def _eval_bumps(params, X, Y):
    A, w, cx, cy = params
    out = np.zeros_like(X, dtype=np.float64)
    for a, s, x0, y0 in zip(A, w, cx, cy):
        out += a * np.exp(-((X - x0) ** 2 + (Y - y0) ** 2) / (2.0 * s * s))
    return out


def heat_1d(nt: int = 16, nx: int = 32, nu: float = 0.1, n_ic: int = 32,
            n_bc: int = 16, pred: int = 64, ell=(0.2, 0.1), jitter: float = 1e-8) -> Problem:
    """1D+time heat u_t = nu u_xx on [0,1]^2, IC u(0,x)=sin(pi x), zero Dirichlet.

    Default sizes: 16x32 cells, 32 IC points on linspace(0,1,32), boundary
    points at x in {0,1} for t = linspace(0,1,n_bc+1)[1:] (the corner t=0 is
    left to the IC so that no point is duplicated)."""
    edges = [uniform_edges(0, 1, nt), uniform_edges(0, 1, nx)]
    xs = np.linspace(0, 1, n_ic)
    ic = PointSet((0, 0), [np.array([0.0]), xs], np.sin(np.pi * xs), jitter, "ic")
    tb = np.linspace(0, 1, n_bc + 1)[1:]
    bc = PointSet((0, 0), [tb, np.array([0.0, 1.0])], np.zeros(2 * n_bc), jitter, "bc_x")
    terms = [((1, 0), 1.0), ((0, 2), -nu)]
    grid = [np.linspace(0, 1, pred), np.linspace(0, 1, pred)]
    return Problem(edges, tuple(ell), 1.0, terms, jitter, [ic, bc], grid,
                   name=f"heat1d_{nt}x{nx}", meta={"nu": nu})


def heat_2d(nt: int = 64, nx: int = 64, ny: int = 64, nu: float = 0.05, seed: int = 0,
            n_ic=(64, 64), n_bc=(16, 16), pred=(32, 32, 32), n_bumps: int = 5,
            ell=(0.2, 0.1, 0.1), jitter: float = 1e-8) -> Problem:
    """2D+time heat u_t = nu (u_xx + u_yy) on [0,1]^3.

    IC: seeded sum of Gaussian bumps on an n_ic linspace grid at t=0;
    BC: zero Dirichlet on the faces x in {0,1} and y in {0,1}, on n_bc
    (time x tangential) cell-midpoint grids per face."""
    rng = np.random.default_rng(seed)
    params = gaussian_bumps(rng, n_bumps)
    edges = [uniform_edges(0, 1, nt), uniform_edges(0, 1, nx), uniform_edges(0, 1, ny)]
    xs, ys = np.linspace(0, 1, n_ic[0]), np.linspace(0, 1, n_ic[1])
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    ic = PointSet((0, 0, 0), [np.array([0.0]), xs, ys], _eval_bumps(params, X, Y).ravel(),
                  jitter, "ic")
    tb, sb = _mid(0, 1, n_bc[0]), _mid(0, 1, n_bc[1])
    two = np.array([0.0, 1.0])
    bcx = PointSet((0, 0, 0), [tb, two, sb], np.zeros(n_bc[0] * 2 * n_bc[1]), jitter, "bc_x")
    bcy = PointSet((0, 0, 0), [tb, sb, two], np.zeros(n_bc[0] * 2 * n_bc[1]), jitter, "bc_y")
    terms = [((1, 0, 0), 1.0), ((0, 2, 0), -nu), ((0, 0, 2), -nu)]
    grid = [np.linspace(0, 1, p) for p in pred]
    return Problem(edges, tuple(ell), 1.0, terms, jitter, [ic, bcx, bcy], grid,
                   name=f"heat2d_{nt}x{nx}x{ny}_s{seed}",
                   meta={"nu": nu, "seed": seed, "bumps": params})


def wave_2d(nt: int = 128, nx: int = 128, ny: int = 128, c: float = 1.0, seed: int = 0,
            n_ic=(64, 64), n_bc=(32, 32), pred=(32, 64, 64), width: float = 0.05,
            ic_noise: float = 0.01, ell=(0.05, 0.05, 0.05), jitter: float = 1e-8) -> Problem:
    """2D+time wave u_tt = c^2 (u_xx + u_yy) on [0,1]^3 with reflecting walls.

    IC: one Gaussian bump of the given width (centre U(0.3,0.7)^2) plus
    N(0, ic_noise^2) noise as displacement (noise variance ic_noise^2), zero
    initial velocity u_t(0)=0; BC: zero normal derivative on the four walls on
    n_bc (time x tangential) midpoint grids per wall."""
    rng = np.random.default_rng(seed)
    cx, cy = rng.uniform(0.3, 0.7, 2)
    edges = [uniform_edges(0, 1, nt), uniform_edges(0, 1, nx), uniform_edges(0, 1, ny)]
    xs, ys = np.linspace(0, 1, n_ic[0]), np.linspace(0, 1, n_ic[1])
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    disp = np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * width * width)).ravel()
    if ic_noise > 0:
        disp = disp + rng.normal(0.0, ic_noise, disp.shape)
    nv = ic_noise ** 2 if ic_noise > 0 else jitter
    ic_u = PointSet((0, 0, 0), [np.array([0.0]), xs, ys], disp, nv, "ic_u")
    ic_v = PointSet((1, 0, 0), [np.array([0.0]), xs, ys], np.zeros(disp.size), jitter, "ic_ut")
    tb, sb = _mid(0, 1, n_bc[0]), _mid(0, 1, n_bc[1])
    two = np.array([0.0, 1.0])
    bcx = PointSet((0, 1, 0), [tb, two, sb], np.zeros(n_bc[0] * 2 * n_bc[1]), jitter, "neu_x")
    bcy = PointSet((0, 0, 1), [tb, sb, two], np.zeros(n_bc[0] * 2 * n_bc[1]), jitter, "neu_y")
    c2 = c * c
    terms = [((2, 0, 0), 1.0), ((0, 2, 0), -c2), ((0, 0, 2), -c2)]
    grid = [np.linspace(0, 1, p) for p in pred]
    return Problem(edges, tuple(ell), 1.0, terms, jitter, [ic_u, ic_v, bcx, bcy], grid,
                   name=f"wave2d_{nt}x{nx}x{ny}_s{seed}",
                   meta={"c": c, "seed": seed, "centre": (cx, cy)})


def wave_2d_sine(nt: int = 8, nx: int = 8, ny: int = 8, C=None, c: float = 1.0, T: float = 2.0,
                 n_ic: int = 8, n_bc=(20, 10), pred=(9, 9, 9), ell=(0.6, 0.3, 0.3),
                 jitter: float = 1e-8, seed: Optional[int] = None) -> Problem:
    """The paper's 2D wave benchmark (App. C.3): [0,T]x[0,1]^2, c=1,
    u(0,x,y) = sum_{i,j<=2} C_ij sin(i pi x) sin(j pi y), u_t(0)=0, zero
    Dirichlet walls; IC on an n_ic x n_ic grid, per wall n_bc (time x space)
    uniformly spaced points.  C is drawn from the stated normal law when seeded."""
    if C is None:
        if seed is None:
            C = np.array([[1.0, 0.5], [0.5, 0.0]])
        else:
            rng = np.random.default_rng(seed)
            C = (np.array([1.0, 0.5, 0.5, 0.0]) +
                 rng.normal(size=4) * np.array([0.1, 0.2, 0.2, 0.3])).reshape(2, 2)
    C = np.asarray(C, dtype=np.float64)
    edges = [uniform_edges(0, T, nt), uniform_edges(0, 1, nx), uniform_edges(0, 1, ny)]
    xs = np.linspace(0, 1, n_ic)
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    u0 = np.zeros_like(X)
    for i in range(2):
        for j in range(2):
            u0 += C[i, j] * np.sin((i + 1) * np.pi * X) * np.sin((j + 1) * np.pi * Y)
    ic_u = PointSet((0, 0, 0), [np.array([0.0]), xs, xs], u0.ravel(), jitter, "ic_u")
    ic_v = PointSet((1, 0, 0), [np.array([0.0]), xs, xs], np.zeros(u0.size), jitter, "ic_ut")
    tb = np.linspace(0, T, n_bc[0] + 1)[1:]
    sb = np.linspace(0, 1, n_bc[1] + 2)[1:-1]
    two = np.array([0.0, 1.0])
    bcx = PointSet((0, 0, 0), [tb, two, sb], np.zeros(n_bc[0] * 2 * n_bc[1]), jitter, "bc_x")
    bcy = PointSet((0, 0, 0), [tb, sb, two], np.zeros(n_bc[0] * 2 * n_bc[1]), jitter, "bc_y")
    terms = [((2, 0, 0), 1.0), ((0, 2, 0), -c * c), ((0, 0, 2), -c * c)]
    grid = [np.linspace(0, T, pred[0]), np.linspace(0, 1, pred[1]), np.linspace(0, 1, pred[2])]
    return Problem(edges, tuple(ell), 1.0, terms, jitter, [ic_u, ic_v, bcx, bcy], grid,
                   name=f"wave_sine_{nt}x{nx}x{ny}", meta={"C": C, "c": c, "T": T})


def toy_cos(n: int = 8, ell: float = 1.0, pred: int = 50, jitter: float = 1e-10,
            observe: str = "fvm") -> Problem:
    """Sec. 3 toy problem (Fig. 2): du/dx = cos x on [0, 2 pi], u(0)=u(2 pi)=0.

    The right-hand side of the i-th volume observation is int_{a_i}^{b_i} cos x dx;
    with observe="collocation" it is cos at the centre of cell i."""
    e = uniform_edges(0.0, 2 * np.pi, n)
    if observe == "collocation":
        rhs = np.cos(0.5 * (e[1:] + e[:-1]))
    else:
        rhs = np.sin(e[1:]) - np.sin(e[:-1])
    bc = PointSet((0,), [np.array([0.0, 2 * np.pi])], np.zeros(2), jitter, "bc")
    return Problem([e], (ell,), 1.0, [((1,), 1.0)], jitter, [bc],
                   [np.linspace(0, 2 * np.pi, pred)], rhs=rhs, name=f"toy_cos_{observe}_{n}", observe=observe)


def collocation(prob: Problem) -> Problem:
    """The same homogeneous IBVP observed by collocation at the cell centres."""
    if prob.rhs is not None:
        raise ValueError("only homogeneous problems: give point values of the forcing instead")
    from dataclasses import replace
    return replace(prob, observe="collocation", name=prob.name + "_colloc")


def heat_1d_varcoef(nt: int = 16, nx: int = 32, pred: int = 33, ell=(0.3, 0.2), jitter: float = 1e-10) -> Problem:
    """1D+time heat u_t = nu(x) u_xx with nu piecewise constant per cell
    (nu = 0.05 (1 + x) at the cell centre), built so that
    u*(t, x) = exp(-t) sin(pi x) satisfies every volume observation exactly:
    the right-hand side of cell [t0,t1] x [x0,x1] is
    (nu_V pi^2 - 1) (e^-t0 - e^-t1) (cos pi x0 - cos pi x1) / pi.
    IC u(0, x) = sin(pi x) on nx + 1 points, zero walls at x = 0, 1."""
    te, xe = uniform_edges(0, 1, nt), uniform_edges(0, 1, nx)
    xc = 0.5 * (xe[1:] + xe[:-1])
    nu = 0.05 * (1.0 + xc)
    field = np.tile(nu, (nt, 1))
    It = np.exp(-te[:-1]) - np.exp(-te[1:])
    Ix = (np.cos(np.pi * xe[:-1]) - np.cos(np.pi * xe[1:])) / np.pi
    rhs = (field * np.pi ** 2 - 1.0) * np.outer(It, Ix)
    xs = np.linspace(0, 1, nx + 1)
    ic = PointSet((0, 0), [np.array([0.0]), xs], np.sin(np.pi * xs), jitter, "ic")
    tb = np.linspace(0, 1, nt + 1)[1:]
    bc = PointSet((0, 0), [tb, np.array([0.0, 1.0])], np.zeros(2 * nt), jitter, "bc_x")
    terms = [((1, 0), 1.0), ((0, 2), -1.0)]
    grid = [np.linspace(0, 1, pred), np.linspace(0, 1, pred)]
    return Problem([te, xe], tuple(ell), 1.0, terms, jitter, [ic, bc], grid, rhs=rhs.ravel(),
                   name=f"heat1d_varcoef_{nt}x{nx}", fields=[None, field.ravel()])


def heat_2d_varcoef(nt: int = 16, nx: int = 20, ny: int = 24, seed: int = 0, **kw) -> Problem:
    """The 2D+time heat problem of heat_2d with a piecewise-constant diffusivity
    nu(x, y) = 0.02 + 0.08 * (seeded Gaussian bump) per cell (a synthetic
    stand-in for a depth-dependent coefficient), shared by both second-order terms."""
    p = heat_2d(nt, nx, ny, seed=seed, **kw)
    rng = np.random.default_rng(seed + 7)
    xe, ye = p.edges[1], p.edges[2]
    X, Y = np.meshgrid(0.5 * (xe[1:] + xe[:-1]), 0.5 * (ye[1:] + ye[:-1]), indexing="ij")
    cx, cy = rng.uniform(0.3, 0.7, 2)
    nu = 0.02 + 0.08 * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * 0.2 ** 2))
    field = np.broadcast_to(nu, (nt, nx, ny)).ravel().copy()
    p.terms = [((1, 0, 0), 1.0), ((0, 2, 0), -1.0), ((0, 0, 2), -1.0)]
    p.fields = [None, field, field]
    p.name = p.name + "_varcoef"
    return p


def batch_heat(n_problems: int = 256, lo: int = 16, hi: int = 64, seed: int = 0,
               ell=(0.2, 0.1, 0.1), jitter: float = 1e-8) -> List[Problem]:
    """Batch of independent 2D+time heat IBVPs: each axis size uniform in
    {lo..hi}, nu ~ U(0.01, 0.1), 5-bump IC on an (Nx/2)x(Ny/2) grid, zero
    Dirichlet walls on ceil(Nt/4) x ceil(Ns/4) midpoint grids per face, and an
    (Nt/2)(Nx/2)(Ny/2) prediction grid."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_problems):
        nt, nx, ny = (int(v) for v in rng.integers(lo, hi + 1, 3))
        nu = float(rng.uniform(0.01, 0.1))
        sub = int(rng.integers(0, 2 ** 31 - 1))
        p = heat_2d(nt, nx, ny, nu=nu, seed=sub, n_ic=(nx // 2, ny // 2),
                    n_bc=(-(-nt // 4), -(-max(nx, ny) // 4)),
                    pred=(nt // 2, nx // 2, ny // 2), ell=ell, jitter=jitter)
        p.name = f"batch{k}_" + p.name
        out.append(p)
    return out


def serving_wave_stream(rate: float = 500.0, duration: float = 1.0, lo: int = 32, hi: int = 128,
                        seed: int = 0, n_max: Optional[int] = None,
                        ell=(0.05, 0.05, 0.05), jitter: float = 1e-8):
    """Poisson request stream of 2D+time wave IBVPs: arrival times (s) and problems.

    Per-axis sizes uniform in {lo..hi}, c ~ U(0.5, 2), one random bump as
    displacement; IC grids of max(N/4, 3) points per axis for displacement and
    velocity, reflecting walls on (Nt/8)(Ns/8) grids per face.  The bump is at
    least half an IC grid spacing wide, so that small requests still observe it."""
    rng = np.random.default_rng(seed)
    t, reqs = 0.0, []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t > duration or (n_max is not None and len(reqs) >= n_max):
            break
        nt, nx, ny = (int(v) for v in rng.integers(lo, hi + 1, 3))
        c = float(rng.uniform(0.5, 2.0))
        ns = max(nx, ny)
        n_ic = (max(nx // 4, 3), max(ny // 4, 3))
        p = wave_2d(nt, nx, ny, c=c, seed=int(rng.integers(0, 2 ** 31 - 1)), n_ic=n_ic,
                    width=max(0.05, 0.5 / (min(n_ic) - 1)),
                    n_bc=(max(nt // 8, 1), max(ns // 8, 1)),
                    pred=(nt // 2, nx // 2, ny // 2), ic_noise=0.0, ell=ell, jitter=jitter)
        reqs.append((t, p))
    return reqs


def wave_1d_system(nt: int = 8, nx: int = 8, pred=(9, 9), ell=(0.5, 0.3), jitter: float = 1e-10,
                   n_ic: Optional[int] = None) -> Problem:
    """The 1D wave equation as a first-order system in two outputs (u, v):
        u_t + v_x = 0,   v_t + u_x = 0   on [0,1]^2,
    u(0, x) = sin(pi x), v(0, x) = 0, u(t, 0) = u(t, 1) = 0, solved by
    u = sin(pi x) cos(pi t), v = -cos(pi x) sin(pi t).  Each equation couples
    both components (Sec. 3.3: operators sum_alpha sum_i c_{alpha,i} D^alpha u_i)."""
    te, xe = uniform_edges(0, 1, nt), uniform_edges(0, 1, nx)
    n_ic = nx + 1 if n_ic is None else n_ic
    xs = np.linspace(0, 1, n_ic)
    t0 = np.array([0.0])
    ic_u = PointSet((0, 0), [t0, xs], np.sin(np.pi * xs), jitter, "ic_u", out=0)
    ic_v = PointSet((0, 0), [t0, xs], np.zeros(n_ic), jitter, "ic_v", out=1)
    tb = np.linspace(0, 1, nt + 1)[1:]
    bc = PointSet((0, 0), [tb, np.array([0.0, 1.0])], np.zeros(2 * nt), jitter, "bc_u", out=0)
    terms = [((1, 0), 1.0), ((0, 1), 1.0), ((1, 0), 1.0), ((0, 1), 1.0)]
    grid = [np.linspace(0, 1, pred[0]), np.linspace(0, 1, pred[1])]
    return Problem([te, xe], tuple(ell), 1.0, terms, jitter, [ic_u, ic_v, bc], grid,
                   name=f"wave1d_system_{nt}x{nx}", n_out=2, term_eq=[0, 0, 1, 1], term_out=[0, 1, 1, 0])


def shallow_water_2d(nt: int = 8, nx: int = 8, ny: int = 8, H: float = 1.0, g: float = 1.0, f: float = 0.5,
                     k: float = 0.1, n_ic=(8, 8), n_bc=(4, 4), pred=(4, 5, 5), ell=(0.4, 0.3, 0.3),
                     width: float = 0.15, jitter: float = 1e-8, seed: int = 0, standing: bool = False,
                     depth: Optional[np.ndarray] = None) -> Problem:
    """Linearised 2D shallow-water equations with constant depth H (App. C.4's
    system without its variable bathymetry), outputs (h, u, v):
        h_t + H (u_x + v_y) = 0,   u_t - f v + g h_x + k u = 0,   v_t + f u + g h_y + k v = 0
    on [0,1]^3.  IC: a Gaussian bump of the given width (centre U(0.35,0.65)^2) in h, zero
    velocities; walls: u = 0 at x = 0, 1 and v = 0 at y = 0, 1 on n_bc (time x tangential)
    midpoint grids.  With standing=True the IC is h = cos(pi x) instead: for f = k = 0 the
    solution is the standing wave h = cos(pi x) cos(w t), u = sqrt(g/H) sin(pi x) sin(w t),
    v = 0 with w = pi sqrt(g H).  depth: an (nx, ny) array of per-cell depths H(x, y)
    (App. C.4's bathymetry, piecewise constant per cell and constant in time) multiplying
    the two velocity terms of the h equation instead of the constant H."""
    rng = np.random.default_rng(seed)
    cx, cy = rng.uniform(0.35, 0.65, 2)
    edges = [uniform_edges(0, 1, nt), uniform_edges(0, 1, nx), uniform_edges(0, 1, ny)]
    xs, ys = np.linspace(0, 1, n_ic[0]), np.linspace(0, 1, n_ic[1])
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    h0 = (np.cos(np.pi * X) if standing else np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * width * width))).ravel()
    t0 = np.array([0.0])
    ic_h = PointSet((0, 0, 0), [t0, xs, ys], h0, jitter, "ic_h", out=0)
    ic_u = PointSet((0, 0, 0), [t0, xs, ys], np.zeros(h0.size), jitter, "ic_u", out=1)
    ic_v = PointSet((0, 0, 0), [t0, xs, ys], np.zeros(h0.size), jitter, "ic_v", out=2)
    tb, sb = _mid(0, 1, n_bc[0]), _mid(0, 1, n_bc[1])
    two = np.array([0.0, 1.0])
    wall_u = PointSet((0, 0, 0), [tb, two, sb], np.zeros(n_bc[0] * 2 * n_bc[1]), jitter, "wall_u", out=1)
    wall_v = PointSet((0, 0, 0), [tb, sb, two], np.zeros(n_bc[0] * 2 * n_bc[1]), jitter, "wall_v", out=2)
    terms, eq, out = [], [], []

    def add(alpha, c, e, o):
        if c != 0.0:
            terms.append((alpha, float(c)))
            eq.append(e)
            out.append(o)
    add((1, 0, 0), 1.0, 0, 0); add((0, 1, 0), 1.0 if depth is not None else H, 0, 1)
    add((0, 0, 1), 1.0 if depth is not None else H, 0, 2)
    add((1, 0, 0), 1.0, 1, 1); add((0, 0, 0), -f, 1, 2); add((0, 1, 0), g, 1, 0); add((0, 0, 0), k, 1, 1)
    add((1, 0, 0), 1.0, 2, 2); add((0, 0, 0), f, 2, 1); add((0, 0, 1), g, 2, 0); add((0, 0, 0), k, 2, 2)
    grid = [np.linspace(0, 1, p) for p in pred]
    fields = None
    if depth is not None:
        field = np.broadcast_to(np.asarray(depth, np.float64), (nt, nx, ny)).ravel().copy()
        fields = [field if (e == 0 and o in (1, 2)) else None for e, o in zip(eq, out)]
    return Problem(edges, tuple(ell), 1.0, terms, jitter, [ic_h, ic_u, ic_v, wall_u, wall_v], grid,
                   name=f"swe2d_{nt}x{nx}x{ny}", meta={"H": H, "g": g, "f": f, "k": k, "centre": (cx, cy)},
                   fields=fields, n_out=3, term_eq=eq, term_out=out)
