"""FP64 CPU oracle for GP-FVM (test infrastructure only; see package docstring).

Parity status per function is listed in ``PINS`` at the bottom of this file;
every function here is pinned by at least one ``-m "not gpu"`` test against
something other than itself (quadrature, finite differences, closed-form PDE
solutions, brute-force multi-dimensional quadrature, exact invariants).

Notation: axes are ordered (t, x, y); r = x - x'; s = sqrt(5)/ell; z = s|r|.
A 1D test functional is written as a short list of *atoms* (w, m, x) meaning
w * d^m u(x), where m = -1 denotes the antiderivative U with U' = u.  A cell
[a, b] observed with derivative order alpha (Eq. linop-simplified, Sec. 3.1)
is  int_a^b u^(alpha) = U^(alpha-1)(b) - U^(alpha-1)(a),  i.e. the atoms
(+1, alpha-1, b), (-1, alpha-1, a).  A point functional d^m u(x) is (1, m, x).
For atoms, cov(d^m u(x), d^n u(x')) = (-1)^n k^(m+n)(x - x') with
k^(-1) = K1 (K1' = k, K1(0) = 0) and k^(-2) = K2 (K2'' = k, K2(0) = 0).
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np
import scipy.linalg as sla

SQRT5 = math.sqrt(5.0)

# ----------------------------------------------------------------------------
# 1D Matern-5/2 closed forms (Sec. 3.1: half-integer Matern, q = 2)
# ----------------------------------------------------------------------------
# k(r) = (1 + z + z^2/3) exp(-z) is the q = 2 member of the family
# exp(-sqrt(2q+1) r) p_q(sqrt(2q+1) r) with r measured in lengthscales.
# Derivatives and antiderivatives (derived by hand, pinned by quadrature and
# finite differences in tests/test_oracle_closed_forms.py):
#   k'(r)  = -sgn(r) s z (1 + z)/3 e^-z
#   k''(r) = -s^2 (1 + z - z^2)/3 e^-z
#   k^(3)(r) = sgn(r) s^3 z (3 - z)/3 e^-z      (continuous: ~ s^4 r near 0)
#   k^(4)(r) = s^4 (3 - 5z + z^2)/3 e^-z        (k^(4)(0) = s^4 = 25/ell^4)
# (the third and fourth derivatives are needed only by collocation
# observations of second-order operators)
#   K1(r)  =  sgn(r)/s  [8/3 - (8/3 + 5z/3 + z^2/3) e^-z]
#   K2(r)  =  s^-2 [8z/3 - 5 + (5 + 7z/3 + z^2/3) e^-z]
# Near z = 0 both antiderivatives lose digits to cancellation, so their
# Taylor series are used for z < 1:
#   s K1 / sgn(r) = sum_{k>=1} (-1)^(k+1) (k-2)(k-4) / (3 k!) z^k
#   s^2 K2        = sum_{k>=2} (-1)^k     (k-3)(k-5) / (3 k!) z^k
_SERIES_TERMS = 24
_G1 = np.array([0.0] + [(-1.0) ** (k + 1) * (k - 2) * (k - 4) / (3.0 * math.factorial(k))
                        for k in range(1, _SERIES_TERMS)])
_F2 = np.array([0.0, 0.0] + [(-1.0) ** k * (k - 3) * (k - 5) / (3.0 * math.factorial(k))
                             for k in range(2, _SERIES_TERMS)])
Z_SERIES = 1.0


def _poly(coef: np.ndarray, z: np.ndarray) -> np.ndarray:
    out = np.zeros_like(z)
    for c in coef[::-1]:
        out = out * z + c
    return out


def g1(z):
    """s*K1(r)/sgn(r) as a function of z >= 0."""
    z = np.asarray(z, dtype=np.float64)
    closed = 8.0 / 3.0 - (8.0 / 3.0 + 5.0 * z / 3.0 + z * z / 3.0) * np.exp(-z)
    return np.where(z < Z_SERIES, _poly(_G1, np.minimum(z, Z_SERIES)), closed)


def f2(z):
    """s^2*K2(r) as a function of z >= 0."""
    z = np.asarray(z, dtype=np.float64)
    closed = 8.0 * z / 3.0 - 5.0 + (5.0 + 7.0 * z / 3.0 + z * z / 3.0) * np.exp(-z)
    return np.where(z < Z_SERIES, _poly(_F2, np.minimum(z, Z_SERIES)), closed)


def kderiv(r, ell: float, order: int):
    """k^(order)(r) of the unit-scale 1D Matern-5/2 kernel, order in -2..4."""
    r = np.asarray(r, dtype=np.float64)
    s = SQRT5 / ell
    z = s * np.abs(r)
    e = np.exp(-z)
    sg = np.sign(r)
    if order == 0:
        return (1.0 + z + z * z / 3.0) * e
    if order == 1:
        return -sg * s * z * (1.0 + z) / 3.0 * e
    if order == 2:
        return -s * s * (1.0 + z - z * z) / 3.0 * e
    if order == 3:
        return sg * s ** 3 * z * (3.0 - z) / 3.0 * e
    if order == 4:
        return s ** 4 * (3.0 - 5.0 * z + z * z) / 3.0 * e
    if order == -1:
        return sg * g1(z) / s
    if order == -2:
        return f2(z) / (s * s)
    raise ValueError(f"derivative order {order} outside -2..4")


# ----------------------------------------------------------------------------
# 1D test functionals and their covariances (Eq. linop-simplified, Eq. LkL)
# ----------------------------------------------------------------------------
def cell_family(a: np.ndarray, b: np.ndarray, alpha: int):
    """Stacked 1D FVM functionals int_{a_j}^{b_j} u^(alpha) over cells j."""
    if alpha not in (0, 1, 2):
        raise ValueError("cell derivative order must be 0, 1 or 2")
    return ("cell", np.asarray(a, np.float64), np.asarray(b, np.float64), int(alpha))


def point_family(x: np.ndarray, order: int):
    """Stacked 1D point functionals d^order u(x_j) (order 2 only for the
    collocation operator; Matern-5/2 paths are twice differentiable)."""
    if order not in (0, 1, 2):
        raise ValueError("point derivative order must be 0, 1 or 2")
    return ("point", np.asarray(x, np.float64), int(order))


def _atoms(fam):
    if fam[0] == "cell":
        _, a, b, alpha = fam
        return [(1.0, alpha - 1, b), (-1.0, alpha - 1, a)]
    _, x, m = fam
    return [(1.0, m, x)]


def cov_1d(F, G, ell: float) -> np.ndarray:
    """Matrix cov(F_i, G_j) of two stacked 1D functional families (unit scale).

    Each entry is  sum over atom pairs  w w' (-1)^n k^(m+n)(x - x').  For the
    antiderivative orders (-1, -2) the polynomial part of K1/K2 is summed
    separately from the exponential part: when every atom separation of an
    entry has one sign (the cells are apart), that polynomial part cancels
    exactly (the atom weights of a cell sum to zero), so only the exponential
    part is kept; entries whose separations are all below one z-unit use the
    Taylor series of the full function instead."""
    A, B = _atoms(F), _atoms(G)
    order = A[0][1] + B[0][1]
    if order > 4:
        raise ValueError("total derivative order above 4 is not supported by Matern-5/2 paths")
    s = SQRT5 / ell
    pairs = []
    for (w1, m, x1) in A:
        for (w2, n, x2) in B:
            r = x1[:, None] - x2[None, :]
            pairs.append((w1 * w2 * (-1.0) ** n, r))
    if order >= 0:
        return sum(w * kderiv(r, ell, order) for w, r in pairs)
    zs = [s * np.abs(r) for _, r in pairs]
    zmax = np.max(np.stack(zs), axis=0)
    near = zmax < Z_SERIES
    if order == -1:
        series = sum(w * np.sign(r) * _poly(_G1, np.minimum(z, Z_SERIES)) for (w, r), z in zip(pairs, zs))
        poly_int = sum(w * np.sign(r) for w, r in pairs)  # exact small integers
        expo = sum(-w * np.sign(r) * (8.0 / 3.0 + 5.0 * z / 3.0 + z * z / 3.0) * np.exp(-z)
                   for (w, r), z in zip(pairs, zs))
        far = poly_int * (8.0 / 3.0) + expo
        return np.where(near, series, far) / s
    # order == -2: only I x I
    series = sum(w * _poly(_F2, np.minimum(z, Z_SERIES)) for (w, r), z in zip(pairs, zs))
    rs = np.stack([r for _, r in pairs])
    same = np.all(rs >= 0, axis=0) | np.all(rs <= 0, axis=0)
    wsum = sum(w for w, _ in pairs)
    lin = sum(w * z for (w, _), z in zip(pairs, zs)) * (8.0 / 3.0) - 5.0 * wsum
    expo = sum(w * (5.0 + 7.0 * z / 3.0 + z * z / 3.0) * np.exp(-z) for (w, _), z in zip(pairs, zs))
    far = np.where(same, 0.0, lin) + expo
    return np.where(near, series, far) / (s * s)


# ----------------------------------------------------------------------------
# Observation blocks: tensor grids of d-dimensional functionals
# ----------------------------------------------------------------------------
class Block:
    """A tensor grid of d-dimensional functionals sum_t c_t prod_i F_{t,i}.

    Every functional of the block is indexed by a multi-index over ``shape``
    (row-major); term t contributes c_t times the product over axes of the
    1D functional family F_{t,i} evaluated at that index.  c_t is a scalar or,
    for a piecewise-constant variable coefficient (one value per functional,
    App. C.4 "Variable bathymetry"), an array over the block.  With several
    outputs (Sec. 3.3), term t acts on the component outs[t]."""

    def __init__(self, shape: Sequence[int], terms: List[Tuple[float, list]], name: str = "",
                 outs: Sequence[int] = None):
        self.shape = tuple(int(n) for n in shape)
        self.terms = terms
        self.name = name
        self.outs = [0] * len(terms) if outs is None else [int(o) for o in outs]

    @property
    def size(self) -> int:
        return int(np.prod(self.shape))


def pde_blocks(prob) -> List[Block]:
    """L_PDE of a factorized box scheme (Sec. 4.1): one volume per cell,
    L_V[u] = sum_alpha c_alpha int_V D^alpha u  (Eq. linop-def, Eq. multi-input-fv).
    With collocation observations (Sec. 3: the collocation operator
    L_x[u] = D[u](x)) the functional of a cell is instead D[u] at its centre:
    sum_alpha c_alpha D^alpha u (x_V), point families of order alpha_i.
    With several outputs (Sec. 3.3) equation e is sum over its terms
    c_{alpha,i} D^alpha u_i: one block per equation, in equation order."""
    colloc = getattr(prob, "observe", "fvm") == "collocation"
    fields = getattr(prob, "fields", None)
    eqs = getattr(prob, "term_eq", None) or [0] * len(prob.terms)
    outs = getattr(prob, "term_out", None) or [0] * len(prob.terms)
    blocks = []
    for e in range(max(eqs) + 1):
        terms, touts = [], []
        for k, (alpha, c) in enumerate(prob.terms):
            if eqs[k] != e:
                continue
            if fields is not None and fields[k] is not None:
                c = float(c) * np.asarray(fields[k], np.float64).ravel()
            if colloc:
                fams = [point_family(0.5 * (ed[:-1] + ed[1:]), a) for ed, a in zip(prob.edges, alpha)]
            else:
                fams = [cell_family(ed[:-1], ed[1:], a) for ed, a in zip(prob.edges, alpha)]
            terms.append((c if isinstance(c, np.ndarray) else float(c), fams))
            touts.append(outs[k])
        blocks.append(Block(prob.n_cells, terms, f"pde{e}", touts))
    return blocks


def pde_block(prob) -> Block:
    """The PDE block of a one-equation problem (see pde_blocks)."""
    blocks = pde_blocks(prob)
    if len(blocks) != 1:
        raise ValueError("several equations: use pde_blocks")
    return blocks[0]


def point_block(ps) -> Block:
    """A tensor grid of point functionals d^m u (x) (initial/boundary data) of
    the component ps.out."""
    return Block(ps.shape, [(1.0, [point_family(x, m) for x, m in zip(ps.coords, ps.order)])],
                 ps.name, [getattr(ps, "out", 0)])


def pred_blocks(prob) -> List[Block]:
    """Point evaluations u_j(x) on the prediction grid, one block per output j."""
    return [Block([len(p) for p in prob.pred], [(1.0, [point_family(p, 0) for p in prob.pred])], f"pred{j}",
                  [j]) for j in range(getattr(prob, "n_out", 1))]


def pred_block(prob) -> Block:
    """Point evaluations u(x) on the prediction grid."""
    return pred_blocks(prob)[0]


def block_cov(X: Block, Y: Block, ell: Sequence[float], outputscale: float) -> np.ndarray:
    """Dense cross-covariance  L_X k L_Y'  evaluated entry by entry (Eq. LkL):
    sum over term pairs of c c' times the product over axes of 1D covariances."""
    I = np.unravel_index(np.arange(X.size), X.shape)
    J = np.unravel_index(np.arange(Y.size), Y.shape)
    out = np.zeros((X.size, Y.size))
    for (c1, F), o1 in zip(X.terms, X.outs):
        for (c2, G), o2 in zip(Y.terms, Y.outs):
            if o1 != o2:  # outputs are a priori uncorrelated (Eq. multioutput-cov-def)
                continue
            # a variable coefficient makes the term pair a Hadamard product with
            # the rank-one matrix c1 c2^T (App. C.4)
            prod = np.outer(np.broadcast_to(c1, (X.size,)), np.broadcast_to(c2, (Y.size,))).copy()
            for ax in range(len(X.shape)):
                C = cov_1d(F[ax], G[ax], ell[ax])
                prod *= C[I[ax][:, None], J[ax][None, :]]
            out += prod
    return outputscale * out


# ----------------------------------------------------------------------------
# Dense exact posterior (Sec. 2.1, Eqs. lin-cond-mean / lin-cond-cov)
# ----------------------------------------------------------------------------
def ibvp_blocks(prob):
    """Observation blocks in the order of L_IBVP = (L_IC,BC ; L_PDE) (Sec. 2.2)."""
    return [point_block(s) for s in prob.sets] + pde_blocks(prob)


def noise_diag(prob) -> np.ndarray:
    """Diagonal of Sigma: each point set's noise variance, jitter on volumes."""
    parts = [np.full(s.size, s.noise_var) for s in prob.sets] + [np.full(prob.N, prob.jitter)]
    return np.concatenate(parts)


def observations(prob) -> np.ndarray:
    """y = (y_IC,BC ; y_PDE); y_PDE holds the volume integrals of f (zero if homogeneous)."""
    rhs = np.zeros(prob.N) if prob.rhs is None else np.asarray(prob.rhs, np.float64).ravel()
    return np.concatenate([np.asarray(s.values, np.float64).ravel() for s in prob.sets] + [rhs])


def dense_gram(prob) -> np.ndarray:
    """G = L k L' + Sigma for the stacked IBVP operator, assembled entrywise."""
    blocks = ibvp_blocks(prob)
    rows = [np.hstack([block_cov(X, Y, prob.lengthscale, prob.outputscale) for Y in blocks])
            for X in blocks]
    G = np.vstack(rows)
    G[np.diag_indices_from(G)] += noise_diag(prob)
    return G


def dense_posterior(prob, return_gram: bool = False):
    """Exact posterior mean and variance on the prediction grid.

    m*(x) = L k(x)^T G^-1 y,   v(x) = k(x,x) - || chol(G)^-1 L k(x) ||^2
    (zero prior mean, zero noise mean; G is positive definite so G^+ = G^-1)."""
    G = dense_gram(prob)
    y = observations(prob)
    pbs = pred_blocks(prob)  # one per output: the grid output-major
    Kx = np.vstack([np.hstack([block_cov(X, pb, prob.lengthscale, prob.outputscale) for pb in pbs])
                    for X in ibvp_blocks(prob)])
    L = sla.cholesky(G, lower=True)
    alpha = sla.cho_solve((L, True), y)
    mean = Kx.T @ alpha
    V = sla.solve_triangular(L, Kx, lower=True)
    var = prob.outputscale - np.sum(V * V, axis=0)
    if return_gram:
        return mean, var, G, y, Kx
    return mean, var


# ----------------------------------------------------------------------------
# Kronecker-structured operator (Sec. 4.1, Eq. kronecker-structure)
# ----------------------------------------------------------------------------
def mode_apply(mats: Sequence[np.ndarray], V: np.ndarray) -> np.ndarray:
    """(mats[0] (x) mats[1] (x) ... ) applied to a row-major tensor V:
    one mode product per axis (Van Loan's Kronecker matvec)."""
    out = V
    for ax, A in enumerate(mats):
        out = np.moveaxis(np.tensordot(A, out, axes=([1], [ax])), 0, ax)
    return out


class KronIBVP:
    """The IBVP Gram operator applied through its Kronecker factors.

    G_PP = sum_{a,b} c_a c_b (x)_i A_i^{a_i b_i}   (Eq. kronecker-structure)
    with A_i^{pq} = L_{G_i;p} k^(i) L'_{G_i;q}, evaluated naively pair by pair
    (no sharing of mode products); point-set blocks are Kronecker products of
    rectangular 1D factors; G_BB is assembled densely entrywise.  A
    piecewise-constant variable coefficient c_a (one value per cell) turns
    each Kronecker term into its Hadamard product with the rank-one matrix
    c_a c_b^T (App. C.4), applied as diag(c_a) (x)A diag(c_b).  For a system
    (Sec. 3.3) G_PP has a block per pair of equations, holding the pairs of
    their terms that act on one output, and every set or prediction block meets
    only the terms on its own output."""

    def __init__(self, prob):
        self.prob = prob
        self.ell = prob.lengthscale
        self.s2 = prob.outputscale
        eqs = pde_blocks(prob)
        self.neq = len(eqs)
        self.nout = int(getattr(prob, "n_out", 1))
        self.pde = eqs[0] if self.neq == 1 else None  # the one-equation block
        self.sets = [point_block(s) for s in prob.sets]
        self.pred = pred_blocks(prob)[0]  # the grid (every output is evaluated on it)
        self.shape = prob.n_cells
        self.Nc = int(np.prod(self.shape))
        self.Pp = self.pred.size
        self.P = self.Pp * self.nout
        d = prob.ndim
        # PDE x PDE: (equation e, equation e2, coefficients, factors) for every pair
        # of terms acting on one output (Sec. 3.3: outputs are a priori uncorrelated)
        self.pp = []
        for e, X in enumerate(eqs):
            for e2, Y in enumerate(eqs):
                for (c1, F), o1 in zip(X.terms, X.outs):
                    for (c2, G), o2 in zip(Y.terms, Y.outs):
                        if o1 == o2:
                            self.pp.append((e, e2, (c1, c2), [cov_1d(F[i], G[i], self.ell[i]) for i in range(d)]))
        # PDE x set s (N_i x n_{s,i} factors per term of an equation on the set's output)
        self.pb = []
        for sb in self.sets:
            (_, G), = sb.terms
            self.pb.append([(e, c, [cov_1d(F[i], G[i], self.ell[i]) for i in range(d)])
                            for e, X in enumerate(eqs) for (c, F), o in zip(X.terms, X.outs) if o == sb.outs[0]])
        # PDE x prediction grid of output j, and set x prediction grid (of the set's output)
        (_, Pf), = self.pred.terms
        self.pp_pred = [[(e, c, [cov_1d(F[i], Pf[i], self.ell[i]) for i in range(d)])
                         for e, X in enumerate(eqs) for (c, F), o in zip(X.terms, X.outs) if o == j]
                        for j in range(self.nout)]
        self.b_pred = []
        for sb in self.sets:
            (_, G), = sb.terms
            self.b_pred.append([cov_1d(G[i], Pf[i], self.ell[i]) for i in range(d)])
        # dense G_BB with noise
        if self.sets:
            self.Gbb = np.vstack([np.hstack([block_cov(X, Y, self.ell, self.s2) for Y in self.sets])
                                  for X in self.sets])
            self.Gbb[np.diag_indices_from(self.Gbb)] += np.concatenate(
                [np.full(s.size, s.noise_var) for s in prob.sets])
            self.Lbb = sla.cholesky(self.Gbb, lower=True)
        else:
            self.Gbb = np.zeros((0, 0))
            self.Lbb = np.zeros((0, 0))
        self.yB = np.concatenate([np.asarray(s.values, np.float64).ravel() for s in prob.sets]) \
            if prob.sets else np.zeros(0)
        self.yP = np.zeros(prob.N) if prob.rhs is None else np.asarray(prob.rhs, np.float64).ravel()
        self.offsets = np.cumsum([0] + [s.size for s in self.sets])

    # --- blocks -------------------------------------------------------------
    # Vectors over the PDE observations hold the equations one after another,
    # vectors over the prediction grid the outputs one after another.
    def _cells(self, c):
        """A term coefficient as a scalar or a tensor over the cells."""
        return c.reshape(self.shape) if isinstance(c, np.ndarray) else c

    def _eq(self, v):
        return v.reshape((self.neq,) + tuple(self.shape))

    def Gpp(self, v: np.ndarray) -> np.ndarray:
        V = self._eq(v)
        out = np.zeros_like(V)
        for e, e2, (c1, c2), mats in self.pp:
            out[e] += self._cells(c1) * mode_apply(mats, self._cells(c2) * V[e2])
        return self.s2 * out.ravel() + self.prob.jitter * v

    def Gbp(self, v: np.ndarray) -> np.ndarray:
        """G_BP v: PDE volumes -> point sets."""
        V = self._eq(v)
        parts = []
        for sb, terms in zip(self.sets, self.pb):
            acc = np.zeros(sb.shape)
            for e, c, mats in terms:
                acc += mode_apply([A.T for A in mats], self._cells(c) * V[e])
            parts.append(self.s2 * acc.ravel())
        return np.concatenate(parts) if parts else np.zeros(0)

    def Gpb(self, w: np.ndarray) -> np.ndarray:
        """G_PB w: point sets -> PDE volumes."""
        out = np.zeros((self.neq,) + tuple(self.shape))
        for k, (sb, terms) in enumerate(zip(self.sets, self.pb)):
            W = w[self.offsets[k]:self.offsets[k + 1]].reshape(sb.shape)
            for e, c, mats in terms:
                out[e] += self._cells(c) * mode_apply(mats, W)
        return self.s2 * out.ravel()

    def Hsolve(self, w: np.ndarray) -> np.ndarray:
        """G_BB^-1 w by the Cholesky factor of the IC/BC Gram matrix."""
        if w.size == 0:
            return w
        return sla.cho_solve((self.Lbb, True), w)

    # --- deflated system (Sec. 4.2) ----------------------------------------
    def Ghat(self, v: np.ndarray) -> np.ndarray:
        """Gram matrix of the PDE observations under the IC/BC-conditioned prior:
        G_PP - G_PB G_BB^-1 G_BP (Schur complement)."""
        return self.Gpp(v) - self.Gpb(self.Hsolve(self.Gbp(v)))

    def rhs_hat(self) -> np.ndarray:
        """y_PDE minus the IC/BC-conditioned prior mean of the volume observations."""
        return self.yP - self.Gpb(self.Hsolve(self.yB))

    # --- prediction-side products --------------------------------------------
    def _out(self, b):
        return b.reshape((self.nout,) + tuple(self.pred.shape))

    def KPx(self, x: np.ndarray) -> np.ndarray:
        """L_PDE k(X*)^T x (volumes -> prediction grid of every output)."""
        X = self._eq(x)
        out = np.zeros((self.nout,) + tuple(self.pred.shape))
        for j, terms in enumerate(self.pp_pred):
            for e, c, mats in terms:
                out[j] += mode_apply([A.T for A in mats], self._cells(c) * X[e])
        return self.s2 * out.ravel()

    def KBx(self, w: np.ndarray) -> np.ndarray:
        """L_IC,BC k(X*)^T w (point sets -> prediction grid of their outputs)."""
        out = np.zeros((self.nout,) + tuple(self.pred.shape))
        for k, (sb, mats) in enumerate(zip(self.sets, self.b_pred)):
            W = w[self.offsets[k]:self.offsets[k + 1]].reshape(sb.shape)
            out[sb.outs[0]] += mode_apply([A.T for A in mats], W)
        return self.s2 * out.ravel()

    def KPxT(self, beta: np.ndarray) -> np.ndarray:
        """L_PDE k(X*) beta (prediction grid -> volumes): the adjoint of KPx."""
        B = self._out(beta)
        out = np.zeros((self.neq,) + tuple(self.shape))
        for j, terms in enumerate(self.pp_pred):
            for e, c, mats in terms:
                out[e] += self._cells(c) * mode_apply(mats, B[j])
        return self.s2 * out.ravel()

    def KBxT(self, beta: np.ndarray) -> np.ndarray:
        """L_IC,BC k(X*) beta (prediction grid -> point sets): the adjoint of KBx."""
        B = self._out(beta)
        parts = [self.s2 * mode_apply(mats, B[sb.outs[0]]).ravel() for sb, mats in zip(self.sets, self.b_pred)]
        return np.concatenate(parts) if parts else np.zeros(0)

    def Lhat_k(self, beta: np.ndarray) -> np.ndarray:
        """Lhat k(X*) beta: the cross-covariance of the volume observations with
        the prediction points under the IC/BC-conditioned prior (Sec. 4.2),
        L_PDE k(X*) beta - G_PB G_BB^-1 L_IC,BC k(X*) beta."""
        return self.KPxT(beta) - self.Gpb(self.Hsolve(self.KBxT(beta)))

    def KB_dense(self) -> np.ndarray:
        """L_IC,BC k(X*) as a dense M x P matrix (entrywise), outputs one after another."""
        if not self.sets:
            return np.zeros((0, self.P))
        preds = pred_blocks(self.prob)
        return np.vstack([np.hstack([block_cov(X, Pj, self.ell, self.s2) for Pj in preds]) for X in self.sets])


def cg_itergp(K: KronIBVP, max_iter: int, rtol: float = 0.0, want_var: bool = True,
              reorth: bool = True, keep_dirs: list = None):
    """CG on the deflated system with the IterGP combined posterior (Sec. 4.1/4.2).

    Recurrence (x0 = 0): q = G^ p, eta = p.q, alpha = r.r/eta, x += alpha p,
    r -= alpha q, beta = r'.r'/r.r, p = r' + beta p.  With CG actions the
    IterGP inverse estimate is C_i = sum_j p_j p_j^T / eta_j, so the combined
    posterior variance removes sum_j (Lhat k(x)^T p_j)^2 / eta_j, where
    Lhat k = L_PDE k - G_PB G_BB^-1 L_IC,BC k is the cross-covariance under the
    IC/BC-conditioned prior.  That sum presumes G^-conjugate directions, which
    finite precision loses; following the paper's stabilisation (Sec. 7, full
    reorthogonalisation) each new direction is made G^-conjugate to all
    previous ones: p <- p - sum_j (q_j.p / eta_j) p_j with q_j = G^ p_j.
    Stops when ||r||/||b|| <= rtol or after max_iter iterations."""
    b = K.rhs_hat()
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    bnorm = math.sqrt(rr)
    down = np.zeros(K.P)
    it = 0
    hist = [1.0]
    S, Q, etas = [], [], []
    while it < max_iter and bnorm > 0 and math.sqrt(rr) > rtol * bnorm:
        w = K.Hsolve(K.Gbp(p))
        q = K.Gpp(p) - K.Gpb(w)
        eta = float(p @ q)
        if not eta > 0:
            raise FloatingPointError("CG breakdown: p^T G p <= 0")
        if want_var:
            u = K.KPx(p) - K.KBx(w)
            down += u * u / eta
        a = rr / eta
        x += a * p
        r -= a * q
        rr_new = float(r @ r)
        if keep_dirs is not None:
            keep_dirs.append((p.copy(), eta))
        if reorth:
            S.append(p)
            Q.append(q)
            etas.append(eta)
        p = r + (rr_new / rr) * p
        if reorth:
            c = (np.array(Q) @ p) / np.array(etas)
            p = p - np.array(S).T @ c
        rr = rr_new
        it += 1
        hist.append(math.sqrt(rr) / bnorm if bnorm > 0 else 0.0)
    return x, down, it, hist


def kron_posterior(prob, max_iter: int = 100000, rtol: float = 1e-12, want_var: bool = True,
                   K: KronIBVP = None, reorth: bool = True):
    """Posterior mean and IterGP combined variance on the prediction grid via
    Cholesky (IC/BC) deflation + CG (Sec. 4.2).

    m*(x) = k_B(x)^T G_BB^-1 (y_B - G_BP x_cg) + L_PDE k(x)^T x_cg
    v(x)  = k(x,x) - || L_BB^-1 k_B(x) ||^2 - sum_j (Lhat k(x)^T p_j)^2/eta_j"""
    K = K or KronIBVP(prob)
    x, down, it, hist = cg_itergp(K, max_iter, rtol, want_var, reorth)
    wB = K.Hsolve(K.yB - K.Gbp(x))
    mean = K.KBx(wB) + K.KPx(x)
    var = None
    if want_var:
        KB = K.KB_dense()
        if KB.shape[0]:
            V = sla.solve_triangular(K.Lbb, KB, lower=True)
            var = K.s2 - np.sum(V * V, axis=0) - down
        else:
            var = K.s2 - down
    return dict(mean=mean, var=var, x=x, iters=it, hist=hist, K=K)


def itergp_actions(K: KronIBVP, S: np.ndarray):
    """IterGP combined posterior for an arbitrary action matrix S (N x k) on the
    deflated system: C = S (S^T G^ S)^-1 S^T, x = C b (Sec. 4.1, Wenger et al.'s
    IterGP as the paper uses it).  Unit-vector actions (S = I) reproduce the
    Cholesky posterior; G^-conjugate CG directions reduce C to sum p p^T/eta."""
    b = K.rhs_hat()
    GS = np.column_stack([K.Ghat(S[:, j]) for j in range(S.shape[1])])
    A = S.T @ GS
    Lc = sla.cholesky(0.5 * (A + A.T), lower=True)
    x = S @ sla.cho_solve((Lc, True), S.T @ b)
    wB = K.Hsolve(K.yB - K.Gbp(x))
    mean = K.KBx(wB) + K.KPx(x)
    U = np.column_stack([K.KPx(S[:, j]) - K.KBx(K.Hsolve(K.Gbp(S[:, j]))) for j in range(S.shape[1])])
    Z = sla.solve_triangular(Lc, U.T, lower=True)
    down = np.sum(Z * Z, axis=0)
    KB = K.KB_dense()
    base = K.s2 - (np.sum(sla.solve_triangular(K.Lbb, KB, lower=True) ** 2, axis=0) if KB.shape[0] else 0.0)
    return mean, base - down


def targeted_itergp(K: KronIBVP, max_iter: int, rtol: float, betas, want_var: bool = True):
    """Targeted uncertainty reduction (appendix "Targeted uncertainty reduction").

    First CG with the IterGP downdate (cg_itergp, reorthogonalised); its
    directions p_j with eta_j = p_j^T G^ p_j give the inverse approximation
    C = sum_j p_j p_j^T / eta_j.  Then one more IterGP action per weight vector
    beta (in the appendix a Dir(1, ..., 1) sample over the target points, zero
    on the rest of the prediction grid; the caller draws it):
        t   = Lhat k(X*) beta                 (linear combination of target columns)
        s_i = t - G^ C t                      (residual w.r.t. the inverse approximation:
                                               the action is CG on the target system)
        d_i = s_i - C G^ s_i                  (IterGP: conjugate to every earlier action)
        eta_i = d_i^T G^ d_i,   C <- C + d_i d_i^T / eta_i
        x  <- x + d_i (d_i^T r) / eta_i,  r = b - G^ x      (x stays C b)
        down <- down + (Lhat k(X*)^T d_i)^2 / eta_i
    Returns (x, down, actions s_i, CG directions as (p, eta) pairs)."""
    dirs = []
    x, down, it, hist = cg_itergp(K, max_iter, rtol, want_var, True, dirs)
    D = [d for d, _ in dirs]
    E = [e for _, e in dirs]
    GD = [K.Ghat(d) for d in D]
    b = K.rhs_hat()
    r = b - K.Ghat(x)
    actions = []
    for beta in betas:
        t = K.Lhat_k(np.asarray(beta, np.float64))
        Ct = np.zeros_like(t)
        for d, e in zip(D, E):
            Ct += d * (d @ t) / e
        s = t - K.Ghat(Ct)
        dv = s.copy()
        for d, g, e in zip(D, GD, E):
            dv -= d * (g @ s) / e
        q = K.Ghat(dv)
        eta = float(dv @ q)
        if not eta > 0:
            raise FloatingPointError("targeted action: d^T G d <= 0")
        a = float(dv @ r) / eta
        x = x + a * dv
        r = r - a * q
        if want_var:
            u = K.KPx(dv) - K.KBx(K.Hsolve(K.Gbp(dv)))
            down = down + u * u / eta
        D.append(dv)
        GD.append(q)
        E.append(eta)
        actions.append(s)
    return x, down, actions, dirs


def restriction(shape, factor: int) -> np.ndarray:
    """W (N x N_c): column c is the indicator of the fine cells inside coarse
    cell c, the axes coarsened by `factor` (each axis size divisible by it).
    A coarse volume is the disjoint union of its fine volumes, so its FVM
    observation is the sum of theirs (appendix "Multigrid preconditioners",
    Eq. subdomain-partition): y_coarse = W^T y_fine."""
    shape = tuple(int(n) for n in shape)
    cshape = tuple(n // factor for n in shape)
    if any(n % factor for n in shape):
        raise ValueError("axis sizes must be divisible by the coarsening factor")
    fine = np.indices(shape).reshape(len(shape), -1) // factor
    cidx = np.ravel_multi_index(tuple(fine), cshape)
    W = np.zeros((int(np.prod(shape)), int(np.prod(cshape))))
    W[np.arange(W.shape[0]), cidx] = 1.0
    return W


def multigrid_itergp(K: KronIBVP, factor: int, max_iter: int, rtol: float = 0.0, want_var: bool = True):
    """Multigrid warm start (appendix "Multigrid preconditioners"): the
    IC/BC-conditioned prior is conditioned further, exactly, on the coarse FVM
    observations W^T y (by a Cholesky factorisation), and IterGP continues with
    CG actions on the fine observations.
      A_c = W^T G^ W = L_c L_c^T                 (the coarse observations' Gram)
      x0  = W A_c^-1 W^T b,  r0 = b - G^ x0      (exact solve on the coarse scheme)
      down0 = diag(U^T A_c^-1 U),  U = Lhat k(X*)^T W
    then CG from r0 whose every direction is made G^-conjugate to span W
    (p <- p - W A_c^-1 (G^ W)^T p) and to the earlier directions (Sec. 7), with
    the downdate of each CG action added to down0.
    Returns (x, down, CG iterations, W, directions as (p, eta) pairs)."""
    W = restriction(K.shape, factor)
    b = K.rhs_hat()
    GW = np.column_stack([K.Ghat(W[:, c]) for c in range(W.shape[1])])
    Ac = W.T @ GW
    Lc = sla.cholesky(0.5 * (Ac + Ac.T), lower=True)
    x = W @ sla.cho_solve((Lc, True), W.T @ b)
    r = b - K.Ghat(x)
    down = np.zeros(K.P)
    if want_var:
        U = np.column_stack([K.KPx(W[:, c]) - K.KBx(K.Hsolve(K.Gbp(W[:, c]))) for c in range(W.shape[1])])
        Z = sla.solve_triangular(Lc, U.T, lower=True)
        down = np.sum(Z * Z, axis=0)

    def deflate(v):
        return v - W @ sla.cho_solve((Lc, True), GW.T @ v)

    p = deflate(r.copy())
    rr = float(r @ r)
    bnorm = math.sqrt(float(b @ b))
    S, Q, E, dirs = [], [], [], []
    it = 0
    while it < max_iter and bnorm > 0 and math.sqrt(rr) > rtol * bnorm:
        q = K.Ghat(p)
        eta = float(p @ q)
        if not eta > 0:
            raise FloatingPointError("CG breakdown: p^T G p <= 0")
        if want_var:
            u = K.KPx(p) - K.KBx(K.Hsolve(K.Gbp(p)))
            down += u * u / eta
        a = float(p @ r) / eta
        x += a * p
        r -= a * q
        rr_new = float(r @ r)
        S.append(p)
        Q.append(q)
        E.append(eta)
        dirs.append((p.copy(), eta))
        p = deflate(r + (rr_new / rr) * p)
        c = (np.array(Q) @ p) / np.array(E)
        p = p - np.array(S).T @ c
        rr = rr_new
        it += 1
    return x, down, it, W, dirs


def posterior_from(K: KronIBVP, x: np.ndarray, down: np.ndarray):
    """Posterior mean and IterGP variance on the prediction grid from the
    representer weights x and the downdate (Eqs. lin-cond-mean, lin-cond-cov)."""
    wB = K.Hsolve(K.yB - K.Gbp(x))
    mean = K.KBx(wB) + K.KPx(x)
    KB = K.KB_dense()
    base = K.s2 - (np.sum(sla.solve_triangular(K.Lbb, KB, lower=True) ** 2, axis=0) if KB.shape[0] else 0.0)
    return mean, base - down


def true_residual(K: KronIBVP, x: np.ndarray) -> float:
    b = K.rhs_hat()
    return float(np.linalg.norm(b - K.Ghat(x)) / np.linalg.norm(b))


PINS = {
    "kderiv, g1, f2": "quadrature + finite differences + series/closed-form switch continuity",
    "cov_1d": "adaptive quadrature of the defining integrals; symmetry; Toeplitz; sub-cell additivity",
    "block_cov/dense_gram": "brute-force 3D quadrature of entries; symmetry; positive definiteness",
    "dense_posterior": "heat 1D+t analytic solution with refinement; Fig. 2 toy vs sin x; "
                       "observation interpolation; FVM integrals of the mean reproduce y_PDE",
    "KronIBVP": "equals dense_gram blocks on small grids",
    "cg_itergp/kron_posterior": "deflated == full dense posterior; IterGP at N iterations == "
                                "Cholesky variance; CG variance >= exact and non-increasing",
    "kderiv orders 3, 4 / order-2 point families": "finite differences; the spectral moment k^(4)(0) by "
                                                    "quadrature of the Matern spectral density; collocation "
                                                    "posteriors of the Fig. 2 toy and the 1D heat equation "
                                                    "converge to the analytic solutions",
    "variable coefficients (pde_block / block_cov / KronIBVP)": "Kronecker-with-diagonals == entrywise dense "
                                                                "blocks; constant fields == scalar coefficients; "
                                                                "manufactured variable-coefficient heat solution",
    "restriction/multigrid_itergp": "equals itergp_actions on [W | CG directions]; with no CG step it is the "
                                    "dense posterior of the same IBVP on the coarse cells; converged, the dense "
                                    "fine posterior",
    "KPxT/KBxT/Lhat_k": "adjoint identities against KPx/KBx; entrywise dense cross-covariances (block_cov)",
    "targeted_itergp/posterior_from": "equals itergp_actions on [CG directions | targeted actions]; one action "
                                      "on one point is the Cauchy-Schwarz-optimal single-action reduction; "
                                      "repeated targeted actions reach the exact (Cholesky) variance there",
    "KronIBVP for systems": "every block product equals the dense entrywise blocks (block_cov) of the same "
                            "system; the converged kron_posterior equals dense_posterior",
    "multi-output (pde_blocks / pred_blocks / block_cov outs)": "two decoupled equations == the pair of one-output "
                                                                "posteriors; an unobserved output keeps its prior; "
                                                                "the first-order 1D wave system and the linearised "
                                                                "shallow-water standing wave converge to their analytic "
                                                                "solutions (and not with a term on the wrong component)",
}
