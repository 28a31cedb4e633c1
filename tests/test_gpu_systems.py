"""Systems of PDEs in several outputs (Sec. 3.3, multi-dimensional codomains)
on the GPU against the oracle: the block operators G_PP, G_BP, G_PB against
the dense entrywise blocks, and the converged FP64 posterior of every output
against the dense Cholesky posterior."""
from dataclasses import replace

import numpy as np
import pytest

import gpfvm_workloads as W
import oracle as O

pytestmark = pytest.mark.gpu

RTOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_05020_gb300 import build
    build.build()


def relerr(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


PROBS = {
    "wave1d_system": lambda: W.wave_1d_system(6, 7, pred=(5, 6)),
    "wave1d_system_colloc": lambda: W.collocation(W.wave_1d_system(6, 7, pred=(5, 6))),
    "swe2d": lambda: W.shallow_water_2d(4, 5, 6, f=0.0, k=0.0, n_ic=(4, 5), n_bc=(2, 3), pred=(3, 4, 3)),
    # with Coriolis and drag: 11 terms in 3 equations (App. C.4's system at constant depth)
    "swe2d_coriolis_drag": lambda: W.shallow_water_2d(4, 5, 6, f=0.5, k=0.1, n_ic=(4, 5), n_bc=(2, 3),
                                                      pred=(3, 4, 3)),
    "swe2d_ragged": lambda: W.shallow_water_2d(3, 6, 4, H=0.7, g=1.3, f=0.0, k=0.0, n_ic=(5, 3), n_bc=(2, 2),
                                               pred=(2, 3, 4), ell=(0.5, 0.35, 0.3)),
    # one output observed by two equations (an overdetermined pair on u)
    "two_eq_one_out": lambda: replace(W.heat_1d(5, 6, n_ic=5, n_bc=3, pred=5),
                                      terms=[((1, 0), 1.0), ((0, 2), -0.1), ((1, 0), 2.0), ((0, 2), -0.2)],
                                      n_out=1, term_eq=[0, 0, 1, 1], term_out=[0, 0, 0, 0]),
}


def _gpu(prob, max_iter=2000):
    from paper_2406_05020_gb300 import gpfvm
    pb = gpfvm.Problem(prob, max_iter=max_iter)
    pb.assemble()
    return pb


def _apply(pb, op, v, n_out):
    import torch
    out = torch.full((n_out,), float("nan"), dtype=torch.float64, device="cuda")
    pb.matvec(op, torch.as_tensor(np.ascontiguousarray(v), device="cuda"), out)
    return out.cpu().numpy()


@pytest.mark.parametrize("name", list(PROBS))
def test_system_block_operators_match_dense_blocks(name):
    prob = PROBS[name]()
    pb = _gpu(prob, max_iter=8)
    assert (pb.N, pb.M, pb.P) == (prob.N, prob.M, prob.P)
    eqs = O.pde_blocks(prob)
    sets = [O.point_block(s) for s in prob.sets]
    cov = lambda X, Y: O.block_cov(X, Y, prob.lengthscale, prob.outputscale)  # noqa: E731
    Gpp = np.vstack([np.hstack([cov(X, Y) for Y in eqs]) for X in eqs])
    Gbp = np.vstack([np.hstack([cov(S, Y) for Y in eqs]) for S in sets])
    rng = np.random.default_rng(7)
    v = rng.normal(size=prob.N)
    w = rng.normal(size=prob.M)
    assert relerr(_apply(pb, 0, v, prob.N), Gpp @ v + prob.jitter * v) < 1e-12
    assert relerr(_apply(pb, 2, v, prob.M), Gbp @ v) < 1e-12
    assert relerr(_apply(pb, 3, w, prob.N), Gbp.T @ w) < 1e-12
    # the operator of the FP64 CG: G^ = G_PP - G_PB G_BB^-1 G_BP
    Gbb = np.vstack([np.hstack([cov(S, T) for T in sets]) for S in sets])
    Gbb[np.diag_indices_from(Gbb)] += np.concatenate([np.full(s.size, s.noise_var) for s in prob.sets])
    ghat = Gpp @ v + prob.jitter * v - Gbp.T @ np.linalg.solve(Gbb, Gbp @ v)
    assert relerr(_apply(pb, 1, v, prob.N), ghat) < 1e-10
    pb.close()


@pytest.mark.parametrize("name", list(PROBS))
def test_system_posterior_matches_dense_cholesky(name):
    import torch
    prob = PROBS[name]()
    pb = _gpu(prob)
    code, info = pb.solve(max_iter=2000, rtol=1e-13, reorth=True, want_var=True)
    assert code == 0, info.as_dict()
    m, v = O.dense_posterior(prob)
    mean = torch.empty(pb.P, dtype=torch.float64, device="cuda")
    var = torch.empty_like(mean)
    pb.query(mean, var)
    assert relerr(mean.cpu().numpy(), m) < RTOL
    # per output too (a mix-up of the output blocks would leave the norm intact
    # only if the outputs had equal posteriors)
    Pp = prob.P // prob.n_out
    for j in range(prob.n_out):
        mj = m[j * Pp:(j + 1) * Pp]
        if np.linalg.norm(mj) > 1e-8:
            assert relerr(mean.cpu().numpy()[j * Pp:(j + 1) * Pp], mj) < 1e-9
    assert np.all(var.cpu().numpy() >= v - 1e-9)
    pb.close()


def test_wave_system_reaches_the_analytic_solution():
    """The first-order 1D wave system on 16 x 16 cells: the GPU posterior mean
    is within 1e-3 of u = sin(pi x) cos(pi t), v = -cos(pi x) sin(pi t)."""
    import torch
    prob = W.wave_1d_system(16, 16, pred=(9, 9))
    pb = _gpu(prob)
    code, info = pb.solve(max_iter=2000, rtol=1e-12, reorth=True, want_var=False)
    assert code == 0, info.as_dict()
    mean = torch.empty(pb.P, dtype=torch.float64, device="cuda")
    pb.query(mean, None)
    T, X = np.meshgrid(prob.pred[0], prob.pred[1], indexing="ij")
    exact = np.concatenate([(np.sin(np.pi * X) * np.cos(np.pi * T)).ravel(),
                            (-np.cos(np.pi * X) * np.sin(np.pi * T)).ravel()])
    assert np.abs(mean.cpu().numpy() - exact).max() < 1e-3
    pb.close()


def test_system_limits_are_reported():
    """Systems run FP64 with the dense IC/BC stage; mixed precisions and
    targeted actions are refused with an error, not computed some other way."""
    import torch

    from paper_2406_05020_gb300 import gpfvm
    prob = PROBS["wave1d_system"]()
    pb = _gpu(prob)
    assert int(pb.export(10, 3)[0]) == 0  # dense IC/BC stage
    with pytest.raises(gpfvm.GpfvmError):
        pb.solve(max_iter=50, rtol=1e-8, precision=gpfvm.MIXED_FP32)
    code, _ = pb.solve(max_iter=2000, rtol=1e-10, reorth=True, want_var=True)
    assert code == 0
    with pytest.raises(gpfvm.GpfvmError):
        pb.target(torch.ones((1, pb.P), dtype=torch.float64, device="cuda"))
    pb.close()
