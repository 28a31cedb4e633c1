"""Targeted uncertainty reduction (appendix "Targeted uncertainty reduction")
on the GPU against the oracle's targeted_itergp: FP64 CG with the IterGP
downdate, then one action per Dirichlet weight vector over target points of
the prediction grid, continuing the same IterGP state."""
import numpy as np
import pytest

import gpfvm_workloads as W
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_05020_gb300 import build
    build.build()


def relerr(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def targets(prob, k, seed=0):
    """k Dir(1, ..., 1) weight vectors over the last time slice of the
    prediction grid near the x = 1 wall (zero elsewhere)."""
    shape = tuple(len(g) for g in prob.pred)
    mask = np.zeros(shape, bool)
    if len(shape) == 3:
        mask[-1, shape[1] // 2:, :] = True
    else:
        mask[-1, shape[1] // 2:] = True
    idx = np.flatnonzero(mask.ravel())
    rng = np.random.default_rng(seed)
    out = np.zeros((k, int(np.prod(shape))))
    for a in range(k):
        out[a, idx] = rng.dirichlet(np.ones(idx.size))
    return out, idx


PROBS = {
    "heat1d": lambda: W.heat_1d(),
    "heat2d_ragged": lambda: W.heat_2d(5, 7, 9, n_ic=(4, 3), n_bc=(2, 3), pred=(3, 2, 4), ell=(0.4, 0.3, 0.35)),
    "heat2d_16": lambda: W.heat_2d(16, 16, 16, n_ic=(16, 16), n_bc=(4, 4), pred=(8, 8, 8)),
    "wave2d": lambda: W.wave_2d(6, 9, 5, n_ic=(4, 4), n_bc=(2, 2), pred=(3, 3, 3), ell=(0.3, 0.3, 0.3)),
}


@pytest.mark.parametrize("name", list(PROBS))
def test_targeted_actions_match_oracle(name):
    import torch

    from paper_2406_05020_gb300 import gpfvm
    prob = PROBS[name]()
    K = O.KronIBVP(prob)
    iters, nact = 8, 6
    betas, idx = targets(prob, nact)
    pb = gpfvm.Problem(prob, max_iter=iters + nact)
    pb.assemble()
    code, info = pb.solve(max_iter=iters, rtol=0.0, precision=gpfvm.FP64, reorth=True, want_var=True)
    assert info.iterations == iters
    m0 = torch.empty(pb.P, dtype=torch.float64, device="cuda")
    v0 = torch.empty_like(m0)
    pb.query(m0, v0)
    pb.target(torch.as_tensor(betas, device="cuda"))
    m1 = torch.empty_like(m0)
    v1 = torch.empty_like(m0)
    pb.query(m1, v1)
    x, down, acts, dirs = O.targeted_itergp(K, iters, 0.0, list(betas))
    mean, var = O.posterior_from(K, x, down)
    np.testing.assert_allclose(v1.cpu().numpy(), var, rtol=0, atol=1e-10 * prob.outputscale)
    assert relerr(m1.cpu().numpy(), mean) < 1e-10
    np.testing.assert_allclose(pb.export(5, pb.P), down, rtol=0, atol=1e-10)
    # the actions lower the variance at the targets, never raise it anywhere
    assert np.all(v1.cpu().numpy() <= v0.cpu().numpy() + 1e-12)
    assert (v0.cpu().numpy() - v1.cpu().numpy())[idx].max() > 0
    pb.close()


def test_targeted_actions_c2_full_size():
    """2D+time heat 64^3 converged FP64 solve + 16 targeted actions on the last
    time slice: the variance at the target points drops, the mean moves by no
    more than the solve's tolerance, and the directions stay conjugate
    (every eta > 0)."""
    import torch

    from paper_2406_05020_gb300 import gpfvm
    prob = W.heat_2d(seed=2)
    nact = 16
    betas, idx = targets(prob, nact, seed=1)
    pb = gpfvm.Problem(prob, max_iter=1500)
    pb.assemble()
    code, info = pb.solve(max_iter=1500 - nact, rtol=1e-10, precision=gpfvm.FP64, reorth=True, want_var=True)
    assert code == 0
    k = info.iterations
    m0 = torch.empty(pb.P, dtype=torch.float64, device="cuda")
    v0 = torch.empty_like(m0)
    pb.query(m0, v0)
    pb.target(torch.as_tensor(betas, device="cuda"))
    m1 = torch.empty_like(m0)
    v1 = torch.empty_like(m0)
    pb.query(m1, v1)
    d = (v0 - v1).cpu().numpy()
    assert d.min() >= -1e-12
    assert d[idx].mean() > 10 * max(d.mean(), 1e-300) or d[idx].mean() > 1e-3
    assert relerr(m1.cpu().numpy(), m0.cpu().numpy()) < 1e-8
    assert np.all(pb.export(12, k + nact) > 0) and pb.export(12, k + nact).size == k + nact
    pb.close()
