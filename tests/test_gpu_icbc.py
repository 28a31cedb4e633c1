"""The structured IC/BC stage (set 0 inverted through the eigen-decomposition
of its Kronecker factors, the other sets through the Schur complement) is an
exact reorganisation of the Cholesky conditioning on G_BB (Sec. 4.2): it must
reproduce the dense-Cholesky GPU path and the oracle."""
import os

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


def _run(prob, mode, iters):
    import torch

    from paper_2406_05020_gb300 import gpfvm
    old = os.environ.get("GPFVM_ICBC")
    os.environ["GPFVM_ICBC"] = mode
    try:
        pb = gpfvm.Problem(prob, max_iter=max(iters, 8))
    finally:
        if old is None:
            del os.environ["GPFVM_ICBC"]
        else:
            os.environ["GPFVM_ICBC"] = old
    pb.assemble()
    sweeps = pb.export(9, 6)
    b = pb.export(0, prob.N)
    code, info = pb.solve(max_iter=iters, rtol=0.0, reorth=True, want_var=True)
    mean = torch.empty(pb.P, dtype=torch.float64, device="cuda")
    var = torch.empty_like(mean)
    pb.query(mean, var)
    v = np.random.default_rng(2).normal(size=prob.N)
    out = torch.empty(prob.N, dtype=torch.float64, device="cuda")
    pb.matvec(1, torch.as_tensor(v, device="cuda"), out)
    res = dict(b=b, mean=mean.cpu().numpy(), var=var.cpu().numpy(), ghat=out.cpu().numpy(), v=v, sweeps=sweeps)
    pb.close()
    return res


PROBS = {
    "heat2d_ragged": lambda: W.heat_2d(5, 7, 9, n_ic=(6, 5), n_bc=(2, 3), pred=(3, 2, 4), ell=(0.4, 0.3, 0.35)),
    "heat2d_tiles": lambda: W.heat_2d(17, 33, 70, n_ic=(20, 23), n_bc=(4, 5), pred=(5, 6, 7)),
    "wave2d_neumann": lambda: W.wave_2d(6, 9, 5, n_ic=(5, 6), n_bc=(2, 2), pred=(3, 3, 3), ell=(0.3, 0.3, 0.3)),
    "heat1d_c1": lambda: W.heat_1d(16, 32, n_ic=33),
    "ic_only": lambda: W.heat_2d(4, 6, 5, n_ic=(7, 5), n_bc=(1, 1), pred=(2, 3, 2)),
}


@pytest.mark.parametrize("name", list(PROBS))
def test_structured_icbc_matches_dense_and_oracle(name):
    prob = PROBS[name]()
    iters = min(10, prob.N // 2)
    s = _run(prob, "structured", iters)
    d = _run(prob, "dense", iters)
    K = O.KronIBVP(prob)
    assert relerr(s["b"], K.rhs_hat()) < 1e-10
    assert relerr(s["b"], d["b"]) < 1e-10
    assert relerr(s["ghat"], K.Ghat(s["v"])) < 1e-10
    r = O.kron_posterior(prob, max_iter=iters, rtol=0.0, K=K)
    assert relerr(s["mean"], r["mean"]) < 1e-10
    assert relerr(s["mean"], d["mean"]) < 1e-10
    np.testing.assert_allclose(s["var"], r["var"], atol=1e-10, rtol=0)
    np.testing.assert_allclose(s["var"], d["var"], atol=1e-10, rtol=0)


def test_structured_icbc_c2_full_size():
    """2D+time heat 64^3 geometry (M = 5120): structured vs dense GPU stages."""
    prob = W.heat_2d(seed=4)
    s = _run(prob, "structured", 6)
    d = _run(prob, "dense", 6)
    assert relerr(s["b"], d["b"]) < 1e-10
    assert relerr(s["ghat"], d["ghat"]) < 1e-10
    assert relerr(s["mean"], d["mean"]) < 1e-10
    np.testing.assert_allclose(s["var"], d["var"], atol=1e-10, rtol=0)


def test_eigensolver_sweeps_converge_before_their_caps():
    """Both Jacobi phases stop on their convergence test (FP32 cap 30 sweeps,
    FP64 cap 12) on the full-size 2D+time heat IC grid (64 x 64 points) and on
    the 1D+time IC line."""
    for prob in (W.heat_2d(seed=4), W.heat_1d(16, 32, n_ic=33)):
        sw = _run(prob, "structured", 2)["sweeps"]
        assert len(sw) == 2 * prob.ndim
        for a in range(prob.ndim):
            s32, s64 = sw[2 * a], sw[2 * a + 1]
            if prob.sets[0].coords[a].size == 1:
                continue
            assert 1 <= s32 < 30, sw
            assert 1 <= s64 < 12, sw
