"""Variable coefficients on the GPU (App. C.4: a piecewise-constant
coefficient per cell makes each Kronecker term a Hadamard product with a
rank-one matrix) against the oracle: operators, fixed iterations, converged
posteriors and the mixed-precision solve."""
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
    "heat1d_var": lambda: W.heat_1d_varcoef(6, 9, pred=7),
    "heat2d_var_ragged": lambda: W.heat_2d_varcoef(5, 7, 9, n_ic=(4, 3), n_bc=(2, 3), pred=(3, 2, 4),
                                                   ell=(0.4, 0.3, 0.35)),
    "heat2d_var_16": lambda: W.heat_2d_varcoef(16, 16, 16, n_ic=(16, 16), n_bc=(4, 4), pred=(8, 8, 8)),
}


def _post(pb):
    import torch
    m = torch.empty(pb.P, dtype=torch.float64, device="cuda")
    v = torch.empty_like(m)
    pb.query(m, v)
    return m.cpu().numpy(), v.cpu().numpy()


@pytest.mark.parametrize("name", list(PROBS))
def test_varcoef_operators_match_oracle(name):
    import torch

    from paper_2406_05020_gb300 import gpfvm
    prob = PROBS[name]()
    pb = gpfvm.Problem(prob, max_iter=64)
    pb.assemble()
    K = O.KronIBVP(prob)
    rng = np.random.default_rng(4)
    v, w = rng.normal(size=prob.N), rng.normal(size=prob.M)
    out = torch.empty(prob.N, dtype=torch.float64, device="cuda")
    outm = torch.empty(prob.M, dtype=torch.float64, device="cuda")
    pb.matvec(0, torch.as_tensor(v, device="cuda"), out)
    assert relerr(out.cpu().numpy(), K.Gpp(v)) < 1e-13
    pb.matvec(1, torch.as_tensor(v, device="cuda"), out)
    assert relerr(out.cpu().numpy(), K.Ghat(v)) < 1e-11
    pb.matvec(2, torch.as_tensor(v, device="cuda"), outm)
    assert relerr(outm.cpu().numpy(), K.Gbp(v)) < 1e-13
    pb.matvec(3, torch.as_tensor(w, device="cuda"), out)
    assert relerr(out.cpu().numpy(), K.Gpb(w)) < 1e-13
    assert relerr(pb.export(0, prob.N), K.rhs_hat()) < 1e-11
    pb.matvec(4, torch.as_tensor(v, device="cuda"), out)  # FP32 form
    assert relerr(out.cpu().numpy(), K.Gpp(v)) < 2e-6
    with pytest.raises(gpfvm.GpfvmError):  # no tensor-core form for variable coefficients
        pb.matvec(5, torch.as_tensor(v, device="cuda"), out)
    pb.close()


@pytest.mark.parametrize("name", list(PROBS))
def test_varcoef_fixed_iterations_and_converged_posterior(name):
    from paper_2406_05020_gb300 import gpfvm
    prob = PROBS[name]()
    pb = gpfvm.Problem(prob, max_iter=4000)
    pb.assemble()
    iters = min(8, max(prob.N // 4, 2))
    pb.solve(max_iter=iters, rtol=0.0, reorth=True, want_var=True)
    r = O.kron_posterior(prob, max_iter=iters, rtol=0.0)
    m, v = _post(pb)
    assert relerr(m, r["mean"]) < RTOL
    np.testing.assert_allclose(v, r["var"], atol=RTOL * prob.outputscale, rtol=0)
    code, info = pb.solve(max_iter=4000, rtol=1e-12, reorth=True, want_var=True)
    assert code == 0
    m, v = _post(pb)
    if prob.N + prob.M < 3000:
        md, vd = O.dense_posterior(prob)
        assert relerr(m, md) < 1e-8
        assert np.all(v >= vd - 1e-8)
    code, info = pb.solve(max_iter=4000, rtol=1e-10, precision=gpfvm.MIXED_FP32, reorth=True, want_var=True)
    assert code == 0, info.as_dict()
    m32, _ = _post(pb)
    assert relerr(m32, m) < 1e-6
    pb.close()


def test_varcoef_manufactured_solution_on_gpu():
    """The manufactured variable-coefficient heat problem (u* = e^-t sin pi x)
    solved on the GPU: the posterior mean is within the oracle's discretisation
    error of u* and equals the dense oracle posterior."""
    from paper_2406_05020_gb300 import gpfvm
    prob = W.heat_1d_varcoef(16, 32)
    pb = gpfvm.Problem(prob, max_iter=3000)
    pb.assemble()
    code, info = pb.solve(max_iter=3000, rtol=1e-12, reorth=True, want_var=True)
    assert code == 0
    m, _ = _post(pb)
    T, X = np.meshgrid(prob.pred[0], prob.pred[1], indexing="ij")
    assert np.abs(m - (np.exp(-T) * np.sin(np.pi * X)).ravel()).max() < 5e-3
    md, _ = O.dense_posterior(prob)
    assert relerr(m, md) < 1e-8
    pb.close()
