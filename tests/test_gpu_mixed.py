"""Mixed-precision path (FP32 inner operator + FP64 refinement) against the
FP64 oracle.  Bar: posterior mean within 1e-6 relative of the FP64 oracle
(the accuracy the mixed solves are counted at); the IterGP variance is a
valid combined posterior, i.e. never below the exact variance."""
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


PROBS = {
    "heat1d_c1": lambda: W.heat_1d(),
    "heat2d_ragged": lambda: W.heat_2d(5, 7, 9, n_ic=(4, 3), n_bc=(2, 3), pred=(3, 2, 4), ell=(0.4, 0.3, 0.35)),
    "heat2d_16": lambda: W.heat_2d(16, 16, 16, n_ic=(16, 16), n_bc=(4, 4), pred=(8, 8, 8)),
    "wave2d": lambda: W.wave_2d(6, 9, 5, n_ic=(4, 4), n_bc=(2, 2), pred=(3, 3, 3), ell=(0.3, 0.3, 0.3)),
}


@pytest.mark.parametrize("name", list(PROBS))
def test_mixed_fp32_solve_matches_oracle(name):
    import torch

    from paper_2406_05020_gb300 import gpfvm
    prob = PROBS[name]()
    pb = gpfvm.Problem(prob, max_iter=4000)
    pb.assemble()
    code, info = pb.solve(max_iter=4000, rtol=1e-10, precision=gpfvm.MIXED_FP32, reorth=True, want_var=True)
    assert code == 0, info.as_dict()
    assert info.true_rel_residual <= 1e-10
    mean = torch.empty(pb.P, dtype=torch.float64, device="cuda")
    var = torch.empty_like(mean)
    pb.query(mean, var)
    m, v = O.dense_posterior(prob)
    assert relerr(mean.cpu().numpy(), m) < 1e-6
    assert np.all(var.cpu().numpy() >= v - 1e-7)
    pb.close()


@pytest.mark.parametrize("name", ["heat2d_ragged", "heat2d_16", "wave2d"])
def test_fp32_gram_operator_accuracy(name):
    """op 4 (FP32 mode products) agrees with the FP64 oracle to FP32 accuracy."""
    import torch

    from paper_2406_05020_gb300 import gpfvm
    prob = PROBS[name]()
    pb = gpfvm.Problem(prob, max_iter=8)
    pb.assemble()
    K = O.KronIBVP(prob)
    v = np.random.default_rng(5).normal(size=prob.N)
    out = torch.empty(prob.N, dtype=torch.float64, device="cuda")
    pb.matvec(4, torch.as_tensor(v, device="cuda"), out)
    assert relerr(out.cpu().numpy(), K.Gpp(v)) < 2e-6
    pb.close()


def test_mixed_c2_full_size_against_fp64_path():
    """2D+time heat 64^3 at full size: the mixed solve's mean is within 1e-6 of the
    plain FP64 GPU solve (itself pinned to the oracle by the parity tests)."""
    import torch

    from paper_2406_05020_gb300 import gpfvm
    prob = W.heat_2d(seed=2)
    pb = gpfvm.Problem(prob, max_iter=3000)
    pb.assemble()
    m64 = torch.empty(pb.P, dtype=torch.float64, device="cuda")
    m32 = torch.empty_like(m64)
    code, info = pb.solve(max_iter=1500, rtol=1e-10, precision=gpfvm.FP64, want_var=False)
    assert code == 0
    pb.query(m64)
    code, info = pb.solve(max_iter=3000, rtol=1e-10, precision=gpfvm.MIXED_FP32, want_var=False)
    assert code == 0, info.as_dict()
    pb.query(m32)
    assert relerr(m32.cpu().numpy(), m64.cpu().numpy()) < 1e-6
    pb.close()
