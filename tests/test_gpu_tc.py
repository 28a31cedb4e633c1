"""Tensor-core (tcgen05, split TF32) Gram matvec and the mixed solve that uses
it, against the FP64 oracle.  Split TF32 carries about FP32 accuracy, so the
operator is checked at 5e-6 relative (the lo*lo product is dropped, ~2^-19) and the refined posterior mean at the
1e-6 bar of the mixed solves."""
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
    "heat2d_8": lambda: W.heat_2d(8, 8, 8, n_ic=(4, 4), n_bc=(2, 2), pred=(3, 3, 3), ell=(0.4, 0.3, 0.3)),
    "heat2d_ragged": lambda: W.heat_2d(5, 7, 9, n_ic=(4, 3), n_bc=(2, 3), pred=(3, 2, 4), ell=(0.4, 0.3, 0.35)),
    "heat2d_tiles": lambda: W.heat_2d(17, 33, 70, n_ic=(9, 11), n_bc=(4, 5), pred=(5, 6, 7)),
    "wave2d": lambda: W.wave_2d(12, 20, 36, n_ic=(4, 4), n_bc=(2, 2), pred=(3, 3, 3), ell=(0.3, 0.3, 0.3)),
    "heat1d": lambda: W.heat_1d(16, 32),
    "c2_64": lambda: W.heat_2d(64, 64, 64, seed=0),
}


@pytest.mark.parametrize("name", list(PROBS))
def test_tc_gram_matvec(name):
    import torch

    from paper_2406_05020_gb300 import gpfvm
    prob = PROBS[name]()
    pb = gpfvm.Problem(prob, max_iter=8)
    pb.assemble()
    K = O.KronIBVP(prob)
    rng = np.random.default_rng(9)
    for _ in range(2):
        v = rng.normal(size=prob.N)
        out = torch.full((prob.N,), float("nan"), dtype=torch.float64, device="cuda")
        pb.matvec(5, torch.as_tensor(v, device="cuda"), out)
        assert relerr(out.cpu().numpy(), K.Gpp(v)) < 5e-6  # split TF32 without lo*lo: ~2^-19
    pb.close()


@pytest.mark.parametrize("name", ["heat2d_ragged", "heat2d_tiles", "heat1d"])
def test_mixed_tf32x3_solve(name):
    import torch

    from paper_2406_05020_gb300 import gpfvm
    prob = PROBS[name]()
    pb = gpfvm.Problem(prob, max_iter=4000)
    pb.assemble()
    code, info = pb.solve(max_iter=4000, rtol=1e-10, precision=gpfvm.MIXED_TF32X3, want_var=True)
    assert code == 0, info.as_dict()
    mean = torch.empty(pb.P, dtype=torch.float64, device="cuda")
    var = torch.empty_like(mean)
    pb.query(mean, var)
    m, v = O.dense_posterior(prob) if prob.N + prob.M < 3000 else (None, None)
    if m is None:
        r = O.kron_posterior(prob, rtol=1e-12, want_var=False)
        m = r["mean"]
    assert relerr(mean.cpu().numpy(), m) < 1e-6
    if v is not None:
        assert np.all(var.cpu().numpy() >= v - 1e-7)
    pb.close()


# ---------------------------------------------------------------------------
# bf16 operands (tcgen05 kind::f16).  Split bf16 keeps hi = bf16(x) and
# lo = bf16(x - hi): each operand carries about 16 significant bits (2^-17),
# and dropping lo*lo adds 2^-16 per product, so a product is good to about
# 2e-5; the 9 terms of a three-term operator partly cancel (the split-TF32
# operator shows a 5x growth over its per-product error), hence 2e-4.  One
# bf16 product (8 bits, 2^-9 per operand) is good to about 4e-3 per product:
# bound 2e-2.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("op,tol", [(8, 2e-4), (10, 2e-2)])
@pytest.mark.parametrize("name", ["heat2d_8", "heat2d_ragged", "heat2d_tiles", "wave2d", "heat1d", "c2_64"])
def test_bf16_gram_matvec(name, op, tol):
    import torch

    from paper_2406_05020_gb300 import gpfvm
    prob = PROBS[name]()
    pb = gpfvm.Problem(prob, max_iter=8)
    pb.assemble()
    K = O.KronIBVP(prob)
    rng = np.random.default_rng(9)
    for _ in range(2):
        v = rng.normal(size=prob.N)
        out = torch.full((prob.N,), float("nan"), dtype=torch.float64, device="cuda")
        pb.matvec(op, torch.as_tensor(v, device="cuda"), out)
        assert relerr(out.cpu().numpy(), K.Gpp(v)) < tol
    pb.close()


@pytest.mark.parametrize("name", ["heat2d_ragged", "heat2d_tiles", "heat1d"])
def test_mixed_bf16x3_solve(name):
    """Split-bf16 inner operator + FP64 residual replacement.  Refinement
    converges only while the operator error (about 2e-5) times the
    conditioning of G^ stays below one: on heat2d_tiles the mean reaches the
    1e-6 bar; on the other two (jitter 1e-8, smaller problems, larger
    condition numbers) a run raises the FP64 residual, the divergence guard
    undoes it and the solve reports NOT_CONVERGED with an iterate no worse
    than before that run."""
    import torch

    from paper_2406_05020_gb300 import gpfvm
    prob = PROBS[name]()
    pb = gpfvm.Problem(prob, max_iter=4000)
    pb.assemble()
    code, info = pb.solve(max_iter=4000, rtol=1e-10, precision=gpfvm.MIXED_BF16X3, want_var=True)
    assert code in (0, 1), info.as_dict()
    assert np.isfinite(info.true_rel_residual) and info.true_rel_residual <= 1.0
    mean = torch.empty(pb.P, dtype=torch.float64, device="cuda")
    pb.query(mean)
    if prob.N + prob.M < 3000:
        m, _ = O.dense_posterior(prob)
    else:
        m = O.kron_posterior(prob, rtol=1e-12, want_var=False)["mean"]
    if code == 0:
        assert relerr(mean.cpu().numpy(), m) < 1e-6
    else:
        assert name != "heat2d_tiles"
    pb.close()
