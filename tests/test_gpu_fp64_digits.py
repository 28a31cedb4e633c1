"""FP64 G_PP by exact digit products on the tensor cores (ops 12 / 13) against
the FP64 oracle, and the FP64 solve that uses it.

The digit-product form computes every mode product to about 2^-54 of
K max|a| max|b| (K <= 128 terms), the accuracy class of an FP64 matrix
product, so the operators are held to the bounds of the FP64 FMA forms
(ops 0 / 1) in the parity tests: 1e-13 normwise for G_PP and 1e-11 for G^
against the oracle (whose own FP64 rounding, amplified by the cancellation
between the Kronecker terms, is of order 1e-14 for G_PP)."""
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
    "colloc_heat2d": lambda: W.collocation(W.heat_2d(6, 9, 11, n_ic=(4, 3), n_bc=(2, 3), pred=(3, 2, 4))),
    "c2_64": lambda: W.heat_2d(64, 64, 64, seed=0),
    "wave_128": lambda: W.wave_2d(128, 128, 128, seed=0),
}


def _apply(pb, op, v):
    import torch
    out = torch.full((v.size,), float("nan"), dtype=torch.float64, device="cuda")
    pb.matvec(op, torch.as_tensor(v, device="cuda"), out)
    return out.cpu().numpy()


@pytest.mark.parametrize("name", list(PROBS))
def test_digit_product_gpp_matches_oracle(name):
    from paper_2406_05020_gb300 import gpfvm
    prob = PROBS[name]()
    pb = gpfvm.Problem(prob, max_iter=8)
    pb.assemble()
    K = O.KronIBVP(prob)
    rng = np.random.default_rng(3)
    for scale in (1.0, 1e-150, 1e120):
        v = rng.normal(size=prob.N) * scale
        ref = K.Gpp(v)
        got = _apply(pb, 12, v)
        fma = _apply(pb, 0, v)
        assert relerr(got, ref) < 1e-13, scale
        assert relerr(got, fma) < 1e-13, scale
    pb.close()


@pytest.mark.parametrize("name", ["heat2d_ragged", "heat2d_tiles", "wave2d", "c2_64"])
def test_digit_product_ghat_matches_fma_form(name):
    from paper_2406_05020_gb300 import gpfvm
    prob = PROBS[name]()
    pb = gpfvm.Problem(prob, max_iter=8)
    pb.assemble()
    K = O.KronIBVP(prob)
    rng = np.random.default_rng(4)
    v = rng.normal(size=prob.N)
    got = _apply(pb, 13, v)
    assert relerr(got, _apply(pb, 1, v)) < 1e-11
    assert relerr(got, K.Ghat(v)) < 1e-11
    pb.close()


def test_digit_product_form_needs_two_axes():
    """One axis (a single row of at most 128 cells) keeps the FMA form: ops
    12 / 13 are rejected there and the FP64 solve runs the FMA operator."""
    from paper_2406_05020_gb300 import gpfvm
    prob = W.toy_cos(24)
    pb = gpfvm.Problem(prob, max_iter=8)
    pb.assemble()
    with pytest.raises(gpfvm.GpfvmError):
        _apply(pb, 12, np.ones(prob.N))
    pb.close()


def test_digit_product_dynamic_range_and_special_values():
    """Entries spanning 1e-200 .. 1e100 within one vector (rows scaled by
    their own exponents), an exact zero vector, and a NaN entry that must
    reach the output rather than vanish in the integer arithmetic."""
    from paper_2406_05020_gb300 import gpfvm
    prob = PROBS["heat2d_tiles"]()
    pb = gpfvm.Problem(prob, max_iter=8)
    pb.assemble()
    K = O.KronIBVP(prob)
    rng = np.random.default_rng(5)
    v = rng.normal(size=prob.N) * 10.0 ** rng.uniform(-200, 100, size=prob.N)
    assert relerr(_apply(pb, 12, v), K.Gpp(v)) < 1e-13
    z = _apply(pb, 12, np.zeros(prob.N))
    assert np.all(z == 0.0)
    w = rng.normal(size=prob.N)
    w[prob.N // 3] = np.nan
    out = _apply(pb, 12, w)
    assert np.isnan(out).any()
    pb.close()


@pytest.mark.parametrize("name", ["heat2d_ragged", "heat2d_tiles", "heat1d", "wave2d"])
def test_fp64_solve_with_digit_products_matches_dense(name):
    """The FP64 solve (digit-product G_PP, the default) reaches the dense
    Cholesky posterior mean at the FP64 bar, as the FMA form (fp64_products=1)
    does.  The variance of a converged IterGP run depends on the directions it
    happened to take (rounding-decided, as between any two FP64 orderings),
    so it is checked against the exact posterior variance from above."""
    import torch

    from paper_2406_05020_gb300 import gpfvm
    prob = PROBS[name]()
    res = {}
    for mode in (0, 1):
        pb = gpfvm.Problem(prob, max_iter=4000, fp64_products=mode)
        pb.assemble()
        code, info = pb.solve(max_iter=4000, rtol=1e-12, precision=gpfvm.FP64, want_var=True)
        assert code == 0, info.as_dict()
        mean = torch.empty(pb.P, dtype=torch.float64, device="cuda")
        var = torch.empty_like(mean)
        pb.query(mean, var)
        res[mode] = (mean.cpu().numpy(), var.cpu().numpy(), info.iterations)
        pb.close()
    if prob.N + prob.M < 3000:
        m, var = O.dense_posterior(prob)
    else:
        m, var = O.kron_posterior(prob, rtol=1e-13, want_var=False)["mean"], None
    assert relerr(res[0][0], m) < 1e-10
    assert relerr(res[1][0], m) < 1e-10
    if var is not None:
        for mode in (0, 1):
            assert np.all(res[mode][1] >= var - 1e-7 * max(np.abs(var).max(), 1.0))
