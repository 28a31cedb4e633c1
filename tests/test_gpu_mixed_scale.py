"""The solves are scale-free in the data.

The posterior mean is linear in the observations and the variance does not
depend on them (Sec. 2.1, Eqs. lin-cond-mean and lin-cond-cov), so scaling every observation by a
power of two must scale the mean by exactly that factor and leave the
variance unchanged, at every precision.  With factors 2^-100 and 2^+100 the
late residuals of the mixed-precision refinement lie far outside the normal
FP32 range unless the inner solve normalises its right-hand side."""
import copy

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


def _scaled(prob, f):
    q = copy.deepcopy(prob)
    for s in q.sets:
        s.values = np.asarray(s.values, dtype=np.float64) * f
    if q.rhs is not None:
        q.rhs = np.asarray(q.rhs, dtype=np.float64) * f
    return q


def _solve(prob, precision):
    import torch

    from paper_2406_05020_gb300 import gpfvm
    pb = gpfvm.Problem(prob, max_iter=2000)
    pb.assemble()
    code, info = pb.solve(max_iter=2000, rtol=1e-10, precision=precision, want_var=True, check_every=8,
                          inner_max_iter=400)
    mean = torch.empty(pb.P, dtype=torch.float64, device="cuda")
    var = torch.empty_like(mean)
    if code == 0:
        pb.query(mean, var)
    out = code, info.iterations, mean.cpu().numpy(), var.cpu().numpy()
    pb.close()
    return out


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_mean_scales_with_the_data_and_variance_does_not(precision):
    prob = W.heat_2d(10, 9, 11, n_ic=(5, 5), n_bc=(2, 2), pred=(4, 4, 4), ell=(0.4, 0.3, 0.3))
    code1, it1, m1, v1 = _solve(prob, precision)
    assert code1 == 0
    m_ref, _ = O.dense_posterior(prob)
    assert np.linalg.norm(m1 - m_ref) / np.linalg.norm(m_ref) < 1e-6
    for e in (-100, 100):
        f = 2.0 ** e
        code, it, m, v = _solve(_scaled(prob, f), precision)
        assert code == 0, (e, it)
        assert it == it1
        np.testing.assert_allclose(m / f, m1, rtol=1e-13, atol=1e-13 * np.abs(m1).max())
        np.testing.assert_allclose(v, v1, rtol=0, atol=1e-14)


def test_served_wave_requests_with_tiny_data_converge():
    """A wave request whose observations are 1e-26 (far below FP32's normal
    range after a 1e-10 residual reduction) converges in every precision."""
    prob = W.wave_2d(16, 10, 11, c=1.2, seed=7, n_ic=(3, 3), n_bc=(2, 2), pred=(4, 4, 4), ic_noise=0.0)
    tiny = _scaled(prob, 1e-26)
    ref = [_solve(prob, p) for p in (0, 1, 2)]
    for p, (code0, _, m0, _) in zip((0, 1, 2), ref):
        code, _, m, _ = _solve(tiny, p)
        assert code0 == 0 and code == 0
        assert np.linalg.norm(m / 1e-26 - m0) / np.linalg.norm(m0) < 1e-6
