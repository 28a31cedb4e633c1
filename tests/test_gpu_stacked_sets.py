"""Stacked IC sets: the IC pair of a second-order-in-time problem (u and u_t
observed on one spatial grid at t = 0) is held as one set with two axis-0
points, so the structured IC/BC stage inverts both through one Kronecker
eigenbasis (the cross-covariance of u and u_t at one time is an odd
derivative of the even Matern kernel at 0, hence the 2 x 2 time factor is
diagonal).  This is a reorganisation of the same conditioning on G_BB
(Sec. 4.2): the posterior must equal the unstacked and dense GPU paths and
the oracle."""
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


def _create(prob, env, iters=8):
    from paper_2406_05020_gb300 import gpfvm
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        return gpfvm.Problem(prob, max_iter=max(iters, 8))
    finally:
        for k, v in old.items():
            if v is None:
                del os.environ[k]
            else:
                os.environ[k] = v


def _run(prob, env, iters):
    import torch
    pb = _create(prob, env, iters)
    pb.assemble()
    lay = pb.export(10, 3)
    b = pb.export(0, prob.N)
    code, info = pb.solve(max_iter=iters, rtol=0.0, reorth=True, want_var=True)
    mean = torch.empty(pb.P, dtype=torch.float64, device="cuda")
    var = torch.empty_like(mean)
    pb.query(mean, var)
    v = np.random.default_rng(2).normal(size=prob.N)
    out = torch.empty(prob.N, dtype=torch.float64, device="cuda")
    pb.matvec(1, torch.as_tensor(v, device="cuda"), out)
    res = dict(lay=lay, b=b, mean=mean.cpu().numpy(), var=var.cpu().numpy(), ghat=out.cpu().numpy(), v=v)
    pb.close()
    return res


PROBS = {
    "wave2d_neumann": lambda: W.wave_2d(6, 9, 5, n_ic=(5, 6), n_bc=(2, 2), pred=(3, 3, 3), ell=(0.3, 0.3, 0.3)),
    "wave_sine": lambda: W.wave_2d_sine(6, 7, 8, n_ic=5, n_bc=(3, 2), pred=(4, 3, 3)),
    "wave2d_colloc": lambda: W.collocation(W.wave_2d(6, 9, 5, n_ic=(4, 4), n_bc=(2, 2), pred=(3, 3, 3),
                                                     ell=(0.3, 0.3, 0.3))),
    "wave2d_tiles": lambda: W.wave_2d(12, 20, 36, n_ic=(9, 11), n_bc=(3, 4), pred=(3, 4, 5), ell=(0.3, 0.3, 0.3)),
}


@pytest.mark.parametrize("name", list(PROBS))
def test_stacked_ic_pair_matches_unstacked_dense_and_oracle(name):
    prob = PROBS[name]()
    ic = prob.sets[0].values.size
    assert prob.sets[1].values.size == ic
    iters = min(10, prob.N // 2)
    st = _run(prob, {}, iters)
    un = _run(prob, {"GPFVM_STACK_SETS": "0"}, iters)
    de = _run(prob, {"GPFVM_ICBC": "dense"}, iters)
    # layout: the stacked pair is the eigenbasis block; unstacked, u_t goes to the Schur complement
    assert tuple(st["lay"].astype(int)) == (1, 2 * ic, prob.M - 2 * ic)
    assert tuple(un["lay"].astype(int)) == (1, ic, prob.M - ic)
    assert int(de["lay"][0]) == 0
    K = O.KronIBVP(prob)
    r = O.kron_posterior(prob, max_iter=iters, rtol=0.0, K=K)
    for x in (st, un, de):
        assert relerr(x["b"], K.rhs_hat()) < 1e-10
        assert relerr(x["ghat"], K.Ghat(x["v"])) < 1e-10
        assert relerr(x["mean"], r["mean"]) < 1e-10
        np.testing.assert_allclose(x["var"], r["var"], atol=1e-10, rtol=0)
    assert relerr(st["mean"], un["mean"]) < 1e-10


def test_factors_of_stacked_sets_keep_the_callers_numbering():
    """gpfvm_factor takes the caller's set numbers: on axis 0 each set of a
    stacked pair gets its own row / column (its own derivative order)."""
    prob = PROBS["wave2d_neumann"]()
    pb = _create(prob, {})
    pb.assemble()
    K = O.KronIBVP(prob)
    pde = O.pde_block(prob)
    fam = [sb.terms[0][1] for sb in K.sets]
    for i in range(prob.ndim):
        for s, G in enumerate(fam):
            for c1, F in pde.terms:
                ref = O.cov_1d(F[i], G[i], prob.lengthscale[i])
                a = F[i][3] if F[i][0] == "cell" else F[i][2]
                got = pb.factor(i, 0, a, 1, s, ref.shape)
                np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())
            for s2, G2 in enumerate(fam):
                ref = O.cov_1d(G[i], G2[i], prob.lengthscale[i])
                got = pb.factor(i, 1, s, 1, s2, ref.shape)
                np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-14 * max(np.abs(ref).max(), 1e-300))
    pb.close()


def test_wave_128_ic_pair_is_stacked():
    """The 128^3 wave problem: both 64 x 64 IC sets in the eigenbasis block,
    only the 4096 wall points in the Schur complement."""
    prob = W.wave_2d(128, 128, 128, seed=0)
    pb = _create(prob, {})
    lay = pb.export(10, 3)
    pb.close()
    assert tuple(lay.astype(int)) == (1, 8192, 4096)
