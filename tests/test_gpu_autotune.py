"""The mode-product autotuner (gpfvm_autotune): it times the solver's own
operator under each plan policy, keeps the fastest, and caches the choice per
size class; the operator it leaves behind computes the same product."""
import numpy as np
import pytest

import gpfvm_workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_05020_gb300 import build
    build.build()


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec,op,tol", [(0, 1, 1e-13), (1, 6, 1e-6), (2, 7, 2e-6), (3, 9, 1e-4)])
def test_autotune_picks_caches_and_keeps_the_operator(prec, op, tol):
    import torch

    from paper_2406_05020_gb300 import gpfvm
    sizes = [(40, 36, 44), (42, 34, 41)]  # one size class (axis sizes rounded up to 16)
    v = None
    cached_flags = []
    for k, (nt, nx, ny) in enumerate(sizes):
        prob = W.heat_2d(nt, nx, ny, n_ic=(nx // 2, ny // 2), n_bc=(-(-nt // 4), -(-max(nx, ny) // 4)),
                         pred=(nt // 2, nx // 2, ny // 2), seed=k)
        pb = gpfvm.Problem(prob, max_iter=16)
        pb.assemble()
        v = torch.as_tensor(np.random.default_rng(k).normal(size=prob.N), device="cuda")
        ref = torch.empty_like(v)
        pb.matvec(op, v, ref)
        cached, ms, choice = pb.autotune(prec)
        cached_flags.append(cached)
        if not cached:
            assert len(ms) == (8 if prec >= 2 else 4) and all(m > 0 for m in ms)
            assert ms[choice_index(choice, prec)] == min(ms)
        out = torch.empty_like(v)
        pb.matvec(op, v, out)
        assert relerr(out.cpu().numpy(), ref.cpu().numpy()) < tol
        pb.close()
    assert cached_flags[1] is True


def choice_index(choice, prec):
    """Position of the chosen candidate in the timing list: grouping policy
    major, tile policy (-1, 0, 1, 2) minor."""
    tile, grp = choice // 3 - 1, choice % 3
    return grp * 4 + (tile + 1)


def test_autotuned_solve_matches_untuned():
    """A converged FP64 solve with the tuned plans gives the untuned posterior."""
    import torch

    from paper_2406_05020_gb300 import gpfvm
    prob = W.heat_2d(24, 20, 28, n_ic=(10, 14), n_bc=(6, 7), pred=(12, 10, 14), seed=3)
    mean = []
    for tune in (False, True):
        pb = gpfvm.Problem(prob, max_iter=3000)
        pb.assemble()
        if tune:
            pb.autotune(0)
        code, info = pb.solve(max_iter=3000, rtol=1e-10, precision=gpfvm.FP64, want_var=False)
        assert code == 0
        m = torch.empty(pb.P, dtype=torch.float64, device="cuda")
        pb.query(m)
        mean.append(m.cpu().numpy())
        pb.close()
    assert relerr(mean[1], mean[0]) < 1e-10
