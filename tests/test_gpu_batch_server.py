"""Batched and served execution (many independent IBVPs on one GPU).

A problem's result must be the same alone and in the mix: every problem runs
the same kernels with fixed-order reductions on its own stream, so the
batched and served results are compared with the individual solves exactly
(up to 1e-14 relative), and against the oracle at the mixed-precision bar."""
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


def _alone(prob, opts):
    import torch

    from paper_2406_05020_gb300 import gpfvm
    pb = gpfvm.Problem(prob, max_iter=opts.max_iter)
    pb.assemble()
    code, info = pb.solve(opts)
    mean = torch.empty(pb.P, dtype=torch.float64, device="cuda")
    var = torch.empty_like(mean)
    pb.query(mean, var)
    out = (code, mean.cpu().numpy(), var.cpu().numpy(), info.iterations)
    pb.close()
    return out


@pytest.mark.parametrize("precision", [0, 2])
def test_batch_of_uneven_problems_equals_individual_solves(precision):
    import torch

    from paper_2406_05020_gb300 import gpfvm
    probs = W.batch_heat(6, lo=6, hi=14, seed=3)
    opts = gpfvm.solve_opts(max_iter=3000, rtol=1e-10, precision=precision, want_var=True, check_every=8,
                            inner_max_iter=400)
    alone = [_alone(p, opts) for p in probs]
    pbs = [gpfvm.Problem(p, max_iter=3000) for p in probs]
    for pb in pbs:
        pb.assemble()
    code, infos = gpfvm.solve_batch(pbs, opts)
    assert code == 0
    for pb, prob, ref, info in zip(pbs, probs, alone, infos):
        mean = torch.empty(pb.P, dtype=torch.float64, device="cuda")
        var = torch.empty_like(mean)
        pb.query(mean, var)
        assert info.iterations == ref[3]
        assert relerr(mean.cpu().numpy(), ref[1]) < 1e-14
        np.testing.assert_allclose(var.cpu().numpy(), ref[2], rtol=0, atol=1e-14)
        if prob.N + prob.M < 2500:
            m, v = O.dense_posterior(prob)
            assert relerr(mean.cpu().numpy(), m) < 1e-6
        pb.close()


def test_server_same_result_alone_and_in_the_mix():
    from paper_2406_05020_gb300 import gpfvm
    reqs = W.serving_wave_stream(rate=500.0, duration=0.05, lo=8, hi=16, seed=5, n_max=6)
    assert len(reqs) >= 3
    kw = dict(max_iter=3000, rtol=1e-10, precision=2, want_var=True, check_every=8, inner_max_iter=400)
    srv = gpfvm.Server(max_slots=3, steps_per_tick=8, **kw)
    tickets = [srv.submit(p) for _, p in reqs]
    guard = 0
    while srv.step() > 0:
        guard += 1
        assert guard < 100000
    opts = gpfvm.solve_opts(**kw)
    for t, (_, prob) in zip(tickets, reqs):
        code, mean, var, info = srv.poll(t)
        assert code == 0, info.as_dict()
        ref = _alone(prob, opts)
        assert relerr(mean, ref[1]) < 1e-14
        np.testing.assert_allclose(var, ref[2], rtol=0, atol=1e-14)
        assert info.latency_ms > 0
    srv.close()


def test_server_isolates_bad_and_oversized_requests():
    from paper_2406_05020_gb300 import gpfvm
    good = W.heat_2d(6, 7, 8, n_ic=(4, 4), n_bc=(2, 2), pred=(3, 3, 3), ell=(0.4, 0.3, 0.3))
    bad = W.heat_2d(6, 7, 8, n_ic=(4, 4), n_bc=(2, 2), pred=(3, 3, 3), ell=(0.4, 0.3, 0.3))
    bad.sets[0].values = bad.sets[0].values.copy()
    bad.sets[0].values[3] = np.nan
    big = W.heat_2d(60, 60, 60, n_ic=(8, 8), n_bc=(2, 2), pred=(3, 3, 3))
    srv = gpfvm.Server(max_slots=2, memory_budget=400 * 1024 * 1024, steps_per_tick=8, max_iter=2000, rtol=1e-10,
                       precision=1, want_var=False, inner_max_iter=400)
    with pytest.raises(gpfvm.GpfvmError) as e:
        srv.submit(bad)  # NaN data is rejected at submission
    assert e.value.code == -1
    t_big = srv.submit(big)
    t_good = srv.submit(good)
    guard = 0
    while srv.step() > 0:
        guard += 1
        assert guard < 100000
    code_big, *_ = srv.poll(t_big, want_var=False)
    code_good, mean, _, info = srv.poll(t_good, want_var=False)
    assert code_big == -2  # cannot fit the memory budget
    assert code_good == 0
    m, _ = O.dense_posterior(good)
    assert relerr(mean, m) < 1e-6
    srv.close()


@pytest.mark.parametrize("precision,reorth", [(0, 1), (2, 1), (2, 2)])
def test_batch_graph_at_c4_sizes_equals_individual_solves(precision, reorth):
    """The uneven heat batch at its own sizes (axis sizes 16..64) as ONE graph
    launch (device-driven refinement in every problem's loop) gives every
    problem's individual, host-driven solve: same iterations, mean and variance
    to 1e-14."""
    import torch

    from paper_2406_05020_gb300 import gpfvm
    probs = W.batch_heat(256, lo=16, hi=64, seed=0)[:5]
    opts = gpfvm.solve_opts(max_iter=3000, rtol=1e-10, precision=precision, reorth=reorth, want_var=True,
                            inner_max_iter=400, inner_rtol=1e-2)
    alone = [_alone(p, opts) for p in probs]
    pbs = [gpfvm.Problem(p, max_iter=3000) for p in probs]
    for pb in pbs:
        pb.assemble()
    code, infos, launches = gpfvm.solve_batch_graph(pbs, opts)
    assert code == 0, [i.as_dict() for i in infos]
    assert launches > 0
    for pb, prob, ref, info in zip(pbs, probs, alone, infos):
        mean = torch.empty(pb.P, dtype=torch.float64, device="cuda")
        var = torch.empty_like(mean)
        pb.query(mean, var)
        assert ref[0] == 0 and info.status == 0
        assert info.iterations == ref[3]
        assert relerr(mean.cpu().numpy(), ref[1]) < 1e-14
        np.testing.assert_allclose(var.cpu().numpy(), ref[2], rtol=0, atol=1e-14)
        pb.close()


def test_server_at_c5_sizes_same_result_alone_and_in_the_mix():
    """Served wave requests from the lower end of the serving size range
    (axis sizes 32..40), bounded-memory refinement (reorth 2): each result is
    the same alone and in the mix."""
    from paper_2406_05020_gb300 import gpfvm
    reqs = W.serving_wave_stream(rate=500.0, duration=1.0, lo=32, hi=40, seed=7, n_max=3)
    kw = dict(max_iter=12000, rtol=1e-10, precision=2, reorth=2, want_var=True, inner_max_iter=400)
    srv = gpfvm.Server(max_slots=3, **kw)
    tickets = [srv.submit(p) for _, p in reqs]
    guard = 0
    while srv.step() > 0:
        guard += 1
        assert guard < 10000000
    opts = gpfvm.solve_opts(**kw)
    for t, (_, prob) in zip(tickets, reqs):
        code, mean, var, info = srv.poll(t)
        ref = _alone(prob, opts)
        assert code == ref[0] and code in (0, 1), info.as_dict()
        assert relerr(mean, ref[1]) < 1e-14
        np.testing.assert_allclose(var, ref[2], rtol=0, atol=1e-14)
    srv.close()
