"""The seeded synthetic workloads: sizes, determinism, and data that the
observations actually see (host-only)."""
import numpy as np

import gpfvm_workloads as W


def test_served_requests_are_seeded_and_within_size_bounds():
    a = W.serving_wave_stream(rate=500.0, duration=0.05, lo=8, hi=16, seed=5, n_max=6)
    b = W.serving_wave_stream(rate=500.0, duration=0.05, lo=8, hi=16, seed=5, n_max=6)
    assert len(a) == len(b) > 0
    t_prev = 0.0
    for (ta, pa), (tb, pb) in zip(a, b):
        assert ta == tb and pa.n_cells == pb.n_cells
        assert ta > t_prev
        t_prev = ta
        assert all(8 <= n <= 16 for n in pa.n_cells)
        np.testing.assert_array_equal(pa.sets[0].values, pb.sets[0].values)


def test_served_requests_observe_their_initial_bump():
    # the IC grid must resolve the bump even for the smallest requests
    for _, p in W.serving_wave_stream(rate=500.0, duration=0.05, lo=8, hi=16, seed=5, n_max=12):
        assert np.abs(p.sets[0].values).max() > 0.1
        assert all(len(c) >= 3 for c in p.sets[0].coords[1:])


def test_batch_sizes_are_uneven_and_bounded():
    probs = W.batch_heat(16, lo=6, hi=14, seed=3)
    sizes = {p.n_cells for p in probs}
    assert len(sizes) > 1
    assert all(6 <= n <= 14 for p in probs for n in p.n_cells)
