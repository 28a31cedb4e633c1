"""The allocation-free Kronecker Gram matvec (gpfvm_kron_matvec_noalloc).

Callers that cannot allocate device memory when they need a Gram product --
frameworks whose allocator owns the whole device, real-time loops that must
stay out of the driver's allocator -- use this entry point: its intermediates
live in a fixed static device array.
These tests check it through the C ABI against the regular entry point
(gpfvm_gram_matvec, op 0, whose intermediates live in memory allocated at
problem creation), on two calls in a row, and check that requests beyond the
static capacity are refused.  This file is collected last on purpose."""
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


def _pp_terms(pb, prob):
    """The (coefficient, per-axis factor) list of G_PP as device tensors,
    one tensor per distinct factor so that equal factors share a pointer."""
    import torch
    cache = {}
    terms = []
    for a, ca in prob.terms:
        for b, cb in prob.terms:
            fs = []
            for i in range(prob.ndim):
                key = (i, a[i], b[i])
                if key not in cache:
                    n = prob.n_cells[i]
                    host = pb.factor(i, 0, a[i], 0, b[i], (n, n))
                    cache[key] = torch.as_tensor(host, dtype=torch.float64, device="cuda").contiguous()
                fs.append(cache[key])
            terms.append((ca * cb, fs))
    return terms


@pytest.mark.parametrize("mk", [
    lambda: W.heat_2d(17, 33, 70, n_ic=(9, 11), n_bc=(4, 5), pred=(5, 6, 7)),
    lambda: W.heat_2d(64, 64, 64, seed=0),
    lambda: W.heat_1d(16, 32),
    lambda: W.toy_cos(40),  # one axis: a single level, no intermediates
])
def test_noalloc_matches_regular_matvec_twice(mk):
    import torch

    from paper_2406_05020_gb300 import gpfvm
    prob = mk()
    pb = gpfvm.Problem(prob, max_iter=8)
    pb.assemble()
    terms = _pp_terms(pb, prob)
    rng = np.random.default_rng(11)
    for call in range(2):
        v = torch.as_tensor(rng.normal(size=prob.N), dtype=torch.float64, device="cuda")
        ref = torch.empty_like(v)
        out = torch.full_like(v, float("nan"))
        pb.matvec(0, v, ref)
        gpfvm.kron_matvec_noalloc(list(prob.n_cells), terms, prob.outputscale, prob.jitter, v, out,
                                  stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.isfinite(o)), call
        assert np.linalg.norm(o - r) / np.linalg.norm(r) < 1e-13, call
    pb.close()


def test_noalloc_rejects_requests_beyond_capacity():
    import ctypes as C

    import torch

    from paper_2406_05020_gb300 import gpfvm
    # three 128-point axes with 4 distinct last-axis and 4 distinct first-axis
    # factors need 8 * 128^3 doubles of intermediates (> 4,194,304): the C entry
    # point refuses before anything is launched, so the tiny stand-in tensors
    # (called through the raw C ABI, past the binding's size checks) are never read
    dummy = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in range(8)]
    facs = [dummy[k % 4] if i == 0 else (dummy[0] if i == 1 else dummy[4 + k % 4])
            for k in range(4) for i in range(3)]
    v = torch.zeros(1, dtype=torch.float64, device="cuda")
    n = (C.c_int * 3)(128, 128, 128)
    ptrs = (C.c_void_p * 12)(*[f.data_ptr() for f in facs])
    coef = (C.c_double * 4)(1.0, 1.0, 1.0, 1.0)
    code = gpfvm.lib().gpfvm_kron_matvec_noalloc(3, n, 4, ptrs, coef, 1.0, 0.0, C.c_void_p(v.data_ptr()),
                                                 C.c_void_p(v.data_ptr()), None)
    assert code == -9
    torch.cuda.synchronize()
