"""Thin ctypes binding of libgpfvm (include/gpfvm.h).

Argument marshalling only: every step of the GP-FVM path runs in the CUDA
library.  Device buffers are torch tensors (float64, cuda), passed by pointer;
the CUDA stream is torch's current stream unless one is given.  If the library
has not been built the import of this module fails loudly -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libgpfvm.so")

MAX_DIM, MAX_TERMS, MAX_SETS, MAX_OUTPUTS = 3, 16, 8, 4
OK, NOT_CONVERGED = 0, 1
FP64, MIXED_FP32, MIXED_TF32X3, MIXED_BF16X3, MIXED_BF16 = 0, 1, 2, 3, 4

_lib = None


def lib():
    """Loads libgpfvm.so; raises if it is missing (build with __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgpfvm.so not found at {LIB_PATH}: run paper_2406_05020_gb300.build.build()")
        _lib = C.CDLL(LIB_PATH)
        _declare(_lib)
    return _lib


class PointSet(C.Structure):
    _fields_ = [("order", C.c_int * MAX_DIM), ("n_pts", C.c_int * MAX_DIM),
                ("coords", C.POINTER(C.c_double) * MAX_DIM), ("values", C.POINTER(C.c_double)),
                ("noise_var", C.c_double)]


class Desc(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n_cells", C.c_int * MAX_DIM), ("edges", C.POINTER(C.c_double) * MAX_DIM),
                ("lengthscale", C.c_double * MAX_DIM), ("outputscale", C.c_double), ("n_terms", C.c_int),
                ("alpha", (C.c_int * MAX_DIM) * MAX_TERMS), ("coef", C.c_double * MAX_TERMS),
                ("rhs", C.POINTER(C.c_double)), ("jitter", C.c_double), ("n_sets", C.c_int),
                ("sets", PointSet * MAX_SETS), ("n_pred", C.c_int * MAX_DIM),
                ("pred", C.POINTER(C.c_double) * MAX_DIM), ("observe", C.c_int),
                ("coef_field", C.POINTER(C.c_double) * MAX_TERMS), ("fp64_products", C.c_int),
                ("n_outputs", C.c_int), ("term_eq", C.c_int * MAX_TERMS), ("term_out", C.c_int * MAX_TERMS),
                ("set_out", C.c_int * MAX_SETS)]


class SolveOpts(C.Structure):
    _fields_ = [("max_iter", C.c_int), ("rtol", C.c_double), ("precision", C.c_int), ("reorth", C.c_int),
                ("want_var", C.c_int), ("check_every", C.c_int), ("inner_max_iter", C.c_int),
                ("inner_rtol", C.c_double), ("inner_reorth_first", C.c_int), ("coarse", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("status", C.c_int), ("rel_residual", C.c_double),
                ("true_rel_residual", C.c_double), ("t_assemble_ms", C.c_double), ("t_solve_ms", C.c_double),
                ("t_query_ms", C.c_double), ("latency_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerOpts(C.Structure):
    _fields_ = [("max_slots", C.c_int), ("memory_budget", C.c_int64), ("solve", SolveOpts),
                ("steps_per_tick", C.c_int)]


P = C.c_void_p
D = C.POINTER(C.c_double)

# name -> (restype, argtypes); every symbol declared in include/gpfvm.h
SIGNATURES = {
    "gpfvm_create": (C.c_int, [C.POINTER(Desc), C.c_int, C.POINTER(P)]),
    "gpfvm_destroy": (None, [P]),
    "gpfvm_sizes": (C.c_int, [P, C.POINTER(C.c_int64)]),
    "gpfvm_assemble": (C.c_int, [P, P]),
    "gpfvm_gram_matvec": (C.c_int, [P, C.c_int, P, P, P]),
    "gpfvm_gram_matvec_bench": (C.c_int, [P, C.c_int, P, P, C.c_int, P, D]),
    "gpfvm_solve": (C.c_int, [P, C.POINTER(SolveOpts), C.POINTER(SolveInfo), P]),
    "gpfvm_query": (C.c_int, [P, P, P, P]),
    "gpfvm_solve_host": (C.c_int, [P, D, C.POINTER(SolveOpts), D, D, C.POINTER(SolveInfo), P]),
    "gpfvm_export": (C.c_int64, [P, C.c_int, D, C.c_int64, P]),
    "gpfvm_factor": (C.c_int64, [P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, D, C.c_int64, P]),
    "gpfvm_solve_batch": (C.c_int, [C.POINTER(P), C.c_int, C.POINTER(SolveOpts), C.POINTER(SolveInfo), P]),
    "gpfvm_solve_batch_graph": (C.c_int, [C.POINTER(P), C.c_int, C.POINTER(SolveOpts), C.POINTER(SolveInfo), P,
                                          C.POINTER(C.c_int64)]),
    "gpfvm_server_create": (C.c_int, [C.POINTER(ServerOpts), C.POINTER(P)]),
    "gpfvm_server_submit": (C.c_int, [P, C.POINTER(Desc), C.POINTER(C.c_int64)]),
    "gpfvm_server_step": (C.c_int, [P]),
    "gpfvm_server_poll": (C.c_int, [P, C.c_int64, D, D, C.POINTER(SolveInfo)]),
    "gpfvm_server_destroy": (None, [P]),
    "gpfvm_set_values": (C.c_int, [P, P, P]),
    "gpfvm_target": (C.c_int, [P, P, C.c_int, P]),
    "gpfvm_autotune": (C.c_int, [P, C.c_int, P, D, C.c_int]),
    "gpfvm_launch_count": (C.c_int64, []),
    "gpfvm_kron_matvec_noalloc": (C.c_int, [C.c_int, C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_void_p), D,
                                            C.c_double, C.c_double, P, P, P]),
    "gpfvm_strerror": (C.c_char_p, [C.c_int]),
    "gpfvm_version": (C.c_char_p, []),
}


def _declare(L):
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


class GpfvmError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        super().__init__(f"{where}: {lib().gpfvm_strerror(code).decode()} ({code})")


def _check(code, where):
    if code < 0:
        raise GpfvmError(code, where)
    return code


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(D)


def _dev(t, n: int, name: str):
    """Checks a device tensor handed to the library as a raw pointer: float64,
    contiguous, on the current CUDA device, with exactly n elements (the C ABI
    cannot check sizes, so a wrong one would become an out-of-bounds access)."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch tensor")
    if t.dtype != torch.float64:
        raise TypeError(f"{name}: expected float64, got {t.dtype}")
    if not t.is_cuda or t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name}: must live on the current CUDA device")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if t.numel() != n:
        raise ValueError(f"{name}: expected {n} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


def _disjoint(a, b, name: str):
    a0, b0 = a.data_ptr(), b.data_ptr()
    if a0 < b0 + 8 * b.numel() and b0 < a0 + 8 * a.numel():
        raise ValueError(f"{name}: input and output memory overlap")


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def make_desc(prob):
    """Builds a gpfvm_desc from a problem statement (gpfvm_workloads.Problem or
    any object with the same attributes).  Returns (desc, keepalive)."""
    keep = []

    def arr(x):
        a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
        keep.append(a)
        return _dptr(a)

    d = Desc()
    d.ndim = prob.ndim
    for i in range(prob.ndim):
        d.n_cells[i] = len(prob.edges[i]) - 1
        d.edges[i] = arr(prob.edges[i])
        d.lengthscale[i] = float(prob.lengthscale[i])
        d.n_pred[i] = len(prob.pred[i])
        d.pred[i] = arr(prob.pred[i])
    d.outputscale = float(prob.outputscale)
    if len(prob.terms) > MAX_TERMS:
        raise ValueError("too many operator terms")
    d.n_terms = len(prob.terms)
    for k, (alpha, c) in enumerate(prob.terms):
        for i in range(prob.ndim):
            d.alpha[k][i] = int(alpha[i])
        d.coef[k] = float(c)
    d.rhs = arr(np.ravel(prob.rhs)) if prob.rhs is not None else None
    d.observe = 1 if getattr(prob, "observe", "fvm") == "collocation" else 0
    fields = getattr(prob, "fields", None)
    if fields is not None:
        shared = {}  # terms sharing one array share one pointer (one field on the device)
        for k, f in enumerate(fields):
            if f is None:
                continue
            if id(f) not in shared:
                shared[id(f)] = arr(np.ravel(f))
            d.coef_field[k] = shared[id(f)]
    d.jitter = float(prob.jitter)
    if len(prob.sets) > MAX_SETS:
        raise ValueError("too many point sets")
    d.n_sets = len(prob.sets)
    for s, ps in enumerate(prob.sets):
        for i in range(prob.ndim):
            d.sets[s].order[i] = int(ps.order[i])
            d.sets[s].n_pts[i] = len(ps.coords[i])
            d.sets[s].coords[i] = arr(ps.coords[i])
        d.sets[s].values = arr(np.ravel(ps.values))
        d.sets[s].noise_var = float(ps.noise_var)
    n_out = int(getattr(prob, "n_out", 1))
    term_eq = getattr(prob, "term_eq", None)
    term_out = getattr(prob, "term_out", None)
    if n_out < 1 or n_out > MAX_OUTPUTS:
        raise ValueError(f"n_out must be 1..{MAX_OUTPUTS}")
    for name, lst in (("term_eq", term_eq), ("term_out", term_out)):
        if lst is not None and len(lst) != len(prob.terms):
            raise ValueError(f"{name}: one entry per operator term")
    if n_out > 1 or (term_eq is not None and max(term_eq) > 0):  # a system (Sec. 3.3)
        d.n_outputs = n_out
        for k in range(len(prob.terms)):
            d.term_eq[k] = int(term_eq[k]) if term_eq is not None else 0
            d.term_out[k] = int(term_out[k]) if term_out is not None else 0
        for s, ps in enumerate(prob.sets):
            d.set_out[s] = int(getattr(ps, "out", 0))
    return d, keep


def solve_opts(max_iter=2000, rtol=1e-10, precision=FP64, reorth=True, want_var=True, check_every=16,
               inner_max_iter=0, inner_rtol=1e-2, inner_reorth_first=False, coarse=0):
    o = SolveOpts()
    o.max_iter, o.rtol, o.precision = int(max_iter), float(rtol), int(precision)
    o.reorth, o.want_var, o.check_every = int(reorth), int(want_var), int(check_every)
    o.inner_max_iter, o.inner_rtol = int(inner_max_iter), float(inner_rtol)
    o.inner_reorth_first = int(inner_reorth_first)
    o.coarse = int(coarse)
    return o


class Problem:
    """One GP-FVM problem resident on the GPU (create/assemble/solve/query)."""

    def __init__(self, prob, max_iter: int = 2000, fp64_products: int = 0):
        """fp64_products: 0 = FP64 G_PP by exact digit products on the tensor
        cores where the problem allows it, 1 = FP64 FMA (gpfvm_desc)."""
        self.prob = prob
        self.desc, self._keep = make_desc(prob)
        self.desc.fp64_products = int(fp64_products)
        h = P()
        _check(lib().gpfvm_create(C.byref(self.desc), int(max_iter), C.byref(h)), "gpfvm_create")
        self.h = h
        sz = (C.c_int64 * 4)()
        _check(lib().gpfvm_sizes(self.h, sz), "gpfvm_sizes")
        self.N, self.M, self.P, self.cap = (int(v) for v in sz)
        self.info = SolveInfo()

    def close(self):
        if getattr(self, "h", None):
            lib().gpfvm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def assemble(self, stream=None):
        return _check(lib().gpfvm_assemble(self.h, _stream(stream)), "gpfvm_assemble")

    def _op_sizes(self, op: int):
        if not 0 <= op <= 13:
            raise ValueError(f"unknown operator {op}")
        if op == 2:
            return self.N, self.M
        if op == 3:
            return self.M, self.N
        return self.N, self.N

    def matvec(self, op: int, v, out, stream=None):
        """out = op(v) on device tensors (see gpfvm_gram_matvec)."""
        nin, nout = self._op_sizes(op)
        pv, po = _dev(v, nin, "v"), _dev(out, nout, "out")
        _disjoint(v, out, "matvec")
        return _check(lib().gpfvm_gram_matvec(self.h, int(op), pv, po, _stream(stream)), "gpfvm_gram_matvec")

    def matvec_bench(self, op: int, v, out, reps: int = 50, stream=None) -> float:
        """Device ms of one application of op (graph replays; see gpfvm_gram_matvec_bench)."""
        nin, nout = self._op_sizes(op)
        pv, po = _dev(v, nin, "v"), _dev(out, nout, "out")
        _disjoint(v, out, "matvec_bench")
        ms = C.c_double(0.0)
        _check(lib().gpfvm_gram_matvec_bench(self.h, int(op), pv, po, int(reps), _stream(stream), C.byref(ms)),
               "gpfvm_gram_matvec_bench")
        return ms.value

    def solve(self, opts: Optional[SolveOpts] = None, stream=None, **kw):
        opts = opts or solve_opts(**kw)
        self.info = SolveInfo()
        code = _check(lib().gpfvm_solve(self.h, C.byref(opts), C.byref(self.info), _stream(stream)), "gpfvm_solve")
        return code, self.info

    def query(self, mean, var=None, stream=None):
        pm = _dev(mean, self.P, "mean")
        pv = _dev(var, self.P, "var") if var is not None else None
        if var is not None:
            _disjoint(mean, var, "query")
        return _check(lib().gpfvm_query(self.h, pm, pv, _stream(stream)), "gpfvm_query")

    def autotune(self, precision: int, stream=None):
        """Picks the fastest mode-product plan policy for this problem's operator
        (cached per size class; see gpfvm_autotune).  Returns (cached, ms per
        timed candidate, choice)."""
        rep = np.full(16, np.nan)
        code = _check(lib().gpfvm_autotune(self.h, int(precision), _stream(stream), _dptr(rep), rep.size),
                      "gpfvm_autotune")
        vals = rep[~np.isnan(rep)]
        return bool(code == 1), list(vals[:-1]), int(vals[-1]) if vals.size else None

    def target(self, betas, stream=None):
        """Targeted uncertainty reduction: one IterGP action per row of betas
        (device tensor, n_actions x P weights on the prediction grid; see gpfvm_target)."""
        n = int(betas.shape[0]) if betas.dim() == 2 else 1
        return _check(lib().gpfvm_target(self.h, _dev(betas, n * self.P, "betas"), n, _stream(stream)),
                      "gpfvm_target")

    def solve_host(self, values: Optional[np.ndarray], opts: SolveOpts, mean: np.ndarray,
                   var: Optional[np.ndarray] = None, stream=None):
        vals = None if values is None else np.ascontiguousarray(values, dtype=np.float64)
        self.info = SolveInfo()
        code = _check(lib().gpfvm_solve_host(self.h, _dptr(vals) if vals is not None else None, C.byref(opts),
                                             _dptr(mean), _dptr(var) if var is not None else None,
                                             C.byref(self.info), _stream(stream)), "gpfvm_solve_host")
        return code, self.info

    def set_values(self, values_dev, stream=None):
        """New point-set values (device tensor of M doubles) on the assembled problem."""
        return _check(lib().gpfvm_set_values(self.h, _dev(values_dev, self.M, "values"), _stream(stream)),
                      "gpfvm_set_values")

    def export(self, what: int, n: int) -> np.ndarray:
        out = np.empty(max(n, 1))
        k = _check(lib().gpfvm_export(self.h, int(what), _dptr(out), out.size, _stream(None)), "gpfvm_export")
        return out[:k]

    def factor(self, axis, kind_a, arg_a, kind_b, arg_b, shape) -> np.ndarray:
        out = np.empty(int(np.prod(shape)))
        k = _check(lib().gpfvm_factor(self.h, axis, kind_a, arg_a, kind_b, arg_b, _dptr(out), out.size,
                                      _stream(None)), "gpfvm_factor")
        return out[:k].reshape(shape)


def solve_batch(problems, opts: SolveOpts, stream=None):
    arr = (P * len(problems))(*[p.h for p in problems])
    infos = (SolveInfo * len(problems))()
    code = _check(lib().gpfvm_solve_batch(arr, len(problems), C.byref(opts), infos, _stream(stream)),
                  "gpfvm_solve_batch")
    return code, list(infos)


def solve_batch_graph(problems, opts: SolveOpts, stream=None):
    """The batch as one graph launch (gpfvm_solve_batch_graph): (code, infos, kernels executed)."""
    arr = (P * len(problems))(*[p.h for p in problems])
    infos = (SolveInfo * len(problems))()
    nl = C.c_int64(0)
    code = _check(lib().gpfvm_solve_batch_graph(arr, len(problems), C.byref(opts), infos, _stream(stream),
                                                C.byref(nl)), "gpfvm_solve_batch_graph")
    return code, list(infos), int(nl.value)


def kron_matvec_noalloc(dims, terms, scale, diag, v, out, stream=None):
    """out = scale * sum_k c_k (F_k0 (x) ...) v + diag * v without any device
    allocation; terms = [(c_k, [F_k0, F_k1, ...])] with device tensors F."""
    ndim = len(dims)
    total = int(np.prod(dims))
    pv, po = _dev(v, total, "v"), _dev(out, total, "out")
    _disjoint(v, out, "kron_matvec_noalloc")
    for _, fs in terms:
        if len(fs) != ndim:
            raise ValueError("kron_matvec_noalloc: one factor per axis")
        for i, f in enumerate(fs):
            _dev(f, int(dims[i]) ** 2, f"factor on axis {i}")
    n = (C.c_int * ndim)(*dims)
    ptrs = (C.c_void_p * (len(terms) * ndim))(*[f.data_ptr() for _, fs in terms for f in fs])
    coef = np.ascontiguousarray([c for c, _ in terms], dtype=np.float64)
    return _check(lib().gpfvm_kron_matvec_noalloc(ndim, n, len(terms), ptrs, _dptr(coef), float(scale),
                                                  float(diag), pv, po, _stream(stream)), "gpfvm_kron_matvec_noalloc")


class Server:
    """Continuous-batching serving loop (gpfvm_server_*)."""

    def __init__(self, max_slots=8, memory_budget=0, steps_per_tick=16, **solve_kw):
        o = ServerOpts()
        o.max_slots, o.memory_budget, o.steps_per_tick = int(max_slots), int(memory_budget), int(steps_per_tick)
        o.solve = solve_opts(**solve_kw)
        self.opts = o
        h = P()
        _check(lib().gpfvm_server_create(C.byref(o), C.byref(h)), "gpfvm_server_create")
        self.h = h
        self._keep = {}

    def submit(self, prob) -> int:
        d, keep = make_desc(prob)
        t = C.c_int64()
        _check(lib().gpfvm_server_submit(self.h, C.byref(d), C.byref(t)), "gpfvm_server_submit")
        self._keep[t.value] = (d, keep, prob)
        return t.value

    def step(self) -> int:
        return _check(lib().gpfvm_server_step(self.h), "gpfvm_server_step")

    def poll(self, ticket: int, want_var: bool = True):
        """(code, mean, var, info); code 2 = still pending."""
        prob = self._keep[ticket][2]
        P_ = int(np.prod([len(x) for x in prob.pred]))
        mean = np.empty(P_)
        var = np.empty(P_) if want_var else None
        info = SolveInfo()
        code = lib().gpfvm_server_poll(self.h, int(ticket), _dptr(mean), _dptr(var) if var is not None else None,
                                       C.byref(info))
        return code, mean, var, info

    def close(self):
        if getattr(self, "h", None):
            lib().gpfvm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def launch_count() -> int:
    return int(lib().gpfvm_launch_count())


def version() -> str:
    return lib().gpfvm_version().decode()
