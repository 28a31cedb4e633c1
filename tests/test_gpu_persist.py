"""Persistent execution of the Gram operators (one cooperative launch per
application, GPFVM_PERSIST=1) against the launch-by-launch execution: the
same device code per tile, GEMV row and tensor-core tile, so the operators,
the solves of every precision and the posteriors are bit-identical."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
import gpfvm_workloads as W
from paper_2406_05020_gb300 import build, gpfvm
build.build()
probs = {"heat": W.heat_2d(17, 33, 70, n_ic=(9, 11), n_bc=(4, 5), pred=(5, 6, 7)),
         "wave": W.wave_2d(16, 10, 11, c=1.2, seed=7, n_ic=(3, 3), n_bc=(2, 2), pred=(4, 4, 4), ic_noise=0.0,
                           width=0.25),
         "heat1d": W.heat_1d(16, 32, n_ic=32)}
out = {}
for name, prob in probs.items():
    pb = gpfvm.Problem(prob, max_iter=3000)
    pb.assemble()
    v = torch.as_tensor(np.random.default_rng(1).normal(size=prob.N), device="cuda")
    o = torch.empty_like(v)
    ops = {}
    for op in (0, 1, 4, 5, 6, 7):
        try:
            pb.matvec(op, v, o)
            ops[op] = o.cpu().numpy().tolist()
        except gpfvm.GpfvmError:
            ops[op] = None
    sol = {}
    for prec in (0, 1, 2):
        try:
            code, info = pb.solve(max_iter=3000, rtol=1e-10, precision=prec, want_var=True, inner_max_iter=400)
        except gpfvm.GpfvmError as e:
            sol[prec] = ["error", e.code]
            continue
        mean = torch.empty(pb.P, dtype=torch.float64, device="cuda")
        var = torch.empty_like(mean)
        pb.query(mean, var)
        sol[prec] = [code, info.iterations, mean.cpu().numpy().tolist(), var.cpu().numpy().tolist()]
    out[name] = {"ops": ops, "sol": sol}
    pb.close()
print(json.dumps(out))
""".replace("ROOT", repr(ROOT))


def _run(persist):
    env = dict(os.environ)
    env.pop("GPFVM_PERSIST", None)
    if persist:
        env["GPFVM_PERSIST"] = "1"
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_persistent_operators_and_solves_are_bit_identical():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    a = _run(False)
    b = _run(True)
    for name in a:
        for op in a[name]["ops"]:
            assert a[name]["ops"][op] == b[name]["ops"][op], (name, op)
        for prec in a[name]["sol"]:
            sa, sb = a[name]["sol"][prec], b[name]["sol"][prec]
            assert sa[0] == 0, (name, prec, sa[:2])
            assert sa == sb, (name, prec, sa[:2], sb[:2])
