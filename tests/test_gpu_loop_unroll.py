"""Device-side CG loops with one, two or three iterations per WHILE pass
(GPFVM_LOOP_UNROLL): the same kernels run in the same order and every kernel
of an iteration does nothing once the run is done, so solves of every
precision, iteration counts and posteriors are bit-identical."""
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
prob = W.heat_2d(17, 33, 70, n_ic=(9, 11), n_bc=(4, 5), pred=(5, 6, 7))
pb = gpfvm.Problem(prob, max_iter=3000)
pb.assemble()
out = {}
for prec in (0, 1, 2):
    code, info = pb.solve(max_iter=3000, rtol=1e-10, precision=prec, want_var=True, inner_max_iter=400)
    mean = torch.empty(pb.P, dtype=torch.float64, device="cuda")
    var = torch.empty_like(mean)
    pb.query(mean, var)
    out[prec] = [code, info.iterations, mean.cpu().numpy().tolist(), var.cpu().numpy().tolist()]
pb.close()
print(json.dumps(out))
""".replace("ROOT", repr(ROOT))


def _run(unroll):
    env = dict(os.environ)
    env["GPFVM_LOOP_UNROLL"] = str(unroll)
    env.pop("GPFVM_HOST_LOOP", None)
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_loop_unroll_is_bit_identical():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    runs = {u: _run(u) for u in (1, 2, 3)}
    for prec in runs[1]:
        assert runs[1][prec][0] == 0, (prec, runs[1][prec][:2])
        for u in (2, 3):
            assert runs[u][prec] == runs[1][prec], (prec, u, runs[u][prec][:2], runs[1][prec][:2])
