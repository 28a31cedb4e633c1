"""Device-side CG loops (graph WHILE nodes) and their host-driven form.

GPFVM_HOST_LOOP=1 replays the same captured iteration pass by pass from the
host (the form per-kernel profilers can attribute); both forms must give the
same iterations and bit-identical posteriors."""
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
prob = W.heat_2d(10, 9, 11, n_ic=(5, 5), n_bc=(2, 2), pred=(4, 4, 4), ell=(0.4, 0.3, 0.3))
out = {}
for prec in (0, 1, 2):
    pb = gpfvm.Problem(prob, max_iter=2000)
    pb.assemble()
    code, info = pb.solve(max_iter=2000, rtol=1e-10, precision=prec, want_var=True, inner_max_iter=400)
    mean = torch.empty(pb.P, dtype=torch.float64, device="cuda")
    var = torch.empty_like(mean)
    pb.query(mean, var)
    out[prec] = [code, info.iterations, mean.cpu().numpy().tolist(), var.cpu().numpy().tolist()]
    pb.close()
print(json.dumps(out))
""".replace("ROOT", repr(ROOT))


def _run(host_loop):
    env = dict(os.environ)
    env.pop("GPFVM_HOST_LOOP", None)
    if host_loop:
        env["GPFVM_HOST_LOOP"] = "1"
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_host_driven_loop_equals_device_loop():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = _run(False)
    host = _run(True)
    for prec in ("0", "1", "2"):
        assert dev[prec][0] == 0 and host[prec][0] == 0
        assert dev[prec][1] == host[prec][1]
        assert dev[prec][2] == host[prec][2]
        assert dev[prec][3] == host[prec][3]
