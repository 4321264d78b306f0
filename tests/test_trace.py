"""NVTX trace ranges of the solver (domain "irk").

A small NVTX tool library (tests/nvtx_probe.c, built here with the C
compiler) is attached through NVTX_INJECTION64_PATH in a child process.  It
counts the ranges by name and by "parent>name" and flags pops without a push.
On the CPU the create range is pushed and popped before the missing device is
reported.  On the GPU the host-driven loop (no graphs) must show one range per
step, Newton iteration, block solve and V-cycle, matching the solver's own
counters.  With graphs, each step must be one "step_graph" range.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import ctypes, json, sys
import numpy as np
from paper_2101_01776_gb300 import binding as B
mode, probe = sys.argv[1], sys.argv[2]
out = {}
if mode == "cpu":
    try:
        B.IrkSolver(np.zeros(64), op="diffusion1d", n=64, stages=2)
        out["created"] = True
    except B.IrkError as e:
        out["created"] = False
else:
    import workloads
    u0 = workloads.random_fourier_2d(64, seed=3)
    graphs = int(mode == "graph")
    with B.IrkSolver(u0, op="burgers2d", n=64, nu=5e-3, stages=2, use_graphs=graphs) as sol:
        st = sol.step(0.0, 2e-3, 3)
    out["stats"] = {k: getattr(st, k) for k in ("steps", "newton_its", "vcycles")}
P = ctypes.CDLL(probe)
P.probe_count.argtypes = [ctypes.c_char_p]
keys = sys.argv[3].split(",")
out["counts"] = {k: P.probe_count(k.encode()) for k in keys}
out["errors"], out["depth"], out["max_depth"] = P.probe_errors(), P.probe_depth(), P.probe_max_depth()
print(json.dumps(out))
"""


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    from paper_2101_01776_gb300 import build
    build.build()
    cuda_root = os.path.dirname(os.path.dirname(build.nvcc()))
    lib = str(tmp_path_factory.mktemp("nvtx") / "libnvtx_probe.so")
    src = os.path.join(ROOT, "tests", "nvtx_probe.c")
    subprocess.run(["gcc", "-O1", "-shared", "-fPIC", "-I", os.path.join(cuda_root, "include"), src,
                    "-o", lib, "-lpthread"], check=True)
    return lib


def run_child(mode, probe, keys):
    env = dict(os.environ, NVTX_INJECTION64_PATH=probe)
    r = subprocess.run([sys.executable, "-c", CHILD, mode, probe, ",".join(keys)], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_create_range_without_device(probe):
    import torch
    if torch.cuda.is_available():
        pytest.skip("checks the path that reports a missing device")
    out = run_child("cpu", probe, ["irk_create", ">irk_create"])
    assert out["created"] is False
    assert out["counts"] == {"irk_create": 1, ">irk_create": 1}
    assert out["errors"] == 0 and out["depth"] == 0 and out["max_depth"] == 1


@pytest.mark.gpu
def test_host_loop_ranges_match_counters(probe):
    keys = ["irk_step", ">irk_step", "irk_step>step", "step>newton", "newton>newton_iteration",
            "newton_iteration>block_solves", "vcycle", "block_solves>vcycle", "step_graph"]
    out = run_child("host", probe, keys)
    c, st = out["counts"], out["stats"]
    assert st["steps"] == 3
    assert c["irk_step"] == 1 and c[">irk_step"] == 1 and c["irk_step>step"] == 3
    assert c["step>newton"] == 3 and c["step_graph"] == 0
    # one loop pass per Newton update plus the converged check of each step
    assert c["newton>newton_iteration"] == st["newton_its"] + st["steps"]
    assert c["newton_iteration>block_solves"] == st["newton_its"]
    assert c["vcycle"] == st["vcycles"] > 0
    assert c["block_solves>vcycle"] == st["vcycles"]
    assert out["errors"] == 0 and out["depth"] == 0 and out["max_depth"] >= 5


@pytest.mark.gpu
def test_graph_step_ranges(probe):
    out = run_child("graph", probe, ["irk_step>step", "step>step_graph", "step>newton"])
    c = out["counts"]
    assert out["stats"]["steps"] == 3
    assert c["irk_step>step"] == 3 and c["step>step_graph"] == 3 and c["step>newton"] == 0
    assert out["errors"] == 0 and out["depth"] == 0
