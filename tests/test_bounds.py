"""The bounds-checked debug build (-DIRK_BOUNDS, _lib/libirk_bounds.so).

In that build the kernels' index checks record out-of-range indices in device
records instead of reaching memory (no trap, no assert).  irk_step, the
stage-residual and Jacobian entry points and the allocation-free residual
then fail on any recorded hit.  The CPU test builds the library and checks
that it exports the same C ABI and identifies as the bounds build.  The GPU
tests check two things in child processes that load it through IRK_LIBRARY:
- the checker itself, through the one-thread self-test;
- a zero hit count over the small-grid parity cases (n = 8..64, where every
  multigrid tile is a boundary tile and the coarse levels are a few points
  wide), which compare each entry point with the oracle.
"""
import ctypes
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bounds_lib():
    from paper_2101_01776_gb300 import build
    return build.build(bounds=True)


def gpu_available():
    import torch
    return torch.cuda.is_available()


def test_bounds_build_exports_the_abi(bounds_lib):
    from test_capi_host import declared_functions
    lib = ctypes.CDLL(bounds_lib)
    for name in declared_functions():
        assert hasattr(lib, name), name
    lib.irk_debug_bounds.restype = ctypes.c_longlong
    lib.irk_debug_bounds.argtypes = [ctypes.c_int, ctypes.c_char_p, ctypes.c_size_t]
    if not gpu_available():
        # a bounds build: it tries to read the device records (and fails without a device)
        buf = ctypes.create_string_buffer(128)
        assert lib.irk_debug_bounds(0, buf, len(buf)) == -2
        assert b"could not be read" in buf.value


def test_normal_build_is_not_a_bounds_build():
    from paper_2101_01776_gb300 import build
    build.build()
    from paper_2101_01776_gb300 import binding as B
    if B._LIB_PATH != build.LIB:
        pytest.skip("the binding loaded another build")
    hits, msg = B.irk_debug_bounds(selftest=True)
    assert hits == -1 and msg == "not a bounds-checked build"


SELFTEST = r"""
from paper_2101_01776_gb300 import binding as B
import numpy as np
assert B.irk_debug_bounds()[0] == 0
hits, msg = B.irk_debug_bounds(selftest=True)
assert hits == 1 and "blas.cu" in msg and "index 1 outside [0, 1)" in msg, (hits, msg)
assert B.irk_debug_bounds() == (0, "")
u0 = np.random.default_rng(5).standard_normal((2, 16, 16)) * 0.5
with B.IrkSolver(u0, op="burgers2d", n=16, nu=2e-2, stages=3) as sol:
    sol.step(0.0, 1e-2, 2)
assert B.irk_debug_bounds()[0] == 0
print("ok")
"""

PARITY_CASES = ("stage_residual or stage_jacobian or burgers2d_parity or vsf_parity or sdirk_parity "
                "or radau_lobatto_2d or device_buffers or edge_cases or vsf_block_triangular "
                "or solver_variants or mixed_precision or graph_path or bad_warm_start "
                "or failed_step or linear_diffusion_pade_per_mode")


def child_env(lib):
    return dict(os.environ, IRK_LIBRARY=lib)


@pytest.mark.gpu
def test_bounds_selftest_records_one_hit(bounds_lib):
    if not gpu_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, "-c", SELFTEST], cwd=ROOT, env=child_env(bounds_lib),
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout[-2000:] + r.stderr[-2000:]


@pytest.mark.gpu
def test_small_grid_parity_cases_record_no_hit(bounds_lib):
    if not gpu_available():
        pytest.skip("no CUDA device")
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
           "tests/test_gpu_parity.py", "tests/test_zz_no_alloc.py", "-k", PARITY_CASES]
    r = subprocess.run(cmd, cwd=ROOT, env=child_env(bounds_lib), capture_output=True, text=True,
                       timeout=1200)
    tail = r.stdout[-3000:] + r.stderr[-2000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout and " failed" not in r.stdout, tail
