"""The serving runtime's HBM pool allocator on the host (no GPU).

The first-fit allocator (csrc/pool.h) decides admission by free HBM.
tests/pool_check.cpp drives it with random alloc/release sequences against a
brute-force granule map and checks, after every operation, four things:
- first fit in address order;
- alignment and the budget bound;
- failure exactly when no free run fits;
- a coalesced free list and exact usage.
At the end it checks that full release restores one free block.
"""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_pool_allocator_against_brute_force_model(tmp_path):
    exe = str(tmp_path / "pool_check")
    subprocess.run(["g++", "-O1", "-std=c++17", "-Wall", "-I",
                    os.path.join(ROOT, "paper_2101_01776_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "pool_check.cpp"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
