"""CPU checks of the host planning code: the persistent thread pool, the
tcgen05 H_eff psi planner (operand deduplication, split-plane layout, tiles,
item chunks and reductions) and the launch plan of the batched Jacobi
eigensolver, through a small C++ program compiled against the package
sources (tests/cpp/host_planning_check.cpp).  No device calls."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2503_20700_gb300", "csrc")


def test_host_pool_planners(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("CUDA headers not found")
    exe = str(tmp_path / "host_planning_check")
    subprocess.run([cxx, "-std=c++17", "-O2", "-pthread", "-I", CSRC, "-I", cuda_inc,
                    os.path.join(ROOT, "tests", "cpp", "host_planning_check.cpp"),
                    os.path.join(CSRC, "hpsi_tc_plan.cpp"), os.path.join(CSRC, "host_pool.cpp"),
                    "-o", exe], check=True, timeout=300)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "host planning checks passed" in r.stdout
