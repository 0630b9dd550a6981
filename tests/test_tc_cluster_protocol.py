"""CPU model check of the clustered tcgen05 contraction's synchronisation
protocol (tests/tc_cluster_model.py) over plans made by the real planner:
no cluster of any plan deadlocks or meets a buffer hazard under random
schedules of its roles and completions.  A variant of the protocol without
the converters' in-order acknowledgement of the piece-read barrier, which
lets a converter fall two parity phases behind, is found faulty by the
same model.  No device calls."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import tc_cluster_model as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2503_20700_gb300", "csrc")


@pytest.fixture(scope="module")
def dumper(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("CUDA headers not found")
    exe = str(tmp_path_factory.mktemp("tcplan") / "tc_plan_dump")
    subprocess.run([cxx, "-std=c++17", "-O2", "-pthread", "-I", CSRC, "-I", cuda_inc,
                    os.path.join(ROOT, "tests", "cpp", "tc_plan_dump.cpp"),
                    os.path.join(CSRC, "hpsi_tc_plan.cpp"), os.path.join(CSRC, "host_pool.cpp"),
                    "-o", exe], check=True, timeout=300)
    return exe


def problem(seed, n_blocks, max_dim, max_items):
    """Random sector blocks and items (sizes only; a few identity factors)."""
    rng = np.random.default_rng(seed)
    out = [str(n_blocks)]
    op = 0
    for _ in range(n_blocks):
        m, n = (int(x) for x in rng.integers(1, max_dim, 2))
        cnt = int(rng.integers(1, max_items + 1))
        out.append("%d %d %d" % (m, n, cnt))
        for _ in range(cnt):
            ida = int(rng.random() < 0.1)
            idb = 0 if ida else int(rng.random() < 0.1)
            ka = m if ida else int(rng.integers(1, max_dim))
            kb = n if idb else int(rng.integers(1, max_dim))
            out.append("%d %d %d %d %d %d %d %d %d" % (ka, kb, ida, idb, rng.integers(0, 2), rng.integers(0, 2),
                                                       op, op + 1, op + 2))
            op += 3
    return "\n".join(out) + "\n"


def plan_of(dumper, tmp_path, text, ncta, cand=0):
    f = tmp_path / "problem.txt"
    f.write_text(text)
    r = subprocess.run([dumper, str(f), str(ncta), str(cand)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    plan = M.parse_plan(r.stdout)
    assert plan["check"] == "ok", plan["check"]
    return plan


CASES = [(9, 4, 300, 60), (1, 6, 700, 40), (2, 5, 600, 25), (3, 3, 1100, 12), (4, 8, 150, 8)]


@pytest.mark.parametrize("seed,nb,dim,items", CASES)
@pytest.mark.parametrize("ncta", [6, 24, 152])
def test_cluster_protocol_has_no_deadlock_or_hazard(dumper, tmp_path, seed, nb, dim, items, ncta):
    plan = plan_of(dumper, tmp_path, problem(seed, nb, dim, items), ncta)
    C = plan["cluster"]
    shared = sum(1 for lst in plan["lists"] for e in lst if e[2] > 1)
    for k in range(len(plan["lists"]) // C):
        for sched in range(2):
            for drain in (1024, 0):
                status, info = M.run_cluster(plan, k, seed=sched, drain_terms=drain)
                assert status == "ok", (k, sched, drain, status, info)
    if dim > 256:
        assert shared > 0  # the plans exercise groups that share stage 1


@pytest.mark.parametrize("cand", [1, 2, 3, 4, 5])
def test_cluster_protocol_under_every_schedule_candidate(dumper, tmp_path, cand):
    """The autotuner's other schedules (finer and coarser item chunks, block
    order, 128-wide tiles, clusters of four CTAs sharing stage 1 by groups of
    up to four tiles) keep the protocol free of deadlocks and hazards."""
    widest = 0
    for seed, nb, dim, items in CASES[:4]:
        plan = plan_of(dumper, tmp_path, problem(seed, nb, dim, items), 24, cand)
        C = plan["cluster"]
        widest = max([widest] + [e[2] for lst in plan["lists"] for e in lst])
        for k in range(len(plan["lists"]) // C):
            status, info = M.run_cluster(plan, k, seed=seed, drain_terms=1024)
            assert status == "ok", (cand, seed, k, status, info)
    if C == 4:
        assert widest == 4  # groups of four tiles share stage 1


def test_model_finds_the_unacknowledged_protocol_faulty(dumper, tmp_path):
    plan = plan_of(dumper, tmp_path, problem(9, 4, 300, 60), 152)
    C = plan["cluster"]
    bad = 0
    for k in range(len(plan["lists"]) // C):
        status, _ = M.run_cluster(plan, k, seed=0, ack=False)
        bad += status != "ok"
    assert bad > 0
