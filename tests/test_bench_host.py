"""Host logic of bench.py on the CPU: the warm-up ramp, the synthetic sector-
block problem of the kernel-only mode, and the N > 1 replica path (max of
the device times and sum of the FLOPs over ranks) on two gloo ranks."""
import os
import socket

import numpy as np
import pytest

import bench


def test_ramp_ends_at_target_and_doubles():
    assert bench.ramp(256, 3) == [64, 128, 256]
    assert bench.ramp(2048, 4) == [512, 1024, 2048, 2048]
    assert bench.ramp(16, 3) == [16, 16, 16]


def test_full_sweep_estimate_scales_measured_bond_steps():
    # 57 of the 76 bond steps of a 40-site sweep measured in 95 s
    assert bench.full_sweep_estimate(95.0, 57, 40) == pytest.approx(95.0 * 76 / 57)
    assert bench.full_sweep_estimate(10.0, 2 * (10 - 2), 10) == pytest.approx(10.0)
    assert bench.full_sweep_estimate(1.0, 0, 10) is None


def test_hpsi_problem_offsets_and_flops():
    A, P, B, clen, blocks, items, flops = bench.hpsi_problem(3, 4, 10, 30, 5)
    fl = 0.0
    for (c_off, m, n, ldc, ib, cnt) in blocks:
        assert ldc == n and c_off + m * n <= clen
        for it in items[ib:ib + cnt]:
            a_off, p_off, b_off, lda, ldp, ldb, ta, tb, ka, kb, a_id, b_id, alpha = it
            assert p_off + ka * kb <= P.size and ldp == kb
            if a_id:
                assert ka == m
            else:
                assert a_off + m * ka <= A.size and lda == (m if ta else ka)
                fl += 2.0 * m * ka * kb
            assert not b_id and b_off + n * kb <= B.size and ldb == (n if tb else kb)
            fl += 2.0 * m * n * kb
    assert fl == flops


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _replica(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    r, w, dist = bench.dist_init(world)
    assert (r, w) == (rank, world)
    # rank r "took" 1 + r seconds and did 10 * (r + 1) FLOPs
    t = bench.allmax(dist, 1.0 + rank)
    f = bench.allsum(dist, 10.0 * (rank + 1))
    bench.barrier(dist)
    out.put((rank, t, f))
    dist.destroy_process_group()


def test_replicas_take_max_time_and_sum_flops_over_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_replica, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2.0, 30.0), (1, 2.0, 30.0)]


def test_parse_ramp_and_bond_defaults():
    assert bench.parse_ramp("64:4,256:4,1024:4") == [(64, 4), (256, 4), (1024, 4)]
    assert bench.parse_ramp("") == []
    # the default step is the middle-bond product at D = 2048
    src = open(os.path.join(os.path.dirname(bench.__file__), "bench.py")).read()
    assert 'ap.add_argument("--mode", default="bond"' in src
    assert 'ap.add_argument("--D", type=int, default=2048)' in src


def test_initial_state_is_aufbau_for_cholesky_workloads():
    import workloads as W
    wl = bench.workload("cas8")
    occ, path = bench.initial_state(wl)
    assert sum(occ) == 8 and path[0] == 0 and occ == W.aufbau_state(wl["h"], 8, 0)[0]
    wl = bench.workload("naphthalene")
    assert bench.initial_state(wl) == (None, None)


def test_profiled_traffic_only_for_the_profiled_kernel():
    """The roofline's DRAM traffic comes from the committed ncu launch list
    only while the kernel source is the one that list was taken on."""
    import argparse
    import hashlib
    import bench
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = os.path.join(root, "paper_2503_20700_gb300", "csrc", "hpsi_tc.cu")
    prof = os.path.join(root, "profiles", "launch_list_cas40_D2048_bond19.md")
    a = argparse.Namespace(traffic=None)
    v, where = bench.profiled_traffic(a, True)
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    if os.path.exists(prof) and sha in open(prof).read():
        assert v is not None and v > 0 and where.endswith("launch_list_cas40_D2048_bond19.md")
    else:
        assert v is None
    assert bench.profiled_traffic(a, False) == (None, None)
    assert bench.profiled_traffic(argparse.Namespace(traffic=5.0), False) == (5.0, "--traffic")
