"""Benchmark of the spin-adapted DMRG hot path (H_eff psi TFLOP/s at D, sweep time).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--mode bond|sweep] [--workload cas40|casN|pentacene|naphthalene]
                    [--D 2048] [--precision split-tc|split|split-all|fp64]

--mode bond (default): a step is one H_eff psi product at the middle bond of
the workload at bond dimension D, inside the Davidson solve of that bond.
The state is brought there by a ramp of sweeps (D 256 then 1024, Davidson
capped), one L->R half-sweep at D and an R->L part down to the bond next to
the middle one; the W warm-up products and the K timed products then run at
the middle bond on the same blocks (dmrg_bond_solve).  The FP64 arm times
float64 products at the same bond on the same vector, and the precision of
the split result is reported as its float64 residual.

--mode sweep: a step is one full two-site sweep (L->R then R->L: blocking,
Davidson with H_eff psi, decimation, renormalisation) at D, after W warm-up
sweeps that ramp D.

The library's work stays in HBM; the timed region is bracketed by a barrier
and a device synchronisation, and its device time comes from CUDA events
the library records on its stream.  With N > 1 GPUs every rank runs an
independent replica (replicas only) and ``value`` is the sum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H_eff·ψ TFLOP/s & sweep time at D=2048, split-FP32 vs FP64, at ΔE≤1e-6 Eh"
L2_BYTES = 129 * 1024 * 1024


def workload(name, seed=20250326):
    import workloads as W
    if name == "cas40":
        h, L = W.cholesky_random(40, 160, seed=seed)
        return dict(h=h, chol=L, eri=None, n_elec=40, two_s=0, e_core=0.0,
                    desc="random Cholesky CAS(40,40), rank 160, singlet")
    if name == "pentacene":
        h, eri, ec = W.ppp_acene(5)
        return dict(h=h, chol=None, eri=eri, n_elec=22, two_s=0, e_core=ec,
                    desc="PPP pentacene pi-system, 22 sites/electrons, singlet")
    if name == "naphthalene":
        h, eri, ec = W.ppp_acene(2)
        return dict(h=h, chol=None, eri=eri, n_elec=10, two_s=0, e_core=ec,
                    desc="PPP naphthalene pi-system, 10 sites/electrons, singlet")
    if name.startswith("cas"):
        n = int(name[3:])
        h, L = W.cholesky_random(n, 4 * n, seed=seed)
        return dict(h=h, chol=L, eri=None, n_elec=n, two_s=0, e_core=0.0,
                    desc=f"random Cholesky CAS({n},{n}), rank {4 * n}, singlet")
    raise SystemExit(f"unknown workload {name}")


def ramp(D, W):
    """Bond dimensions of the W warm-up sweeps, ending at D."""
    seq = []
    d = max(16, D // 4)
    for _ in range(W):
        seq.append(min(d, D))
        d *= 2
    if seq:
        seq[-1] = D
    return seq


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during a region."""

    def __init__(self, device):
        self.device = device
        self.samples = []
        self._stop = threading.Event()
        self._proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self._proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, ValueError):
            self._proc = None
        return self

    def _read(self):
        for line in self._proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self._proc:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self._proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def dist_init(n_gpus):
    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo", init_method="env://")
        return rank, world, dist
    return 0, 1, None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def allmax(dist, x):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allsum(dist, x):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def oracle_sample(seconds_budget=15.0):
    """The CPU oracle on a bounded sample: sweeps of the random Cholesky
    active space at n=8 (the full-space oracle cannot hold 40 orbitals), D=12."""
    import workloads as W
    from oracle.dmrg import OracleDMRG
    h, L = W.cholesky_random(8, 32, seed=20250326)
    eri = W.eri_from_cholesky(L)
    o = OracleDMRG(h, eri, 8, 0, D=12)
    t0 = time.perf_counter()
    sweeps = 0
    while time.perf_counter() - t0 < seconds_budget and sweeps < 6:
        o.sweep(1)
        sweeps += 1
    wall = time.perf_counter() - t0
    tf = o.heff_flops / max(o.heff_seconds, 1e-12) / 1e12
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": tf, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
            "sample": (f"{sweeps} oracle sweep(s) of cholesky_random(8, 32) at D=12 "
                       f"({o.heff_calls} H_eff applications, executed FLOPs of the full-space "
                       f"H_eff application / their time; {wall:.1f} s wall)")}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    res = []
    # each step a bounded sample, so that the whole run stays within minutes
    per_step = max(1.0, min(10.0, 90.0 / max(1, args.steps)))
    for _ in range(args.warmup):
        oracle_sample(min(3.0, per_step))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        res.append(oracle_sample(per_step))
    wall = time.perf_counter() - t0
    v = float(np.mean([r["value"] for r in res]))
    cb = dict(res[-1])
    cb["value"] = v
    line = {"metric": METRIC, "value": v, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": wall * 1000 / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "oracle sample: cholesky_random(8, 32), D=12 (CPU oracle)"},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def hpsi_problem(seed, n_blocks, dim_lo, dim_hi, items_per_block):
    """Synthetic sector-block H_eff psi contraction with the shape mix of the
    middle bonds of the Cholesky workloads (sector dimensions dim_lo..dim_hi,
    a few percent identity factors), as flat float64 host arrays and the
    block/item tuples of ops.hpsi_contract."""
    rng = np.random.default_rng(seed)
    dims = rng.integers(dim_lo, dim_hi + 1, size=n_blocks * 2)
    A_parts, P_parts, B_parts, blocks, items = [], [], [], [], []
    ao = po = bo = co = 0
    flops = 0.0
    for b in range(n_blocks):
        m, n = int(dims[2 * b]), int(dims[2 * b + 1])
        ib = len(items)
        for _ in range(items_per_block):
            ka = m if rng.random() < 0.02 else int(rng.integers(dim_lo, dim_hi + 1))
            kb = n if rng.random() < 0.02 else int(rng.integers(dim_lo, dim_hi + 1))
            a_id, b_id = int(ka == m and rng.random() < 0.5), 0
            ta, tb = int(rng.integers(0, 2)), int(rng.integers(0, 2))
            if a_id:
                a_entry = (0, 1, 0)
            else:
                a = rng.standard_normal((ka, m) if ta else (m, ka))
                a_entry = (ao, a.shape[1], ta)
                A_parts.append(a.ravel())
                ao += a.size
                flops += 2.0 * m * ka * kb
            bm = rng.standard_normal((kb, n) if tb else (n, kb))
            B_parts.append(bm.ravel())
            b_entry = (bo, bm.shape[1], tb)
            bo += bm.size
            flops += 2.0 * m * n * kb
            P_parts.append(rng.standard_normal(ka * kb))
            items.append((a_entry[0], po, b_entry[0], a_entry[1], kb, b_entry[1], a_entry[2], b_entry[2],
                          ka, kb, a_id, b_id, float(rng.standard_normal())))
            po += ka * kb
        blocks.append((co, m, n, n, ib, len(items) - ib))
        co += m * n
    return (np.concatenate(A_parts), np.concatenate(P_parts), np.concatenate(B_parts), co, blocks, items,
            flops)


def run_hpsi_only(args):
    """The H_eff psi contraction alone (dmrg_hpsi_contract, one launch per
    step) on the synthetic sector blocks; device time from CUDA events."""
    import paper_2503_20700_gb300 as pkg
    pkg.load()
    prec = {"split": 1, "split-tc": 4, "split-all-tc": 4, "split-all": 1, "fp64": 0}[args.precision]
    if args.hpsi_shape == "large":
        # sector dimensions of the middle bonds at D = 1024 .. 2048 (300 .. 600)
        A, P, B, clen, blocks, items, flops = hpsi_problem(7, 8, 300, 600, 30)
    else:
        A, P, B, clen, blocks, items, flops = hpsi_problem(7, 16, 100, 250, 80)
    C = np.zeros(clen)
    W, K = max(3, args.warmup), max(1, args.steps)
    for _ in range(W):
        pkg.ops.hpsi_contract(A, P, B, C, blocks, items, precision=prec)
    ms = []
    for _ in range(K):
        pkg.ops.hpsi_contract(A, P, B, C, blocks, items, precision=prec)
        ms.append(pkg.ops.last_contract_ms())
    t = float(np.median(ms))
    achieved = flops / (t / 1000.0) / 1e12
    pk, src = peaks()
    peak = pk["bf16_tflops"] * (1.1 / 2.25) / 3.0 if prec else 1.25
    nbytes = 8.0 * (A.size + P.size + B.size + 2 * clen)
    print(json.dumps({"mode": "hpsi-only", "shape": args.hpsi_shape, "precision": args.precision,
                      "value": achieved, "unit": "TFLOP/s",
                      "ms_per_launch": t, "steps": K, "warmup": W, "algorithmic_flops": flops,
                      "operand_bytes": nbytes, "blocks": len(blocks), "items": len(items),
                      "roofline": {"bound": "tensor" if prec else "alu", "achieved": achieved, "peak": peak,
                                   "unit": "TFLOP/s", "frac": achieved / peak,
                                   "peak_source": ("3xTF32 effective peak = burst bf16 (%s) x 1.1/2.25 / 3" % src)
                                   if prec else "FP64 nominal 1.25 TFLOP/s"}}))
    return 0


def initial_state(wl):
    """Aufbau occupation for the Cholesky workloads (their h_pp grow along the
    chain), the even-spread default state for the half-filled PPP models."""
    import workloads as W
    if wl["chol"] is not None:
        return W.aufbau_state(wl["h"], wl["n_elec"], wl["two_s"])
    return None, None


def tc_peak(prec, pk, src, pkg):
    if prec != pkg.FP64:
        # 3xTF32: three TF32 tensor products per algorithmic product; TF32 peak =
        # measured dense bf16 peak x the nominal TF32/BF16 ratio (1.1/2.25)
        return (pk["bf16_tflops_sustained"] * (1.1 / 2.25) / 3.0,
                f"3xTF32 effective peak = sustained bf16 ({src}) x 1.1/2.25 / 3")
    return 1.25, "FP64 nominal 1.25 TFLOP/s (no measured FP64 peak)"


def profiled_traffic(args, mode_default):
    """DRAM bytes per contraction launch for the roofline: --traffic, else, on
    the default workload, the figure of the committed ncu launch list of the
    same command, if that list was taken on the kernel source as it is now
    (its sha256 is recorded in the summary); else None."""
    if args.traffic is not None:
        return args.traffic, "--traffic"
    if not mode_default:
        return None, None
    import hashlib
    here = os.path.dirname(os.path.abspath(__file__))
    prof = os.path.join(here, "profiles", "launch_list_cas40_D2048_bond19.md")
    src = os.path.join(here, "paper_2503_20700_gb300", "csrc", "hpsi_tc.cu")
    try:
        text = open(prof).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None, None
    if sha not in text:
        return None, None
    for line in text.splitlines():
        if line.startswith("traffic_bytes_per_launch:"):
            return float(line.split(":", 1)[1]), os.path.relpath(prof, here)
    return None, None


def full_sweep_estimate(seconds, bonds, n):
    """Wall time of a full sweep (L->R over bonds 0..n-3, R->L over n-2..1:
    2(n-2) bond steps) extrapolated from `seconds` measured over `bonds` bond
    steps of the same bond dimension and Davidson cap."""
    return seconds * 2.0 * (n - 2) / bonds if bonds > 0 else None


def parse_ramp(text):
    out = []
    for part in text.split(","):
        if part.strip():
            d, it = part.split(":")
            out.append((int(d), int(it)))
    return out


def run_bond(args, pkg, prec, rank, world, dist, device):
    wl = workload(args.workload)
    n = wl["h"].shape[0]
    mid = n // 2 - 1 if args.bond < 0 else args.bond
    W, K = max(3, args.warmup), max(1, args.steps)
    ramp_list = parse_ramp(args.ramp)
    occ, path = initial_state(wl)
    barrier(dist)
    t_job0 = time.perf_counter()
    g = pkg.DMRG(wl["h"], eri=wl["eri"], chol=wl["chol"], n_elec=wl["n_elec"], two_s=wl["two_s"],
                 D=ramp_list[0][0] if ramp_list else args.D, e_core=wl["e_core"], precision=prec,
                 tol=args.tol, device=device, verbose=args.verbose, occ=occ, two_s_right=path)
    flops_job = 0.0
    products = 0  # H_eff psi products before the timed region (one contraction launch each)
    t_ramp0 = time.perf_counter()
    ramp_energies = []
    for d, it in ramp_list:
        g.set_bond_dim(d)
        g.set_davidson(it, args.tol)
        ramp_energies.append(g.sweep(1)[0])
        flops_job += g.stats()["hpsi_flops"]
        products += g.stats()["hpsi_calls"]
    t_ramp = time.perf_counter() - t_ramp0
    # at the target D: one L->R half-sweep, then R->L down to the bond next to
    # the middle one, with the Davidson cap of the approach
    g.set_bond_dim(args.D)
    g.set_davidson(args.approach_iters, args.tol)
    t_app0 = time.perf_counter()
    g.sweep_part(0, n - 3)
    flops_job += g.stats()["hpsi_flops"]
    products += g.stats()["hpsi_calls"]
    app_ms = g.sweep_device_ms()
    # wall seconds per phase of the D=2048 bonds of the approach (the parts of
    # a sweep besides the H_eff psi products: blocking, planning, decimation,
    # renormalisation), summed over both parts
    app_phases = dict(g.phases())
    app_bonds = n - 2
    app_products = g.stats()["hpsi_calls"]
    g.sweep_part(1, mid + 1)
    flops_job += g.stats()["hpsi_flops"]
    products += g.stats()["hpsi_calls"]
    app_ms += g.sweep_device_ms()
    for k, v in g.phases().items():
        app_phases[k] = app_phases.get(k, 0.0) + v
    app_bonds += (n - 2) - (mid + 1) + 1
    app_products += g.stats()["hpsi_calls"]
    t_app = time.perf_counter() - t_app0
    left, right = g.block_dims()
    left_u1, right_u1 = g.block_dims_u1()  # the same blocks in U(1) states (D~)
    # schedule autotuning at the middle bond (split tcgen05 path): each
    # candidate schedule computes one product of a Davidson solve of the bond
    # and the fastest is kept for its sector histogram
    schedule = None
    if prec in (pkg.SPLIT_HPSI_TC, pkg.SPLIT_ALL_TC) and not args.no_autotune:
        cands = pkg.tc_shape_candidates()
        g.set_tc_autotune(True)
        g.bond_solve(mid, 1, prec, max_iter=1, tol=args.tol, min_calls=len(cands), check64=False)
        products += len(cands)
        info = g.tc_schedule()
        schedule = {"picked": {"tile_n": info["shape"][0], "chunks_per_cta": info["shape"][1],
                               "order": info["shape"][2], "cluster": info["shape"][3]},
                    "candidates": [{"tile_n": c[0], "chunks_per_cta": c[1], "order": c[2], "cluster": c[3],
                                    "ms": t} for c, t in zip(cands, info["ms"])]}
    # warm-up products at the middle bond
    g.bond_solve(mid, 1, prec, max_iter=max(1, W - 1), tol=args.tol, min_calls=W, check64=False)
    # ---- timed region: K products inside the Davidson solve of the middle bond
    barrier(dist)
    g.profile(True)
    l0 = g.launch_count()
    with Clocks(device) as clk:
        t0 = time.perf_counter()
        res = g.bond_solve(mid, 1, prec, max_iter=max(1, K - 1), tol=args.tol, min_calls=K, check64=False)
        wall = time.perf_counter() - t0
    launches = g.launch_count() - l0
    k_ms, k_launch = res["contraction_ms"], res["contraction_launches"]
    k_flops = res["calls"] * res["flops_per_call"]
    s_ms, s_launch = res["split_ms"], res["calls"]
    flops_job += res["calls"] * res["flops_per_call"]
    kernel_ms = {name: g.kernel_stats(i)[0]
                 for i, name in enumerate(["gemm", "hpsi", "place", "eigh_subspace", "eigh_batched",
                                           "split"])}
    dev_s = res["ms_total"] / 1000.0
    t_max = allmax(dist, dev_s)
    flops_all = allsum(dist, res["calls"] * res["flops_per_call"])
    value = flops_all / t_max / 1e12
    # ---- FP64 arm: one float64 product at the same bond on the split
    # result's vector; it also gives the float64 Rayleigh quotient and residual
    fp64 = None
    chk = g.bond_check64()
    res["energy_rq64"], res["residual64"] = chk["energy_rq64"], chk["residual64"]
    if prec != pkg.FP64:
        v64 = chk["flops"] / (chk["ms"] / 1000.0) / 1e12
        fp64 = {"value": v64, "unit": "TFLOP/s", "calls": 1, "ms_per_call": chk["ms"],
                "speedup_split_over_fp64": value / v64, "kernel": "hpsi_f64_kernel"}
        if args.fp64_converge:
            e_split_rq = res["energy_rq64"]
            rc = g.bond_solve(mid, 1, pkg.FP64, max_iter=200, tol=args.tol, min_calls=0)
            fp64["converged"] = {"energy": rc["energy_rq64"], "residual64": rc["residual64"],
                                 "iterations": rc["iterations"],
                                 "delta_e_split_minus_fp64": e_split_rq - rc["energy_rq64"]}
    mem_now, mem_peak = g.memory()
    _ = g.energy()
    t_job = allmax(dist, time.perf_counter() - t_job0)
    barrier(dist)

    pk, src = peaks()
    default_workload = (args.workload == "cas40" and args.D == 2048 and args.bond < 0 and
                        args.precision == "split-tc" and args.ramp == "64:4,256:4,1024:4")
    traffic, traffic_src = profiled_traffic(args, default_workload)
    peak_tf, peak_note = tc_peak(prec, pk, src, pkg)
    achieved = k_flops / (k_ms / 1000.0) / 1e12 if k_ms > 0 else 0.0
    roof = {"bound": "tensor" if prec != pkg.FP64 else "alu", "achieved": achieved, "peak": peak_tf,
            "unit": "TFLOP/s", "frac": achieved / peak_tf, "traffic": traffic, "traffic_source": traffic_src,
            "kernel": {pkg.FP64: "hpsi_f64_kernel", pkg.SPLIT_HPSI_TC: "hpsi_tc_kernel",
                       pkg.SPLIT_ALL_TC: "hpsi_tc_kernel"}.get(prec, "hpsi_tf32x3_kernel"),
            "launches": k_launch, "avg_launch_ms": k_ms / max(1, k_launch), "peak_source": peak_note,
            "what": "algorithmic FLOPs of the contraction launches (kernel and chunk reduction) / their "
                    "CUDA-event time; the psi splits are timed apart (split_ms)",
            "split_ms": s_ms, "split_launches": s_launch}
    e2e = None
    if not args.no_e2e:
        h2d = wl["h"].nbytes + (wl["eri"].nbytes if wl["eri"] is not None else wl["chol"].nbytes)
        e2e = {"value": allsum(dist, flops_job) / t_job / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": 8, "seconds": t_job,
               "what": ("whole job through the public API: dmrg_init from host integrals (h2d once), "
                        f"ramp sweeps {ramp_list}, the approach to bond {mid} at D={args.D}, W={W} warm-up "
                        f"and K={K} timed products, the FP64 arm, energy read back (d2h); all H_eff psi "
                        "FLOPs / wall time")}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(15.0)
    if rank == 0:
        ms_sorted = sorted(res["call_ms"])
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": K,
                "warmup": W, "ms_per_step": t_max * 1000.0 / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "tf32x3" if prec != pkg.FP64 else "f64", "data": "synthetic",
                "config": {"workload": f"{wl['desc']}: H_eff psi at the middle bond {mid} at D={args.D}",
                           "D": args.D, "bond": mid, "ramp": ramp_list, "approach_davidson_iters": args.approach_iters,
                           "schedule": schedule,
                           "precision": args.precision, "davidson_tol": args.tol,
                           "parallelism": "replicas" if world > 1 else "single",
                           "l2": ("operators larger than L2" if mem_peak > 4 * L2_BYTES
                                  else "working set below L2 size")},
                "step": "one H_eff psi product inside the Davidson solve of the bond",
                "flops_per_step": res["flops_per_call"], "psi_dim": res["dim"],
                "ms_median": ms_sorted[len(ms_sorted) // 2] if ms_sorted else None,
                "davidson_iters": res["iterations"],
                "precision_check": {"energy_split": res["energy"], "energy_rq64": res["energy_rq64"],
                                    "delta_e_eval": res["energy"] - res["energy_rq64"],
                                    "residual64": res["residual64"], "ritz_gap": res["gap"],
                                    "delta_e_bound": (res["residual64"] ** 2 / res["gap"]) if res["gap"] > 0 else None},
                "fp64": fp64, "ramp_energies": ramp_energies, "ramp_seconds": t_ramp,
                "approach_seconds": t_app, "approach_device_ms": app_ms,
                "sweep_seconds_estimate": {
                    "value": full_sweep_estimate(t_app, app_bonds, n),
                    "what": (f"a full sweep at D={args.D} with the approach's Davidson cap "
                             f"({args.approach_iters} iterations per bond), extrapolated from the "
                             f"{app_bonds} bond steps of the approach measured at that D "
                             f"(of {2 * (n - 2)} in a sweep); not a converged sweep")},
                "approach_phases": {"bonds": app_bonds, "products": app_products,
                                    "seconds": {k: app_phases[k] for k in
                                                ("enlarge", "plan", "davidson", "decimate", "renormalize",
                                                 "guess")}},
                "block_dims_left": left.tolist(), "block_dims_right": right.tolist(),
                "block_dims_u1_left": left_u1.tolist(), "block_dims_u1_right": right_u1.tolist(),
                "wall_seconds": wall, "hpsi_tflops_kernel": achieved, "device_mem_peak_gb": mem_peak / 1e9,
                "kernel_ms": kernel_ms, "clocks": clk.summary(), "e2e": e2e, "gpu_launches": launches,
                "launches_before_timed": l0, "contraction_launches_before_timed": products + W,
                "roofline": roof, "cpu_baseline": cpu}
        print(json.dumps(line))
    g.close()
    return 0


def run_sweep(args, pkg, prec, rank, world, dist, device):
    wl = workload(args.workload)
    W, K = max(3, args.warmup), max(1, args.steps)
    ds = ramp(args.D, W)
    occ, path = initial_state(wl)
    # the whole job runs through the public API from host integrals: its wall
    # time (dmrg_init with the host->device copy of the integrals, every sweep,
    # the final energy read back) is the end-to-end figure
    barrier(dist)
    t_job0 = time.perf_counter()
    g = pkg.DMRG(wl["h"], eri=wl["eri"], chol=wl["chol"], n_elec=wl["n_elec"], two_s=wl["two_s"],
                 D=ds[0], e_core=wl["e_core"], precision=prec, tol=args.tol, device=device,
                 verbose=args.verbose, occ=occ, two_s_right=path,
                 tc_autotune=prec in (pkg.SPLIT_HPSI_TC, pkg.SPLIT_ALL_TC) and not args.no_autotune)
    flops_job = 0.0
    for d in ds:
        g.set_bond_dim(d)
        g.sweep(1)
        flops_job += g.stats()["hpsi_flops"]
    # ---- timed region
    barrier(dist)
    g.profile(True)
    l0 = g.launch_count()
    flops, dev_ms, energies = 0.0, 0.0, []
    with Clocks(device) as clk:
        t0 = time.perf_counter()
        phases = None
        for _ in range(K):
            e, _ = g.sweep(1)
            st = g.stats()
            ph = g.phases()
            phases = ph if phases is None else {k: phases[k] + ph[k] for k in ph}
            flops += st["hpsi_flops"]
            dev_ms += g.sweep_device_ms()
            energies.append(e)
        wall = time.perf_counter() - t0
    launches = g.launch_count() - l0
    k_ms, k_flops, k_launch = g.kernel_stats(1)
    s_ms, _, s_launch = g.kernel_stats(5)
    kernel_ms = {name: g.kernel_stats(i)[0]
                 for i, name in enumerate(["gemm", "hpsi", "place", "eigh_subspace", "eigh_batched",
                                           "split"])}
    mem_now, mem_peak = g.memory()
    flops_job += flops
    _ = g.energy()
    t_job = allmax(dist, time.perf_counter() - t_job0)
    barrier(dist)
    t_max = allmax(dist, dev_ms / 1000.0)
    flops_all = allsum(dist, flops)
    value = flops_all / t_max / 1e12
    pk, src = peaks()
    peak_tf, peak_note = tc_peak(prec, pk, src, pkg)
    achieved = k_flops / (k_ms / 1000.0) / 1e12 if k_ms > 0 else 0.0
    roof = {"bound": "tensor" if prec != pkg.FP64 else "alu", "achieved": achieved,
            "peak": peak_tf, "unit": "TFLOP/s", "frac": achieved / peak_tf, "traffic": args.traffic,
            "traffic_source": "--traffic" if args.traffic is not None else None,
            "kernel": {pkg.FP64: "hpsi_f64_kernel", pkg.SPLIT_HPSI_TC: "hpsi_tc_kernel",
                       pkg.SPLIT_ALL_TC: "hpsi_tc_kernel"}.get(prec, "hpsi_tf32x3_kernel"),
            "launches": k_launch, "avg_launch_ms": k_ms / max(1, k_launch), "peak_source": peak_note,
            "split_ms": s_ms, "split_launches": s_launch}
    e2e = None
    if not args.no_e2e:
        h2d = wl["h"].nbytes + (wl["eri"].nbytes if wl["eri"] is not None else wl["chol"].nbytes)
        e2e = {"value": allsum(dist, flops_job) / t_job / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": 8, "seconds": t_job,
               "what": ("whole job through the public API: dmrg_init from host integrals (h2d once), "
                        f"{len(ds)} warm-up sweeps at D={ds} and {K} timed sweep(s), energy read back (d2h)")}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(15.0)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": K,
                "warmup": W, "ms_per_step": t_max * 1000.0 / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "tf32x3" if prec != pkg.FP64 else "f64", "data": "synthetic",
                "config": {"workload": f"{wl['desc']}: full sweeps at D={args.D}", "D": args.D, "warmup_D": ds,
                           "precision": args.precision, "davidson_tol": args.tol,
                           "parallelism": "replicas" if world > 1 else "single",
                           "l2": ("operators larger than L2" if mem_peak > 4 * L2_BYTES
                                  else "working set below L2 size")},
                "step": "one full sweep", "sweep_energy": energies[-1], "sweep_energies": energies,
                "sweep_seconds": t_max / K, "wall_seconds": wall,
                "hpsi_tflops_kernel": achieved, "device_mem_peak_gb": mem_peak / 1e9,
                "phase_seconds": phases, "kernel_ms": kernel_ms, "davidson_iters": st["davidson_iters"],
                "clocks": clk.summary(), "e2e": e2e, "gpu_launches": launches,
                "roofline": roof, "cpu_baseline": cpu}
        print(json.dumps(line))
    g.close()
    return 0


def run_casscf(args, pkg, prec, rank, world, dist, device):
    """The CAS-SCF gradient step at the configuration size: 200 orbitals (20
    core, CAS(30,30), 150 virtual), Cholesky ERIs of rank 600.  A small
    orbital rotation U = exp(-kappa) and the integral transformation (timed
    on the device: float64 GEMMs), the active-space problem, DMRG on the
    CAS(30,30) ramped to D=1024, the spin-free RDMs from the float64
    measurement pass and the generalised-Fock orbital gradient.  (Their
    parity with the oracle at this size is a GPU test, not part of the bench.)"""
    import workloads as W
    from paper_2503_20700_gb300 import ops
    nb, ncore, ncas, rk = 200, 20, 30, 600
    h, L = W.cholesky_random(nb, rk, seed=20250326)
    rng = np.random.default_rng(20250326)
    K = 0.01 * rng.standard_normal((nb, nb))
    K = K - K.T
    t_job0 = time.perf_counter()
    R = ops.rotation(K, device)
    hr, Lr = ops.transform(R, h, L, device)
    tr_ms, tr_flops = ops.casscf_last_kernel_ms()
    e_core, h_act, eri_act = ops.active_space(hr, Lr, ncore, ncas, device)
    occ, path = W.aufbau_state(h_act, ncas, 0)
    ramp_list = parse_ramp(args.ramp)
    g = pkg.DMRG(h_act, eri=eri_act, n_elec=ncas, two_s=0, D=ramp_list[0][0], e_core=e_core, precision=prec,
                 tol=args.tol, device=device, occ=occ, two_s_right=path)
    t0 = time.perf_counter()
    energies = []
    for d, it in ramp_list + [(1024, args.approach_iters)] * max(1, args.steps):
        g.set_bond_dim(d)
        g.set_davidson(it, args.tol)
        energies.append(g.sweep(1)[0])
    t_dmrg = time.perf_counter() - t0
    t0 = time.perf_counter()
    gamma, Gamma = g.rdm12()
    t_rdm = time.perf_counter() - t0
    g.close()
    t0 = time.perf_counter()
    grad = ops.orbital_gradient(hr, Lr, ncore, ncas, gamma, Gamma, device)
    t_grad = time.perf_counter() - t0
    gr_ms, gr_flops = ops.casscf_last_kernel_ms()
    t_job = time.perf_counter() - t_job0
    pk, src = peaks()
    tr_bytes = 2.0 * (L.nbytes + h.nbytes)  # algorithmic: read h and L, write h' and L'
    if rank == 0:
        print(json.dumps({
            "mode": "casscf", "config": {"workload": "random Cholesky, 200 orbitals (20 core, CAS(30,30), 150 "
                                                     "virtual), rank 600", "D": 1024, "precision": args.precision,
                                         "ramp": ramp_list, "sweeps_at_D": max(1, args.steps)},
            "transform": {"ms": tr_ms, "fp64_tflops": tr_flops / (tr_ms / 1e3) / 1e12 if tr_ms > 0 else None,
                          "gb_per_s": tr_bytes / (tr_ms / 1e3) / 1e9 if tr_ms > 0 else None, "algorithmic_bytes": tr_bytes,
                          "algorithmic_flops": tr_flops,
                          "bound": "fp64 alu", "fp64_peak_note": "nominal 1.25 TFLOP/s FP64 (no measured FP64 peak)"},
            "dmrg": {"seconds": t_dmrg, "energies": energies, "rdm_seconds": t_rdm,
                     "trace_gamma": float(np.trace(gamma))},
            "gradient": {"seconds": t_grad, "kernel_ms": gr_ms, "max_abs": float(np.abs(grad).max())},
            "job_seconds": t_job, "peaks_source": src}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="bond", choices=["bond", "sweep", "casscf"])
    ap.add_argument("--workload", default="cas40")
    ap.add_argument("--D", type=int, default=2048)
    ap.add_argument("--bond", type=int, default=-1, help="bond of --mode bond (default: the middle one)")
    ap.add_argument("--ramp", default="64:4,256:4,1024:4",
                    help="--mode bond: sweeps before the target D, as D:davidson_iters,...")
    ap.add_argument("--approach-iters", type=int, default=2,
                    help="--mode bond: Davidson cap of the half-sweeps at the target D")
    ap.add_argument("--fp64-converge", action="store_true",
                    help="--mode bond: also converge the float64 Davidson at the bond (slow at large D)")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per contraction launch from an ncu capture of the same kernel")
    ap.add_argument("--precision", default="split-tc",
                    choices=["split", "split-tc", "split-all-tc", "split-all", "fp64"],
                    help="split-tc: 3xTF32 H_eff psi on tcgen05, renormalisation in FP64; "
                         "split-all-tc: the renormalisation U^T O U on tcgen05 too; "
                         "split: the H_eff psi products on mma.sync; split-all: mma.sync 3xTF32 also in "
                         "renormalisation; fp64: all FP64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="bond mode: keep the default schedule of the tcgen05 launch (no timing of candidates)")
    ap.add_argument("--tol", type=float, default=1e-7)
    ap.add_argument("--verbose", type=int, default=0, help="library diagnostics on stderr (2: H_eff psi shapes)")
    ap.add_argument("--hpsi-only", action="store_true",
                    help="time the H_eff psi contraction alone on synthetic sector blocks (kernel roofline)")
    ap.add_argument("--hpsi-shape", default="small", choices=["small", "large"],
                    help="--hpsi-only: sector dimensions 100-250 (small) or 300-600 (large)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.hpsi_only:
        return run_hpsi_only(args)

    import paper_2503_20700_gb300 as pkg
    pkg.load()
    rank, world, dist = dist_init(args.gpus)
    device = int(os.environ.get("LOCAL_RANK", "0"))
    prec = {"split": pkg.SPLIT_HPSI, "split-tc": pkg.SPLIT_HPSI_TC, "split-all-tc": pkg.SPLIT_ALL_TC,
            "split-all": pkg.SPLIT_TF32, "fp64": pkg.FP64}[args.precision]
    rc = {"bond": run_bond, "sweep": run_sweep, "casscf": run_casscf}[args.mode](args, pkg, prec, rank, world,
                                                                                 dist, device)
    if dist is not None:
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
