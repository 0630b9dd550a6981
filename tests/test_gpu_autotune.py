"""The autotuned batching of the tcgen05 H_eff psi launch (every sector block
of one product in one persistent launch, its schedule picked by timing).

Each candidate schedule (tile width, item chunks per CTA, task order) is
checked element by element against numpy on ragged sector blocks: the
schedule only moves work between CTAs and changes the FP32 summation order,
so every candidate must stay within the split tolerance and be bitwise
reproducible.  A DMRG run with autotuning on must still match the float64
oracle at the split-precision target, and a bond solve with enough products
must time every candidate and keep the fastest."""
import numpy as np
import pytest

import workloads as W
from oracle.dmrg import OracleDMRG
from test_gpu_dmrg import random_hpsi_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2503_20700_gb300 as p
    p.load()
    return p


EDGE_SHAPES = [
    (130, 257, [(1, 256), (15, 257), (16, 32), (17, 33), (300, 512), (33, 513)]),
    (7, 1, [(16, 16), (40, 17), (5, 255), (257, 1)]),
    (256, 300, [(64, 48), (129, 288), (31, 600), (2, 31)]),
    (1, 16, [(260, 270)]),
    (129, 129, [(130, 140), (8, 128)]),
]


def test_every_schedule_candidate_against_numpy(pkg):
    cands = pkg.tc_shape_candidates()
    problems = [random_hpsi_problem(np.random.default_rng(9), 4, 300, 300),
                random_hpsi_problem(np.random.default_rng(23), 0, 0, 0, shapes=EDGE_SHAPES)]
    try:
        for k, shape in enumerate(cands):
            pkg.set_kernel_tc_shape(k)
            for A, P, B, clen, blocks, items, refs in problems:
                C1 = np.zeros(clen)
                C2 = np.zeros(clen)
                pkg.ops.hpsi_contract(A, P, B, C1, blocks, items, precision=4)
                pkg.ops.hpsi_contract(A, P, B, C2, blocks, items, precision=4)
                assert np.array_equal(C1, C2), shape
                for off, m, n, ref in refs:
                    scale = np.abs(ref).max()
                    got = C1[off:off + m * n].reshape(m, n)
                    assert np.abs(got - ref).max() < 3e-5 * scale, (shape, m, n)
    finally:
        pkg.set_kernel_tc_shape(0)


def test_autotuned_sweeps_match_oracle(pkg):
    h, L = W.cholesky_random(8, 32, seed=20250326)
    eri = W.eri_from_cholesky(L)
    o = OracleDMRG(h, eri, 8, 0, D=16)
    eo = o.sweep(3)
    g = pkg.DMRG(h, eri=eri, n_elec=8, two_s=0, D=16, precision=pkg.SPLIT_HPSI_TC, tol=1e-10,
                 rq64_every_bond=True, tc_autotune=True)
    eg = [g.sweep()[0] for _ in range(3)]
    info = g.tc_schedule()
    g.close()
    assert abs(eg[-1] - eo[-1]) < 1e-6
    assert np.abs(np.array(eg) - np.array(eo)).max() < 1e-5
    assert info["shape"] in pkg.tc_shape_candidates()
    assert any(t >= 0 for t in info["ms"])


def test_bond_solve_times_every_candidate_and_keeps_the_fastest(pkg):
    h, L = W.cholesky_random(12, 48, seed=3)
    occ, path = W.aufbau_state(h, 12, 0)
    g = pkg.DMRG(h, chol=L, n_elec=12, two_s=0, D=64, precision=pkg.SPLIT_HPSI_TC, tol=1e-8,
                 occ=occ, two_s_right=path)
    g.sweep(2)
    info0 = g.tc_schedule()
    assert info0["shape"] == pkg.tc_shape_candidates()[0]  # autotuning off: the default
    assert all(t < 0 for t in info0["ms"])
    n, mid = 12, 5
    g.sweep_part(0, n - 3)
    g.sweep_part(1, mid + 1)
    g.set_tc_autotune(True)
    cands = pkg.tc_shape_candidates()
    # the candidates are timed on the first products of the (converging) solve
    r = g.bond_solve(mid, 1, pkg.SPLIT_HPSI_TC, max_iter=80, tol=1e-7, min_calls=len(cands) + 2,
                     check64=True)
    info = g.tc_schedule()
    g.close()
    assert len(info["ms"]) == len(cands) and all(t > 0 for t in info["ms"])
    assert info["shape"] == cands[int(np.argmin(info["ms"]))]
    assert r["residual64"] < 1e-3
    # the split Davidson eigenvalue is first order in the products' rounding
    assert abs(r["energy"] - r["energy_rq64"]) < 1e-5 * abs(r["energy"])
