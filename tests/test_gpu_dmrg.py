"""GPU parity: the CUDA path (through the C-ABI) against the CPU oracle.

Tolerances: float64 path 1e-8 Eh per sweep energy (the requirement for the
FP64 GPU path); split-FP32 (3xTF32) path 1e-6 Eh against the float64 path.
"""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle.dmrg import OracleDMRG
from oracle.fci import fci

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def pkg():
    import paper_2503_20700_gb300 as p
    p.load()
    return p


def _case(name):
    if name == "hub6":
        h, eri, ec = W.hubbard_chain(6, u=4.0)
        return h, eri, ec, 6, 0, 8, 3
    if name == "benzene_ppp":
        h, eri, ec = W.ppp_acene(1)
        return h, eri, ec, 6, 0, 10, 3
    if name == "rand6_s0":
        h, L = W.cholesky_random(6, 12, seed=1)
        return h, W.eri_from_cholesky(L), 0.0, 6, 0, 8, 3
    if name == "rand6_s2":
        h, L = W.cholesky_random(6, 12, seed=1)
        return h, W.eri_from_cholesky(L), 0.0, 6, 2, 8, 3
    if name == "rand7_s1":
        h, L = W.cholesky_random(7, 14, seed=3)
        return h, W.eri_from_cholesky(L), 0.0, 7, 1, 12, 3
    if name == "rand8_n6":
        h, L = W.cholesky_random(8, 16, seed=2)
        return h, W.eri_from_cholesky(L), 0.0, 6, 0, 10, 2
    if name == "rand8_n10":
        h, L = W.cholesky_random(8, 16, seed=2)
        return h, W.eri_from_cholesky(L), 0.0, 10, 0, 10, 2
    raise KeyError(name)


@pytest.mark.parametrize("name", ["hub6", "benzene_ppp", "rand6_s0", "rand6_s2", "rand7_s1",
                                  "rand8_n6", "rand8_n10"])
def test_sweep_energies_match_oracle(pkg, name):
    h, eri, ec, N, S, D, sw = _case(name)
    g = pkg.DMRG(h, eri=eri, n_elec=N, two_s=S, D=D, e_core=ec)
    eg = [g.sweep()[0] for _ in range(sw)]
    bg = g.bond_energies()
    o = OracleDMRG(h, eri, N, S, D=D, e_core=ec)
    eo = o.sweep(sw)
    bo = np.array([b[3] for b in o.record.bond_energies])
    assert np.abs(np.array(eg) - np.array(eo)).max() < 1e-8
    assert len(bg) == len(bo)
    assert np.abs(bg - bo).max() < 1e-8


def test_exact_at_full_bond_dimension(pkg):
    h, L = W.cholesky_random(6, 12, seed=1)
    eri = W.eri_from_cholesky(L)
    e_fci, _, _ = fci(h, eri, 6, 0)
    g = pkg.DMRG(h, eri=eri, n_elec=6, two_s=0, D=500)
    e = [g.sweep()[0] for _ in range(3)]
    assert e[-1] == pytest.approx(e_fci, abs=1e-9)


def test_cholesky_input_equals_eri_input(pkg):
    h, L = W.cholesky_random(6, 12, seed=4)
    eri = W.eri_from_cholesky(L)
    e1 = pkg.DMRG(h, eri=eri, n_elec=6, D=8).sweep(2)[0]
    e2 = pkg.DMRG(h, chol=L, n_elec=6, D=8).sweep(2)[0]
    assert e1 == pytest.approx(e2, abs=1e-11)


def test_naphthalene_d64_against_oracle_and_fci(pkg):
    """PPP naphthalene, D=64, 4 sweeps (the plain FP64 workload)."""
    path = os.path.join(GOLD, "naphthalene_ppp_d64.json")
    if not os.path.exists(path):
        pytest.skip("golden file missing")
    gold = json.load(open(path))
    h, eri, ec = W.ppp_acene(2)
    g = pkg.DMRG(h, eri=eri, n_elec=10, two_s=0, D=64, e_core=ec)
    eg = [g.sweep()[0] for _ in range(4)]
    assert np.abs(np.array(eg) - np.array(gold["e_dmrg_sweeps"])).max() < 1e-8
    assert eg[-1] >= gold["e_fci"] - 1e-10          # variational bound
    assert eg[-1] - gold["e_fci"] < 1e-3            # D=64 is close to FCI here


@pytest.mark.parametrize("prec,tol", [("SPLIT_HPSI", 1e-6), ("SPLIT_HPSI_TC", 1e-6), ("SPLIT_TF32", 3e-5)])
def test_split_precision_sweep_energy(pkg, prec, tol):
    """Sweep energy of the split (3xTF32) paths against the float64 path.  The
    sweep energy is the float64 Rayleigh quotient of the split-converged
    eigenvector, so with float64 renormalisation the difference is second
    order (<= 1e-6 Eh); with split renormalisation (SPLIT_TF32) the operators
    themselves carry the ~1e-7 relative rounding and the bound is first order."""
    h, L = W.cholesky_random(8, 16, seed=2)
    eri = W.eri_from_cholesky(L)
    e64 = pkg.DMRG(h, eri=eri, n_elec=8, D=16).sweep(3)[0]
    e32 = pkg.DMRG(h, eri=eri, n_elec=8, D=16, precision=getattr(pkg, prec)).sweep(3)[0]
    assert abs(e32 - e64) < tol


@pytest.mark.parametrize("prec", ["SPLIT_HPSI", "SPLIT_HPSI_TC"])
def test_split_sweep_drift_from_same_state(pkg, prec):
    """One sweep in split precision against the same sweep in float64, both
    from the same converged float64 state (identical history in two
    contexts): the energy drift is within 1e-6 Eh."""
    h, L = W.cholesky_random(16, 64, seed=20250326)
    out = []
    for p in (pkg.FP64, getattr(pkg, prec)):
        g = pkg.DMRG(h, chol=L, n_elec=16, D=64, precision=pkg.FP64)
        for d in (16, 32, 64):
            g.set_bond_dim(d)
            g.sweep(1)
        g.set_precision(p)
        out.append(g.sweep(1)[0])
        g.close()
    assert abs(out[1] - out[0]) < 1e-6


def test_bad_arguments_return_einval(pkg):
    h = np.zeros((4, 4))
    eri = np.zeros((4, 4, 4, 4))
    with pytest.raises(pkg.DmrgError) as ei:
        pkg.DMRG(h, eri=eri, n_elec=4, two_s=1)
    assert ei.value.status == pkg.DMRG_EINVAL
    with pytest.raises(pkg.DmrgError) as ei:
        pkg.DMRG(h, eri=eri, n_elec=9)
    assert ei.value.status == pkg.DMRG_EINVAL


# ---------------------------------------------------------------- kernels
def _random_groups(rng, n_groups, max_dim, max_k, max_segs):
    A_parts, B_parts, groups, segs, refs = [], [], [], [], []
    a_off = b_off = c_off = 0
    C_len = 0
    for g in range(n_groups):
        m = int(rng.integers(1, max_dim))
        n = int(rng.integers(1, max_dim))
        ns = int(rng.integers(1, max_segs + 1))
        ref = np.zeros((m, n))
        sb = len(segs)
        for _ in range(ns):
            k = int(rng.integers(1, max_k))
            ta, tb = int(rng.integers(0, 2)), int(rng.integers(0, 2))
            a = rng.standard_normal((k, m) if ta else (m, k))
            b = rng.standard_normal((n, k) if tb else (k, n))
            alpha = float(rng.standard_normal())
            ref += alpha * (a.T if ta else a) @ (b.T if tb else b)
            segs.append((a_off, b_off, k, a.shape[1], b.shape[1], ta, tb, alpha))
            A_parts.append(a.ravel())
            B_parts.append(b.ravel())
            a_off += a.size
            b_off += b.size
        groups.append((c_off, m, n, n, sb, ns))
        refs.append((c_off, m, n, ref))
        c_off += m * n
    return (np.concatenate(A_parts), np.concatenate(B_parts), c_off, groups, segs, refs)


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-6)])
def test_grouped_gemm_against_numpy(pkg, prec, tol):
    rng = np.random.default_rng(7)
    # ragged sizes spanning several 64x64 tiles with tails
    A, B, clen, groups, segs, refs = _random_groups(rng, 24, 200, 300, 4)
    C0 = rng.standard_normal(clen)
    C = C0.copy()
    pkg.ops.grouped_gemm(A, B, C, groups, segs, precision=prec)
    for off, m, n, ref in refs:
        got = C[off:off + m * n].reshape(m, n) - C0[off:off + m * n].reshape(m, n)
        scale = np.abs(ref).max() + 1e-300
        assert np.abs(got - ref).max() <= tol * scale * 10


def test_grouped_gemm_rejects_out_of_range(pkg):
    A = np.zeros(10)
    B = np.zeros(10)
    C = np.zeros(10)
    with pytest.raises(pkg.DmrgError):
        pkg.ops.grouped_gemm(A, B, C, [(0, 4, 4, 4, 0, 1)], [(0, 0, 4, 4, 4, 0, 0, 1.0)])


def test_eigh_against_numpy(pkg):
    rng = np.random.default_rng(3)
    mats = []
    for n in (1, 2, 5, 17, 64, 150):
        x = rng.standard_normal((n, n))
        mats.append(x + x.T)
    res = pkg.ops.eigh_batched(mats)
    for M, (w, V) in zip(mats, res):
        ref = np.sort(np.linalg.eigvalsh(M))[::-1]
        assert np.abs(w - ref).max() < 1e-11 * max(1.0, np.abs(ref).max())
        assert np.abs(V @ M - w[:, None] * V).max() < 1e-10 * max(1.0, np.abs(ref).max())
        assert np.abs(V @ V.T - np.eye(len(w))).max() < 1e-12


def test_eigh_cooperative_groups_density_matrices(pkg):
    """Matrices above 112 go to the cooperative multi-CTA Jacobi: a batch of
    density-matrix-like (PSD, rank-deficient, fast-decaying) and indefinite
    matrices of several sizes, with small ones mixed in."""
    rng = np.random.default_rng(8)
    mats = []
    for n in (97, 130, 257, 40, 400, 3):
        x = rng.standard_normal((n, max(1, n // 2))) * np.exp(-np.arange(max(1, n // 2)) / 8.0)
        mats.append(x @ x.T)
    y = rng.standard_normal((211, 211))
    mats.append(y + y.T)
    res = pkg.ops.eigh_batched(mats)
    for M, (w, V) in zip(mats, res):
        ref = np.sort(np.linalg.eigvalsh(M))[::-1]
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(w - ref).max() < 1e-11 * scale
        assert np.abs(V @ M - w[:, None] * V).max() < 1e-10 * scale
        assert np.abs(V @ V.T - np.eye(len(w))).max() < 1e-11


def test_eigh_batches_larger_than_one_launch(pkg):
    """More matrices than one CTA per SM: several cooperative launches, group
    sizes from the cost model (mid-size matrices split over CTA groups, small
    ones on one CTA), density-matrix-like and indefinite, sizes 1..160."""
    rng = np.random.default_rng(12)
    mats = []
    for k in range(190):
        n = int(rng.integers(1, 161))
        if k % 3:
            x = rng.standard_normal((n, max(1, n // 3))) * np.exp(-np.arange(max(1, n // 3)) / 6.0)
            mats.append(x @ x.T)
        else:
            y = rng.standard_normal((n, n))
            mats.append(y + y.T)
    res = pkg.ops.eigh_batched(mats)
    for M, (w, V) in zip(mats, res):
        ref = np.sort(np.linalg.eigvalsh(M))[::-1]
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(w - ref).max() < 1e-11 * scale
        assert np.abs(V @ M - w[:, None] * V).max() < 1e-10 * scale
        assert np.abs(V @ V.T - np.eye(len(w))).max() < 1e-11


def random_hpsi_problem(rng, n_blocks, max_dim, max_items, big=False, shapes=None):
    """Sector-block contraction sigma += alpha op(A) P op(B)^T with ragged
    sizes (several tiles and tails), both transposes, identities.  With
    `shapes` = [(m, n, [(ka, kb), ...]), ...] the block and item sizes are
    the given ones (no identities)."""
    A_parts, P_parts, B_parts = [], [], []
    ao = po = bo = co = 0
    blocks, items, refs = [], [], []
    if shapes is not None:
        n_blocks = len(shapes)
    for bi in range(n_blocks):
        if shapes is not None:
            m, n, kk = shapes[bi]
        else:
            m = int(rng.integers(1, max_dim))
            n = int(rng.integers(1, max_dim))
            kk = [None] * int(rng.integers(1, max_items + 1))
        ib = len(items)
        ref = np.zeros((m, n))
        for kab in kk:
            if kab is not None:
                a_id = b_id = 0
                ka, kb = kab
            else:
                a_id = int(rng.random() < 0.15)
                b_id = int(rng.random() < 0.15) if not a_id else 0
                ka = m if a_id else int(rng.integers(1, max_dim))
                kb = n if b_id else int(rng.integers(1, max_dim))
            ta, tb = int(rng.integers(0, 2)), int(rng.integers(0, 2))
            alpha = float(rng.standard_normal())
            Pm = rng.standard_normal((ka, kb))
            if a_id:
                Am = np.eye(m)
                a_entry = (0, 1, 0)
            else:
                a = rng.standard_normal((ka, m) if ta else (m, ka))
                Am = a.T if ta else a
                a_entry = (ao, a.shape[1], ta)
                A_parts.append(a.ravel())
                ao += a.size
            if b_id:
                Bt = np.eye(n)
                b_entry = (0, 1, 0)
            else:
                b = rng.standard_normal((kb, n) if tb else (n, kb))
                Bt = b if tb else b.T          # op(B)^T, kb x n
                b_entry = (bo, b.shape[1], tb)
                B_parts.append(b.ravel())
                bo += b.size
            ref += alpha * Am @ Pm @ Bt
            items.append((a_entry[0], po, b_entry[0], a_entry[1], kb, b_entry[1], a_entry[2],
                          b_entry[2], ka, kb, a_id, b_id, alpha))
            P_parts.append(Pm.ravel())
            po += Pm.size
        blocks.append((co, m, n, n, ib, len(items) - ib))
        refs.append((co, m, n, ref))
        co += m * n
    cat = lambda v: np.concatenate(v) if v else np.zeros(1)
    return cat(A_parts), cat(P_parts), cat(B_parts), co, blocks, items, refs


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 3e-6), (4, 3e-6)])
def test_fused_hpsi_against_numpy(pkg, prec, tol):
    rng = np.random.default_rng(11)
    A, P, B, clen, blocks, items, refs = random_hpsi_problem(rng, 12, 150, 6)
    C0 = rng.standard_normal(clen)
    C = C0.copy()
    pkg.ops.hpsi_contract(A, P, B, C, blocks, items, precision=prec)
    for off, m, n, ref in refs:
        got = (C - C0)[off:off + m * n].reshape(m, n)
        assert np.abs(got - ref).max() <= tol * (np.abs(ref).max() + 1e-300) * 10


def test_fused_hpsi_many_items_split_into_chunks(pkg):
    """Blocks with hundreds of items: the launch splits them into chunks whose
    partial tiles are reduced in a fixed order; results are bitwise
    reproducible between two launches."""
    rng = np.random.default_rng(5)
    A, P, B, clen, blocks, items, refs = random_hpsi_problem(rng, 3, 70, 400)
    C1 = np.zeros(clen)
    C2 = np.zeros(clen)
    pkg.ops.hpsi_contract(A, P, B, C1, blocks, items, precision=0)
    pkg.ops.hpsi_contract(A, P, B, C2, blocks, items, precision=0)
    assert np.array_equal(C1, C2)
    for off, m, n, ref in refs:
        assert np.abs(C1[off:off + m * n].reshape(m, n) - ref).max() < 1e-11 * np.abs(ref).max()


def test_fused_hpsi_tcgen05_chunks_and_tails(pkg):
    """tcgen05 kernel (128 x 256 sigma tiles): blocks spanning several row and
    column tiles with ragged tails, hundreds of items split into chunks;
    bitwise reproducible, and equal to the mma.sync kernel within the split
    tolerance."""
    rng = np.random.default_rng(9)
    A, P, B, clen, blocks, items, refs = random_hpsi_problem(rng, 4, 300, 300)
    C1 = np.zeros(clen)
    C2 = np.zeros(clen)
    C3 = np.zeros(clen)
    pkg.ops.hpsi_contract(A, P, B, C1, blocks, items, precision=4)
    pkg.ops.hpsi_contract(A, P, B, C2, blocks, items, precision=4)
    pkg.ops.hpsi_contract(A, P, B, C3, blocks, items, precision=1)
    assert np.array_equal(C1, C2)
    for off, m, n, ref in refs:
        scale = np.abs(ref).max()
        got = C1[off:off + m * n].reshape(m, n)
        assert np.abs(got - ref).max() < 3e-5 * scale
        assert np.abs(got - C3[off:off + m * n].reshape(m, n)).max() < 3e-5 * scale


@pytest.mark.parametrize("drain", [0, 1024])
def test_fused_hpsi_tcgen05_super_chunk_edges(pkg, drain):
    """tcgen05 kernel at the edges of its blocking: inner dimensions of psi
    (kb) at and around the 256-column stage-1 width, the 32-column pieces and
    the 16-deep k-blocks; ka of 1, 15, 16, 17 and more than 256; sigma tiles
    of one column and of 256 plus a tail; drains after every item and after
    1024 terms.  Bitwise reproducible, within the split tolerance of numpy."""
    rng = np.random.default_rng(23)
    shapes = [
        (130, 257, [(1, 256), (15, 257), (16, 32), (17, 33), (300, 512), (33, 513)]),
        (7, 1, [(16, 16), (40, 17), (5, 255), (257, 1)]),
        (256, 300, [(64, 48), (129, 288), (31, 600), (2, 31)]),
        (1, 16, [(260, 270)]),
    ]
    A, P, B, clen, blocks, items, refs = random_hpsi_problem(rng, 0, 0, 0, shapes=shapes)
    pkg.set_kernel_tc_drain_terms(drain)
    try:
        C1 = np.zeros(clen)
        C2 = np.zeros(clen)
        pkg.ops.hpsi_contract(A, P, B, C1, blocks, items, precision=4)
        pkg.ops.hpsi_contract(A, P, B, C2, blocks, items, precision=4)
    finally:
        pkg.set_kernel_tc_drain_terms(1024)
    assert np.array_equal(C1, C2)
    for off, m, n, ref in refs:
        scale = np.abs(ref).max()
        got = C1[off:off + m * n].reshape(m, n)
        assert np.abs(got - ref).max() < 3e-5 * scale


def test_heff_at_a_bond_is_symmetric_and_linear(pkg):
    """The device H_eff at a bond, applied to chosen vectors (dmrg_bond_apply):
    <x|H y> = <H x|y> and H(2x - 3y) = 2Hx - 3Hy in float64 to 1e-12
    relative (the reduced multiplet basis is orthonormal, so H_eff is
    symmetric); the split tcgen05 product on the same vector agrees with
    float64 within the split tolerance; wrong lengths are rejected."""
    n, mid = 10, 4
    h, L = W.cholesky_random(n, 40, seed=4)
    occ, path = W.aufbau_state(h, n, 0)
    g = pkg.DMRG(h, chol=L, n_elec=n, two_s=0, D=48, tol=1e-8, occ=occ, two_s_right=path)
    g.sweep(1)
    g.sweep_part(0, n - 3)
    g.sweep_part(1, mid + 1)
    r = g.bond_solve(mid, 1, pkg.FP64, max_iter=30, tol=1e-8, min_calls=0, check64=False)
    dim = g.bond_apply(None)
    assert dim == r["dim"] and dim > 100
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal(dim), rng.standard_normal(dim)
    Hx, Hy = g.bond_apply(x), g.bond_apply(y)
    assert abs(x @ Hy - Hx @ y) < 1e-12 * np.linalg.norm(Hx) * np.linalg.norm(y)
    H2 = g.bond_apply(2.0 * x - 3.0 * y)
    assert np.abs(H2 - (2.0 * Hx - 3.0 * Hy)).max() < 1e-12 * np.abs(H2).max()
    Tx = g.bond_apply(x, pkg.SPLIT_HPSI_TC)
    assert np.abs(Tx - Hx).max() < 3e-5 * np.abs(Hx).max()
    with pytest.raises(pkg.DmrgError) as ei:
        g.bond_apply(np.zeros(dim + 1))
    assert ei.value.status == pkg.DMRG_EINVAL
    g.close()
