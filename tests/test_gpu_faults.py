"""Failure detection in the allowed forms: every error comes back as a status
code and leaves the context usable.

* DMRG_ENOCONV: a Davidson cap of one iteration with a tolerance no bond can
  reach, with strict_convergence on; the sweep completes first.
* DMRG_ENOMEM: a device-memory budget the context cannot stay under.
* DMRG_ETIMEOUT: a wait bound of 0 on the device waits (a wait not complete
  at its first probe gives up; the kernel sets its error flag, waits for its
  own copies, frees its tensor memory and returns), in the tcgen05 H_eff psi
  kernel's mbarrier waits and in the group barrier of the cooperative
  eigensolver; with the bound restored the same calls succeed.
No test faults, traps or hangs the GPU.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2503_20700_gb300 as p
    p.load()
    return p


def _small():
    h, L = W.cholesky_random(8, 32, seed=3)
    return h, W.eri_from_cholesky(L)


def test_strict_convergence_returns_enoconv_after_the_sweep(pkg):
    h, eri = _small()
    g = pkg.DMRG(h, eri=eri, n_elec=8, D=12, max_iter=1, tol=1e-14, strict_convergence=True)
    with pytest.raises(pkg.DmrgError) as ei:
        g.sweep(1)
    assert ei.value.status == pkg.DMRG_ENOCONV
    e_capped = g.energy()                    # the sweep completed: its energy is there
    assert np.isfinite(e_capped)
    g.set_davidson(200, 1e-10)
    e, _ = g.sweep(1)                        # the context is still usable
    assert e <= e_capped + 1e-9
    g.close()


def test_budget_returns_enomem_and_frees(pkg):
    h, eri = _small()
    g = pkg.DMRG(h, eri=eri, n_elec=8, D=16)
    g.close()
    with pytest.raises(pkg.DmrgError) as ei:
        g2 = pkg.DMRG(h, eri=eri, n_elec=8, D=16, hbm_budget_bytes=64 * 1024)
        g2.sweep(1)
    assert ei.value.status == pkg.DMRG_ENOMEM
    # a budget that fits runs normally
    g3 = pkg.DMRG(h, eri=eri, n_elec=8, D=16, hbm_budget_bytes=2 << 30)
    g3.sweep(1)
    g3.close()


def test_zero_wait_bound_times_out_tcgen05_kernel_and_context_recovers(pkg):
    h, eri = _small()
    g = pkg.DMRG(h, eri=eri, n_elec=8, D=12, precision=pkg.SPLIT_HPSI_TC, wait_timeout_s=0.0)
    with pytest.raises(pkg.DmrgError) as ei:
        g.sweep(1)
    assert ei.value.status == pkg.DMRG_ETIMEOUT
    g.set_wait_timeout(2.0)
    e1, _ = g.sweep(1)
    e2, _ = g.sweep(1)
    assert np.isfinite(e1) and e2 <= e1 + 1e-6
    g.close()


def test_zero_wait_bound_times_out_eigensolver_group_barrier(pkg):
    """Matrices above the shared-memory size run on CTA groups that meet at a
    bounded group barrier every rotation round."""
    rng = np.random.default_rng(4)
    mats = []
    for n in (300, 260, 240):
        x = rng.standard_normal((n, n))
        mats.append(x + x.T)
    try:
        pkg.set_kernel_wait_timeout(0.0)
        with pytest.raises(pkg.DmrgError) as ei:
            pkg.ops.eigh_batched(mats)
        assert ei.value.status == pkg.DMRG_ETIMEOUT
    finally:
        pkg.set_kernel_wait_timeout(2.0)
    res = pkg.ops.eigh_batched(mats)
    for M, (w, V) in zip(mats, res):
        assert np.abs(w - np.sort(np.linalg.eigvalsh(M))[::-1]).max() < 1e-10 * np.abs(w).max()


def test_zero_wait_bound_times_out_kernel_level_contraction(pkg):
    rng = np.random.default_rng(8)
    m = n = 200
    ka = kb = 96
    A = rng.standard_normal(m * ka)
    P = rng.standard_normal(ka * kb)
    B = rng.standard_normal(n * kb)
    blocks = [(0, m, n, n, 0, 3)]
    items = [(0, 0, 0, ka, kb, kb, 0, 0, ka, kb, 0, 0, 0.5)] * 3
    try:
        pkg.set_kernel_wait_timeout(0.0)
        C = np.zeros(m * n)
        with pytest.raises(pkg.DmrgError) as ei:
            pkg.ops.hpsi_contract(A, P, B, C, blocks, items, precision=4)
        assert ei.value.status == pkg.DMRG_ETIMEOUT
    finally:
        pkg.set_kernel_wait_timeout(2.0)
    C = np.zeros(m * n)
    pkg.ops.hpsi_contract(A, P, B, C, blocks, items, precision=4)
    ref = 1.5 * A.reshape(m, ka) @ P.reshape(ka, kb) @ B.reshape(n, kb).T
    assert np.abs(C.reshape(m, n) - ref).max() < 3e-5 * np.abs(ref).max()


def test_debug_bounds_checks_plans_without_changing_results(pkg):
    h, eri = _small()
    a = pkg.DMRG(h, eri=eri, n_elec=8, D=12, precision=pkg.SPLIT_HPSI_TC)
    b = pkg.DMRG(h, eri=eri, n_elec=8, D=12, precision=pkg.SPLIT_HPSI_TC, debug_bounds=True)
    ea = [a.sweep()[0] for _ in range(2)]
    eb = [b.sweep()[0] for _ in range(2)]
    a.close()
    b.close()
    assert ea == eb


def test_budget_stages_blocks_to_pinned_host_memory_bit_identically(pkg):
    """A device budget below what the stored blocks of a sweep need (PPP
    octacene, 34 sites, D=64): stored blocks go to pinned host memory on the
    side stream and come back ahead of their bond; the energies are
    bit-identical to the unbudgeted run."""
    h, eri, ec = W.ppp_acene(8)
    ref = pkg.DMRG(h, eri=eri, n_elec=34, D=64, e_core=ec)
    e_ref = [ref.sweep()[0] for _ in range(2)]
    md = ref.memory_detail()
    _, peak = ref.memory()
    ref.close()
    # room for a bond's working memory, the MPS tensors and three quarters of
    # the right blocks a sweep ends with: in the middle of a sweep the left
    # blocks built so far come on top, so blocks have to be staged out
    stored = md["stored_device"] + md["stored_host"]
    assert stored > 6 * md["max_block"]
    budget = md["max_bond_extra"] + md["mps"] + int(0.75 * stored) + (8 << 20)
    g = pkg.DMRG(h, eri=eri, n_elec=34, D=64, e_core=ec, hbm_budget_bytes=budget)
    e = [g.sweep()[0] for _ in range(2)]
    st = g.memory_detail()
    _, peak_b = g.memory()
    g.close()
    assert e == e_ref
    assert st["staged_out"] > 0 and st["staged_in"] > 0
    assert peak_b <= budget
