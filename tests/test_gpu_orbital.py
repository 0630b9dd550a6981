"""GPU parity of the orbital-ordering step (Sec. II "Numerical procedure")
against the oracle, through the C-ABI.

The device measurement pass evaluates the orbital invariants in float64 and
the library assembles the one- and two-orbital reduced density matrices; they
are compared element by element with the oracle's (dense Fock-space) ones: at
untruncated D against the exact (FCI) state, and at truncated D against the
oracle's own DMRG state after the same sweeps, to the RDM bar of 1e-7.  The
entropies, the mutual information and the Fiedler ordering follow."""
import numpy as np
import pytest

import workloads as W
from oracle import orbital as OB
from oracle.dmrg import OracleDMRG
from oracle.fci import fci

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2503_20700_gb300 as p
    p.load()
    return p


def oracle_rdms(states, psi, n, two_s):
    vecs = OB.multiplet(states, psi, n, two_s)
    r1 = np.array([OB.one_orbital_rdm(vecs, n, p) for p in range(n)])
    r2 = np.zeros((n, n, 16, 16))
    for p in range(n):
        for q in range(p + 1, n):
            r2[p, q] = OB.two_orbital_rdm(vecs, n, p, q)
    return r1, r2


@pytest.mark.parametrize("n,n_elec,two_s,seed", [(6, 6, 0, 3), (7, 7, 1, 5), (6, 6, 2, 1)])
def test_orbital_rdms_exact_at_full_bond_dimension(pkg, n, n_elec, two_s, seed):
    h, L = W.cholesky_random(n, 2 * n, seed=seed)
    eri = W.eri_from_cholesky(L)
    e, x, H = fci(h, eri, n_elec, two_s)
    g = pkg.DMRG(h, eri=eri, n_elec=n_elec, two_s=two_s, D=400, tol=1e-11)
    g.sweep(2)
    r1, r2 = g.orbital_rdms()
    s1, mi = g.orbital_entanglement()
    g.close()
    o1, o2 = oracle_rdms(H.ops.states, x, n, two_s)
    assert np.abs(r1 - o1).max() < 1e-8
    assert np.abs(r2 - o2).max() < 1e-8
    os1, omi = OB.orbital_entanglement(H.ops.states, x, n, two_s)
    assert np.abs(s1 - os1).max() < 1e-7
    assert np.abs(mi - omi).max() < 1e-7


def test_orbital_rdms_match_oracle_at_truncated_bond_dimension(pkg):
    h, L = W.cholesky_random(8, 32, seed=20250326)
    eri = W.eri_from_cholesky(L)
    o = OracleDMRG(h, eri, 8, 0, D=12)
    o.sweep(3)
    g = pkg.DMRG(h, eri=eri, n_elec=8, two_s=0, D=12, tol=1e-10)
    g.sweep(3)
    r1, r2 = g.orbital_rdms()
    s1, mi = g.orbital_entanglement()
    g.close()
    o1, o2 = oracle_rdms(o.states, o.psi_full, 8, 0)
    assert np.abs(r1 - o1).max() < 1e-7
    assert np.abs(r2 - o2).max() < 1e-7
    os1, omi = OB.orbital_entanglement(o.states, o.psi_full, 8, 0)
    assert np.abs(s1 - os1).max() < 1e-6
    assert np.abs(mi - omi).max() < 1e-6
    # the ordering from the device's mutual information, by the device's
    # Fiedler vector, is the oracle's
    assert list(pkg.fiedler_order(mi)) == list(OB.fiedler_order(omi))


def test_fiedler_order_of_a_shuffled_chain(pkg):
    rng = np.random.default_rng(7)
    for n in (2, 3, 9, 40):
        perm = rng.permutation(n)
        pos = np.argsort(perm)
        I = np.exp(-np.abs(pos[:, None] - pos[None, :]).astype(float))
        np.fill_diagonal(I, 0.0)
        order = pkg.fiedler_order(I)
        if n > 2:
            assert list(order) == list(OB.fiedler_order(I))
            assert list(order) in (list(perm), list(perm[::-1]))
    with pytest.raises(pkg.DmrgError):
        pkg.fiedler_order(np.array([[0.0, 1.0], [0.5, 0.0]]))


def test_ordering_step_recovers_a_shuffled_chain(pkg):
    """The ordering procedure on a Hubbard chain whose sites were shuffled:
    the order the device finds from a D=16 state is the oracle's from the
    same algorithm, and the reordered problem has a much lower energy at the
    same small D."""
    n = 8
    h, eri, _ = W.hubbard_chain(n, t=-1.0, u=4.0)
    perm = np.random.default_rng(3).permutation(n)
    hs, es, _ = pkg.permute_orbitals(perm, h, eri)
    order, s1, mi = pkg.order_orbitals(hs, eri=es, n_elec=n, two_s=0, D_steps=(16,), sweeps_per_step=2,
                                       tol=1e-10)
    o = OracleDMRG(hs, es, n, 0, D=16)
    o.sweep(2)
    os1, omi = OB.orbital_entanglement(o.states, o.psi_full, n, 0)
    assert np.abs(mi - omi).max() < 1e-6
    assert list(order) == list(OB.fiedler_order(omi))
    chain = perm[order]
    assert sum(abs(int(a) - int(b)) == 1 for a, b in zip(chain[:-1], chain[1:])) >= n - 2
    g1 = pkg.DMRG(hs, eri=es, n_elec=n, two_s=0, D=16, tol=1e-10)
    e_shuffled = g1.sweep(2)[0]
    g1.close()
    ho, eo, _ = pkg.permute_orbitals(order, hs, es)
    g2 = pkg.DMRG(ho, eri=eo, n_elec=n, two_s=0, D=16, tol=1e-10)
    e_ordered = g2.sweep(2)[0]
    g2.close()
    assert e_ordered < e_shuffled - 0.3


@pytest.mark.parametrize("n_elec,two_s", [(3, 1), (4, 0), (2, 2)])
def test_orbital_rdms_on_three_orbitals(pkg, n_elec, two_s):
    """The smallest chain the pass takes: its only bond is also the last, so
    the single-orbital values of all three sites and the pairs (0,1), (0,2),
    (1,2) are all measured there (x in L(1), s on site 1, y on site 2)."""
    n = 3
    h, L = W.cholesky_random(n, 6, seed=12)
    eri = W.eri_from_cholesky(L)
    e, x, H = fci(h, eri, n_elec, two_s)
    g = pkg.DMRG(h, eri=eri, n_elec=n_elec, two_s=two_s, D=64, tol=1e-12)
    g.sweep(2)
    r1, r2 = g.orbital_rdms()
    g.close()
    o1, o2 = oracle_rdms(H.ops.states, x, n, two_s)
    assert np.abs(r1 - o1).max() < 1e-8
    assert np.abs(r2 - o2).max() < 1e-8
