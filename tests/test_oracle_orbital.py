"""Pins of the oracle's orbital entanglement and Fiedler ordering (CPU).

The one- and two-orbital reduced density matrices are checked against facts
fixed independently of their construction:
  * a product state (one determinant of site orbitals) has no entanglement;
  * the Hubbard dimer has closed-form one-orbital weights, and its two-orbital
    state is pure, so I_12 = 2 s_1;
  * rho_pq reproduces the spin-free 1- and 2-RDM elements of the same state
    (oracle.rdm, pinned against FCI elsewhere) through operators written here
    on a separate 4-mode Jordan-Wigner space: hopping, density-density,
    pair transfer and exchange (spin-flip) elements;
  * traces, marginals, positivity, spin symmetry of the averaged multiplet,
    subadditivity and the Araki-Lieb bound I_pq <= 2 min(s_p, s_q);
  * the Fiedler order of a chain's mutual information, shuffled, is the chain.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import orbital as OB
from oracle.dmrg import OracleDMRG
from oracle.fci import fci
from oracle.rdm import rdm12


def four_modes():
    """16 x 16 matrices of a+ for the modes (p up, p dn, q up, q dn) on the
    local states a = 4 d_p + d_q, d = 2 n_up + n_dn, with the creators of
    |a> applied in that mode order."""
    def occ(a):
        dp, dq = divmod(a, 4)
        return [dp >> 1, dp & 1, dq >> 1, dq & 1]

    def index(o):
        return 4 * (2 * o[0] + o[1]) + (2 * o[2] + o[3])

    cr = []
    for m in range(4):
        M = np.zeros((16, 16))
        for a in range(16):
            o = occ(a)
            if o[m]:
                continue
            sign = (-1) ** sum(o[:m])
            o2 = list(o)
            o2[m] = 1
            M[index(o2), a] = sign
        cr.append(M)
    return cr


def expect(rho, X):
    return float(np.trace(rho @ X))


def test_product_state_has_no_entanglement():
    n = 5
    occ = [2, 1, 0, 2, 1]  # digits: updn, dn, empty, updn, dn
    idx = sum(d * 4 ** (n - 1 - p) for p, d in enumerate([3, 1, 0, 3, 1]))
    vecs = [OB.full_vector([idx], [1.0], n)]
    for p in range(n):
        assert OB.entropy(OB.one_orbital_rdm(vecs, n, p)) == pytest.approx(0.0, abs=1e-14)
        for q in range(p + 1, n):
            assert OB.entropy(OB.two_orbital_rdm(vecs, n, p, q)) == pytest.approx(0.0, abs=1e-12)
    assert sum(occ) == 6


@pytest.mark.parametrize("u", [0.5, 4.0, 10.0])
def test_hubbard_dimer_closed_form(u):
    h, eri, _ = W.hubbard_chain(2, t=-1.0, u=u)
    e, x, H = fci(h, eri, 2, 0)
    # covalent (a) and ionic (b) weights of the singlet ground state:
    # H = [[0, -2t], [-2t, U]] on the two singlets, t = 1
    b2 = 1.0 / (1.0 + (2.0 / e) ** 2)  # b/a = -e / (2t)
    a2 = 1.0 - b2
    vecs = OB.multiplet(H.ops.states, x, 2, 0)
    r1 = OB.one_orbital_rdm(vecs, 2, 0)
    assert np.allclose(r1, [b2 / 2, a2 / 2, a2 / 2, b2 / 2], atol=1e-10)
    s1 = -(b2 * math.log(b2 / 2) + a2 * math.log(a2 / 2))
    s, I = OB.orbital_entanglement(H.ops.states, x, 2, 0)
    assert s == pytest.approx([s1, s1], abs=1e-9)
    assert I[0, 1] == pytest.approx(2 * s1, abs=1e-9)  # the two orbitals are the whole (pure) state


def _random_state(n, n_elec, two_s, seed):
    h, L = W.cholesky_random(n, 2 * n, seed=seed)
    eri = W.eri_from_cholesky(L)
    e, x, H = fci(h, eri, n_elec, two_s)
    return h, eri, x, H


@pytest.mark.parametrize("n_elec,two_s", [(6, 0), (5, 1)])
def test_two_orbital_rdm_reproduces_spin_free_rdms(n_elec, two_s):
    n = 6
    h, eri, x, H = _random_state(n, n_elec, two_s, seed=11)
    gamma, Gamma = rdm12(H.ops, x / np.linalg.norm(x))
    vecs = OB.multiplet(H.ops.states, x, n, two_s)
    cr = four_modes()
    an = [M.T for M in cr]
    up_p, dn_p, up_q, dn_q = 0, 1, 2, 3
    hop = cr[up_p] @ an[up_q] + cr[dn_p] @ an[dn_q]
    num_p = cr[up_p] @ an[up_p] + cr[dn_p] @ an[dn_p]
    num_q = cr[up_q] @ an[up_q] + cr[dn_q] @ an[dn_q]
    P_, Q_ = (up_p, dn_p), (up_q, dn_q)
    # Gamma~_pqrs = sum_{s,t} <a+_{p s} a+_{q t} a_{r t} a_{s s}> for orbitals (p, q, r, s) in {P, Q}
    def g2(o1, o2, o3, o4):
        X = np.zeros((16, 16))
        for s in range(2):
            for t in range(2):
                X += cr[o1[s]] @ cr[o2[t]] @ an[o3[t]] @ an[o4[s]]
        return X
    for p in range(n):
        r1 = OB.one_orbital_rdm(vecs, n, p)
        assert r1.sum() == pytest.approx(1.0, abs=1e-12)
        assert r1[1] == pytest.approx(r1[2], abs=1e-12)  # up and dn alike in the averaged multiplet
        assert r1[1] + r1[2] + 2 * r1[3] == pytest.approx(gamma[p, p], abs=1e-10)
        assert r1[3] == pytest.approx(Gamma[p, p, p, p] / 2, abs=1e-10)
        for q in range(p + 1, n):
            rho = OB.two_orbital_rdm(vecs, n, p, q)
            assert np.allclose(rho, rho.T, atol=1e-13)
            assert np.linalg.eigvalsh(rho).min() > -1e-12
            assert np.trace(rho) == pytest.approx(1.0, abs=1e-12)
            R = rho.reshape(4, 4, 4, 4)
            assert np.allclose(np.einsum("acbc->ab", R), np.diag(r1), atol=1e-12)
            assert np.allclose(np.einsum("cacb->ab", R), np.diag(OB.one_orbital_rdm(vecs, n, q)), atol=1e-12)
            assert expect(rho, hop) == pytest.approx(gamma[p, q], abs=1e-10)
            assert expect(rho, num_p @ num_q) == pytest.approx(Gamma[p, q, q, p], abs=1e-10)
            assert expect(rho, g2(P_, P_, Q_, Q_)) == pytest.approx(Gamma[p, p, q, q], abs=1e-10)
            assert expect(rho, g2(P_, Q_, P_, Q_)) == pytest.approx(Gamma[p, q, p, q], abs=1e-10)
            assert expect(rho, g2(P_, P_, P_, Q_)) == pytest.approx(Gamma[p, p, p, q], abs=1e-10)
            assert expect(rho, g2(P_, Q_, Q_, Q_)) == pytest.approx(Gamma[p, q, q, q], abs=1e-10)


def test_mutual_information_bounds_and_symmetry():
    n = 6
    h, eri, x, H = _random_state(n, 6, 0, seed=4)
    s, I = OB.orbital_entanglement(H.ops.states, x, n, 0)
    assert np.allclose(I, I.T) and np.all(np.diag(I) == 0)
    assert np.all(s >= -1e-14) and np.all(s <= math.log(4) + 1e-12)
    for p in range(n):
        for q in range(p + 1, n):
            assert I[p, q] >= -1e-12                          # subadditivity
            assert I[p, q] <= 2 * min(s[p], s[q]) + 1e-12     # Araki-Lieb
    assert I.max() > 1e-3


def test_fiedler_order_recovers_a_shuffled_chain():
    rng = np.random.default_rng(2)
    for n in (5, 8, 12):
        perm = rng.permutation(n)            # orbital perm[k] sits at chain position k
        pos = np.argsort(perm)
        I = np.exp(-np.abs(pos[:, None] - pos[None, :]).astype(float))
        np.fill_diagonal(I, 0.0)
        order = OB.fiedler_order(I)
        assert sorted(order) == list(range(n))
        assert list(order) in (list(perm), list(perm[::-1]))
        assert order[0] < order[-1]


def test_full_bond_dimension_dmrg_state_has_the_fci_entanglement():
    n = 6
    h, eri, x, H = _random_state(n, 6, 0, seed=9)
    s_f, I_f = OB.orbital_entanglement(H.ops.states, x, n, 0)
    o = OracleDMRG(h, eri, 6, 0, D=400)
    o.sweep(2)
    s_d, I_d = OB.orbital_entanglement(o.states, o.psi_full, n, 0)
    assert np.abs(s_d - s_f).max() < 1e-7
    assert np.abs(I_d - I_f).max() < 1e-7
