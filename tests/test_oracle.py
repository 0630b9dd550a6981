"""Pins of the CPU oracle against closed forms, brute force and invariants.

Nothing here touches the CUDA path.  Each test ties one oracle function to
something other than itself: a textbook closed form, an exhaustive dense
diagonalisation, an operator identity, or a finite difference.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import workloads as W
from oracle import casscf as C
from oracle.dmrg import OracleDMRG, dbss_dimension, select_multiplets
from oracle.fci import Hamiltonian, fci
from oracle.rdm import Gamma_su2, energy_from_rdms, gamma_su2, rdm12
from oracle.su2 import cg, wigner6j_bruteforce


# ---------------------------------------------------------------- SU(2)
def test_cg_known_values():
    # <1/2 1/2, 1/2 -1/2 | 0 0> = 1/sqrt(2), <1/2 -1/2, 1/2 1/2 | 0 0> = -1/sqrt(2)
    assert cg(1, 1, 1, -1, 0, 0) == pytest.approx(1 / math.sqrt(2), abs=1e-15)
    assert cg(1, -1, 1, 1, 0, 0) == pytest.approx(-1 / math.sqrt(2), abs=1e-15)
    assert cg(1, 1, 1, -1, 2, 0) == pytest.approx(1 / math.sqrt(2), abs=1e-15)
    assert cg(1, 1, 1, 1, 2, 2) == pytest.approx(1.0, abs=1e-15)
    # <1 1, 1/2 -1/2 | 1/2 1/2> = sqrt(2/3)
    assert cg(2, 2, 1, -1, 1, 1) == pytest.approx(math.sqrt(2 / 3), abs=1e-15)


@pytest.mark.parametrize("j1,j2", [(1, 1), (2, 1), (3, 2), (4, 4), (5, 2)])
def test_cg_orthonormal(j1, j2):
    rows = []
    for J in range(abs(j1 - j2), j1 + j2 + 1, 2):
        for M in range(-J, J + 1, 2):
            rows.append([cg(j1, m1, j2, m2, J, M)
                         for m1 in range(-j1, j1 + 1, 2) for m2 in range(-j2, j2 + 1, 2)])
    U = np.array(rows)
    assert np.allclose(U @ U.T, np.eye(len(rows)), atol=1e-13)


def test_6j_special_value():
    # {a b c; 0 c b} = (-1)^(a+b+c) / sqrt((2b+1)(2c+1))
    for a, b, c in [(1, 1, 0), (1, 1, 2), (2, 1, 1), (3, 2, 1), (4, 2, 2)]:
        val = wigner6j_bruteforce(a, b, c, 0, c, b)
        ref = (-1) ** ((a + b + c) // 2) / math.sqrt((b + 1) * (c + 1))
        assert val == pytest.approx(ref, abs=1e-13)


# ---------------------------------------------------------------- inputs
def test_acene_geometry_sizes():
    for rings, nsite, nbond in [(2, 10, 11), (5, 22, 26), (20, 82, 101)]:
        xy, bonds = W.acene_geometry(rings)
        assert len(xy) == nsite and len(bonds) == nbond
        d = np.linalg.norm(xy[:, None] - xy[None], axis=-1)
        assert np.all(d[np.triu_indices(nsite, 1)] > 1.39)


def test_cholesky_random_symmetry_psd():
    h, L = W.cholesky_random(8, 16, seed=3)
    eri = W.eri_from_cholesky(L)
    assert np.allclose(h, h.T)
    for perm in ["qprs", "pqsr", "rspq", "srqp"]:
        assert np.allclose(eri, np.einsum("pqrs->" + perm, eri))
    w = np.linalg.eigvalsh(eri.reshape(64, 64))
    assert w.min() > -1e-12


def test_initial_state_path():
    occ, path = W.initial_product_state(6, 6, 0)
    assert occ == [1] * 6 and path[0] == 0 and path[6] == 0
    assert all(abs(path[i] - path[i + 1]) == 1 for i in range(6))
    occ, path = W.initial_product_state(5, 7, 1)
    assert occ == [2, 2, 1, 1, 1] and path[0] == 1


# ---------------------------------------------------------------- FCI
def test_fci_hubbard_dimer_closed_form():
    for u in (0.5, 4.0, 10.0):
        h, eri, _ = W.hubbard_chain(2, t=-1.0, u=u)
        e, _, _ = fci(h, eri, 2, 0)
        assert e == pytest.approx((u - math.sqrt(u * u + 16.0)) / 2, abs=1e-10)
        e3, _, _ = fci(h, eri, 2, 2)          # triplet: no double occupancy
        assert e3 == pytest.approx(0.0, abs=1e-10)


def test_fci_huckel_sum_of_orbital_energies():
    xy, bonds = W.acene_geometry(1)
    h, eri, ec = W.ppp_integrals(xy, bonds, u_ev=0.0)    # U = V = 0
    e, _, _ = fci(h, eri, 6, 0, e_core=ec)
    w = np.linalg.eigvalsh(h)
    assert e == pytest.approx(2 * w[:3].sum() + ec, abs=1e-10)


def test_fci_matches_dense_diagonalisation():
    h, L = W.cholesky_random(4, 6, seed=2)
    eri = W.eri_from_cholesky(L)
    H = Hamiltonian(h, eri, 4, 0)
    dense = np.stack([H.apply(col) for col in np.eye(H.dim)], 1)
    assert np.allclose(dense, dense.T, atol=1e-13)
    # ground state over all spins present in Sz = 0 vs projected singlet
    s2 = np.stack([H.ops.apply_s2(col) for col in np.eye(H.dim)], 1)
    w, v = np.linalg.eigh(dense + 50.0 * s2)   # penalise S > 0
    e, _, _ = fci(h, eri, 4, 0)
    assert e == pytest.approx(w[0], abs=1e-9)


# ---------------------------------------------------------------- RDMs
@pytest.fixture(scope="module")
def rand5():
    h, L = W.cholesky_random(5, 10, seed=4)
    eri = W.eri_from_cholesky(L)
    e, x, H = fci(h, eri, 5, 1)
    g, G = rdm12(H.ops, x)
    return h, eri, e, x, H, g, G


def test_rdm_traces_and_symmetries(rand5):
    h, eri, e, x, H, g, G = rand5
    N = 5
    assert np.trace(g) == pytest.approx(N, abs=1e-10)
    assert np.einsum("pqqp->", G) == pytest.approx(N * (N - 1), abs=1e-9)
    assert np.allclose(np.einsum("pqqs->ps", G), (N - 1) * g, atol=1e-10)
    assert np.allclose(G, np.einsum("pqrs->qpsr", G), atol=1e-12)
    assert np.allclose(G, np.einsum("pqrs->srqp", G), atol=1e-12)
    occ = np.linalg.eigvalsh(g)
    assert occ.min() > -1e-10 and occ.max() < 2 + 1e-10
    assert energy_from_rdms(h, eri, g, G) == pytest.approx(e, abs=1e-10)


def test_spin_coupled_rdms(rand5):
    """Eq. rdm1_su2 exactly; the two-channel 2-RDM fixes the constant c1.

    With the spinor coupling of Eq. rdm1_su2 and standard Clebsch-Gordan
    coefficients the spin-free 2-RDM is sqrt(3) Gamma^(1) - Gamma^(0); the
    printed 2 sqrt(3) does not reproduce Gamma~ in this convention.
    """
    h, eri, e, x, H, g, G = rand5
    n, st = 5, H.ops.states
    gc = np.array([[gamma_su2(n, st, x, p, q) for q in range(n)] for p in range(n)])
    assert np.allclose(-math.sqrt(2) * gc, g, atol=1e-13)
    rng = np.random.default_rng(0)
    for _ in range(12):
        p, q, r, s = rng.integers(0, n, 4)
        g0 = Gamma_su2(n, st, x, p, q, r, s, 0)
        g1 = Gamma_su2(n, st, x, p, q, r, s, 2)
        assert math.sqrt(3) * g1 - g0 == pytest.approx(G[p, q, r, s], abs=1e-12)


# ---------------------------------------------------------------- DMRG
@pytest.mark.parametrize("case", ["hub6", "rand6_s0", "rand6_s2", "benzene"])
def test_dmrg_exact_at_full_bond_dimension(case):
    if case == "hub6":
        h, eri, ec = W.hubbard_chain(6, u=4.0); N, S = 6, 0
    elif case == "benzene":
        h, eri, ec = W.ppp_acene(1); N, S = 6, 0
    else:
        h, L = W.cholesky_random(6, 12, seed=1); eri = W.eri_from_cholesky(L); ec = 0.0
        N, S = 6, (0 if case == "rand6_s0" else 2)
    e_fci, _, _ = fci(h, eri, N, S, e_core=ec)
    d = OracleDMRG(h, eri, N, S, D=400, e_core=ec)
    es = d.sweep(3)
    assert es[-1] == pytest.approx(e_fci, abs=1e-9)


def test_dmrg_variational_and_monotone():
    h, L = W.cholesky_random(6, 12, seed=1)
    eri = W.eri_from_cholesky(L)
    e_fci, _, _ = fci(h, eri, 6, 0)
    es = []
    for D in (2, 4, 8):
        d = OracleDMRG(h, eri, 6, 0, D=D)
        es.append(d.sweep(3)[-1])
        left, right = d.bond_dims()
        assert max(x for x in left + right if x is not None) <= D
    assert es[0] >= es[1] - 1e-10 >= es[2] - 2e-10
    assert es[2] >= e_fci - 1e-10


def test_dmrg_bases_are_orthonormal_spin_multiplets():
    h, L = W.cholesky_random(6, 12, seed=1)
    eri = W.eri_from_cholesky(L)
    d = OracleDMRG(h, eri, 6, 2, D=6)
    d.sweep(1)
    from oracle.dmrg import _splus
    for b in d.left[1:5] + d.right[2:6]:
        if b is None:
            continue
        assert np.allclose(b.vecs.T @ b.vecs, np.eye(b.m), atol=1e-12)
        nsites = int(round(math.log(b.vecs.shape[0], 4)))
        Sp = _splus(nsites)
        Sp_b = b.vecs.T @ (Sp @ b.vecs)
        Sz = np.diag(0.5 * b.two_m)
        S2 = Sp_b.T @ Sp_b + Sz @ Sz + Sz
        jj = 0.5 * b.two_j
        assert np.allclose(S2, np.diag(jj * (jj + 1)), atol=1e-10)


def test_heff_hermitian():
    h, L = W.cholesky_random(6, 12, seed=5)
    eri = W.eri_from_cholesky(L)
    d = OracleDMRG(h, eri, 6, 0, D=5)
    d.sweep(1)
    i = 2
    Lb, Rb = d._blocks(i)
    m = int(d._mask(Lb, Rb, 0).sum())
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal(m), rng.standard_normal(m)
    lhs = x @ d.heff_apply(i, y)
    rhs = d.heff_apply(i, x) @ y
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_selection_rule_ties_and_threshold():
    cands = [(0.5, 2, 0, 0), (0.2, 3, 1, 0), (0.2, 1, 1, 0), (0.1, 2, 2, 0), (1e-13, 2, 0, 1)]
    assert select_multiplets(cands, 2) == [0, 2]         # tie broken by N asc
    assert select_multiplets(cands, 10) == [0, 2, 1, 3]  # below 1e-12 dropped


def test_dbss_dimension_rule_by_hand():
    """Fewest multiplets with discarded weight <= target, clamped to [D_min, D]."""
    lam = [0.6, 0.3, 0.09, 0.009, 0.001]
    assert dbss_dimension(lam, 10, 1, 0.0101) == 3      # discards 0.009 + 0.001
    assert dbss_dimension(lam, 10, 1, 0.0099) == 4      # 0.01 is above the target
    assert dbss_dimension(lam, 10, 1, 0.5) == 1
    assert dbss_dimension(lam, 2, 1, 0.0099) == 2       # D_max caps
    assert dbss_dimension(lam, 10, 4, 0.5) == 4         # D_min floors
    assert dbss_dimension(list(reversed(lam)), 10, 1, 0.0101) == 3  # order-free
    assert dbss_dimension(lam, 10, 1, 0.0) == 5


def test_dbss_sweeps_bound_discarded_weight_and_reach_fci():
    h, L = W.cholesky_random(6, 12, seed=1)
    eri = W.eri_from_cholesky(L)
    e_fci, _, _ = fci(h, eri, 6, 0)
    fixed = OracleDMRG(h, eri, 6, 0, D=6)
    e_fixed = fixed.sweep(3)
    same = OracleDMRG(h, eri, 6, 0, D=6, trunc_target=0.0)
    assert same.sweep(3) == e_fixed                    # target 0: fixed D
    d = OracleDMRG(h, eri, 6, 0, D=400, D_min=2, trunc_target=1e-3)
    es = d.sweep(3)
    assert max(d.record.trunc[1:]) <= 1e-3 + 1e-15      # the bound, after the first sweep
    assert es[-1] >= e_fci - 1e-10
    assert min(d.kept) >= 2 and max(d.kept) < 400
    finer = OracleDMRG(h, eri, 6, 0, D=400, D_min=2, trunc_target=1e-6)
    e_finer = finer.sweep(3)[-1]
    assert e_fci - 1e-10 <= e_finer < es[-1]             # a smaller target is closer to FCI
    assert max(finer.kept) > max(d.kept)
    tight = OracleDMRG(h, eri, 6, 0, D=400, D_min=1, trunc_target=1e-14)
    assert tight.sweep(3)[-1] == pytest.approx(e_fci, abs=1e-9)


# ---------------------------------------------------------------- CAS-SCF
def test_rotation_convention_matches_manybody_exponential():
    n = 3
    h, L = W.cholesky_random(n, 5, seed=7)
    eri = W.eri_from_cholesky(L)
    e, x, H = fci(h, eri, 2, 0)
    rng = np.random.default_rng(0)
    K = np.zeros((n, n))
    for p in range(n):
        for q in range(p):
            K[p, q] = 0.3 * rng.normal()
            K[q, p] = -K[p, q]
    eye = np.eye(H.dim)
    kap = np.zeros((H.dim, H.dim))
    for j in range(H.dim):
        for p in range(n):
            for q in range(p):
                H.ops.apply_e(p, q, eye[:, j], kap[:, j], K[p, q])
                H.ops.apply_e(q, p, eye[:, j], kap[:, j], -K[p, q])
    U = scipy.linalg.expm(-kap)
    Hm = np.stack([H.apply(c) for c in eye], 1)
    e_mb = x @ U.T @ Hm @ U @ x
    g, G = rdm12(H.ops, x)
    assert C.casscf_energy(h, L, 0, n, g, G, K=K) == pytest.approx(e_mb, abs=1e-12)


def _cas_problem(nb=7, nc=1, na=3, seed=11):
    h, L = W.cholesky_random(nb, 10, seed=seed)
    fi = C.inactive_fock(h, L, nc)
    a = slice(nc, nc + na)
    eri_a = np.einsum("ktu,kvw->tuvw", L[:, a, a], L[:, a, a])
    e, x, H = fci(fi[a, a], eri_a, 2, 0)
    g, G = rdm12(H.ops, x)
    return h, L, nc, na, g, G, e


def test_orbital_gradient_matches_finite_differences():
    h, L, nc, na, g, G, _ = _cas_problem()
    nb = h.shape[0]
    grad = C.orbital_gradient(h, L, nc, na, g, G)
    eps = 1e-5
    for p in range(nb):
        for q in range(p):
            if nc <= p < nc + na and nc <= q < nc + na:
                assert grad[p, q] == 0.0
                continue
            K = np.zeros((nb, nb))
            K[p, q], K[q, p] = eps, -eps
            fd = (C.casscf_energy(h, L, nc, na, g, G, K=K)
                  - C.casscf_energy(h, L, nc, na, g, G, K=-K)) / (2 * eps)
            assert grad[p, q] == pytest.approx(fd, rel=1e-5, abs=1e-8)
    assert np.allclose(grad, -grad.T)


def test_casscf_energy_at_zero_rotation_is_cas_energy():
    h, L, nc, na, g, G, e_act = _cas_problem()
    fi = C.inactive_fock(h, L, nc)
    e_core = float(np.trace(h[:nc, :nc]) + np.trace(fi[:nc, :nc]))
    assert C.casscf_energy(h, L, nc, na, g, G) == pytest.approx(e_core + e_act, abs=1e-10)


def test_transform_preserves_energy_under_active_rotation():
    """Rotations inside the active space leave the CAS-CI energy unchanged
    when the RDMs are rotated with them (a property of the exact CAS)."""
    h, L, nc, na, g, G, _ = _cas_problem()
    nb = h.shape[0]
    K = np.zeros((nb, nb))
    K[nc + 1, nc] = 0.2
    K[nc, nc + 1] = -0.2
    R = C.rotation_matrix(K)
    Ra = R[nc:nc + na, nc:nc + na]
    g2 = Ra.T @ g @ Ra
    G2 = np.einsum("ap,bq,cr,ds,abcd->pqrs", Ra, Ra, Ra, Ra, G)
    e0 = C.casscf_energy(h, L, nc, na, g, G)
    e1 = C.casscf_energy(h, L, nc, na, g2, G2, K=K)
    assert e1 == pytest.approx(e0, abs=1e-10)


# ---------------------------------------------------------------- DMRG-SCF
def _fci_solver(n_elec, two_s=0):
    def solve(h_act, eri_act, e_core):
        e, x, H = fci(h_act, eri_act, n_elec, two_s, e_core=e_core)
        g, G = rdm12(H.ops, x)
        return e, g, G
    return solve


def test_dmrg_scf_converges_to_a_minimum_of_the_cas_energy():
    """The macro loop (exact CI in the active space) reaches the paper's
    thresholds, lowers the energy, and ends at a local minimum: a direct
    minimisation of the CAS-CI energy over the non-redundant rotations from
    the final orbitals finds nothing lower."""
    import scipy.optimize
    h, L = W.cholesky_random(7, 14, seed=5, sigma_h=0.2)
    nc, na, ne = 1, 4, 4
    es, gs, U = C.dmrg_scf(h, L, nc, na, _fci_solver(ne))
    assert gs[-1] < 1e-3 and abs(es[-1] - es[-2]) < 1e-7
    assert es[-1] < es[0]
    assert np.allclose(U.T @ U, np.eye(7), atol=1e-12)
    h2, L2 = C.transform(h, L, U)
    mask = C.rotation_mask(7, nc, na)
    idx = np.argwhere(mask > 0)

    def cas_energy(x):
        K = np.zeros((7, 7))
        K[idx[:, 0], idx[:, 1]] = x
        h3, L3 = C.transform(h2, L2, C.rotation_matrix(K - K.T))
        fi = C.inactive_fock(h3, L3, nc)
        a = slice(nc, nc + na)
        e_core = float(np.trace(h3[:nc, :nc]) + np.trace(fi[:nc, :nc]))
        eri = np.einsum("ktu,kvw->tuvw", L3[:, a, a], L3[:, a, a])
        return fci(fi[a, a], eri, ne, 0, e_core=e_core)[0]

    assert cas_energy(np.zeros(len(idx))) == pytest.approx(es[-1], abs=1e-9)
    res = scipy.optimize.minimize(cas_energy, np.zeros(len(idx)), method="BFGS", options={"gtol": 1e-6})
    assert res.fun > es[-1] - 1e-6
