"""CPU check of the library's assembly of the one- and two-orbital reduced
density matrices from their SU(2) invariants (dmrg_orbital_rdms_from_invariants,
host-only).

The invariants [S_a of p (x) S_b of q]^0 are built here independently: the
spinor components of a+ and a~ on a separate four-mode Jordan-Wigner space,
coupled left to right with the oracle's Clebsch-Gordan coefficients (Racah
closed form).  Their expectation values in the oracle's rho_pq (and rho_p)
of random states -- singlet and doublet, multiplet-averaged -- go into the
library, which must return the same matrices.  This pins the library's
invariant tables, coupling convention and solve on the CPU; the device pass
that measures the invariants is checked against the oracle in
test_gpu_orbital.py."""
import numpy as np
import pytest

import workloads as W
from oracle import orbital as OB
from oracle.fci import fci
from oracle.su2 import cg

STRINGS = [((1,), ()), ((0,), ()), ((1, 0), (0,)), ((1, 0), (2,)), ((1, 1), (0,)), ((0, 0), (0,)),
           ((1, 1, 0), (0, 1)), ((0, 0, 1), (0, 1)), ((1, 1, 0, 0), (0, 1, 0))]
PAIRS = [(2, 2), (2, 8), (8, 2), (8, 8), (3, 3), (0, 1), (0, 7), (6, 1), (6, 7),
         (1, 0), (1, 6), (7, 0), (7, 6), (4, 5), (5, 4)]


def modes(orbs):
    """Creators of the 2*orbs modes (orbital-major, up before down) on the
    local states indexed by the occupation bits, first mode most significant."""
    M = 2 * orbs
    dim = 1 << M
    cr = []
    for m in range(M):
        A = np.zeros((dim, dim))
        for a in range(dim):
            bit = 1 << (M - 1 - m)
            if a & bit:
                continue
            before = sum((a >> (M - 1 - k)) & 1 for k in range(m))
            A[a | bit, a] = (-1) ** before
        cr.append(A)
    return cr


def spinor(cr, orb, dag):
    """Components {2m: matrix}: a+(+1/2) = a+_up, a+(-1/2) = a+_dn,
    a~(+1/2) = a_dn, a~(-1/2) = -a_up."""
    up, dn = cr[2 * orb], cr[2 * orb + 1]
    if dag:
        return {1: up, -1: dn}
    return {1: dn.T, -1: -up.T}


def couple(A, ka, B, kb, K):
    out = {}
    for Q in range(-K, K + 1, 2):
        acc = 0.0
        for qa, Ma in A.items():
            qb = Q - qa
            if qb in B:
                c = cg(ka, qa, kb, qb, K, Q)
                if c:
                    acc = acc + c * (Ma @ B[qb])
        out[Q] = acc
    return out


def string_op(cr, orb, a):
    dag, kl = STRINGS[a]
    T, k = spinor(cr, orb, dag[0]), 1
    for d, k2 in zip(dag[1:], kl):
        T = couple(T, k, spinor(cr, orb, d), 1, k2)
        k = k2
    return T, k


def invariant(cr, a, b):
    dim = cr[0].shape[0]
    if a is None and b is None:
        return np.eye(dim)
    if b is None:
        T, k = string_op(cr, 0, a)
        assert k == 0
        return T[0]
    if a is None:
        T, k = string_op(cr, 1, b)
        assert k == 0
        return T[0]
    X, kx = string_op(cr, 0, a)
    Y, ky = string_op(cr, 1, b)
    return couple(X, kx, Y, ky, 0)[0]


@pytest.fixture(scope="module")
def lib():
    import paper_2503_20700_gb300 as p
    from paper_2503_20700_gb300 import build as b
    import os
    if not os.path.exists(p.lib_path()):
        b.build()
    p.load()
    return p


@pytest.mark.parametrize("n_elec,two_s,seed", [(6, 0, 3), (5, 1, 8), (6, 2, 1)])
def test_library_assembles_oracle_rdms_from_independent_invariants(lib, n_elec, two_s, seed):
    n = 6
    h, L = W.cholesky_random(n, 2 * n, seed=seed)
    e, x, H = fci(h, W.eri_from_cholesky(L), n_elec, two_s)
    vecs = OB.multiplet(H.ops.states, x, n, two_s)
    cr1, cr2 = modes(1), modes(2)
    s1 = [invariant(cr1, 2, None), invariant(cr1, 8, None)]
    s2 = [invariant(cr2, a, b) for a, b in PAIRS]
    rho1 = np.array([np.diag(OB.one_orbital_rdm(vecs, n, p)) for p in range(n)])
    inv1 = np.array([[np.trace(r @ M) for M in s1] for r in rho1])
    inv2 = np.zeros((n, n, len(PAIRS)))
    rho2 = np.zeros((n, n, 16, 16))
    for p in range(n):
        for q in range(p + 1, n):
            rho2[p, q] = OB.two_orbital_rdm(vecs, n, p, q)
            inv2[p, q] = [np.trace(rho2[p, q] @ M) for M in s2]
    r1, r2 = lib.orbital_rdms_from_invariants(inv1, inv2)
    assert np.abs(r1 - np.array([np.diag(r) for r in rho1])).max() < 1e-12
    assert np.abs(r2 - rho2).max() < 1e-12
