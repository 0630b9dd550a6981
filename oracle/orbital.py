"""Orbital entanglement and the quantum-information orbital ordering (oracle).

TEST INFRASTRUCTURE ONLY.  Sec. II "Numerical procedure": before the large
DMRG-SCF runs, a few low-bond-dimension DMRG runs (D = 16, 32, 64) fix an
orbital ordering from quantum-information measures of the state (the cited
works of Legeza et al. and Barcza et al.).  Written from the definitions:

* one-orbital reduced density matrix rho_p: the state restricted to orbital
  p, a 4 x 4 matrix over the local states (0, dn, up, updn) (diagonal for a
  state of fixed N and S_z);
* two-orbital reduced density matrix rho_pq (p != q): the 16 x 16 matrix over
  the local states |d_p d_q> with Tr(rho_pq X) = <X> for every operator X
  built from the four modes of p and q (fermionic operators in the
  Jordan-Wigner order of the full space, p before q);
* for a spin multiplet S > 0 both are averaged over the 2S+1 states M of the
  multiplet (the SU(2)-invariant reduced states);
* von Neumann entropies s_p = -Tr rho_p ln rho_p, s_pq likewise, and the
  mutual information I_pq = s_p + s_q - s_pq (p != q), I_pp = 0;
* the ordering: the orbitals sorted by the Fiedler vector (eigenvector of
  the second-smallest eigenvalue) of the graph Laplacian L = diag(I 1) - I,
  the minimiser of sum_pq I_pq (x_p - x_q)^2 over unit vectors orthogonal to
  the constant one, the spectral relaxation of placing strongly entangled
  orbitals next to each other.

Dense vectors over the whole 4^n Fock space (n <= 10); the basis and the
Jordan-Wigner order are those of ``oracle.fock``.
"""
from __future__ import annotations

import numpy as np

from .fock import _mode_value, digits, mode_occupations


def full_vector(states, coef, n):
    """Dense 4^n vector of a sector vector (full indices ``states``)."""
    x = np.zeros(4 ** n)
    x[np.asarray(states, dtype=np.int64)] = coef
    return x


class Modes:
    """Creation and annihilation of single modes on dense 4^n vectors."""

    def __init__(self, n):
        self.n = n
        idx = np.arange(4 ** n, dtype=np.int64)
        self.occ = mode_occupations(digits(idx, n))  # (4^n, 2n)
        self.before = np.cumsum(self.occ, axis=1) - self.occ  # occupied modes before each mode

    def annihilate(self, mode, x):
        """a_mode x."""
        y = np.zeros_like(x)
        src = np.nonzero(self.occ[:, mode] == 1)[0]
        sign = np.where(self.before[src, mode] % 2 == 0, 1.0, -1.0)
        y[src - _mode_value(self.n, mode)] = sign * x[src]
        return y

    def create(self, mode, x):
        """a+_mode x."""
        y = np.zeros_like(x)
        src = np.nonzero(self.occ[:, mode] == 0)[0]
        sign = np.where(self.before[src, mode] % 2 == 0, 1.0, -1.0)
        y[src + _mode_value(self.n, mode)] = sign * x[src]
        return y

    def empty_projector(self, modes, x):
        """Projector onto states with all ``modes`` empty."""
        keep = np.all(self.occ[:, modes] == 0, axis=1)
        return np.where(keep, x, 0.0)


LOCAL = [(0, 0), (0, 1), (1, 0), (1, 1)]  # digit d -> (n_up, n_dn): 0 empty, 1 dn, 2 up, 3 updn


def multiplet(states, psi, n, two_s):
    """The 2S+1 dense vectors |S, M> (M = S, S-1, ..., -S) of the multiplet
    whose highest-weight state is the sector vector ``psi`` (2 S_z = two_s),
    by repeated S- = sum_p a+_{p dn} a_{p up}, each normalised."""
    md = Modes(n)
    v = full_vector(states, psi, n)
    v = v / np.linalg.norm(v)
    out = [v]
    for _ in range(two_s):
        w = np.zeros_like(v)
        for p in range(n):
            w += md.create(2 * p + 1, md.annihilate(2 * p, v))
        v = w / np.linalg.norm(w)
        out.append(v)
    return out


def one_orbital_rdm(vecs, n, p):
    """Diagonal of rho_p over the local states (0, dn, up, updn), averaged
    over the given multiplet vectors."""
    idx = np.arange(4 ** n, dtype=np.int64)
    d = digits(idx, n)[:, p]
    out = np.zeros(4)
    for v in vecs:
        for k in range(4):
            out[k] += np.sum(v[d == k] ** 2)
    return out / len(vecs)


def two_orbital_rdm(vecs, n, p, q):
    """rho_pq (16 x 16, p < q) over the local states a = 4 d_p + d_q, averaged over
    the multiplet vectors.  With |a> = A_a |vac> (A_a the product of the
    creators of the occupied modes among p-up, p-dn, q-up, q-dn in that
    order) and P the projector onto those four modes empty,
        rho_ab = <psi| A_b P A_a^+ |psi> = (P A_b^+ psi) . (P A_a^+ psi),
    so that Tr(rho X) = <X> for every operator X of the four modes."""
    assert p < q
    md = Modes(n)
    modes = [2 * p, 2 * p + 1, 2 * q, 2 * q + 1]
    rho = np.zeros((16, 16))
    for v in vecs:
        cols = []
        for a in range(16):
            da, db = divmod(a, 4)  # digits of p and of q
            occ = [LOCAL[da][0], LOCAL[da][1], LOCAL[db][0], LOCAL[db][1]]
            w = v
            # A_a^+ = product of annihilators in the reverse order of the creators
            for k in range(3, -1, -1):
                if occ[k]:
                    w = md.annihilate(modes[k], w)
            cols.append(md.empty_projector(modes, w))
        V = np.array(cols)
        rho += V @ V.T
    return rho / len(vecs)


def entropy(rho):
    """von Neumann entropy -Tr rho ln rho (eigenvalues below 1e-14 dropped)."""
    w = np.linalg.eigvalsh(0.5 * (rho + rho.T)) if rho.ndim == 2 else np.asarray(rho)
    w = w[w > 1e-14]
    return float(-(w * np.log(w)).sum())


def orbital_entanglement(states, psi, n, two_s):
    """One-orbital entropies s (n) and mutual information I (n x n)."""
    vecs = multiplet(states, psi, n, two_s)
    s1 = np.array([entropy(one_orbital_rdm(vecs, n, p)) for p in range(n)])
    I = np.zeros((n, n))
    for p in range(n):
        for q in range(p + 1, n):
            I[p, q] = I[q, p] = s1[p] + s1[q] - entropy(two_orbital_rdm(vecs, n, p, q))
    return s1, I


def fiedler_order(I):
    """Orbitals sorted by the Fiedler vector of the Laplacian diag(I 1) - I.
    The vector's sign is fixed so that its first orbital (in the returned
    order) is the smaller of the two ends; equal components keep index order."""
    I = np.asarray(I, dtype=np.float64)
    L = np.diag(I.sum(1)) - I
    w, V = np.linalg.eigh(L)
    f = V[:, 1]
    order = np.argsort(f, kind="stable")
    if order[0] > order[-1]:
        order = np.argsort(-f, kind="stable")
    return order


def permute_integrals(h, eri, order):
    """Integrals in the new site order: site k holds orbital order[k]."""
    o = np.asarray(order)
    return h[np.ix_(o, o)], eri[np.ix_(o, o, o, o)]
