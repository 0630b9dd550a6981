"""Orbital rotation, integral transformation and the CAS-SCF gradient (oracle).

TEST INFRASTRUCTURE ONLY.  Sec. II.A of the paper: orbitals are rotated by
U = exp(-kappa^) with kappa^ = sum_{p>q} kappa_pq (e_pq - e_qp), the energy
is E = <Psi| U+ H U |Psi>, and the orbital gradient is obtained from the
one- and two-particle RDMs (Eqs. onerdm, twordm).  Active-active rotations
are left out, as the paper does (Sec. II.C).

Conventions (pinned by the tests against a full Fock-space matrix exponential
and against finite differences):
* ``K`` is the real antisymmetric matrix with K[p, q] = kappa_pq for p > q.
* With U = exp(-kappa^) the rotated Hamiltonian U+ H U has the integrals
  h' = R^T h R and L'^k = R^T L^k R with R = expm(-K) (checked against the
  many-body exponential of kappa^ on the full Fock space).
* Orbitals are ordered core (ncore), active (ncas), virtual (rest).
* Gamma~ is in the paper's operator order, Gamma~_pqrs = <a+_p a+_q a_r a_s>
  summed over spins as in Eq. twordm; the chemists'-order 2-RDM is
  d_pqrs = Gamma~_prsq.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def rotation_matrix(K):
    """R = expm(-K) for an antisymmetric K (library matrix exponential)."""
    K = np.asarray(K, float)
    return scipy.linalg.expm(-K)


def transform(h, L, R):
    """h' = R^T h R and L'^k = R^T L^k R."""
    h2 = R.T @ h @ R
    L2 = np.einsum("rp,krs,sq->kpq", R, L, R, optimize=True)
    return h2, L2


def _eri(L):
    k, n, _ = L.shape
    m = L.reshape(k, n * n)
    return (m.T @ m).reshape(n, n, n, n)


def inactive_fock(h, L, ncore):
    """F^I_pq = h_pq + sum_i [2 (pq|ii) - (pi|iq)] over core orbitals i."""
    c = slice(0, ncore)
    J = np.einsum("kpq,kii->pq", L, L[:, c, c])
    K = np.einsum("kpi,kiq->pq", L[:, :, c], L[:, c, :])
    return h + 2.0 * J - K


def casscf_energy(h, L, ncore, ncas, gamma, Gamma, K=None, e_nuc=0.0):
    """E(kappa) with the RDMs held fixed (closed-shell core).

    E = sum_i (h'_ii + F^I'_ii) + sum_tu F^I'_tu gamma~_tu
        + 1/2 sum_tuvw (tu|vw)' Gamma~_tvwu + e_nuc.
    """
    if K is not None:
        h, L = transform(h, L, rotation_matrix(K))
    fi = inactive_fock(h, L, ncore)
    e = float(np.trace(h[:ncore, :ncore]) + np.trace(fi[:ncore, :ncore]))
    a = slice(ncore, ncore + ncas)
    e += float(np.einsum("tu,tu->", fi[a, a], gamma))
    la = L[:, a, a]
    eri_a = np.einsum("ktu,kvw->tuvw", la, la)
    e += 0.5 * float(np.einsum("tuvw,tvwu->", eri_a, Gamma))
    return e + e_nuc


def generalized_fock(h, L, ncore, ncas, gamma, Gamma):
    """Generalised Fock matrix F (nb x nb), textbook closed-shell-core form.

    F_iq = 2 (F^I_qi + F^A_qi)                       i core
    F_tq = sum_u gamma~_tu F^I_qu + sum_uvw d_tuvw (qu|vw)   t active
    F_aq = 0                                          a virtual
    with F^A_pq = sum_tu gamma~_tu [(pq|tu) - 1/2 (pt|uq)] and
    d_tuvw = Gamma~_tvwu (chemists' order).
    """
    nb = h.shape[0]
    a = slice(ncore, ncore + ncas)
    fi = inactive_fock(h, L, ncore)
    la_pq = L                              # (k, p, q)
    # F^A
    w = np.einsum("ktu,tu->k", L[:, a, a], gamma)
    fa = np.einsum("k,kpq->pq", w, L)
    fa -= 0.5 * np.einsum("kpt,tu,kuq->pq", L[:, :, a], gamma, L[:, a, :], optimize=True)
    F = np.zeros((nb, nb))
    F[:ncore, :] = 2.0 * (fi[:, :ncore] + fa[:, :ncore]).T
    d = np.einsum("tvwu->tuvw", Gamma)
    # (qu|vw) with u,v,w active
    quvw = np.einsum("kqu,kvw->quvw", la_pq[:, :, a], L[:, a, a], optimize=True)
    F[a, :] = (gamma @ fi[:, a].T) + np.einsum("tuvw,quvw->tq", d, quvw, optimize=True)
    return F


def orbital_gradient(h, L, ncore, ncas, gamma, Gamma):
    """G[p, q] = dE/dkappa_pq (p > q) as an antisymmetric matrix.

    G = 2 (F - F^T) with the generalised Fock matrix; active-active entries
    are set to zero (those rotations are neglected).  Core-core and
    virtual-virtual entries vanish identically.
    """
    F = generalized_fock(h, L, ncore, ncas, gamma, Gamma)
    G = 2.0 * (F - F.T)
    a = slice(ncore, ncore + ncas)
    G[a, a] = 0.0
    return G
