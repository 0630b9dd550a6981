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


# ---------------------------------------------------------------- DMRG-SCF
def fock_diagonals(h, L, ncore, ncas, gamma, Gamma):
    """Diagonals of F^I, F^A and of the generalised Fock matrix F."""
    a = slice(ncore, ncore + ncas)
    fi = inactive_fock(h, L, ncore)
    w = np.einsum("ktu,tu->k", L[:, a, a], gamma)
    fa = np.einsum("k,kpq->pq", w, L)
    fa -= 0.5 * np.einsum("kpt,tu,kuq->pq", L[:, :, a], gamma, L[:, a, :], optimize=True)
    F = generalized_fock(h, L, ncore, ncas, gamma, Gamma)
    return np.diag(fi).copy(), np.diag(fa).copy(), np.diag(F).copy()


def diagonal_hessian(h, L, ncore, ncas, gamma, Gamma, floor=0.05):
    """Approximate diagonal orbital Hessian H[p, q] (p > q) of the
    closed-shell-core CAS-SCF energy, one value per non-redundant rotation,
    floored at `floor` (the step of a quasi-Newton update):
      core i - virtual a:   4 (f_aa - f_ii)
      active t - virtual a: 2 n_t f_aa - 2 F_tt
      core i - active t:    4 (f_tt - f_ii) + 2 n_t f_ii - 2 F_tt
    with f = F^I + F^A, n_t = gamma~_tt and F the generalised Fock matrix.
    Active-active pairs and the rest are 0 (no step)."""
    nb = h.shape[0]
    fi, fa, Fd = fock_diagonals(h, L, ncore, ncas, gamma, Gamma)
    f = fi + fa
    H = np.zeros((nb, nb))
    for p in range(nb):
        for q in range(p):
            pc, pa = p < ncore, ncore <= p < ncore + ncas
            qc, qa = q < ncore, ncore <= q < ncore + ncas
            if pc or (pa and qa):
                continue          # p > q: p core implies q core; active-active redundant
            if not pa and qc:      # virtual - core
                v = 4.0 * (f[p] - f[q])
            elif not pa and qa:    # virtual - active
                t = q - ncore
                v = 2.0 * gamma[t, t] * f[p] - 2.0 * Fd[q]
            elif pa and qc:        # active - core
                t = p - ncore
                v = 4.0 * (f[p] - f[q]) + 2.0 * gamma[t, t] * f[q] - 2.0 * Fd[p]
            else:
                continue
            H[p, q] = max(v, floor)
    return H


def rotation_mask(nb, ncore, ncas):
    """Non-redundant rotations: p > q in different classes (core, active,
    virtual); core-core, active-active and virtual-virtual rotations are left
    out (the last two do not change a CAS energy; active-active rotations are
    not used, Sec. II.C)."""
    cls = np.array([0 if p < ncore else (1 if p < ncore + ncas else 2) for p in range(nb)])
    m = (cls[:, None] != cls[None, :]) & np.tril(np.ones((nb, nb), bool), -1)
    return m.astype(float)


def dmrg_scf(h, L, ncore, ncas, solver, max_iter=60, e_tol=1e-7, g_tol=1e-3, memory=8, max_step=0.5):
    """DMRG-SCF macro iterations (Sec. II.A; thresholds of the paper: energy
    change 1e-7, gradient 1e-3).  The active-space problem of the current
    orbitals is solved by `solver(h_act, eri_act, e_core)` -> (E, gamma~,
    Gamma~); the orbital gradient g = dE/dkappa (non-redundant p > q) comes
    from the RDMs; the step x = -H^-1 g is a limited-memory BFGS step (the
    last `memory` pairs of steps and gradient changes, two-loop recursion)
    with the diagonal Hessian above as the initial inverse, its largest
    entry capped at max_step; the orbitals rotate as U <- U expm(-(x - x^T)).
    Stops after an iteration whose energy change is below e_tol with
    max |g| below g_tol.

    Returns (energies, max |g| per iteration, U)."""
    nb = h.shape[0]
    mask = rotation_mask(nb, ncore, ncas)
    U = np.eye(nb)
    energies, gmax = [], []
    S, Y = [], []
    x_prev = g_prev = None
    a = slice(ncore, ncore + ncas)
    for it in range(max_iter):
        h2, L2 = transform(h, L, U)
        fi = inactive_fock(h2, L2, ncore)
        e_core = float(np.trace(h2[:ncore, :ncore]) + np.trace(fi[:ncore, :ncore]))
        eri_a = np.einsum("ktu,kvw->tuvw", L2[:, a, a], L2[:, a, a])
        E, gamma, Gamma = solver(fi[a, a], eri_a, e_core)
        g = mask * orbital_gradient(h2, L2, ncore, ncas, gamma, Gamma)
        energies.append(float(E))
        gmax.append(float(np.abs(g).max()))
        if it > 0 and abs(energies[-1] - energies[-2]) < e_tol and gmax[-1] < g_tol:
            break
        if x_prev is not None:
            y = g - g_prev
            if float(np.sum(x_prev * y)) > 1e-12:
                S.append(x_prev)
                Y.append(y)
                if len(S) > memory:
                    S.pop(0)
                    Y.pop(0)
        Hd = diagonal_hessian(h2, L2, ncore, ncas, gamma, Gamma)
        q = g.copy()
        alpha = []
        for s_i, y_i in zip(reversed(S), reversed(Y)):
            rho = 1.0 / float(np.sum(y_i * s_i))
            al = rho * float(np.sum(s_i * q))
            q = q - al * y_i
            alpha.append((rho, al))
        r = np.where(mask > 0, q / np.where(Hd > 0, Hd, 1.0), 0.0)
        for (s_i, y_i), (rho, al) in zip(zip(S, Y), reversed(alpha)):
            be = rho * float(np.sum(y_i * r))
            r = r + (al - be) * s_i
        x = -r
        big = float(np.abs(x).max())
        if big > max_step:
            x = x * (max_step / big)
        U = U @ rotation_matrix(x - x.T)
        x_prev, g_prev = x, g
    return energies, gmax, U
