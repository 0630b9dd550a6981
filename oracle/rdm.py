"""One- and two-particle reduced density matrices (oracle).

TEST INFRASTRUCTURE ONLY.  Written from Sec. II.A-C:

* spin-free RDMs (Eqs. onerdm, twordm):
      gamma~_pq = <e_pq>,   Gamma~_pqrs = <sum_{s,t} a+_ps a+_qt a_rt a_ss>;
  evaluated on an explicit full-space vector with
      Gamma~_pqrs = <E_sp Psi | E_qr Psi> - delta_qs gamma~_pr,
  which follows from E_ps E_qr = delta_qs E_pr + e_pqrs (anticommutation).
* spin-coupled forms (Eq. rdm1_su2 and the two-channel 2-RDM): built from
  the spinors f+_p = (a+_p,up, a+_p,dn) and f_p = (a_p,dn, -a_p,up) and
  coupled with Clebsch-Gordan coefficients, by direct evaluation of the
  operator products on the full-space vector.
"""
from __future__ import annotations

import numpy as np

from .fock import OneBodyMap, SectorOps, digits, mode_occupations
from .su2 import cg


def rdm12(ops: SectorOps, psi):
    """Spin-free (gamma~, Gamma~) of the normalised sector vector ``psi``."""
    n = ops.n
    phi = np.zeros((n, n, ops.dim))
    for q in range(n):
        for r in range(n):
            ops.apply_e(q, r, psi, phi[q, r])
    gamma = np.einsum("d,qrd->qr", psi, phi)
    # G[s,p,q,r] = <E_sp psi | E_qr psi>
    flat = phi.reshape(n * n, -1)
    G = (flat @ flat.T).reshape(n, n, n, n)
    Gamma = np.einsum("spqr->pqrs", G).copy()
    for q in range(n):
        Gamma[:, q, :, q] -= gamma
    return gamma, Gamma


def energy_from_rdms(h, eri, gamma, Gamma, e_core=0.0):
    """E = sum h_pq gamma~_pq + 1/2 sum (pq|rs) Gamma~_prsq + e_core."""
    return (float(np.einsum("pq,pq->", h, gamma))
            + 0.5 * float(np.einsum("pqrs,prsq->", eri, Gamma)) + e_core)


# ---------- spin-coupled RDMs by direct operator evaluation ----------

def _mode(p, up):
    return 2 * p + (0 if up else 1)


class _Op:
    """Sum of products of single-mode fermion operators, applied to vectors.

    A term is (coef, [(mode, dagger), ...]) acting right-to-left as written
    (the last factor acts first).
    """

    def __init__(self, n):
        self.n = n
        self.terms = []

    def add(self, coef, factors):
        if coef != 0.0:
            self.terms.append((coef, factors))


def _apply_factor(n, idx, amp, mode, dagger):
    occ = mode_occupations(digits(idx, n))
    want = 0 if dagger else 1
    ok = occ[:, mode] == want
    idx, amp, occ = idx[ok], amp[ok], occ[ok]
    sign = np.where(occ[:, :mode].sum(1) % 2 == 0, 1.0, -1.0)
    p, spin = divmod(mode, 2)
    val = (2 if spin == 0 else 1) * 4 ** (n - 1 - p)
    idx = idx + val if dagger else idx - val
    return idx, amp * sign


def expectation(n, states, psi, op: _Op):
    """<psi| op |psi> for a vector on the sorted full indices ``states``."""
    total = 0.0
    for coef, factors in op.terms:
        idx, amp = states.copy(), psi.copy()
        for mode, dag in reversed(factors):
            idx, amp = _apply_factor(n, idx, amp, mode, dag)
            if idx.size == 0:
                break
        if idx.size == 0:
            continue
        j = np.searchsorted(states, idx)
        j = np.minimum(j, len(states) - 1)
        hit = states[j] == idx
        total += coef * float(np.dot(psi[j[hit]], amp[hit]))
    return total


def _fdag(p, comp):
    """Component comp (0 -> m=+1/2, 1 -> m=-1/2) of f+_p: (a+_up, a+_dn)."""
    return [(1.0, (_mode(p, comp == 0), True))]


def _f(p, comp):
    """Component of f_p = (a_dn, -a_up)."""
    return [(1.0, (_mode(p, False), False))] if comp == 0 else [(-1.0, (_mode(p, True), False))]


def _couple(A, B, k2, q2):
    """[A B]^k_q for spin-1/2 tensors A, B given as component lists.

    A[c], B[c]: list of (coef, factors) for components c (0: m=+1/2, 1: -1/2).
    Returns a list of (coef, factors).
    """
    out = []
    for ca, ma in ((0, 1), (1, -1)):
        for cb, mb in ((0, 1), (1, -1)):
            c = cg(1, ma, 1, mb, k2, q2)
            if c == 0.0:
                continue
            for xa, fa in A[ca]:
                for xb, fb in B[cb]:
                    out.append((c * xa * xb, list(fa) + list(fb)))
    return out


def _couple_scalar(X, Y, k2):
    """[X^k Y^k]^0 with X[q], Y[q] given per projection q2 in {-k2..k2}."""
    out = []
    for q2 in range(-k2, k2 + 1, 2):
        c = cg(k2, q2, k2, -q2, 0, 0)
        for xa, fa in X[q2]:
            for xb, fb in Y[-q2]:
                out.append((c * xa * xb, list(fa) + list(fb)))
    return out


def _spinor(fun, p):
    return {0: [(c, [f]) for c, f in fun(p, 0)], 1: [(c, [f]) for c, f in fun(p, 1)]}


def gamma_su2(n, states, psi, p, q):
    """gamma_pq = <[f+_p f_q]_0> (Eq. rdm1_su2)."""
    op = _Op(n)
    for c, fac in _couple(_spinor(_fdag, p), _spinor(_f, q), 0, 0):
        op.add(c, fac)
    return expectation(n, states, psi, op)


def Gamma_su2(n, states, psi, p, q, r, s, k2):
    """Gamma^(k)_pqrs = <[[f+_p f+_q]_k [f_r f_s]_k]_0> for k = k2/2 in {0, 1}."""
    X = {q2: _couple(_spinor(_fdag, p), _spinor(_fdag, q), k2, q2) for q2 in range(-k2, k2 + 1, 2)}
    Y = {q2: _couple(_spinor(_f, r), _spinor(_f, s), k2, q2) for q2 in range(-k2, k2 + 1, 2)}
    op = _Op(n)
    for c, fac in _couple_scalar(X, Y, k2):
        op.add(c, fac)
    return expectation(n, states, psi, op)


def spin_free_from_su2(gamma_c, Gamma0, Gamma1, c1):
    """Spin-free RDMs from the coupled ones: gamma~ = -sqrt(2) gamma and
    Gamma~ = c1 Gamma^(1) - Gamma^(0) (the paper prints c1 = 2 sqrt(3))."""
    return -np.sqrt(2.0) * gamma_c, c1 * Gamma1 - Gamma0
