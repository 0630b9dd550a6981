"""Ab initio Hamiltonian on full-space vectors and exact diagonalisation.

Oracle (test infrastructure only).  Follows Sec. II.A: H = sum_pq h_pq e_pq
+ sum_pqrs V_pqrs e_pqrs with e_pq = sum_s a+_ps a_qs.  The paper's e_pqrs
pairs V with a+_p a+_q a_r a_s; with chemists' integrals (pq|rs) this is the
standard H = sum h_pq E_pq + 1/2 sum (pq|rs) (E_pq E_rs - delta_qr E_ps),
i.e. V_pqrs = 1/2 (ps|qr) in the paper's operator order (the reading of the
garbled normalisation that the tests pin through E(FCI) = <H> from RDMs).

The spin-adapted target is handled by working in the Sz = S sector and
projecting onto total spin S with the Loewdin projector
    P_S = prod_{S' > S} (S^2 - S'(S'+1)) / (S(S+1) - S'(S'+1)).
"""
from __future__ import annotations

import numpy as np

from .fock import SectorOps


class Hamiltonian:
    """H applied inside one (N, 2Sz) sector of the full Fock space."""

    def __init__(self, h, eri, n_elec, two_m, e_core=0.0):
        h = np.asarray(h, dtype=np.float64)
        eri = np.asarray(eri, dtype=np.float64)
        self.n = h.shape[0]
        self.h, self.eri, self.e_core = h, eri, float(e_core)
        self.ops = SectorOps(self.n, n_elec, two_m)
        self.dim = self.ops.dim
        # K_pq = h_pq - 1/2 sum_r (pr|rq)
        self.k = h - 0.5 * np.einsum("prrq->pq", eri)
        self.v = eri.reshape(self.n * self.n, self.n * self.n)

    def apply(self, x):
        """H x (electronic part, without e_core).  x: (dim,) or (dim, m)."""
        n = self.n
        ops = self.ops
        phi = np.zeros((n * n,) + x.shape)
        for r in range(n):
            for s in range(n):
                ops.apply_e(r, s, x, phi[r * n + s])
        chi = np.tensordot(self.v, phi, axes=(1, 0))  # chi_pq = sum_rs (pq|rs) phi_rs
        y = np.zeros_like(x)
        for p in range(n):
            for q in range(n):
                t = 0.5 * chi[p * n + q] + self.k[p, q] * x
                ops.apply_e(p, q, t, y)
        return y


def spin_projector(ops: SectorOps, two_s: int, n_max_spin2: int):
    """Return f(x) applying the Loewdin projector onto spin S = two_s/2."""
    s = 0.5 * two_s
    factors = []
    sp = two_s + 2
    while sp <= n_max_spin2:
        s1 = 0.5 * sp
        factors.append(s1 * (s1 + 1.0))
        sp += 2

    def proj(x):
        y = x
        for f in factors:
            y = (ops.apply_s2(y) - f * y) / (s * (s + 1.0) - f)
        return y
    return proj


def davidson(apply, diag, x0, tol=1e-10, max_iter=500, max_space=24, project=None):
    """Lowest eigenpair of a symmetric operator by Davidson's method (FP64).

    ``apply(X)`` maps (dim, m) -> (dim, m); ``diag`` is the diagonal used in
    the preconditioner (or None); ``project`` (optional) is applied to every
    new search direction (spin projection).  Convergence: ||H x - E x|| < tol
    with ||x|| = 1.  Returns (E, x, n_iter).
    """
    x = np.array(x0, dtype=np.float64)
    if project is not None:
        x = project(x)
    nrm = np.linalg.norm(x)
    if nrm == 0:
        raise ValueError("zero initial vector")
    V = (x / nrm)[:, None]
    HV = apply(V)
    e = None
    for it in range(1, max_iter + 1):
        A = V.T @ HV
        A = 0.5 * (A + A.T)
        w, u = np.linalg.eigh(A)
        e = w[0]
        c = u[:, 0]
        x = V @ c
        hx = HV @ c
        r = hx - e * x
        rn = np.linalg.norm(r)
        if rn < tol:
            return e, x, it
        if V.shape[1] >= max_space:
            # thick restart with the two lowest Ritz vectors
            keep = u[:, :2]
            V = V @ keep
            HV = HV @ keep
            q, rr = np.linalg.qr(V)
            V = q
            HV = HV @ np.linalg.inv(rr)
        if diag is not None:
            den = diag - e
            den[np.abs(den) < 1e-8] = 1e-8
            t = r / den
        else:
            t = r.copy()
        if project is not None:
            t = project(t)
        for _ in range(2):
            t -= V @ (V.T @ t)
        tn = np.linalg.norm(t)
        if tn < 1e-14:
            t = r - V @ (V.T @ r)
            tn = np.linalg.norm(t)
            if tn < 1e-14:
                return e, x, it
        t /= tn
        V = np.concatenate([V, t[:, None]], axis=1)
        HV = np.concatenate([HV, apply(t[:, None])], axis=1)
    raise RuntimeError(f"Davidson did not converge (residual {rn:.3e})")


def fci(h, eri, n_elec, two_s=0, e_core=0.0, tol=1e-10, seed=0):
    """Exact ground state of spin S = two_s/2.  Returns (E_total, x, H).

    ``x`` is the normalised ground state in the Sz = S sector (ordering of
    ``H.ops.states``).
    """
    H = Hamiltonian(h, eri, n_elec, two_s, e_core)
    n = H.n
    proj = spin_projector(H.ops, two_s, min(n_elec, 2 * n - n_elec))
    diag = _diagonal(H)
    rng = np.random.default_rng(seed)
    x0 = rng.standard_normal(H.dim) + 0.1
    e, x, _ = davidson(lambda X: H.apply(X), diag, x0, tol=tol, project=proj)
    return e + H.e_core, x, H


def _diagonal(H: Hamiltonian):
    """Diagonal of H in the determinant basis (for preconditioning only)."""
    from .fock import digits, mode_occupations
    occ = mode_occupations(digits(H.ops.states, H.n)).astype(np.float64)
    nu, nd = occ[:, 0::2], occ[:, 1::2]
    ntot = nu + nd
    d = ntot @ np.diag(H.h)
    J = np.einsum("ppqq->pq", H.eri)
    K = np.einsum("pqqp->pq", H.eri)
    d += 0.5 * np.einsum("sp,pq,sq->s", ntot, J, ntot)
    d -= 0.5 * np.einsum("sp,pq,sq->s", nu, K, nu) + 0.5 * np.einsum("sp,pq,sq->s", nd, K, nd)
    return d
