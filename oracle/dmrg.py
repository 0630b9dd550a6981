"""Spin-adapted two-site DMRG as a plain subspace method (oracle).

TEST INFRASTRUCTURE ONLY.  Written from Sec. II.B-D of the paper (MPS ansatz,
DMRG as variational minimisation over MPS, D counted in SU(2) multiplets) in
its most direct form, with no recoupling coefficients and no renormalised
operators:

* A left block basis (sites 0..a-1) is stored as explicit vectors of the
  4^a-dimensional Fock space of those sites; a right block basis likewise.
  Each basis is a set of complete SU(2) multiplets (all 2j+1 components).
* At bond (i, i+1) the two-site subspace is  L(0..i-1) x site i x site i+1 x
  R(i+2..n-1).  Its vectors are embedded into the full Fock space, the
  Hamiltonian of ``fci.Hamiltonian`` is applied there and the result is
  projected back: H_eff = P^T H P.  The lowest spin-S eigenpair is found by
  Davidson (residual ||H_eff c - E c|| < tol, Sec. II.D) with every search
  direction projected onto spin S.
* Decimation: the spin-averaged reduced density matrix of the enlarged block
  (average over the 2S+1 components of the target multiplet) commutes with
  the block's total spin.  Its highest-weight eigenvectors (S+ v = 0,
  M = j) are found sector by sector; a multiplet's weight is
  lambda = (2j+1) w with w the per-state eigenvalue.  D multiplets are kept
  (the bond dimension counts multiplets, Sec. II.C) and expanded into all
  their components with S-.

Readings fixed here (the paper is silent on them):
* Initial state: the product state of ``workloads.initial_product_state``
  (or a given occupation and spin path, e.g. ``workloads.aufbau_state``),
  coupled from the right; every right block starts as one multiplet.
* Sweep: L->R over bonds 0..n-3 (truncating the left enlarged block after
  each), then R->L over bonds n-2..1 (truncating the right enlarged block).
  The sweep energy is the Davidson eigenvalue of the last bond.
* Selection: multiplets ranked by lambda (descending); lambda < 1e-12 dropped;
  exact ties (relative 1e-9) at the cut broken by (N asc, 2j asc, index asc).
  With a truncation-error target (dynamic block-state selection) the number
  kept is the fewest whose discarded weight is at most the target, clamped
  to [D_min, D].
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .fci import Hamiltonian, davidson
from .fock import SectorOps, full_splus_matrix, sector
from .su2 import cg

SITE_N = np.array([0, 1, 1, 2])          # electrons of site digits 0..3
SITE_2M = np.array([0, -1, 1, 0])        # 2*Sz of site digits
LAMBDA_MIN = 1e-12
TIE_REL = 1e-9


@dataclass
class Basis:
    """Explicit block basis: vecs[full_block_index, k] plus labels of column k."""
    vecs: np.ndarray
    n: np.ndarray        # electrons
    two_m: np.ndarray    # 2 Sz
    two_j: np.ndarray    # 2 S of the multiplet
    mult: np.ndarray     # multiplet id (columns of one multiplet share it)

    @property
    def m(self):
        return self.vecs.shape[1]

    def n_multiplets(self):
        return len(np.unique(self.mult))


def vacuum_basis():
    z = np.zeros(1, dtype=np.int64)
    return Basis(np.ones((1, 1)), z, z.copy(), z.copy(), z.copy())


_SPLUS_CACHE = {}


def _splus(nsites):
    if nsites not in _SPLUS_CACHE:
        _SPLUS_CACHE[nsites] = full_splus_matrix(nsites)
    return _SPLUS_CACHE[nsites]


def initial_right_bases(n, occ, two_s_right):
    """Right bases R(i) (sites i..n-1), i = 0..n, of the product state.

    R(i) is the single multiplet obtained by coupling site i (site first) to
    R(i+1) with Clebsch-Gordan coefficients.  Returns a list indexed by i.
    """
    out = [None] * (n + 1)
    out[n] = vacuum_basis()
    for i in range(n - 1, -1, -1):
        nxt = out[i + 1]
        j2 = two_s_right[i + 1]
        J2 = two_s_right[i]
        o = occ[i]
        if o == 1:
            site = [(1, 2), (-1, 1)]      # (2m, digit)
            s2 = 1
        else:
            site = [(0, 0 if o == 0 else 3)]
            s2 = 0
        dimn = nxt.vecs.shape[0]
        cols, ms = [], []
        for M2 in range(J2, -J2 - 1, -2):
            v = np.zeros(4 * dimn)
            for m2s, d in site:
                Mp = M2 - m2s
                if abs(Mp) > j2:
                    continue
                k = np.nonzero(nxt.two_m == Mp)[0]
                assert len(k) == 1
                c = cg(s2, m2s, j2, Mp, J2, M2)
                v[d * dimn:(d + 1) * dimn] += c * nxt.vecs[:, k[0]]
            v /= np.linalg.norm(v)
            cols.append(v)
            ms.append(M2)
        ne = int(nxt.n[0]) + o
        k = len(cols)
        out[i] = Basis(np.array(cols).T, np.full(k, ne), np.array(ms),
                       np.full(k, J2), np.zeros(k, dtype=np.int64))
    return out


@dataclass
class SweepRecord:
    energies: list = field(default_factory=list)       # per sweep
    trunc: list = field(default_factory=list)          # max discarded weight per sweep
    bond_energies: list = field(default_factory=list)  # (sweep, direction, bond, E)


class OracleDMRG:
    """Two-site SU(2) DMRG on explicit full-space block bases."""

    def __init__(self, h, eri, n_elec, two_s, D, e_core=0.0, tol=1e-10, occ=None, two_s_right=None,
                 trunc_target=0.0, D_min=1):
        from workloads import initial_product_state
        self.h = np.asarray(h, float)
        self.eri = np.asarray(eri, float)
        self.n = self.h.shape[0]
        if self.n < 2:
            raise ValueError("need at least two sites")
        self.n_elec, self.two_s, self.D = n_elec, two_s, D
        self.trunc_target, self.D_min = float(trunc_target), int(D_min)
        self.kept = []  # multiplets kept at each decimation, in sweep order
        self.e_core, self.tol = float(e_core), tol
        # one Hamiltonian per Sz component of the target multiplet
        self.ham = {tm: Hamiltonian(self.h, self.eri, n_elec, tm, e_core)
                    for tm in range(-two_s, two_s + 1, 2)}
        self.H = self.ham[two_s]
        self.states = self.H.ops.states
        if occ is None:
            occ, path = initial_product_state(self.n, n_elec, two_s)
        else:
            path = two_s_right
        self.right = initial_right_bases(self.n, list(occ), list(path))
        self.left = [None] * (self.n + 1)
        self.left[0] = vacuum_basis()
        full0 = self.right[0]
        k = int(np.nonzero(full0.two_m == two_s)[0][0])
        self.psi_full = full0.vecs[self.states, k].copy()
        self.energy = None
        self.record = SweepRecord()
        self.heff_flops = 0.0     # executed flops of the H_eff applications
        self.heff_seconds = 0.0
        self.heff_calls = 0

    # ----- embedding of the two-site subspace -----
    def _blocks(self, i):
        return self.left[i], self.right[i + 2]

    def _mask(self, L, R, two_m):
        nn = (L.n[:, None, None, None] + SITE_N[None, :, None, None]
              + SITE_N[None, None, :, None] + R.n[None, None, None, :])
        mm = (L.two_m[:, None, None, None] + SITE_2M[None, :, None, None]
              + SITE_2M[None, None, :, None] + R.two_m[None, None, None, :])
        return (nn == self.n_elec) & (mm == two_m)

    def _embed(self, L, R, c, states):
        t = np.einsum("la,aijb->lijb", L.vecs, c, optimize=True)
        t = np.einsum("lijb,rb->lijr", t, R.vecs, optimize=True)
        return t.reshape(-1)[states]

    def _project(self, L, R, x, states):
        full = np.zeros(4 ** self.n)
        full[states] = x
        t = full.reshape(L.vecs.shape[0], 4, 4, R.vecs.shape[0])
        t = np.einsum("lijr,rb->lijb", t, R.vecs, optimize=True)
        return np.einsum("lijb,la->aijb", t, L.vecs, optimize=True)

    def heff_apply(self, i, cvec):
        """H_eff c for bond i (electronic part), c given on the sector mask."""
        L, R = self._blocks(i)
        mask = self._mask(L, R, self.two_s)
        c = np.zeros(mask.shape)
        c[mask] = cvec
        y = self.H.apply(self._embed(L, R, c, self.states))
        return self._project(L, R, y, self.states)[mask]

    def _solve_bond(self, i):
        L, R = self._blocks(i)
        mask = self._mask(L, R, self.two_s)
        shape = mask.shape
        ops = self.H.ops
        n_max = min(self.n_elec, 2 * self.n - self.n_elec)
        S = 0.5 * self.two_s
        factors = [0.5 * sp * (0.5 * sp + 1.0) for sp in range(self.two_s + 2, n_max + 1, 2)]

        def embed(v):
            c = np.zeros(shape)
            c[mask] = v
            return self._embed(L, R, c, self.states)

        def proj(v):
            return self._project(L, R, v, self.states)[mask]

        n = self.n
        la, lb = L.vecs.shape[0], R.vecs.shape[0]
        ml, mr = L.vecs.shape[1], R.vecs.shape[1]
        # floating-point operations one application executes (embedding and
        # projection contractions, the E_pq maps and the integral contraction)
        nmap = sum(m.src_pos.size for p in range(n) for q in range(n)
                   for m in self.H.ops.e_maps(p, q))
        fl = (2 * (2.0 * la * ml * 16 * mr + 2.0 * la * 16 * mr * lb)
              + 2 * 2.0 * nmap + 2.0 * n ** 4 * self.H.dim)

        def apply(X):
            import time as _t
            t0 = _t.perf_counter()
            out = np.stack([proj(self.H.apply(embed(X[:, k]))) for k in range(X.shape[1])], 1)
            self.heff_seconds += _t.perf_counter() - t0
            self.heff_flops += fl * X.shape[1]
            self.heff_calls += X.shape[1]
            return out

        def spin_project(v):
            v = v.reshape(-1, 1) if v.ndim == 1 else v
            out = []
            for k in range(v.shape[1]):
                x = embed(v[:, k])
                for f in factors:
                    x = (ops.apply_s2(x) - f * x) / (S * (S + 1.0) - f)
                out.append(proj(x))
            o = np.stack(out, 1)
            return o[:, 0] if o.shape[1] == 1 else o

        c0 = proj(self.psi_full)
        if np.linalg.norm(c0) < 1e-8:
            c0 = np.ones(int(mask.sum()))
        e, cv, _ = davidson(apply, None, c0, tol=self.tol, project=spin_project)
        c = np.zeros(shape)
        c[mask] = cv
        self.psi_full = embed(cv)
        return e + self.e_core, c

    # ----- spin components of the two-site state -----
    def _components(self, i, c):
        """Coefficient tensors of all Sz components M = S..-S of the target."""
        L, R = self._blocks(i)
        comps = [c]
        x = self._embed(L, R, c, self.states)
        tm = self.two_s
        while tm > -self.two_s:
            lower = self.ham[tm - 2].ops
            upper = self.ham[tm].ops
            x = lower.apply_sminus_from(upper, x)
            x /= np.linalg.norm(x)
            comps.append(self._project(L, R, x, lower.states))
            tm -= 2
        return comps

    # ----- decimation -----
    def _decimate(self, enl_vecs, enl_n, enl_m, rho, nsites, D):
        """Select D multiplets of an enlarged block and build its new basis.

        enl_vecs: explicit enlarged-block basis (4^nsites x d); rho: spin-averaged
        density matrix in those coordinates.  Returns (Basis, discarded weight).
        """
        sp_full = _splus(nsites)
        Sp = enl_vecs.T @ (sp_full @ enl_vecs)      # S+ in enlarged coordinates
        cands = []
        for ne in np.unique(enl_n):
            for tm in np.unique(enl_m[enl_n == ne]):
                if tm < 0:
                    continue
                cols = np.nonzero((enl_n == ne) & (enl_m == tm))[0]
                rows = np.nonzero((enl_n == ne) & (enl_m == tm + 2))[0]
                if len(rows):
                    blk = Sp[np.ix_(rows, cols)]
                    u, s, vt = np.linalg.svd(blk)
                    rank = int((s > 1e-10).sum())
                    W = vt[rank:].T
                else:
                    W = np.eye(len(cols))
                if W.shape[1] == 0:
                    continue
                r = W.T @ rho[np.ix_(cols, cols)] @ W
                w, vec = np.linalg.eigh(0.5 * (r + r.T))
                order = np.argsort(-w, kind="stable")
                for rank_in, k in enumerate(order):
                    lam = (tm + 1) * w[k]
                    hw = np.zeros(len(enl_n))
                    hw[cols] = W @ vec[:, k]
                    cands.append((lam, int(ne), int(tm), rank_in, hw))
        total = sum(c[0] for c in cands)
        if self.trunc_target > 0.0:
            D = dbss_dimension([c[0] for c in cands], D, self.D_min, self.trunc_target)
        kept = select_multiplets([(c[0], c[1], c[2], c[3]) for c in cands], D)
        self.kept.append(len(kept))
        disc = total - sum(cands[k][0] for k in kept)
        vecs, nn, mm, jj, mid = [], [], [], [], []
        for mid_k, k in enumerate(kept):
            lam, ne, tj, _, hw = cands[k]
            v = hw
            for tm in range(tj, -tj - 1, -2):
                vecs.append(v)
                nn.append(ne)
                mm.append(tm)
                jj.append(tj)
                mid.append(mid_k)
                v = Sp.T @ v
                nv = np.linalg.norm(v)
                if tm > -tj:
                    v = v / nv
        V = np.array(vecs).T if vecs else np.zeros((len(enl_n), 0))
        basis = Basis(enl_vecs @ V, np.array(nn), np.array(mm), np.array(jj), np.array(mid))
        return basis, max(disc, 0.0)

    def _truncate_left(self, i, comps):
        L = self.left[i]
        enl_vecs = np.kron(L.vecs, np.eye(4))
        enl_n = (L.n[:, None] + SITE_N[None, :]).reshape(-1)
        enl_m = (L.two_m[:, None] + SITE_2M[None, :]).reshape(-1)
        d = enl_vecs.shape[1]
        rho = np.zeros((d, d))
        for c in comps:
            C = c.reshape(d, -1)
            rho += C @ C.T
        rho /= len(comps)
        self.left[i + 1], disc = self._decimate(enl_vecs, enl_n, enl_m, rho, i + 1, self.D)
        return disc

    def _truncate_right(self, i, comps):
        R = self.right[i + 2]
        enl_vecs = np.kron(np.eye(4), R.vecs)
        enl_n = (SITE_N[:, None] + R.n[None, :]).reshape(-1)
        enl_m = (SITE_2M[:, None] + R.two_m[None, :]).reshape(-1)
        d = enl_vecs.shape[1]
        rho = np.zeros((d, d))
        for c in comps:
            C = c.reshape(-1, d)
            rho += C.T @ C
        rho /= len(comps)
        self.right[i + 1], disc = self._decimate(enl_vecs, enl_n, enl_m, rho,
                                                 self.n - i - 1, self.D)
        return disc

    def sweep(self, n_sweeps=1, D=None):
        """Run full sweeps; returns the list of sweep energies (incl. e_core)."""
        if D is not None:
            self.D = D
        n = self.n
        for _ in range(n_sweeps):
            sw = len(self.record.energies)
            tmax = 0.0
            for i in range(0, n - 2):
                e, c = self._solve_bond(i)
                self.record.bond_energies.append((sw, "LR", i, e))
                tmax = max(tmax, self._truncate_left(i, self._components(i, c)))
            for i in range(n - 2, 0, -1):
                e, c = self._solve_bond(i)
                self.record.bond_energies.append((sw, "RL", i, e))
                tmax = max(tmax, self._truncate_right(i, self._components(i, c)))
            self.energy = e
            self.record.energies.append(e)
            self.record.trunc.append(tmax)
        return list(self.record.energies)

    def bond_dims(self):
        """Multiplet counts of the current left (0..n-2) and right bases."""
        return ([b.n_multiplets() if b is not None else None for b in self.left],
                [b.n_multiplets() if b is not None else None for b in self.right])


def dbss_dimension(lams, D_max, D_min, target):
    """Dynamic block-state selection (Sec. II.D, fixed truncation error): the
    fewest multiplets, taken in decreasing weight, whose discarded weight
    sum(lams) - sum(kept) is at most `target`, clamped to [D_min, D_max]."""
    lams = sorted(lams, reverse=True)
    total = sum(lams)
    kept, k = 0.0, 0
    while k < len(lams) and total - kept > target:
        kept += lams[k]
        k += 1
    return max(D_min, min(D_max, k))


def select_multiplets(cands, D):
    """Indices of the kept multiplets.  cands: list of (lambda, N, 2j, rank)."""
    idx = [k for k, c in enumerate(cands) if c[0] >= LAMBDA_MIN]
    idx.sort(key=lambda k: (-cands[k][0], cands[k][1], cands[k][2], cands[k][3]))
    if len(idx) <= D:
        return idx
    lam_d = cands[idx[D - 1]][0]
    hi = [k for k in idx if cands[k][0] > lam_d * (1 + TIE_REL)]
    tie = [k for k in idx if abs(cands[k][0] - lam_d) <= lam_d * TIE_REL]
    tie.sort(key=lambda k: (cands[k][1], cands[k][2], cands[k][3]))
    return hi + tie[:D - len(hi)]


