"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only *constructs inputs*: integrals of model Hamiltonians, and the
occupation pattern of the initial product state.  It holds none of the DMRG,
RDM or CAS-SCF arithmetic, so both the CPU oracle and the CUDA path may import
it without sharing method code.

Workloads (all energies returned in Hartree, integrals in chemists' notation
(pq|rs), row-major float64):

* ``ppp_acene(n_rings)`` -- Pariser-Parr-Pople model of the pi-system of a
  linear acene C_{4n+2}H_{2n+4} (naphthalene n=2: 10 sites, pentacene n=5:
  22 sites, icosacene n=20: 82 sites).  The paper studies this acene series
  with CAS(4n+2, 4n+2) active spaces (Sec. III, Fig. "pah"); the PPP model is
  the synthetic stand-in for its B3LYP/cc-pVDZ pi orbitals, which cannot be
  generated here.
* ``cholesky_random(n, rank, seed)`` -- random Cholesky-form active space:
  (pq|rs) = sum_k L^k_pq L^k_rs, 8-fold symmetric and positive semidefinite.
* ``initial_product_state(n, n_elec, two_s)`` -- occupations and the
  intermediate-spin path of the deterministic product state that starts the
  sweeps; ``aufbau_state(h, n_elec, two_s)`` the same for an occupation by
  orbital energy.
"""
from __future__ import annotations

import math

import numpy as np

HARTREE_EV = 27.211386245988          # CODATA 2018, eV per Hartree
COULOMB_EV_ANGSTROM = 14.397          # e^2 / (4 pi eps0) in eV * Angstrom
DEFAULT_SEED = 20250326

__all__ = [
    "HARTREE_EV", "DEFAULT_SEED", "acene_geometry", "ppp_integrals", "ppp_acene",
    "cholesky_random", "eri_from_cholesky", "initial_product_state",
    "aufbau_state", "spin_path", "hubbard_chain",
]


def acene_geometry(n_rings: int, bond: float = 1.40):
    """Carbon positions (Angstrom) of a linear acene with ideal hexagons.

    Rings share vertical edges and are fused along x.  Sites are ordered
    lexicographically in (x, y), i.e. zig-zag along the long axis.  Returns
    ``(xy, bonds)`` with ``bonds`` the list of site pairs at distance ``bond``.
    """
    if n_rings < 1:
        raise ValueError("n_rings must be >= 1")
    pts = []
    dx = math.sqrt(3.0) * bond
    for k in range(n_rings):
        cx = k * dx
        for a in range(6):
            ang = math.radians(30.0 + 60.0 * a)
            pts.append((round(cx + bond * math.cos(ang), 6),
                        round(bond * math.sin(ang), 6)))
    uniq = sorted(set(pts))
    xy = np.array(uniq, dtype=np.float64)
    assert len(xy) == 4 * n_rings + 2
    d = np.linalg.norm(xy[:, None, :] - xy[None, :, :], axis=-1)
    bonds = [(i, j) for i in range(len(xy)) for j in range(i + 1, len(xy))
             if abs(d[i, j] - bond) < 1e-4]
    return xy, bonds


def ppp_integrals(xy, bonds, t_ev: float = -2.4, u_ev: float = 11.26):
    """PPP Hamiltonian as (h, eri, e_core) in Hartree.

    H = sum_<ij>,s t c+_is c_js + U sum_i n_i^up n_i^dn
        + 1/2 sum_{i!=j} V_ij (n_i - 1)(n_j - 1),
    with the Ohno potential V_ij = U / sqrt(1 + (U r_ij / 14.397)^2).
    In integral form: (ii|ii) = U, (ii|jj) = V_ij, h_ij = t on bonds,
    h_ii = -sum_{j!=i} V_ij and e_core = 1/2 sum_{i!=j} V_ij.
    """
    n = len(xy)
    r = np.linalg.norm(xy[:, None, :] - xy[None, :, :], axis=-1)
    v = u_ev / np.sqrt(1.0 + (u_ev * r / COULOMB_EV_ANGSTROM) ** 2)
    h = np.zeros((n, n))
    for i, j in bonds:
        h[i, j] = h[j, i] = t_ev
    off = v.copy()
    np.fill_diagonal(off, 0.0)
    h[np.diag_indices(n)] = -off.sum(axis=1)
    eri = np.zeros((n, n, n, n))
    for i in range(n):
        for j in range(n):
            eri[i, i, j, j] = v[i, j]
    e_core = 0.5 * off.sum()
    return h / HARTREE_EV, eri / HARTREE_EV, e_core / HARTREE_EV


def ppp_acene(n_rings: int, t_ev: float = -2.4, u_ev: float = 11.26):
    """PPP integrals of the linear acene with ``n_rings`` rings (4n+2 sites)."""
    xy, bonds = acene_geometry(n_rings)
    return ppp_integrals(xy, bonds, t_ev, u_ev)


def hubbard_chain(n: int, t: float = -1.0, u: float = 4.0, periodic: bool = False):
    """Hubbard chain in integral form: h_{i,i+1} = t, (ii|ii) = U, e_core = 0."""
    h = np.zeros((n, n))
    for i in range(n - 1):
        h[i, i + 1] = h[i + 1, i] = t
    if periodic and n > 2:
        h[0, n - 1] = h[n - 1, 0] = t
    eri = np.zeros((n, n, n, n))
    for i in range(n):
        eri[i, i, i, i] = u
    return h, eri, 0.0


def cholesky_random(n: int, rank: int, seed: int = DEFAULT_SEED,
                    decay: float = 6.0, sigma_h: float = 0.5):
    """Random Cholesky-form active space ``(h, L)``.

    L^k_pq = s exp(-|p-q|/decay) (G + G^T)/sqrt(2) with G ~ N(0,1) i.i.d. and
    s = sqrt(0.5/rank) (so the mean (pp|pp) is about 0.5 Eh);
    h = sigma_h (H + H^T)/sqrt(2) with H ~ N(0,1), plus a diagonal shift
    linspace(-2, -0.5, n) Eh (lowest orbital first).  ``L`` has shape
    (rank, n, n), each L^k symmetric, so (pq|rs) = sum_k L^k_pq L^k_rs is
    8-fold symmetric and positive semidefinite.
    """
    rng = np.random.default_rng(seed)
    hh = rng.standard_normal((n, n))
    h = sigma_h * (hh + hh.T) / math.sqrt(2.0)
    h[np.diag_indices(n)] += np.linspace(-2.0, -0.5, n)
    p = np.arange(n)
    env = np.exp(-np.abs(p[:, None] - p[None, :]) / decay)
    g = rng.standard_normal((rank, n, n))
    s = math.sqrt(0.5 / rank)
    L = s * env[None, :, :] * (g + g.transpose(0, 2, 1)) / math.sqrt(2.0)
    return h, L


def eri_from_cholesky(L):
    """(pq|rs) = sum_k L^k_pq L^k_rs as a dense (n,n,n,n) array."""
    rank, n, _ = L.shape
    m = L.reshape(rank, n * n)
    return (m.T @ m).reshape(n, n, n, n)


def initial_product_state(n: int, n_elec: int, two_s: int):
    """Deterministic product state that starts the DMRG sweeps.

    Returns ``(occ, two_s_right)``: ``occ[p]`` in {0, 1, 2} is the occupation
    of site p, and ``two_s_right[i]`` (length n+1) is twice the spin of the
    block of sites i..n-1 when the sites are coupled one by one from the right
    end (site i coupled in front of the block i+1..n-1), with
    ``two_s_right[n] = 0`` and ``two_s_right[0] = two_s``.

    Electrons are spread as evenly as possible: with n_elec <= n the first
    n_elec sites are singly occupied; otherwise the first n_elec - n sites are
    doubly occupied and the rest singly.  Scanning from the right end, the
    singly occupied sites first couple up to the target spin, then alternate
    (S+1/2, S, S+1/2, ...), so every intermediate spin is as small as the
    path allows.  Each right block of this state is a single SU(2) multiplet.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    if not (0 <= n_elec <= 2 * n):
        raise ValueError("n_elec out of range")
    if two_s < 0 or (n_elec - two_s) % 2 != 0:
        raise ValueError("two_s has the wrong parity for n_elec")
    if n_elec <= n:
        occ = [1] * n_elec + [0] * (n - n_elec)
    else:
        occ = [2] * (n_elec - n) + [1] * (2 * n - n_elec)
    return occ, spin_path(occ, two_s)


def aufbau_state(h, n_elec: int, two_s: int):
    """Closed-shell-like product state by orbital energy (``occ``, ``two_s_right``).

    The orbitals with the lowest diagonal one-electron integrals h_pp take the
    electrons: (n_elec - two_s)/2 of them doubly occupied, the next two_s
    singly occupied (ties by orbital index).  Sites keep their chain order;
    only the occupation pattern follows h_pp.  For the random Cholesky active
    spaces, whose h_pp grow along the chain on average, this start is near the
    ground state's charge distribution, where the even-spread state puts one
    electron on every orbital and leaves the sweeps to move charge between the
    halves of the chain one bond at a time.
    """
    d = np.asarray(np.diag(h), dtype=np.float64)
    n = d.size
    if not (0 <= n_elec <= 2 * n) or two_s < 0 or (n_elec - two_s) % 2 != 0:
        raise ValueError("bad n_elec / two_s")
    n_double = (n_elec - two_s) // 2
    if n_double + two_s > n:
        raise ValueError("two_s too large for this filling")
    order = sorted(range(n), key=lambda p: (d[p], p))
    occ = [0] * n
    for p in order[:n_double]:
        occ[p] = 2
    for p in order[n_double:n_double + two_s]:
        occ[p] = 1
    return occ, spin_path(occ, two_s)


def spin_path(occ, two_s: int):
    """Doubled spins of the right blocks of a product state (length n+1).

    Scanning from the right end, the singly occupied sites first couple up to
    the target spin, then alternate (S+1/2, S, S+1/2, ...), so every
    intermediate spin is as small as the path allows."""
    n = len(occ)
    n_single = sum(1 for o in occ if o == 1)
    if two_s > n_single or (n_single - two_s) % 2 != 0:
        raise ValueError("two_s not reachable from this occupation")
    path = [0] * (n + 1)
    seen = 0
    cur = 0
    for i in range(n - 1, -1, -1):
        if occ[i] == 1:
            seen += 1
            if seen <= two_s:
                cur += 1
            else:
                cur = cur + 1 if cur == two_s else cur - 1
        path[i] = cur
    assert path[0] == two_s, (path, two_s)
    return path
