"""Fock space of n spatial orbitals (oracle; test infrastructure only).

Basis and ordering.  Each site p carries a digit d_p in {0,1,2,3}: 0 empty,
1 one spin-down electron, 2 one spin-up electron, 3 doubly occupied (the site
labelling of Sec. II.B).  A basis state has full index
    idx = sum_p d_p 4^(n-1-p)
(site 0 most significant, so a left block of sites 0..a-1 times a right block
is a Kronecker product in numpy C order).  The state is
    prod_{modes in order} (a+_mode)^(occ) |vac>
with the mode order (0 up, 0 down, 1 up, 1 down, ...), i.e. Jordan-Wigner
ordering by site, up before down within a site.
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np


def digits(idx: np.ndarray, n: int) -> np.ndarray:
    """Digits d_p of full indices, shape (len(idx), n)."""
    idx = np.asarray(idx, dtype=np.int64)
    out = np.empty((idx.size, n), dtype=np.int64)
    rem = idx.copy()
    for p in range(n - 1, -1, -1):
        out[:, p] = rem % 4
        rem //= 4
    return out


def mode_occupations(dig: np.ndarray) -> np.ndarray:
    """Occupations of the 2n modes in Jordan-Wigner order, shape (S, 2n)."""
    s, n = dig.shape
    occ = np.empty((s, 2 * n), dtype=np.int64)
    occ[:, 0::2] = (dig >> 1) & 1   # up
    occ[:, 1::2] = dig & 1          # down
    return occ


def quantum_numbers(idx: np.ndarray, n: int):
    """(N, 2*Sz) of full-space basis states."""
    occ = mode_occupations(digits(idx, n))
    nu = occ[:, 0::2].sum(1)
    nd = occ[:, 1::2].sum(1)
    return nu + nd, nu - nd


@lru_cache(maxsize=None)
def sector(n: int, n_elec: int, two_m: int) -> np.ndarray:
    """Sorted full indices of all states with N = n_elec and 2*Sz = two_m."""
    if (n_elec + two_m) % 2 or abs(two_m) > n_elec:
        return np.zeros(0, dtype=np.int64)
    n_up = (n_elec + two_m) // 2
    n_dn = (n_elec - two_m) // 2
    if n_up < 0 or n_dn < 0 or n_up > n or n_dn > n:
        return np.zeros(0, dtype=np.int64)
    # enumerate all 4^n states in chunks (n <= 12 in practice)
    total = 4 ** n
    keep = []
    chunk = 1 << 20
    for start in range(0, total, chunk):
        idx = np.arange(start, min(total, start + chunk), dtype=np.int64)
        nn, mm = quantum_numbers(idx, n)
        keep.append(idx[(nn == n_elec) & (mm == two_m)])
    return np.concatenate(keep)


def _mode_value(n: int, mode: int) -> int:
    p, spin = divmod(mode, 2)
    return (2 if spin == 0 else 1) * 4 ** (n - 1 - p)


class OneBodyMap:
    """Action of a+_{mode_c} a_{mode_a} from sector ``src`` into ``dst``.

    ``apply(x)`` returns y = (a+_c a_a) x with x indexed by ``src`` states and
    y by ``dst`` states.  Signs follow the Jordan-Wigner order above.
    """

    def __init__(self, n, src, dst, mode_c, mode_a):
        occ = mode_occupations(digits(src, n))
        ok = occ[:, mode_a] == 1
        occ2 = occ.copy()
        occ2[:, mode_a] = 0
        if mode_c != mode_a:
            ok &= occ2[:, mode_c] == 0
        pos = np.nonzero(ok)[0]
        # sign of a_a: parity of occupied modes before mode_a
        s1 = occ[pos, :mode_a].sum(1)
        occ2 = occ2[pos]
        s2 = occ2[:, :mode_c].sum(1)
        sign = np.where((s1 + s2) % 2 == 0, 1.0, -1.0)
        new = src[pos] - _mode_value(n, mode_a) + _mode_value(n, mode_c)
        j = np.searchsorted(dst, new)
        assert np.all(dst[np.minimum(j, len(dst) - 1)] == new)
        self.src_pos = pos
        self.dst_pos = j
        self.sign = sign

    def apply_add(self, x, y, coef=1.0):
        """y += coef * (a+_c a_a) x (rows of 2-D arrays are states)."""
        if self.src_pos.size:
            if x.ndim == 1:
                y[self.dst_pos] += coef * self.sign * x[self.src_pos]
            else:
                y[self.dst_pos] += (coef * self.sign)[:, None] * x[self.src_pos]


class SectorOps:
    """E_pq maps inside one (N, 2Sz) sector and S+ into the next sector."""

    def __init__(self, n: int, n_elec: int, two_m: int):
        self.n, self.n_elec, self.two_m = n, n_elec, two_m
        self.states = sector(n, n_elec, two_m)
        self.dim = len(self.states)
        self._e = {}
        self._sp = None

    def e_maps(self, p, q):
        key = (p, q)
        if key not in self._e:
            self._e[key] = [OneBodyMap(self.n, self.states, self.states, 2 * p + s, 2 * q + s)
                            for s in (0, 1)]
        return self._e[key]

    def apply_e(self, p, q, x, y=None, coef=1.0):
        """y += coef * E_pq x  with E_pq = sum_s a+_ps a_qs."""
        if y is None:
            y = np.zeros_like(x)
        for m in self.e_maps(p, q):
            m.apply_add(x, y, coef)
        return y

    def splus_maps(self):
        """Maps of a+_{p up} a_{p down} from this sector to (N, 2Sz + 2)."""
        if self._sp is None:
            dst = sector(self.n, self.n_elec, self.two_m + 2)
            self._sp = (dst, [OneBodyMap(self.n, self.states, dst, 2 * p, 2 * p + 1)
                              for p in range(self.n)]) if len(dst) else (dst, [])
        return self._sp

    def apply_splus(self, x):
        dst, maps = self.splus_maps()
        y = np.zeros((len(dst),) + x.shape[1:])
        for m in maps:
            m.apply_add(x, y)
        return y

    def apply_s2(self, x):
        """S^2 x = (S- S+ + Sz^2 + Sz) x inside the sector."""
        dst, maps = self.splus_maps()
        mz = 0.5 * self.two_m
        out = (mz * mz + mz) * x
        if maps:
            t = np.zeros((len(dst),) + x.shape[1:])
            for m in maps:
                m.apply_add(x, t)
            for m in maps:  # S- = (S+)^T for real matrices
                if m.src_pos.size:
                    if x.ndim == 1:
                        out[m.src_pos] += m.sign * t[m.dst_pos]
                    else:
                        out[m.src_pos] += m.sign[:, None] * t[m.dst_pos]
        return out

    def apply_sminus_from(self, upper: "SectorOps", x):
        """S- applied to a vector of the sector (N, 2Sz+2) given by ``upper``.

        ``upper`` must be the sector directly above this one; the result lives
        in this sector.  Uses S- = (S+)^T with S+ mapping self -> upper.
        """
        dst, maps = self.splus_maps()
        assert np.array_equal(dst, upper.states)
        out = np.zeros((self.dim,) + x.shape[1:])
        for m in maps:
            if m.src_pos.size:
                if x.ndim == 1:
                    out[m.src_pos] += m.sign * x[m.dst_pos]
                else:
                    out[m.src_pos] += m.sign[:, None] * x[m.dst_pos]
        return out


def full_splus_matrix(n: int):
    """S+ = sum_p a+_{p up} a_{p down} on the whole 4^n space as a scipy CSR."""
    import scipy.sparse as sp
    idx = np.arange(4 ** n, dtype=np.int64)
    rows, cols, vals = [], [], []
    for p in range(n):
        m = OneBodyMap(n, idx, idx, 2 * p, 2 * p + 1)
        rows.append(m.dst_pos)
        cols.append(m.src_pos)
        vals.append(m.sign)
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    return sp.csr_matrix((vals, (rows, cols)), shape=(4 ** n, 4 ** n))
