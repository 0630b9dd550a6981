"""Clebsch-Gordan coefficients (oracle; test infrastructure only).

Racah's closed form for <j1 m1 j2 m2 | J M> in the Condon-Shortley phase
convention, with all angular momenta passed as twice their value (integers).
The oracle uses it only to build the explicit spin multiplet of the initial
product state (Sec. II.C: SU(2)-adapted MPS); the tests also use it to pin the
recoupling coefficients of the CUDA path by brute-force sums over m.
"""
from __future__ import annotations

from functools import lru_cache
from math import factorial, sqrt


def _f(x2: int) -> int:
    """factorial of x where x2 = 2x must be even and non-negative."""
    assert x2 % 2 == 0 and x2 >= 0, x2
    return factorial(x2 // 2)


@lru_cache(maxsize=None)
def cg(j1: int, m1: int, j2: int, m2: int, J: int, M: int) -> float:
    """<j1/2 m1/2, j2/2 m2/2 | J/2 M/2> (arguments doubled)."""
    if m1 + m2 != M:
        return 0.0
    if abs(m1) > j1 or abs(m2) > j2 or abs(M) > J:
        return 0.0
    if (j1 + m1) % 2 or (j2 + m2) % 2 or (J + M) % 2:
        return 0.0
    if J < abs(j1 - j2) or J > j1 + j2 or (j1 + j2 + J) % 2:
        return 0.0
    pref = (J + 1) * _f(J + j1 - j2) * _f(J - j1 + j2) * _f(j1 + j2 - J) / _f(j1 + j2 + J + 2)
    pref *= _f(J + M) * _f(J - M) * _f(j1 - m1) * _f(j1 + m1) * _f(j2 - m2) * _f(j2 + m2)
    s = 0.0
    k = 0
    while True:
        a = j1 + j2 - J - 2 * k
        b = j1 - m1 - 2 * k
        c = j2 + m2 - 2 * k
        d = J - j2 + m1 + 2 * k
        e = J - j1 - m2 + 2 * k
        if a < 0 or b < 0 or c < 0:
            break
        if d >= 0 and e >= 0:
            s += (-1) ** k / (factorial(k) * _f(a) * _f(b) * _f(c) * _f(d) * _f(e))
        k += 1
    return sqrt(pref) * s


def wigner6j_bruteforce(j1, j2, j3, j4, j5, j6) -> float:
    """{j1 j2 j3; j4 j5 j6} (doubled) from a sum of four CG products over m.

    Uses the defining relation of the 6j symbol as the overlap of two coupling
    schemes of three angular momenta:
        <(j1 j2)j3, j4; j5 | j1, (j2 j4)j6; j5>
          = (-1)^(j1+j2+j4+j5) sqrt((2j3+1)(2j6+1)) {j1 j2 j3; j4 j5 j6}.
    The overlap is evaluated by summing CG products over all projections
    (slow, test use only).
    """
    def tri(a, b, c):
        return abs(a - b) <= c <= a + b and (a + b + c) % 2 == 0
    if not (tri(j1, j2, j3) and tri(j1, j5, j6) and tri(j4, j2, j6) and tri(j4, j5, j3)):
        return 0.0
    M = j5
    ov = 0.0
    for m1 in range(-j1, j1 + 1, 2):
        for m2 in range(-j2, j2 + 1, 2):
            m4 = M - m1 - m2
            if abs(m4) > j4:
                continue
            m3 = m1 + m2
            m6 = m2 + m4
            if abs(m3) > j3 or abs(m6) > j6:
                continue
            a = cg(j1, m1, j2, m2, j3, m3) * cg(j3, m3, j4, m4, j5, M)
            b = cg(j2, m2, j4, m4, j6, m6) * cg(j1, m1, j6, m6, j5, M)
            ov += a * b
    ph = (j1 + j2 + j4 + j5) // 2
    return ov * (-1) ** ph / sqrt((j3 + 1) * (j6 + 1))
