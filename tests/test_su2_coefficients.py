"""The library's SU(2) coefficients (csrc/su2.cpp: Racah closed forms for
Clebsch-Gordan and 6j, the 9j as a sum of 6j's, and the tensor-product
coefficient of two coupled subsystems) against sympy's exact values, on the
CPU.  Every case is evaluated twice, so the memoised value is checked too.

The tensor-product coefficient of [X^{kx} (x) Y^{ky}]^k between |(j1' j2') J'>
and |(j1 j2) J> is sqrt((J+1)(k+1)(j1'+1)(j2'+1)) times the 9j symbol
{j1' j1 kx; j2' j2 ky; J' J k} (doubled arguments)."""
import os
import random
import shutil
import subprocess

import pytest

sympy = pytest.importorskip("sympy")
from sympy import Rational, sqrt  # noqa: E402
from sympy.physics.wigner import clebsch_gordan, wigner_6j, wigner_9j  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2503_20700_gb300", "csrc")


def h(x):
    return Rational(x, 2)


def exact(f, *args):
    """sympy's value; zero where it rejects the arguments (an odd doubled sum
    or a broken triangle), which is where the symbols vanish."""
    try:
        return f(*args)
    except ValueError:
        return 0


def tri(a, b, c):
    return abs(a - b) <= c <= a + b and (a + b + c) % 2 == 0


def draw(rng, n, hi, ok, tries=2000):
    """n doubled spins below hi; mostly drawn until ok(...) holds (nonzero
    symbols), one in five left as drawn (zeros from broken triangles)."""
    v = [rng.randrange(0, hi) for _ in range(n)]
    if rng.random() < 0.2:
        return v
    for _ in range(tries):
        if ok(v):
            return v
        v = [rng.randrange(0, hi) for _ in range(n)]
    return v


def cases(seed=11):
    rng = random.Random(seed)
    out = []
    ok6 = lambda a: tri(a[0], a[1], a[2]) and tri(a[0], a[4], a[5]) and tri(a[3], a[1], a[5]) and tri(a[3], a[4], a[2])
    ok9 = lambda a: (tri(a[0], a[1], a[2]) and tri(a[3], a[4], a[5]) and tri(a[6], a[7], a[8]) and
                     tri(a[0], a[3], a[6]) and tri(a[1], a[4], a[7]) and tri(a[2], a[5], a[8]))
    for _ in range(120):
        a = draw(rng, 6, 9, ok6)
        out.append(("6j", a, float(exact(wigner_6j, *map(h, a)))))
    for _ in range(40):
        a = draw(rng, 9, 6, ok9, tries=20000)
        out.append(("9j", a, float(exact(wigner_9j, *map(h, a)))))
    for _ in range(120):
        j1, j2, J = draw(rng, 3, 9, lambda v: tri(*v))
        m1 = rng.randrange(-j1, j1 + 1, 2) if j1 else 0
        m2 = rng.randrange(-j2, j2 + 1, 2) if j2 else 0
        M = m1 + m2 if rng.random() < 0.8 else m1 + m2 + 2
        out.append(("cg", [j1, m1, j2, m2, J, M], float(exact(clebsch_gordan, h(j1), h(j2), h(J), h(m1), h(m2), h(M)))))
    # tensor-product coefficients with the site/block spins of the sweep:
    # block spins up to 3, site spins 0 or 1/2, operator ranks 0, 1/2, 1
    for _ in range(80):
        def okt(v):
            return ok9(v) and v[4] in (0, 1) and v[3] in (0, 1) and v[2] <= 2 and v[5] <= 2 and v[8] <= 2
        v = draw(rng, 9, 7, okt, tries=20000)
        j1p, j1, kx, j2p, j2, ky, Jp, J, k = v
        val = sqrt((J + 1) * (k + 1) * (j1p + 1) * (j2p + 1)) * exact(wigner_9j, *map(h, v))
        out.append(("tp", v, float(val)))
    # repeats (memo hits)
    out += out[:30]
    return out


def test_su2_coefficients_against_sympy(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "su2_check")
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", CSRC, os.path.join(ROOT, "tests", "cpp", "su2_check.cpp"),
                    os.path.join(CSRC, "su2.cpp"), "-o", exe], check=True, timeout=300)
    cs = cases()
    assert sum(1 for _, _, x in cs if x != 0.0) > 150  # the cases are not all trivial zeros
    text = "\n".join(f"{k} {' '.join(map(str, a))} {x!r}" for k, a, x in cs) + "\n"
    r = subprocess.run([exe], input=text, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
