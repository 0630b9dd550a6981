"""The C-ABI library builds, loads and exports every declared entry point.

No compute call is made here (this suite also runs on machines without a
GPU); argument validation paths that return before touching the device are
exercised.
"""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import paper_2503_20700_gb300 as p
    from paper_2503_20700_gb300 import build as b
    if not os.path.exists(p.lib_path()):
        b.build()
    return p.load()


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(\w+)\s*\([^;{]*\)\s*;", txt)
    return sorted(set(n for n in names if n.startswith(("dmrg_", "casscf_"))))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "dmrg_init" in names and "dmrg_grouped_gemm" in names
    for n in names:
        assert hasattr(lib, n), n


def test_library_links_no_host_fallback():
    """The product library links only the CUDA backend (no host compute path)."""
    import paper_2503_20700_gb300 as p
    out = subprocess.run(["nm", "-DC", p.lib_path()], capture_output=True, text=True).stdout
    assert "CpuBackend" not in out


def test_init_validates_before_touching_the_device(lib):
    import paper_2503_20700_gb300 as p
    h = np.zeros((4, 4))
    eri = np.zeros((4, 4, 4, 4))
    for kw in [dict(n_elec=4, two_s=1), dict(n_elec=9), dict(n_elec=4, two_s=-2)]:
        with pytest.raises(p.DmrgError) as ei:
            p.DMRG(h, eri=eri, **kw)
        assert ei.value.status == p.DMRG_EINVAL


def test_default_opts(lib):
    import paper_2503_20700_gb300 as p
    o = p.Opts()
    lib.dmrg_default_opts(ctypes.byref(o))
    assert o.D == 64 and o.precision == 0 and o.davidson_tol == 1e-10


def test_schedule_candidates_listed_without_a_device(lib):
    """The autotuner's candidate schedules of the tcgen05 launch are host data:
    the default (256-wide tiles, four item chunks per CTA, longest first,
    clusters of two) comes first, every tile width is a multiple of 16 up to
    256, clusters have two or four CTAs, and the kernel-level shape setter
    rejects an index outside the list."""
    import paper_2503_20700_gb300 as p
    c = p.tc_shape_candidates()
    assert c[0] == (256, 4, 0, 2) and len(set(c)) == len(c) >= 2
    assert any(cl == 4 for *_, cl in c)
    for tn, ch, order, cl in c:
        assert tn % 16 == 0 and 16 <= tn <= 256 and ch >= 1 and order in (0, 1) and cl in (2, 4)
    for bad in (-1, len(c)):
        with pytest.raises(p.DmrgError) as ei:
            p.set_kernel_tc_shape(bad)
        assert ei.value.status == p.DMRG_EINVAL


def test_fiedler_order_validates_on_the_host(lib):
    """Input checks of dmrg_fiedler_order return before any device work:
    a non-symmetric or non-finite mutual information is rejected, and fewer
    than three orbitals keep their order."""
    import paper_2503_20700_gb300 as p
    with pytest.raises(p.DmrgError) as ei:
        p.fiedler_order(np.array([[0.0, 1.0, 0.2], [0.5, 0.0, 0.1], [0.2, 0.1, 0.0]]))
    assert ei.value.status == p.DMRG_EINVAL
    bad = np.zeros((3, 3))
    bad[0, 1] = bad[1, 0] = np.nan
    with pytest.raises(p.DmrgError):
        p.fiedler_order(bad)
    assert list(p.fiedler_order(np.array([[0.0, 0.3], [0.3, 0.0]]))) == [0, 1]
