"""GPU parity of the reduced density matrices (a7): the measurement pass of the
CUDA path (dmrg_rdm12 through the C-ABI) against the oracle's RDMs of the same
two-site state, plus the identities every spin-free RDM satisfies.

Tolerance: 1e-7 max-abs (float64 path)."""
import numpy as np
import pytest

import workloads as W
from oracle.dmrg import OracleDMRG
from oracle.fci import fci
from oracle.rdm import energy_from_rdms, rdm12

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2503_20700_gb300 as p
    p.load()
    return p


def _case(name):
    if name == "rand3":
        h, L = W.cholesky_random(3, 6, seed=1)
        return h, W.eri_from_cholesky(L), 0.0, 3, 1, 4
    if name == "rand5_doublet":
        h, L = W.cholesky_random(5, 10, seed=1)
        return h, W.eri_from_cholesky(L), 0.0, 5, 1, 6
    if name == "rand6_singlet":
        h, L = W.cholesky_random(6, 12, seed=1)
        return h, W.eri_from_cholesky(L), 0.0, 6, 0, 8
    if name == "rand6_triplet":
        h, L = W.cholesky_random(6, 12, seed=1)
        return h, W.eri_from_cholesky(L), 0.0, 6, 2, 8
    if name == "hub6":
        h, eri, ec = W.hubbard_chain(6, u=4.0)
        return h, eri, ec, 6, 0, 8
    if name == "rand7_n5":
        h, L = W.cholesky_random(7, 14, seed=3)
        return h, W.eri_from_cholesky(L), 0.0, 5, 1, 10
    raise KeyError(name)


@pytest.mark.parametrize("name", ["rand3", "rand5_doublet", "rand6_singlet", "rand6_triplet", "hub6",
                                  "rand7_n5"])
def test_rdms_match_oracle(pkg, name):
    h, eri, ec, N, S, D = _case(name)
    g = pkg.DMRG(h, eri=eri, n_elec=N, two_s=S, D=D, e_core=ec)
    e = g.sweep(2)[0]
    g1, g2 = g.rdm12()
    o = OracleDMRG(h, eri, N, S, D=D, e_core=ec)
    eo = o.sweep(2)[-1]
    o1, o2 = rdm12(o.H.ops, o.psi_full)
    assert abs(e - eo) < 1e-8
    assert np.abs(g1 - o1).max() < 1e-7
    assert np.abs(g2 - o2).max() < 1e-7


def test_rdms_exact_at_full_bond_dimension(pkg):
    """Untruncated D: the RDMs are those of the FCI ground state."""
    h, L = W.cholesky_random(5, 10, seed=4)
    eri = W.eri_from_cholesky(L)
    g = pkg.DMRG(h, eri=eri, n_elec=4, two_s=0, D=64)
    g.sweep(3)
    g1, g2 = g.rdm12()
    e_fci, x, H = fci(h, eri, 4, 0)
    f1, f2 = rdm12(H.ops, x)
    assert np.abs(g1 - f1).max() < 1e-7
    assert np.abs(g2 - f2).max() < 1e-7


@pytest.mark.parametrize("D", [32, 64])
def test_rdm_identities_naphthalene(pkg, D):
    """Larger than the oracle reaches in seconds: traces, partial traces,
    index symmetries, occupations and the energy of the state from its RDMs."""
    h, eri, ec = W.ppp_acene(2)
    n, N = 10, 10
    g = pkg.DMRG(h, eri=eri, n_elec=N, two_s=0, D=D, e_core=ec)
    e = g.sweep(3)[0]
    g1, g2 = g.rdm12()
    assert abs(np.trace(g1) - N) < 1e-9
    assert np.abs(g1 - g1.T).max() < 1e-10
    occ = np.linalg.eigvalsh(g1)
    assert occ.min() > -1e-9 and occ.max() < 2 + 1e-9
    assert abs(np.einsum("pqqp->", g2) - N * (N - 1)) < 1e-8
    assert np.abs(np.einsum("pqqs->ps", g2) - (N - 1) * g1).max() < 1e-9
    assert np.abs(g2 - g2.transpose(1, 0, 3, 2)).max() < 1e-10
    assert np.abs(g2 - g2.transpose(3, 2, 1, 0)).max() < 1e-10
    assert abs(energy_from_rdms(h, eri, g1, g2, ec) - e) < 1e-8


def test_rdm_before_sweep_is_a_state_error(pkg):
    h, L = W.cholesky_random(4, 8, seed=1)
    g = pkg.DMRG(h, eri=W.eri_from_cholesky(L), n_elec=4, D=8)
    with pytest.raises(pkg.DmrgError) as ei:
        g.rdm12()
    assert ei.value.status == pkg.DMRG_ESTATE


def test_dmrg_energy_autograd_hellmann_feynman(pkg):
    """DMRGEnergy's backward (gamma~, 1/2 Gamma~) against central finite
    differences of the DMRG energy at untruncated D, for perturbations of h
    and of (pq|rs) that keep their symmetries."""
    torch = pytest.importorskip("torch")
    from paper_2503_20700_gb300.autograd import DMRGEnergy
    n, N = 4, 4
    h, L = W.cholesky_random(n, 8, seed=5)
    eri = W.eri_from_cholesky(L)
    ht = torch.tensor(h, requires_grad=True)
    et = torch.tensor(eri, requires_grad=True)
    E = DMRGEnergy.apply(ht, et, N, 0, 64, 3)
    E.backward()
    gh, ge = ht.grad.numpy(), et.grad.numpy()

    def energy(hh, ee):
        g = pkg.DMRG(hh, eri=ee, n_elec=N, two_s=0, D=64)
        e = g.sweep(3)[0]
        g.close()
        return e

    eps = 1e-4
    for p, q in [(0, 0), (0, 1), (1, 3)]:
        d = np.zeros((n, n))
        d[p, q] += 1.0
        if p != q:
            d[q, p] += 1.0
        fd = (energy(h + eps * d, eri) - energy(h - eps * d, eri)) / (2 * eps)
        assert abs(fd - (gh * d).sum()) < 1e-6
    for p, q, r, s in [(0, 0, 1, 1), (0, 1, 2, 3), (1, 2, 1, 3)]:
        d = np.zeros((n,) * 4)
        for a, b, c, e in {(p, q, r, s), (q, p, r, s), (p, q, s, r), (q, p, s, r),
                           (r, s, p, q), (s, r, p, q), (r, s, q, p), (s, r, q, p)}:
            d[a, b, c, e] = 1.0
        fd = (energy(h, eri + eps * d) - energy(h, eri - eps * d)) / (2 * eps)
        assert abs(fd - (ge * d).sum()) < 1e-6
