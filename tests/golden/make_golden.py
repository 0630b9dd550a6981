"""Write the stored expected values of tests/golden/ by calling the oracle only.

Usage: python tests/golden/make_golden.py [name ...]
Each fixture is a small JSON file: the workload recipe, and the oracle's
energies (Hartree).  Nothing here imports or runs the CUDA path.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle.dmrg import OracleDMRG  # noqa: E402
from oracle.fci import fci  # noqa: E402


def naphthalene():
    """PPP naphthalene (10 sites/electrons, singlet): FCI and D=64 DMRG, 4 sweeps."""
    h, eri, ec = W.ppp_acene(2)
    t = time.time()
    e_fci, _, _ = fci(h, eri, 10, 0, e_core=ec, tol=1e-11)
    d = OracleDMRG(h, eri, 10, 0, D=64, e_core=ec, tol=1e-10)
    es = d.sweep(4)
    return {"workload": "PPP naphthalene pi-system, t=-2.4 eV, U=11.26 eV, Ohno, 1.40 A hexagons",
            "n": 10, "n_elec": 10, "two_s": 0, "D": 64, "sweeps": 4,
            "e_fci": e_fci, "e_dmrg_sweeps": es, "max_trunc": d.record.trunc,
            "seconds": time.time() - t}


def random8():
    """Random Cholesky CAS(8,8) rank 16 seed 2: FCI and D=12 DMRG, 3 sweeps."""
    h, L = W.cholesky_random(8, 16, seed=2)
    eri = W.eri_from_cholesky(L)
    e_fci, _, _ = fci(h, eri, 8, 0, tol=1e-11)
    d = OracleDMRG(h, eri, 8, 0, D=12, tol=1e-10)
    es = d.sweep(3)
    return {"workload": "cholesky_random(8, 16, seed=2)", "n": 8, "n_elec": 8, "two_s": 0,
            "D": 12, "sweeps": 3, "e_fci": e_fci, "e_dmrg_sweeps": es}


def ordering_hubbard8():
    """The ordering step (Sec. II "Numerical procedure") on a Hubbard chain of
    8 sites (t = -1, U = 4, half filling) whose sites were shuffled: two D=16
    sweeps in the shuffled order, the orbital entropies and mutual
    information of that state, and its Fiedler order."""
    import numpy as np
    from oracle import orbital as OB
    n = 8
    h, eri, _ = W.hubbard_chain(n, t=-1.0, u=4.0)
    perm = np.random.default_rng(3).permutation(n)
    hs, es = OB.permute_integrals(h, eri, perm)
    d = OracleDMRG(hs, es, n, 0, D=16, tol=1e-10)
    energies = d.sweep(2)
    s1, mi = OB.orbital_entanglement(d.states, d.psi_full, n, 0)
    return {"workload": "hubbard_chain(8, t=-1, u=4), sites shuffled by default_rng(3).permutation(8)",
            "perm": [int(x) for x in perm], "D": 16, "sweeps": 2, "e_dmrg_sweeps": energies,
            "s1": s1.tolist(), "mutual": mi.tolist(), "order": [int(x) for x in OB.fiedler_order(mi)]}


FIXTURES = {"naphthalene_ppp_d64": naphthalene, "random8_d12": random8, "ordering_hubbard8": ordering_hubbard8}

if __name__ == "__main__":
    names = sys.argv[1:] or list(FIXTURES)
    for name in names:
        out = FIXTURES[name]()
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump(out, f, indent=1)
        print(name, out.get("e_dmrg_sweeps"), out.get("e_fci"))
