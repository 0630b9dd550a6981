"""The stored expected values of tests/golden/ come from the oracle: the small
fixture is regenerated here by the same script (oracle only) and must match
what is committed; every stored DMRG energy respects the variational bound
of the stored FCI energy."""
import importlib.util
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden")


def _make_golden():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLD, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_random8_fixture_reproduces_from_the_oracle():
    stored = json.load(open(os.path.join(GOLD, "random8_d12.json")))
    out = _make_golden().random8()
    assert abs(out["e_fci"] - stored["e_fci"]) < 1e-9
    np.testing.assert_allclose(out["e_dmrg_sweeps"], stored["e_dmrg_sweeps"], rtol=0, atol=1e-9)


def test_stored_dmrg_energies_are_variational():
    for name in ("random8_d12", "naphthalene_ppp_d64"):
        d = json.load(open(os.path.join(GOLD, name + ".json")))
        es = d["e_dmrg_sweeps"]
        assert all(e >= d["e_fci"] - 1e-9 for e in es), name
        assert all(b <= a + 1e-9 for a, b in zip(es, es[1:])), name  # sweeps do not raise the energy


def test_ordering_fixture_reproduces_and_recovers_the_chain():
    """The ordering-step fixture regenerates from the oracle, and its stored
    Fiedler order places the shuffled chain's neighbours next to each other
    (at most one break)."""
    stored = json.load(open(os.path.join(GOLD, "ordering_hubbard8.json")))
    out = _make_golden().ordering_hubbard8()
    np.testing.assert_allclose(out["s1"], stored["s1"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(out["mutual"], stored["mutual"], rtol=0, atol=1e-9)
    assert out["order"] == stored["order"]
    chain = [stored["perm"][k] for k in stored["order"]]
    assert sum(abs(a - b) == 1 for a, b in zip(chain[:-1], chain[1:])) >= len(chain) - 2
