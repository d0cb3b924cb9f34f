"""The stored oracle solves (tests/golden/oracle_<name>.json, written by
tests/golden/make_golden.py from oracle/ alone) still describe the current synthetic
workloads: same workload name and basis sizes as the seeded generators give now, a converged
status at the solve tolerance ||R||_F <= 1e-8 (Algorithm 3's stopping test), and an energy equal
to the sum of its stored terms (kinetic, local, Hartree, exchange-correlation, nonlocal)."""
import importlib.util
import json
import os

import pytest

from oracle.model import Model

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


def _workloads():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.WORKLOADS


WORKLOADS = _workloads()
STORED = sorted(n for n in WORKLOADS if os.path.exists(os.path.join(GOLDEN, f"oracle_{n}.json")))


def test_some_solves_are_stored():
    assert "diamond_k444" in STORED and "diamond64_ec5" in STORED


@pytest.mark.parametrize("name", STORED)
def test_stored_solve_matches_its_workload(name):
    with open(os.path.join(GOLDEN, f"oracle_{name}.json")) as fh:
        g = json.load(fh)
    cfg = WORKLOADS[name]()
    assert g["workload"] == cfg["name"]
    assert g["natoms"] == len(cfg["Z"])
    assert g["status"] == "converged" and g["rnorm"] <= 1e-8
    terms = g["terms"]
    assert set(terms) >= {"kin", "loc", "hartree", "xc", "nl"}
    total = terms["kin"] + terms["loc"] + terms["hartree"] + terms["xc"] + terms["nl"]
    assert abs(total - g["E"]) <= 1e-10 * max(1.0, abs(g["E"]))
    assert g["iterations"] > 0 and g["band_applications"] > 0
    if cfg["N"] <= 48:  # basis sizes per k-point (cheap to rebuild at these grids)
        assert list(Model(cfg).nk) == list(g["nk"])
