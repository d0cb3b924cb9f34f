"""Full-size parity: the 8-atom diamond workload (64 k-points, 48^3, 16 bands, the benchmark
configuration) solved on the GPU reaches the oracle's converged energy (stored in
tests/golden/oracle_diamond_k444.json by tests/golden/make_golden.py, which calls only the
oracle) within 1e-8 Ha/atom in FP64 and 1e-6 Ha/atom in mixed precision, with the oracle's
iteration count."""
import json
import os

import numpy as np
import pytest

import synth
from tests.conftest import ROOT, ensure_library

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
ensure_library()
import paper_2503_16225_gb300 as E  # noqa: E402

GOLD = json.load(open(os.path.join(ROOT, "tests", "golden", "oracle_diamond_k444.json")))


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-6)])
def test_diamond_k444_solve_matches_oracle(precision, tol):
    cfg = synth.config_diamond(2, kgrid=(4, 4, 4))
    s = E.System(cfg, E.eacg_default_params(precision=precision))
    assert s.nk == GOLD["nk"]
    raw = synth.raw_coefficients(cfg["seed"], s.nk, s.p, s.n_max)
    E.eacg_set_psi(s.h, torch.from_numpy(raw).cuda())
    r = E.eacg_solve(s.h)
    assert r.status == 0 and r.rnorm <= 1e-8
    assert abs(r.E - GOLD["E"]) <= tol * GOLD["natoms"]
    assert abs(r.iterations - GOLD["iterations"]) <= 3
    assert r.warm_iterations == GOLD["warm_iterations"] or precision == 1
    # the converged orbitals are orthonormal at every k-point
    phi = s.block()
    E.eacg_get_psi(s.h, phi)
    g = torch.einsum("kin,kjn->kij", phi.conj(), phi).cpu().numpy()
    assert np.abs(g - np.eye(s.p)[None]).max() < 1e-12
    s.close()
