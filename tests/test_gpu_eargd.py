"""EARGD on the GPU (eacg_params.method = 1) against the oracle's EARGD: the first
energy-adaptive steps (energies, Barzilai-Borwein / backtracked step sizes) follow the oracle's
history, and whole solves reach the oracle's minimiser (FP64: 1e-8 Ha per atom, mixed: 1e-6)."""
import numpy as np
import pytest

import synth
from oracle import earcg
from oracle.model import Model
from tests.conftest import ensure_library
from tests.small_models import small

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
ensure_library()
import paper_2503_16225_gb300 as E  # noqa: E402


def _start(model, cfg, n_max):
    raw = synth.raw_coefficients(cfg["seed"], model.nk, model.p, n_max)
    return raw, [raw[k, :, :model.nk[k]].T.copy() for k in range(model.K)]


def test_eargd_steps_follow_the_oracle():
    """The warm-up steps, then the first energy-adaptive EARGD steps (BB step sizes after the
    non-monotone backtracking), follow the oracle's history."""
    cfg = synth.config_two_atom(1)
    model = Model(cfg)
    s = E.System(cfg, E.eacg_default_params(method=1))
    try:
        raw, psi0 = _start(model, cfg, s.n_max)
        E.eacg_set_psi(s.h, torch.from_numpy(raw).cuda())
        ores = earcg.solve(model, psi0, earcg.Params(method=1, max_outer=40))
        ea = [h for h in ores.history[1:] if h["phase"] == "ea"]
        assert len(ea) >= 4, "the comparison must reach the energy-adaptive phase"
        n_ea = 0
        for h in ores.history[1:]:
            info = E.eacg_step(s.h)
            assert abs(info.E - h["E"]) <= 1e-9 * max(1.0, abs(h["E"]))
            assert abs(info.tau - h["tau_acc"]) <= 1e-6 * abs(h["tau_acc"])
            if h["phase"] == "ea":
                assert info.phase == 1 and info.beta == 0.0
                n_ea += 1
                if n_ea == 6 or info.converged:
                    break
    finally:
        s.close()


@pytest.mark.parametrize("name,cfg", [("two_atom", synth.config_two_atom(1)),
                                      ("small_nl", small(nproj=4, kgrid=(2, 1, 1), nb=3))])
@pytest.mark.parametrize("precision", [0, 1])
def test_eargd_solve_reaches_the_oracle_minimiser(name, cfg, precision):
    model = Model(cfg)
    s = E.System(cfg, E.eacg_default_params(method=1, precision=precision))
    try:
        raw, psi0 = _start(model, cfg, s.n_max)
        E.eacg_set_psi(s.h, torch.from_numpy(raw).cuda())
        r = E.eacg_solve(s.h)
        assert r.status == 0 and r.rnorm <= 1e-8
        ores = earcg.solve(model, psi0, earcg.Params(method=1))
        assert ores.status == "converged"
        nat = max(1, len(cfg["Z"]))
        assert abs(r.E - ores.E) <= (1e-8 if precision == 0 else 1e-6) * nat
        phi = s.block()
        E.eacg_get_psi(s.h, phi)
        got = phi.cpu().numpy()
        for k in range(model.K):
            g = got[k, :, :model.nk[k]].T
            np.testing.assert_allclose(g.conj().T @ g, np.eye(model.p), atol=1e-12)
    finally:
        s.close()
