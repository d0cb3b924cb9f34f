"""The SCF initial guess of the experiments (Sec. 5.2) through the C ABI against the FP64 CPU
oracle: the density differences of every step (1e-6 relative), the number of steps, the
orbital subspace of the guess, the closed-form (1 - alpha) decay for a density-independent
Hamiltonian, and EARCG continuing from the guess to the oracle's minimiser."""
import numpy as np
import pytest

import synth
from oracle import earcg, scf
from oracle.model import Model
from tests.conftest import ensure_library
from tests.small_models import small, start

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
ensure_library()
import paper_2503_16225_gb300 as E  # noqa: E402


def to_dev(s, blocks):
    t = torch.zeros((s.K, s.p, s.n_max), dtype=torch.complex128)
    for k, b in enumerate(blocks):
        t[k, :, :b.shape[0]] = torch.from_numpy(np.ascontiguousarray(b.T))
    return t.cuda()


def angle(A, B):
    sv = np.linalg.svd(A.conj().T @ B, compute_uv=False)
    return float(np.arccos(np.clip(sv.min(), -1.0, 1.0)))


def test_two_atom_scf_guess_and_solve():
    cfg = synth.config_two_atom(1)
    m = Model(cfg)
    raw = synth.raw_coefficients(cfg["seed"], m.nk, m.p)
    psi0 = [raw[k, :, :n].T.copy() for k, n in enumerate(m.nk)]
    Phi_o, steps_o, hist_o, _ = scf.scf_guess(m, psi0, tol=0.1, alpha=0.5)
    s = E.System(cfg)
    try:
        hist = E.eacg_scf_guess(s.h, to_dev(s, psi0), tol=0.1, alpha=0.5, eig_tol=1e-10)
        assert len(hist) == steps_o
        np.testing.assert_allclose(hist, hist_o, rtol=1e-6, atol=1e-8)
        phi = s.block()
        E.eacg_get_psi(s.h, phi)
        got = phi.cpu().numpy()
        for k in range(m.K):
            assert angle(got[k, :, :m.nk[k]].T, Phi_o[k]) <= 1e-6
        r = E.eacg_solve(s.h)
        assert r.status == 0 and r.rnorm <= 1e-8
        ores = earcg.solve(m, psi0)
        assert abs(r.E - ores.E) <= 1e-8 * len(cfg["Z"])
    finally:
        s.close()


def test_density_independent_hamiltonian_decays_by_one_minus_alpha():
    cfg = small(a=7.0, N=16, ecut=3.0, nb=2, nproj=4, hartree=0, xc=0, kgrid=(2, 1, 1))
    m = Model(cfg)
    _, steps_o, hist_o, _ = scf.scf_guess(m, start(m), tol=1e-3, alpha=0.5)
    s = E.System(cfg)
    try:
        hist = E.eacg_scf_guess(s.h, to_dev(s, start(m)), tol=1e-3, alpha=0.5, eig_tol=1e-10)
        assert len(hist) == steps_o
        np.testing.assert_allclose(hist, hist_o, rtol=1e-6, atol=1e-8)
        for a, b in zip(hist, hist[1:]):
            assert abs(b - 0.5 * a) <= 1e-6 * hist[0]
        with pytest.raises(E.EacgError):
            E.eacg_scf_guess(s.h, to_dev(s, start(m)), alpha=0.0)
    finally:
        s.close()
