"""Solves with more than 64 bands, against the FP64 CPU oracle: the 64-atom diamond supercell
(128 bands, 256 s/p projectors, positions jittered) at Ecut 5 Ha on a 48^3 grid, Gamma.

Above 64 bands the p x p kernels (Jacobi eigen-decomposition, inverse, Lyapunov solve,
pivoted Cholesky) keep their matrices in a global scratch of the system instead of shared
memory, and run 1024 threads per k-point.  Checked through the C ABI:
  * the polar factor of eacg_set_psi (Sec. 3.1) against the oracle's Psi (Psi^* Psi)^{-1/2};
  * the retraction and its transport (Sec. 3.2, Prop. 1) at a random tangent;
  * the energy-adaptive gradient with the FP64 FOM (Algorithm 4, Eq. (5.2)) at the oracle's
    iterate after 50 outer iterations;
  * a converged mixed-precision solve against the stored oracle solve
    (tests/golden/oracle_diamond64_ec5.json, written by tests/golden/make_golden.py).
Tolerances as in the main parity suite."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import earcg
from oracle.manifold import polar, transport_self
from oracle.model import Model
from tests.conftest import ensure_library
from tests.small_models import free_electron

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
ensure_library()
import paper_2503_16225_gb300 as E  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_diamond64_ec5.json")


def config():
    return synth.config_diamond_supercell(2, ecut=5.0, N=48)


@pytest.fixture(scope="module")
def sup():
    cfg = config()
    model = Model(cfg)
    s = E.System(cfg, E.eacg_default_params())
    yield cfg, model, s
    s.close()


def to_dev(s, blocks):
    t = torch.zeros((s.K, s.p, s.n_max), dtype=torch.complex128)
    for k, b in enumerate(blocks):
        t[k, :, :b.shape[0]] = torch.from_numpy(np.ascontiguousarray(b.T))
    return t.cuda()


def from_dev(t, model):
    h = t.cpu().numpy()
    return [h[k, :, :model.nk[k]].T.copy() for k in range(model.K)]


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def raw_start(cfg, model, n_max=None):
    return synth.raw_coefficients(cfg["seed"], model.nk, model.p, n_max)


def test_sizes(sup):
    cfg, model, s = sup
    assert s.p == 128 > 64 and s.N == 48 and model.Dvec.size == 256 and s.nk == model.nk


def test_polar_factor_of_set_psi(sup):
    cfg, model, s = sup
    raw = raw_start(cfg, model, s.n_max)
    E.eacg_set_psi(s.h, torch.from_numpy(raw).cuda())
    phi = s.block()
    E.eacg_get_psi(s.h, phi)
    got = from_dev(phi, model)
    want = earcg.lowdin([raw[k, :, :model.nk[k]].T.copy() for k in range(model.K)])
    for k in range(model.K):
        assert rel(got[k], want[k]) < 1e-12
        np.testing.assert_allclose(got[k].conj().T @ got[k], np.eye(model.p), atol=1e-12)


def test_retraction_and_transport(sup):
    cfg, model, s = sup
    raw = raw_start(cfg, model)
    Phi = earcg.lowdin([raw[k, :, :model.nk[k]].T.copy() for k in range(model.K)])
    rng = np.random.default_rng(7)
    eta = []
    for P in Phi:
        Z = rng.standard_normal(P.shape) + 1j * rng.standard_normal(P.shape)
        M = P.conj().T @ Z
        eta.append(0.3 * (Z - P @ (0.5 * (M + M.conj().T))))
    tau = 0.7
    po, to = s.block(), s.block()
    E.eacg_retract(s.h, to_dev(s, Phi), to_dev(s, eta), tau, po, to)
    gp, gt = from_dev(po, model), from_dev(to, model)
    for k in range(model.K):
        assert rel(gp[k], polar(Phi[k] + tau * eta[k])[0]) < 1e-12
        assert rel(gt[k], transport_self(Phi[k], tau, eta[k])) < 1e-11


def test_energy_adaptive_gradient(sup):
    """FP64 FOM at the oracle's iterate after 50 outer iterations (||R|| = 1.6e-2, in the
    energy-adaptive phase).  Bound 1e-5 of max |G|: with 128 bands the shifted systems are
    close to singular for some shifts (Lambda has eigenvalue gaps down to 6e-5), and the
    oracle's own G moves by 7e-8 when Phi is perturbed by 1e-14 and by 3e-5 for 1e-12 (measured
    with the oracle alone), so the GPU's FP64-level rounding (double-float GEMMs, FFTs) is
    amplified the same way; at 6 iterations (||R|| = 1.5) a 1e-14 perturbation already moves G
    by 1.5e-4, which is why the point is taken this late.  A wrong term, sign or preconditioner
    moves G by 1e-2 or more."""
    cfg, model, s = sup
    raw = raw_start(cfg, model)
    Phi = earcg.lowdin([raw[k, :, :model.nk[k]].T.copy() for k in range(model.K)])
    res = earcg.solve(model, Phi, earcg.Params(max_outer=50), warm=True)
    Phi = res.Phi
    pt = earcg.evaluate(model, Phi)
    stats = {"fom_iters": [], "h_cols": 0}
    G = earcg.ea_gradient(model, pt, earcg.Params(), stats)
    g = s.block()
    iters = E.eacg_ea_gradient(s.h, to_dev(s, Phi), g, s.K, 0)
    got = from_dev(g, model)
    Gi = G if iters == stats["fom_iters"] else earcg.ea_gradient(model, pt, earcg.Params(), fixed_iters=iters)
    for k in range(model.K):
        assert abs(iters[k] - stats["fom_iters"][k]) <= 1, (iters, stats["fom_iters"])
        assert rel(got[k], Gi[k]) < 1e-5, rel(got[k], Gi[k])


@pytest.mark.parametrize("precision", [1])
def test_solve_matches_stored_oracle_solve(precision):
    """Mixed precision (FP32 Krylov blocks and projected solves, FP64 energy and retraction):
    the plain-FP64 solve is left out here, its FP64 projected solves of up to 2,300 Krylov
    columns on one SM per k take tens of seconds per outer step (the FP64 gradient itself is
    checked above)."""
    with open(GOLDEN) as fh:
        gold = json.load(fh)
    assert gold["status"] == "converged"
    cfg = config()
    assert gold["workload"] == cfg["name"]
    s = E.System(cfg, E.eacg_default_params(precision=precision))
    try:
        model_nk = s.nk
        raw = synth.raw_coefficients(cfg["seed"], model_nk, s.p, s.n_max)
        E.eacg_set_psi(s.h, torch.from_numpy(raw).cuda())
        r = E.eacg_solve(s.h)
        assert r.status == 0 and r.rnorm <= 1e-8
        tol = 1e-8 if precision == 0 else 1e-6
        assert abs(r.E - gold["E"]) <= tol * gold["natoms"], (r.E, gold["E"])
        phi = s.block()
        E.eacg_get_psi(s.h, phi)
        h = phi.cpu().numpy()[0, :, :model_nk[0]].T
        np.testing.assert_allclose(h.conj().T @ h, np.eye(s.p), atol=1e-11)
    finally:
        s.close()


def test_more_bands_than_the_dense_limit_are_refused():
    """p = EACG_MAX_BANDS_DENSE + 1 (free electrons in a 12 bohr cell, 691 plane waves): the
    transforms take it, the calls that decompose p x p matrices return EACG_EUNSUPPORTED."""
    cfg = free_electron(a=12.0, N=32, ecut=4.0, nb=E.EACG_MAX_BANDS_DENSE + 1)
    s = E.System(cfg, E.eacg_default_params())
    try:
        assert s.p == E.EACG_MAX_BANDS_DENSE + 1 and min(s.nk) >= s.p
        with pytest.raises(E.EacgError) as err:
            E.eacg_set_psi(s.h, s.block())
        assert err.value.code == 9
    finally:
        s.close()
