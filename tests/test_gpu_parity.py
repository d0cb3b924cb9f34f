"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bit-exact: basis index maps.  FP64 arithmetic: relative 1e-11 on H psi, rho, V and
the energy terms (rounding of FFTs and reductions of ~1e4-1e6 terms, ~1e-15 each);
the FOM-based gradient compares to 1e-8 (iterative solve amplifies rounding) with
identical per-k iteration counts.  FP32 transforms: relative 5e-6 on H psi (FP32
unit roundoff 6e-8 times log2(N^3) butterfly levels and the V range).  Solves: energy
within 1e-8 Ha per atom (FP64) / 1e-6 Ha per atom (mixed) and orbital subspace
angle <= 1e-6."""
import math

import numpy as np
import pytest

import synth
from oracle import earcg
from oracle.manifold import polar, transport_self
from oracle.model import Model
from tests.conftest import ensure_library
from tests.small_models import small

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
ensure_library()
import paper_2503_16225_gb300 as E  # noqa: E402


def _configs():
    return {
        "small_nl": small(nproj=4, kgrid=(2, 1, 1), nb=3),
        "small_lda": small(nproj=4, kgrid=(2, 1, 1), nb=3, xc=2),   # exchange + PW92 correlation
        "small_p1": small(nproj=1, kgrid=(1, 1, 1), nb=1, N=16),
        "small_odd": small(nproj=0, kgrid=(3, 1, 1), nb=5, ecut=4.0, N=24),
        "two_atom": synth.config_two_atom(1),
        "diamond_k2": synth.config_diamond(2, kgrid=(2, 2, 2)),
    }


CFG = _configs()


@pytest.fixture(scope="module", params=list(CFG))
def pair(request):
    cfg = CFG[request.param]
    model = Model(cfg)
    s = E.System(cfg)
    yield request.param, cfg, model, s
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


def start_blocks(model, cfg, n_max):
    raw = synth.raw_coefficients(cfg["seed"], model.nk, model.p, n_max)
    return raw, earcg.lowdin([raw[k, :, :model.nk[k]].T.copy() for k in range(model.K)])


def test_basis_is_bit_exact(pair):
    name, cfg, model, s = pair
    assert s.nk == model.nk
    m = s.basis().cpu().numpy()
    for k in range(model.K):
        assert np.array_equal(m[k, :model.nk[k]], model.basis[k])


def test_density_and_potential(pair):
    name, cfg, model, s = pair
    _, Phi = start_blocks(model, cfg, s.n_max)
    rho = s.grid()
    E.eacg_density(s.h, to_dev(s, Phi), rho, 0)
    rho_o = model.density(Phi)
    assert rel(rho.cpu().numpy(), rho_o) < 1e-11
    v = s.grid()
    E.eacg_get_potential(s.h, v)
    assert rel(v.cpu().numpy(), model.potentials(rho_o)[0]) < 1e-11


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 5e-6)])
def test_apply_H(pair, prec, tol):
    name, cfg, model, s = pair
    _, Phi = start_blocks(model, cfg, s.n_max)
    E.eacg_density(s.h, to_dev(s, Phi), None, 0)
    vtot = model.potentials(model.density(Phi))[0]
    rng = np.random.default_rng(5)
    C = [rng.standard_normal(P.shape) + 1j * rng.standard_normal(P.shape) for P in Phi]
    out = s.block()
    E.eacg_apply_H(s.h, to_dev(s, C), out, prec)
    got = from_dev(out, model)
    for k in range(model.K):
        assert rel(got[k], model.apply_H(k, C[k], vtot)) < tol
    # padding stays zero
    h = out.cpu().numpy()
    for k in range(model.K):
        assert np.all(h[k, :, model.nk[k]:] == 0)


def test_fp64_transforms_in_double_float_and_plain_fp64(pair):
    """The FP64-accurate transforms in double-float arithmetic (default) and on the FP64 pipe
    give the oracle's density and H psi to 1e-11, and each other's to 1e-13 (the double-float
    pairs carry about 48 significant bits, so both are rounding-level copies of the exact
    transform)."""
    name, cfg, model, s = pair
    _, Phi = start_blocks(model, cfg, s.n_max)
    rng = np.random.default_rng(8)
    C = [rng.standard_normal(P.shape) + 1j * rng.standard_normal(P.shape) for P in Phi]
    rho_o = model.density(Phi)
    vtot = model.potentials(rho_o)[0]
    got = {}
    for df in (1, 0):
        s2 = E.System(cfg, E.eacg_default_params(df_transforms=df))
        try:
            rho = s2.grid()
            E.eacg_density(s2.h, to_dev(s2, Phi), rho, 0)
            out = s2.block()
            E.eacg_apply_H(s2.h, to_dev(s2, C), out, 0)
            got[df] = (rho.cpu().numpy(), from_dev(out, model))
        finally:
            s2.close()
        assert rel(got[df][0], rho_o) < 1e-11, df
        for k in range(model.K):
            assert rel(got[df][1][k], model.apply_H(k, C[k], vtot)) < 1e-11, (df, k)
    assert rel(got[1][0], got[0][0]) < 1e-13
    for k in range(model.K):
        assert rel(got[1][1][k], got[0][1][k]) < 1e-13


def test_energy_lambda_residual(pair):
    name, cfg, model, s = pair
    _, Phi = start_blocks(model, cfg, s.n_max)
    lam = torch.zeros((s.K, s.p, s.p), dtype=torch.complex128, device="cuda")
    res = s.block()
    terms, rn = E.eacg_energy(s.h, to_dev(s, Phi), lam, res, 0)
    pt = earcg.evaluate(model, Phi)
    want = pt.terms
    for got, key in zip(terms[:5], ("kin", "loc", "hartree", "xc", "nl")):
        assert abs(got - want[key]) <= 1e-11 * max(1.0, abs(want[key])), key
    assert abs(terms[5] - pt.E) <= 1e-11 * max(1.0, abs(pt.E))
    assert abs(rn - pt.rnorm) <= 1e-10 * pt.rnorm
    L = lam.cpu().numpy()
    for k in range(model.K):
        # column-major p x p on the device
        assert rel(L[k].T, pt.Lam[k]) < 1e-11
    assert rel(np.concatenate([r.ravel() for r in from_dev(res, model)]),
               np.concatenate([r.ravel() for r in pt.R])) < 1e-9


def test_retraction_and_transport(pair):
    name, cfg, model, s = pair
    _, Phi = start_blocks(model, cfg, s.n_max)
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


def test_energy_adaptive_gradient(pair):
    name, cfg, model, s = pair
    if name == "diamond_k2":
        pytest.skip("covered by the smaller models (the oracle FOM at 8 k-points takes a minute)")
    _, Phi = start_blocks(model, cfg, s.n_max)
    # a point a few warm-up iterations in, where the shifted operator is the paper's regime
    res = earcg.solve(model, [P.copy() for P in Phi], earcg.Params(max_outer=6), warm=True)
    Phi = res.Phi
    pt = earcg.evaluate(model, Phi)
    stats = {"fom_iters": [], "h_cols": 0}
    G = earcg.ea_gradient(model, pt, earcg.Params(), stats)
    g = s.block()
    iters = E.eacg_ea_gradient(s.h, to_dev(s, Phi), g, s.K, 0)
    assert iters == stats["fom_iters"]
    got = from_dev(g, model)
    for k in range(model.K):
        assert rel(got[k], G[k]) < 1e-8


def test_energy_adaptive_gradient_fp32_krylov(pair):
    """Mixed mode: the FOM in FP32 (Krylov blocks, transforms, projected solves) gives, element
    by element, the oracle's gradient after the same number of FOM iterations per k.  Bound
    5e-3 of max |G|: the projected shifted systems (A - s_m) have eigenvalues down to mu = 0.01
    against |A| ~ Ecut, so FP32 rounding (6e-8) in the Krylov blocks, Gram matrices and
    transforms is amplified by ~|A| / mu ~ 1e3; an emulation of the FOM with every block
    rounded to FP32 gives 6e-4 on the 32-band tensor-core model, the GPU (with FP32 transforms
    and chunk sums as well) up to 1.5e-3.  The bound stays five times below the FOM's own
    2.5e-2 stopping tolerance, while a wrong term, sign or preconditioner moves G by O(1e-2)
    or more.  The FOM's stopping test picks the oracle's iteration count or one apart."""
    name, cfg, model, s = pair
    if name == "diamond_k2":
        pytest.skip("covered by the smaller models")
    _, Phi = start_blocks(model, cfg, s.n_max)
    res = earcg.solve(model, [P.copy() for P in Phi], earcg.Params(max_outer=6), warm=True)
    Phi = res.Phi
    pt = earcg.evaluate(model, Phi)
    stats = {"fom_iters": [], "h_cols": 0}
    G = earcg.ea_gradient(model, pt, earcg.Params(), stats)
    g = s.block()
    iters = E.eacg_ea_gradient(s.h, to_dev(s, Phi), g, s.K, 1)
    got = from_dev(g, model)
    Gi = earcg.ea_gradient(model, pt, earcg.Params(), fixed_iters=iters)
    for k in range(model.K):
        assert abs(iters[k] - stats["fom_iters"][k]) <= 1, (iters, stats["fom_iters"])
        assert rel(got[k], Gi[k]) < 5e-3, (k, iters[k], rel(got[k], Gi[k]))
        if iters[k] == stats["fom_iters"][k]:
            assert rel(got[k], G[k]) < 5e-3
        # tangent to the manifold at Phi (Cor. 1 form)
        M = Phi[k].conj().T @ got[k]
        assert np.abs(M + M.conj().T).max() < 1e-2 * max(1.0, np.abs(got[k]).max())


def _angle(A, B):
    s = np.linalg.svd(A.conj().T @ B, compute_uv=False)
    return float(np.arccos(np.clip(s.min(), -1.0, 1.0)))


@pytest.mark.parametrize("name", ["small_nl", "small_lda", "small_p1", "two_atom"])
@pytest.mark.parametrize("precision", [0, 1])
def test_solve_matches_oracle(name, precision):
    cfg = CFG[name]
    model = Model(cfg)
    s = E.System(cfg, E.eacg_default_params(precision=precision))
    raw, _ = start_blocks(model, cfg, s.n_max)
    E.eacg_set_psi(s.h, torch.from_numpy(raw).cuda())
    r = E.eacg_solve(s.h)
    assert r.status == 0 and r.rnorm <= 1e-8
    ores = earcg.solve(model, [raw[k, :, :model.nk[k]].T.copy() for k in range(model.K)])
    assert ores.status == "converged"
    nat = max(1, len(cfg["Z"]))
    tol = 1e-8 if precision == 0 else 1e-6
    assert abs(r.E - ores.E) <= tol * nat
    phi = s.block()
    E.eacg_get_psi(s.h, phi)
    got = from_dev(phi, model)
    for k in range(model.K):
        assert _angle(got[k], ores.Phi[k]) <= 1e-6
        np.testing.assert_allclose(got[k].conj().T @ got[k], np.eye(model.p), atol=1e-12)
    # the oracle's own residual at the GPU's minimiser
    assert earcg.evaluate(model, got).rnorm <= 2e-8
    s.close()


def test_step_sequence_matches_oracle_history():
    """The first iterations (energies, steps) follow the oracle's history closely."""
    cfg = CFG["two_atom"]
    model = Model(cfg)
    s = E.System(cfg)
    raw, _ = start_blocks(model, cfg, s.n_max)
    E.eacg_set_psi(s.h, torch.from_numpy(raw).cuda())
    ores = earcg.solve(model, [raw[k, :, :model.nk[k]].T.copy() for k in range(model.K)],
                       earcg.Params(max_outer=5))
    for h in ores.history[1:]:
        info = E.eacg_step(s.h)
        assert abs(info.E - h["E"]) <= 1e-9 * max(1.0, abs(h["E"]))
        assert abs(info.tau - h["tau"]) <= 1e-6 * abs(h["tau"])
    s.close()
