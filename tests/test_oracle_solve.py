"""Whole-iteration pins of the oracle's EARCG (Algorithm 3): closed-form free-electron
energies, dense diagonalisation of linear models, self-consistency (Aufbau) of the
converged nonlinear state, monotone energy and Remark 4's O(||R||^2) estimate."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import earcg, fom
from oracle.manifold import polar
from oracle.model import Model
from tests.small_models import free_electron, small, start


def _check_history(res):
    E = [h["E"] for h in res.history]
    for e0, e1 in zip(E, E[1:]):
        assert e1 <= e0 + 1e-12 * abs(e0)


def test_free_electron_closed_shell_energy():
    """V = 0, p = 7 at Gamma: the 7 lowest 1/2|G|^2 are 0 and six times b^2/2, so
    E = f * 3 b^2 = 6 b^2 and Lambda has eigenvalues {0, b^2/2 (x6)}."""
    m = Model(free_electron(a=6.0, N=16, ecut=4.0, nb=7))
    res = earcg.solve(m, start(m))
    assert res.status == "converged"
    b2 = m.b ** 2
    assert abs(res.E - 6.0 * b2) < 1e-10
    lam = np.linalg.eigvalsh(res.point.Lam[0])
    np.testing.assert_allclose(lam, [0.0] + [0.5 * b2] * 6, atol=1e-9)
    _check_history(res)


def test_linear_model_matches_dense_diagonalisation():
    """Hartree and exchange off: E = f sum_k w_k sum_{i<=p} lambda_ik of the explicit matrix."""
    cfg = small(a=7.0, N=16, ecut=3.0, nb=2, nproj=4, hartree=0, xc=0, kgrid=(2, 1, 1))
    m = Model(cfg)
    res = earcg.solve(m, start(m))
    assert res.status == "converged"
    want = 0.0
    for k in range(m.K):
        w = np.linalg.eigvalsh(m.dense_H(k, m.vloc))
        assert w[m.p] - w[m.p - 1] > 1e-3        # gap: unique minimiser
        want += m.kw[k] * m.occ * w[:m.p].sum()
        np.testing.assert_allclose(np.linalg.eigvalsh(res.point.Lam[k]), w[:m.p], atol=1e-9)
    assert abs(res.E - want) < 1e-10 * max(1.0, abs(want))
    _check_history(res)


@pytest.fixture(scope="module")
def two_atom_solution():
    cfg = synth.config_two_atom(1)
    m = Model(cfg)
    raw = synth.raw_coefficients(cfg["seed"], m.nk, m.p)
    res = earcg.solve(m, [raw[k, :, :m.nk[k]].T.copy() for k in range(m.K)])
    return m, res


def test_two_atom_converges_monotonically(two_atom_solution):
    m, res = two_atom_solution
    assert res.status == "converged"
    assert res.rnorm <= 1e-8
    _check_history(res)
    Phi = res.Phi[0]
    np.testing.assert_allclose(Phi.conj().T @ Phi, np.eye(m.p), atol=1e-13)
    # the energy-adaptive phase takes few iterations from ||R|| = 1e-2 (paper: ~7-10, Sec. 5.3)
    assert res.iterations - res.warm_iterations <= 15


@pytest.fixture(scope="module")
def small_nonlinear_solution():
    """A small gapped nonlinear model (Hartree + exchange + projectors), n ~ 10^2."""
    cfg = small(a=7.0, N=16, ecut=3.0, nb=2, nproj=4, kgrid=(1, 1, 1))
    m = Model(cfg)
    res = earcg.solve(m, start(m))
    return m, res


def test_converged_state_is_self_consistent_ground_state(small_nonlinear_solution):
    """At the converged Phi, the eigenvalues of Lambda are the p lowest eigenvalues of the
    dense H_Phi built from rho(Phi) (Aufbau principle, Sec. 2.1) and there is a gap."""
    m, res = small_nonlinear_solution
    assert res.status == "converged"
    _check_history(res)
    w = np.linalg.eigvalsh(m.dense_H(0, res.point.vtot))
    np.testing.assert_allclose(np.linalg.eigvalsh(res.point.Lam[0]), w[:m.p], atol=1e-8)
    assert w[m.p] - w[m.p - 1] > 1e-3
    assert abs(m.integrate(res.point.rho) - m.occ * m.p) < 1e-10


def test_remark4_shifted_inverse_overlap_is_quadratic_in_the_residual(small_nonlinear_solution):
    """|| Phi^* X - mu^{-1} I ||_F = O(||R||^2) near the minimiser (Remark 4)."""
    m, res = small_nonlinear_solution
    rng = np.random.default_rng(8)
    P0 = res.Phi[0]
    Z = rng.standard_normal(P0.shape) + 1j * rng.standard_normal(P0.shape)
    W = Z - P0 @ (0.5 * (P0.conj().T @ Z + Z.conj().T @ P0))
    W /= np.linalg.norm(W)
    mu = 0.01
    out = []
    for eps in (2e-3, 1e-3):
        Phi = [polar(P0 + eps * W)[0]]
        pt = earcg.evaluate(m, Phi)
        H = m.dense_H(0, pt.vtot)
        Sig = pt.Lam[0] - mu * np.eye(m.p)
        X = sla.solve_sylvester(H, -Sig, Phi[0])
        out.append((pt.rnorm, np.linalg.norm(Phi[0].conj().T @ X - np.eye(m.p) / mu)))
    (r1, d1), (r2, d2) = out
    ratio = math.log(d1 / d2) / math.log(r1 / r2)
    assert 1.7 < ratio < 2.3


# ----------------------------------------------------------------------------- EARGD
def test_bb_step_closed_form():
    """y = c s: both Barzilai-Borwein quotients equal 1/c (the secant of a c-scaled identity)."""
    m = Model(small(nb=2))
    rng = np.random.default_rng(2)
    s = [rng.standard_normal((n, m.p)) + 1j * rng.standard_normal((n, m.p)) for n in m.nk]
    for c in (0.5, 3.0):
        y = [c * x for x in s]
        assert abs(earcg.bb_step(m, s, y, True) - 1.0 / c) < 1e-12
        assert abs(earcg.bb_step(m, s, y, False) - 1.0 / c) < 1e-12


def test_eargd_linear_model_matches_dense_diagonalisation():
    """EARGD reaches the same minimiser as the explicit eigenvalue problem."""
    cfg = small(a=7.0, N=16, ecut=3.0, nb=2, nproj=4, hartree=0, xc=0, kgrid=(2, 1, 1))
    m = Model(cfg)
    res = earcg.solve(m, start(m), earcg.Params(method=1))
    assert res.status == "converged"
    want = sum(m.kw[k] * m.occ * np.linalg.eigvalsh(m.dense_H(k, m.vloc))[:m.p].sum() for k in range(m.K))
    assert abs(res.E - want) < 1e-10 * max(1.0, abs(want))


def test_eargd_monotone_limit_and_agreement_with_earcg(two_atom_solution):
    """nm_rho = 0 makes the reference value the current energy: the energy-adaptive phase then
    decreases monotonically; either way EARGD ends at EARCG's energy (unique minimiser)."""
    m, ref = two_atom_solution
    cfg = synth.config_two_atom(1)
    raw = synth.raw_coefficients(cfg["seed"], m.nk, m.p)
    psi0 = [raw[k, :, :m.nk[k]].T.copy() for k in range(m.K)]
    for rho in (0.85, 0.0):
        res = earcg.solve(m, psi0, earcg.Params(method=1, nm_rho=rho))
        assert res.status == "converged"
        assert abs(res.E - ref.E) < 1e-9
        if rho == 0.0:
            E = [h["E"] for h in res.history if h["phase"] == "ea"]
            for e0, e1 in zip(E, E[1:]):
                assert e1 <= e0 + 1e-12 * abs(e0)
