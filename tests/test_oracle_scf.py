"""Pins of the oracle's SCF initial guess (Sec. 5.2): the closed-form geometric decay of the
density difference for a Hamiltonian that does not depend on the density, and agreement of the
tight SCF fixed point with the EARCG minimiser (two independent routes to the ground state)."""
import numpy as np
import pytest

import synth
from oracle import earcg, scf
from oracle.model import Model
from tests.small_models import small, start


def test_linear_model_density_difference_decays_by_one_minus_alpha():
    """V independent of rho: every step returns the ground-state density rho_gs, so
    rho_out - rho_in shrinks by exactly (1 - alpha) per step and Phi diagonalises H."""
    m = Model(small(a=7.0, N=16, ecut=3.0, nb=2, nproj=4, hartree=0, xc=0, kgrid=(2, 1, 1)))
    for alpha in (0.5, 0.8):
        Phi, steps, hist, _ = scf.scf_guess(m, start(m), tol=1e-6, alpha=alpha)
        assert steps == len(hist) and hist[-1] < 1e-6 <= hist[-2]
        for a, b in zip(hist, hist[1:]):
            assert abs(b - (1 - alpha) * a) <= 1e-9 * hist[0]
        want = sum(m.kw[k] * m.occ * np.linalg.eigvalsh(m.dense_H(k, m.vloc))[:m.p].sum() for k in range(m.K))
        assert abs(m.energy(Phi) - want) < 1e-10


def _two_atom():
    cfg = synth.config_two_atom(1)
    m = Model(cfg)
    raw = synth.raw_coefficients(cfg["seed"], m.nk, m.p)
    return m, [raw[k, :, :n].T.copy() for k, n in enumerate(m.nk)]


def test_tight_scf_fixed_point_is_the_earcg_minimiser():
    """Hartree + exchange, gapped: SCF to ||drho|| < 1e-9 and EARCG to ||R|| < 1e-8 reach the
    same energy and density (the self-consistent ground state is the energy minimiser)."""
    m, psi0 = _two_atom()
    Phi, steps, hist, _ = scf.scf_guess(m, psi0, tol=1e-9, alpha=0.5)
    res = earcg.solve(m, psi0)
    assert res.status == "converged"
    assert abs(m.energy(Phi) - res.E) < 1e-9
    assert scf.density_difference(m, m.density(Phi), m.density(res.Phi)) < 1e-6


def test_paper_tolerance_stops_at_the_first_step_below_it():
    m, psi0 = _two_atom()
    Phi, steps, hist, rho_in = scf.scf_guess(m, psi0, tol=0.1, alpha=0.5)
    assert hist[-1] < 0.1 and all(h >= 0.1 for h in hist[:-1])
    assert scf.density_difference(m, m.density(Phi), rho_in) == pytest.approx(hist[-1], rel=1e-12)
    # EARCG from the SCF guess reaches the same minimiser as from the random start
    res = earcg.solve(m, Phi)
    assert res.status == "converged"
    assert abs(res.E - earcg.solve(m, psi0).E) < 1e-9
