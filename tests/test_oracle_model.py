"""Pins of the oracle's discrete model against closed forms, textbook routines and
invariants (none of them re-derives the oracle's own formula)."""
import math

import numpy as np
import pytest

import synth
from oracle import earcg
from oracle.model import PW92, Model, pairing
from tests.small_models import free_electron, small, start


def test_basis_is_the_cutoff_sphere_brute_force():
    """Every integer triple inside 1/2|k+G|^2 <= Ecut, nothing else, canonical order."""
    cfg = small(kgrid=(2, 1, 1))
    m = Model(cfg)
    for k in range(m.K):
        kf = m.kfrac[k]
        want = []
        for mx in range(-8, 8):
            for my in range(-8, 8):
                for mz in range(-8, 8):
                    e = 0.5 * m.b ** 2 * ((mx + kf[0]) ** 2 + (my + kf[1]) ** 2 + (mz + kf[2]) ** 2)
                    if e <= m.ecut:
                        want.append((mx, my, mz))
        assert np.array_equal(m.basis[k], np.array(want))


def test_grid_orbital_equals_direct_fourier_sum():
    """u(r_j) = Omega^{-1/2} sum_G c_G exp(i G.r_j) evaluated literally on an 8^3 grid."""
    cfg = small(a=5.0, N=8, ecut=2.0, nb=1)
    m = Model(cfg)
    rng = np.random.default_rng(0)
    c = rng.standard_normal((m.nk[0], 1)) + 1j * rng.standard_normal((m.nk[0], 1))
    u = m.to_grid(0, c)[0]
    N = m.N
    j = np.arange(N)
    r = np.stack(np.meshgrid(j, j, j, indexing="ij"), -1).reshape(-1, 3) * (m.a / N)
    G = m.b * m.basis[0]
    direct = (np.exp(1j * r @ G.T) @ c[:, 0]) / math.sqrt(m.omega)
    np.testing.assert_allclose(u.reshape(-1), direct, rtol=0, atol=1e-12)


def test_density_integrates_to_electron_count():
    """Parseval: int rho = f * p for orthonormal orbitals, any weights summing to one."""
    m = Model(small(kgrid=(2, 2, 1), nb=3))
    Phi = earcg.lowdin(start(m))
    rho = m.density(Phi)
    assert abs(m.integrate(rho) - m.occ * m.p) < 1e-11
    assert rho.min() >= 0


def test_local_part_equals_explicit_convolution_matrix():
    """Convolution theorem: the FFT application equals the explicit matrix
    1/2|k+G|^2 delta + V(G - G') + B D B^* built entry by entry."""
    m = Model(small(nproj=4, kgrid=(2, 1, 1), nb=3))
    rng = np.random.default_rng(1)
    v = rng.standard_normal((m.N,) * 3)
    for k in range(m.K):
        C = rng.standard_normal((m.nk[k], 3)) + 1j * rng.standard_normal((m.nk[k], 3))
        np.testing.assert_allclose(m.apply_H(k, C, v), m.dense_H(k, v) @ C, atol=1e-11, rtol=0)
        H = m.dense_H(k, v)
        assert np.abs(H - H.conj().T).max() < 1e-12


def test_free_electron_hamiltonian_is_kinetic_diagonal():
    m = Model(free_electron(kgrid=(2, 1, 1)))
    rng = np.random.default_rng(2)
    v = np.zeros((m.N,) * 3)
    for k in range(m.K):
        C = rng.standard_normal((m.nk[k], 2)) + 0j
        kv = m.b * (m.basis[k] + m.kfrac[k])
        want = 0.5 * (kv ** 2).sum(1)[:, None] * C
        np.testing.assert_allclose(m.apply_H(k, C, v), want, atol=1e-13, rtol=0)


def test_hartree_of_a_single_cosine_density():
    """rho = cos(G0.r) has V_H = 4 pi / |G0|^2 cos(G0.r) (Poisson, closed form)."""
    m = Model(small(a=7.0, N=12))
    N = m.N
    j = np.arange(N)
    X, Y, Zc = np.meshgrid(j, j, j, indexing="ij")
    G0 = m.b * np.array([1, 2, 0])
    ph = (G0[0] * X + G0[1] * Y + G0[2] * Zc) * (m.a / N)
    rho = np.cos(ph)
    vh = m.hartree_potential(rho)
    np.testing.assert_allclose(vh, 4 * math.pi / (G0 @ G0) * np.cos(ph), atol=1e-12)


def test_exchange_potential_is_derivative_of_exchange_energy():
    rho = np.array([1e-3, 0.05, 0.3, 2.0])
    h = 1e-6 * rho
    fd = (Model.exchange_energy_density(rho + h) - Model.exchange_energy_density(rho - h)) / (2 * h)
    np.testing.assert_allclose(Model.exchange_potential(rho), fd, rtol=1e-8)


def test_correlation_potential_is_derivative_of_correlation_energy():
    """V_c = d(rho eps_c)/d rho by central differences (pins eps_c' and the r_s chain rule)."""
    rho = np.array([1e-5, 1e-3, 0.05, 0.3, 2.0, 40.0])
    h = 1e-6 * rho
    fd = (Model.correlation(rho + h)[0] - Model.correlation(rho - h)[0]) / (2 * h)
    np.testing.assert_allclose(Model.correlation(rho)[1], fd, rtol=1e-7)
    e, v = Model.correlation(np.array([0.0, -1e-12]))
    assert np.all(e == 0) and np.all(v == 0)


def _eps_c(rs):
    rho = 3.0 / (4.0 * math.pi * rs ** 3)
    return Model.correlation(np.array([rho]))[0][0] / rho


def test_correlation_high_density_limit():
    """r_s -> 0: eps_c = c0 ln r_s - c1 + o(1) with the exact Gell-Mann-Brueckner coefficient
    c0 = (1 - ln 2) / pi^2 and the second-order constant c1 = 0.046644 Ha that the Perdew-Wang
    fit is built on; with them its beta2 equals 2 A beta1^2."""
    c0 = (1.0 - math.log(2.0)) / math.pi ** 2
    slope = (_eps_c(1e-9) - _eps_c(1e-10)) / math.log(10.0)
    assert abs(slope - c0) < 1e-4 * c0
    assert abs(_eps_c(1e-12) - c0 * math.log(1e-12) + 0.046644) < 2e-5
    A, b1 = PW92["A"], PW92["beta1"]
    assert abs(PW92["beta2"] - 2 * A * b1 * b1) < 1e-4 * PW92["beta2"]


def test_correlation_agrees_with_an_independent_fit_of_the_same_gas():
    """Perdew-Zunger 1981 fit of the same Ceperley-Alder energies (Phys. Rev. B 23, 5048,
    unpolarised: r_s >= 1: gamma / (1 + beta1 sqrt(r_s) + beta2 r_s), gamma = -0.1423,
    beta1 = 1.0529, beta2 = 0.3334; r_s < 1: 0.0311 ln r_s - 0.048 + 0.0020 r_s ln r_s
    - 0.0116 r_s, Ha): the two agree within 1 mHa from r_s = 0.1 to 50."""
    for rs in (0.1, 0.3, 0.5, 1.0, 2.0, 5.0, 10.0, 20.0, 50.0):
        if rs >= 1:
            pz = -0.1423 / (1 + 1.0529 * math.sqrt(rs) + 0.3334 * rs)
        else:
            pz = 0.0311 * math.log(rs) - 0.048 + 0.0020 * rs * math.log(rs) - 0.0116 * rs
        assert abs(_eps_c(rs) - pz) < 1e-3, rs


def test_local_potential_minimum_sits_on_the_atom():
    """A single Gaussian-screened ion placed on a grid point: V_loc is lowest there."""
    a, N = 8.0, 16
    cfg = small(a=a, N=N, pos=((2.0, 3.5, 5.0),), Z=(3,), rc=(0.7,), ecut=6.0)
    m = Model(cfg)
    idx = np.unravel_index(np.argmin(m.vloc), m.vloc.shape)
    assert np.allclose(np.array(idx) * a / N, [2.0, 3.5, 5.0])
    assert abs(m.vloc.mean()) < 1e-12   # neutralising background: no G = 0 term


def test_projectors_are_normalised_orthogonal_and_centred():
    """sum_G |beta(G)|^2 -> 1 for L2-normalised s/p Gaussians (Ecut large), s and p
    orthogonal on the same atom, and the real-space s projector peaks at the atom."""
    R = (1.5, 2.25, 3.0)
    cfg = small(a=9.0, N=36, ecut=30.0, pos=(R,), Z=(1,), rc=(1.0,), nproj=4, width=0.7)
    m = Model(cfg)
    B = m.proj[0]
    gram = B.conj().T @ B
    np.testing.assert_allclose(np.diag(gram).real, 1.0, atol=1e-6)
    np.testing.assert_allclose(gram - np.diag(np.diag(gram)), 0.0, atol=1e-6)
    us = m.to_grid(0, B[:, :1])[0]
    idx = np.unravel_index(np.argmax(np.abs(us)), us.shape)
    assert np.allclose(np.array(idx) * m.a / m.N, R)
    w = m.width
    peak = (math.pi * w * w) ** -0.75
    assert abs(abs(us[idx]) - peak) < 1e-5 * peak   # cutoff and periodic images


def _tangent(Phi, Z):
    return [Z[k] - Phi[k] @ (0.5 * (Phi[k].conj().T @ Z[k] + Z[k].conj().T @ Phi[k])) for k in range(len(Phi))]


@pytest.mark.parametrize("nproj,hartree,xc", [(0, 1, 1), (4, 1, 1), (4, 0, 0), (4, 1, 2)])
def test_energy_derivative_equals_residual_pairing(nproj, hartree, xc):
    """Eq. (2.4)/(2.5): d/dh E(pf(Phi + h W)) at h = 0 equals 2 f <R, W> for tangent W
    (central differences, O(h^2)); pins the factors of every energy term against H."""
    m = Model(small(nproj=nproj, kgrid=(2, 1, 1), nb=2, hartree=hartree, xc=xc))
    Phi = earcg.lowdin(start(m))
    pt = earcg.evaluate(m, Phi)
    rng = np.random.default_rng(3)
    Z = [rng.standard_normal(P.shape) + 1j * rng.standard_normal(P.shape) for P in Phi]
    W = _tangent(Phi, Z)
    want = 2 * m.occ * pairing(m, pt.R, W)
    errs = []
    for h in (2e-4, 1e-4):
        ep = m.energy(earcg.lowdin([Phi[k] + h * W[k] for k in range(m.K)]))
        em = m.energy(earcg.lowdin([Phi[k] - h * W[k] for k in range(m.K)]))
        errs.append(abs((ep - em) / (2 * h) - want))
    assert errs[1] < 1e-4 * abs(want)
    assert errs[1] < errs[0] / 3.0   # second-order convergence


def test_energy_and_density_unitary_invariance():
    m = Model(small(nproj=4, kgrid=(2, 1, 1), nb=3))
    Phi = earcg.lowdin(start(m))
    rng = np.random.default_rng(4)
    U = [np.linalg.qr(rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3)))[0] for _ in range(m.K)]
    PhiU = [Phi[k] @ U[k] for k in range(m.K)]
    np.testing.assert_allclose(m.density(PhiU), m.density(Phi), atol=1e-13)
    assert abs(m.energy(PhiU) - m.energy(Phi)) < 1e-12 * abs(m.energy(Phi))


def test_residual_is_in_the_cotangent_space():
    """Phi^* R = 0 and Lambda Hermitian (Sec. 2.2)."""
    m = Model(small(nproj=4, nb=3))
    pt = earcg.evaluate(m, earcg.lowdin(start(m)))
    for k in range(m.K):
        assert np.abs(pt.Phi[k].conj().T @ pt.R[k]).max() < 1e-12
        assert np.abs(pt.Lam[k] - pt.Lam[k].conj().T).max() == 0.0


def test_synthetic_configs_are_well_formed():
    c1 = synth.config_two_atom(1)
    m = Model(c1)
    assert m.nk == [1503]
    c2 = synth.config_diamond(2, kgrid=(1, 1, 1))
    assert synth.mp_grid(4, 4, 4)[0].shape == (64, 3)
    assert np.all(synth.mp_grid(4, 4, 4)[0] >= -0.5) and np.all(synth.mp_grid(4, 4, 4)[0] < 0.5)
    assert len(c2["pos"]) == 8 and c2["nbands"] == 16


def test_workload_sizes():
    """Plane waves at Gamma of the four crystal workloads: two-atom 1,503 (32^3 grid, 2 bands),
    diamond8 2,945 (48^3, 16 bands), diamond64 23,847 (96^3, 128 bands, 256 projectors),
    diamond216 80,725 (128^3, 432 bands, 864 projectors)."""
    from oracle.model import sphere_basis
    cases = [(synth.config_two_atom(1), 1503, 32, 2, 0),
             (synth.config_diamond(2, kgrid=(1, 1, 1)), 2945, 48, 16, 32),
             (synth.config_diamond_supercell(2), 23847, 96, 128, 256),
             (synth.config_diamond_supercell(3), 80725, 128, 432, 864)]
    for cfg, n, N, p, nproj in cases:
        b = 2 * math.pi / cfg["a"]
        assert len(sphere_basis(cfg["N"], np.zeros(3), cfg["ecut"], b)) == n
        assert cfg["N"] == N and cfg["nbands"] == p
        assert len(cfg["pos"]) * cfg["nproj_per_atom"] == nproj
