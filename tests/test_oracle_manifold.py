"""Pins of the oracle's geometry (Sec. 3.1-3.2), block FOM (App. A), step size
(Algorithm 2) and CG parameter (Sec. 3.4) against closed forms, library routines,
finite differences and crafted scalar functions."""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import earcg, fom
from oracle.manifold import (lyapunov, outer, polar, sf_from, tangent_defect, transport_general,
                             transport_self)
from oracle.model import Model
from tests.small_models import small, start

HERE = os.path.dirname(os.path.abspath(__file__))


def _rand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _stiefel(rng, n, p):
    return np.linalg.qr(_rand(rng, n, p))[0]


def _tangent(Phi, Z):
    M = Phi.conj().T @ Z
    return Z - Phi @ (0.5 * (M + M.conj().T))


def test_polar_factor_properties():
    rng = np.random.default_rng(0)
    Psi = _rand(rng, 40, 5)
    pf, d, V = polar(Psi)
    np.testing.assert_allclose(pf.conj().T @ pf, np.eye(5), atol=1e-13)
    S = sf_from(d, V)
    np.testing.assert_allclose(pf @ S, Psi, atol=1e-12)
    np.testing.assert_allclose(S, S.conj().T, atol=1e-13)
    assert np.linalg.eigvalsh(S).min() > 0
    # library polar decomposition as an independent route
    U, P = sla.polar(Psi, side="right")
    np.testing.assert_allclose(pf, U, atol=1e-12)
    Phi = _stiefel(rng, 40, 5)
    np.testing.assert_allclose(polar(Phi)[0], Phi, atol=1e-13)


def test_lyapunov_matches_library_solver():
    rng = np.random.default_rng(1)
    A = _rand(rng, 6, 6)
    S = A.conj().T @ A + np.eye(6)
    d, V = np.linalg.eigh(S)
    M = _rand(rng, 6, 6)
    X = lyapunov(d, V, M)
    np.testing.assert_allclose(X, sla.solve_continuous_lyapunov(S, M), atol=1e-12)


def test_transport_closed_form_equals_general_form_and_is_tangent():
    rng = np.random.default_rng(2)
    Phi = _stiefel(rng, 30, 4)
    eta = _tangent(Phi, _rand(rng, 30, 4))
    tau = 0.37
    T1 = transport_self(Phi, tau, eta)
    T2 = transport_general(Phi, tau * eta, eta)
    np.testing.assert_allclose(T1, T2, atol=1e-12)
    Phip = polar(Phi + tau * eta)[0]
    assert tangent_defect(Phip, T1) < 1e-12
    g = _tangent(Phi, _rand(rng, 30, 4))
    assert tangent_defect(Phip, transport_general(Phi, tau * eta, g)) < 1e-12


def test_transport_is_the_derivative_of_the_retraction():
    """T_{xi}(eta) = d/dt pf(Phi + xi + t eta) at t = 0 (central differences)."""
    rng = np.random.default_rng(3)
    Phi = _stiefel(rng, 25, 3)
    xi = 0.4 * _tangent(Phi, _rand(rng, 25, 3))
    eta = _tangent(Phi, _rand(rng, 25, 3))
    h = 1e-5
    fd = (polar(Phi + xi + h * eta)[0] - polar(Phi + xi - h * eta)[0]) / (2 * h)
    np.testing.assert_allclose(transport_general(Phi, xi, eta), fd, atol=1e-8)


def test_algorithm3_transports_are_the_retraction_derivatives():
    """earcg.transports (the two transports of each EARCG step, Sec. 3.2; they feed beta,
    Sec. 3.4, and the BB step of EARGD) on two k-blocks of different sizes: T(eta) equals
    the closed form and the central difference of t -> pf(Phi + (tau + t) eta); T(g) equals
    the general Lyapunov form and the central difference of t -> pf(Phi + tau eta + t g).
    A sign slip in the Lyapunov right-hand side, or the old point's Phi where the new one
    belongs, moves T(g) by O(1) against both references."""
    from types import SimpleNamespace
    rng = np.random.default_rng(11)
    tau, h = 0.43, 1e-5
    base, new, eta, g = [], [], [], []
    for n, p in ((27, 3), (19, 3)):
        Phi = _stiefel(rng, n, p)
        e = 0.8 * _tangent(Phi, _rand(rng, n, p))
        base.append(Phi)
        eta.append(e)
        g.append(_tangent(Phi, _rand(rng, n, p)))
        new.append(polar(Phi + tau * e)[0])
    Teta, Tg = earcg.transports(SimpleNamespace(Phi=base), SimpleNamespace(Phi=new), eta, g, tau,
                                SimpleNamespace(K=2))
    for k in range(2):
        Phi, e, gk = base[k], eta[k], g[k]
        np.testing.assert_allclose(Teta[k], transport_self(Phi, tau, e), atol=1e-12)
        fd_eta = (polar(Phi + (tau + h) * e)[0] - polar(Phi + (tau - h) * e)[0]) / (2 * h)
        np.testing.assert_allclose(Teta[k], fd_eta, atol=1e-8)
        np.testing.assert_allclose(Tg[k], transport_general(Phi, tau * e, gk), atol=1e-12)
        fd_g = (polar(Phi + tau * e + h * gk)[0] - polar(Phi + tau * e - h * gk)[0]) / (2 * h)
        np.testing.assert_allclose(Tg[k], fd_g, atol=1e-8)
        # both transports are tangent at the new point (Eq. (2.3))
        assert tangent_defect(new[k], Teta[k]) < 1e-12
        assert tangent_defect(new[k], Tg[k]) < 1e-12


def test_projected_sylvester_matches_library_solver():
    rng = np.random.default_rng(4)
    A = _rand(rng, 9, 9)
    A = A + A.conj().T
    Sig = _rand(rng, 3, 3)
    Sig = Sig + Sig.conj().T - 10 * np.eye(3)
    C = _rand(rng, 9, 3)
    Y = fom.sylvester_projected(A, Sig, C)
    np.testing.assert_allclose(Y, sla.solve_sylvester(A, -Sig, C), atol=1e-11)


def test_orthonormalise_is_rank_revealing():
    rng = np.random.default_rng(5)
    V = _stiefel(rng, 50, 4)
    R = _rand(rng, 50, 3)
    R = np.hstack([R, R[:, :1] * 2.0 + R[:, 1:2], V[:, :1]])   # rank 3 after projecting out V
    Q = fom.orthonormalise(R, V)
    assert Q.shape[1] == 3
    np.testing.assert_allclose(Q.conj().T @ Q, np.eye(3), atol=1e-13)
    assert np.abs(V.conj().T @ Q).max() < 1e-13


def test_pivoted_cholesky_is_qr_with_column_pivoting():
    """On a Gram matrix the pivoted Cholesky is Householder QR with column pivoting (LAPACK
    geqp3): the same pivot order and |L| = |R^*|, so the orthonormalisation is an RRQR."""
    rng = np.random.default_rng(17)
    R = _rand(rng, 40, 7) * np.array([0.3, 2.0, 1.0, 5.0, 0.7, 1.5, 3.0])
    G = R.conj().T @ R
    piv, L = fom.pivoted_cholesky(G, 1.0, 1e-12)
    Qr, Rr, P = sla.qr(R, mode="economic", pivoting=True)
    assert list(P) == piv
    np.testing.assert_allclose(np.abs(L), np.abs(Rr.conj().T), atol=1e-12)
    np.testing.assert_allclose(L @ L.conj().T, G[np.ix_(piv, piv)], atol=1e-11)


def test_pivoted_cholesky_stops_at_the_numerical_rank():
    rng = np.random.default_rng(18)
    B = _rand(rng, 30, 3)
    R = np.hstack([B, B @ _rand(rng, 3, 2)])          # rank 3, five columns
    G = R.conj().T @ R
    piv, L = fom.pivoted_cholesky(G, np.abs(np.diag(G)).max(), 1e-12)
    assert len(piv) == 3
    # the kept columns span range(R)
    Q = np.linalg.solve(L, R[:, piv].conj().T).conj().T
    np.testing.assert_allclose(Q.conj().T @ Q, np.eye(3), atol=1e-12)
    np.testing.assert_allclose(Q @ (Q.conj().T @ R), R, atol=1e-11)


def test_fom_with_tight_tolerance_solves_the_sylvester_equation_exactly():
    """Algorithm 4 with rtol -> 0 reproduces the dense Sylvester solution."""
    m = Model(small(nproj=4, nb=3, ecut=2.0))
    Phi = earcg.lowdin(start(m))
    pt = earcg.evaluate(m, Phi)
    H = m.dense_H(0, pt.vtot)
    mu = 0.01
    Sig = pt.Lam[0] - mu * np.eye(m.p)
    alpha = earcg.kinetic_alpha(m, Phi)[0]
    X, it, rel, _ = fom.fom(lambda V: H @ V, Phi[0], pt.HPhi[0], Sig, mu,
                            fom.tpa_inverse(m.kin[0], alpha), rtol=1e-11, max_iter=200)
    Xd = sla.solve_sylvester(H, -Sig, Phi[0])
    np.testing.assert_allclose(X, Xd, atol=1e-9 * np.abs(Xd).max())


def test_fom_galerkin_condition_and_stopping_rule():
    m = Model(small(nproj=4, nb=3, ecut=2.0))
    Phi = earcg.lowdin(start(m))
    pt = earcg.evaluate(m, Phi)
    H = m.dense_H(0, pt.vtot)
    mu = 0.01
    Sig = pt.Lam[0] - mu * np.eye(m.p)
    alpha = earcg.kinetic_alpha(m, Phi)[0]
    X, it, rel, _ = fom.fom(lambda V: H @ V, Phi[0], pt.HPhi[0], Sig, mu,
                            fom.tpa_inverse(m.kin[0], alpha), rtol=2.5e-2)
    X0 = Phi[0] / mu
    r0 = np.linalg.norm(H @ X0 - X0 @ Sig - Phi[0])
    rj = np.linalg.norm(H @ X - X @ Sig - Phi[0])
    assert rj <= 2.5e-2 * r0 + 1e-12
    assert abs(rj / r0 - rel) < 1e-10


def test_ea_gradient_with_fixed_iteration_counts():
    """ea_gradient(fixed_iters=...) runs exactly the given FOM iteration count per k: with the
    counts the stopping test chose it reproduces the default result bit for bit, and with one
    more iteration per k it gives the iterate of the FOM run for exactly that many iterations
    (Algorithm 4; a Galerkin method, so its residual need not fall monotonically)."""
    m = Model(small(nproj=4, nb=3, ecut=3.0, kgrid=(2, 1, 1)))
    pt = earcg.evaluate(m, earcg.lowdin(start(m)))
    prm = earcg.Params()
    stats = {"fom_iters": [], "h_cols": 0}
    G = earcg.ea_gradient(m, pt, prm, stats)
    its = stats["fom_iters"]
    assert all(i >= 1 for i in its)
    G2 = earcg.ea_gradient(m, pt, prm, fixed_iters=its)
    for a, b in zip(G, G2):
        assert np.array_equal(a, b)
    more = [i + 1 for i in its]
    G3 = earcg.ea_gradient(m, pt, prm, fixed_iters=more)
    for k in range(m.K):
        Sig = pt.Lam[k] - prm.mu * np.eye(m.p)
        alpha = earcg.kinetic_alpha(m, pt.Phi)[k]
        for cap, rtol in ((its[k], prm.fom_rtol), (more[k], 0.0)):
            X, it, rel, _ = fom.fom(lambda V: m.apply_H(k, V, pt.vtot), pt.Phi[k], pt.HPhi[k], Sig, prm.mu,
                                    fom.tpa_inverse(m.kin[k], alpha), rtol=rtol, max_iter=cap)
            assert it == cap
        Gk = pt.Phi[k] - X @ np.linalg.inv(pt.Phi[k].conj().T @ X)
        np.testing.assert_allclose(G3[k], Gk, atol=1e-12 * np.abs(Gk).max())


def test_ea_gradient_with_uniform_shift_is_the_riesz_representative():
    """Cor. 1 with a uniform coercive shift Sigma = -s I and an exact solve: G is tangent
    and g(G, eta) = <(H - Sigma) G, eta> = <R, eta> for tangent eta (Eq. (2.7))."""
    rng = np.random.default_rng(6)
    n, p = 40, 3
    A = _rand(rng, n, n)
    H = A + A.conj().T
    s = -np.linalg.eigvalsh(H).min() + 1.0
    Sig = -s * np.eye(p)
    Phi = _stiefel(rng, n, p)
    X = sla.solve_sylvester(H, -Sig, Phi)
    G = Phi - X @ np.linalg.inv(Phi.conj().T @ X)
    assert tangent_defect(Phi, G) < 1e-11
    R = H @ Phi - Phi @ (Phi.conj().T @ H @ Phi)
    for _ in range(3):
        eta = _tangent(Phi, _rand(rng, n, p))
        lhs = np.vdot(H @ G - G @ Sig, eta).real
        assert abs(lhs - np.vdot(R, eta).real) < 1e-10 * abs(lhs)


def test_shifted_sylvester_operator_spectrum():
    """Proof of Prop. 4: at an eigenbasis, X -> H X - X (Lambda - mu I) has the eigenvalues
    lambda_m - lambda_l + mu (Kronecker sum, checked on a dense matrix)."""
    rng = np.random.default_rng(7)
    n, p, mu = 8, 2, 0.01
    A = _rand(rng, n, n)
    H = A + A.conj().T
    lam, U = np.linalg.eigh(H)
    Phi = U[:, :p]
    Sig = Phi.conj().T @ H @ Phi - mu * np.eye(p)
    L = np.kron(np.eye(p), H) - np.kron(Sig.T, np.eye(n))
    ev = np.sort(np.linalg.eigvals(L).real)
    want = np.sort((lam[:, None] - lam[None, :p] + mu).ravel())
    np.testing.assert_allclose(ev, want, atol=1e-10)


def _prm(**kw):
    return earcg.Params(**kw)


def test_secant_solves_a_quadratic_in_one_step():
    """f(t) = (t - 3)^2: from tau0 = 1 the first secant step lands on the minimiser."""
    f = lambda t: (None, (t - 3.0) ** 2, 2.0 * (t - 3.0))
    tau, _, trials = earcg.modified_secant(f, 9.0, -6.0, 1.0, _prm())
    assert tau == pytest.approx(3.0, abs=1e-14)
    assert trials == 2


def test_secant_accepts_the_initial_step_when_it_is_wolfe():
    f = lambda t: (None, (t - 1.0) ** 2, 2.0 * (t - 1.0))
    tau, _, trials = earcg.modified_secant(f, 1.0, -2.0, 1.0, _prm())
    assert tau == 1.0 and trials == 1


def test_secant_too_big_branch_shrinks_the_interval():
    """A secant point with f > f(0) and f' < 0 (past a hump) resets [a, b] = [0, gamma b]."""
    calls = []

    def g(t):
        calls.append(t)
        if t == 8.0:
            return None, 5.0, -1.0      # first trial: not Wolfe
        if len(calls) == 2:
            return None, 5.0, -0.5      # secant point: f > f0 and f' < 0 -> too big
        return None, (t - 1.0) ** 2 - 1.0, 2.0 * (t - 1.0)

    tau, _, trials = earcg.modified_secant(g, 0.0, -2.0, 8.0, _prm())
    assert calls[2] == 4.0               # tau = gamma * b
    assert tau == pytest.approx(1.0, abs=1e-12)


def test_secant_too_small_branch_expands_the_interval():
    """A secant point left of a (f' decreasing) resets [a, b] = [0, b / gamma]."""
    calls = []

    def g(t):
        calls.append(t)
        if len(calls) == 1:
            return None, -0.1, -30.0    # f' more negative at b than at a: secant gives tau < 0
        return None, (t - 5.0) ** 2 - 25.0, 2.0 * (t - 5.0)

    tau, _, _ = earcg.modified_secant(g, 0.0, -10.0, 1.0, _prm())
    assert calls == [1.0, 2.0, 5.0]      # no evaluation left of a; tau = b / gamma, then secant
    assert tau == pytest.approx(5.0, abs=1e-12)


def test_secant_trial_cap_raises():
    g = lambda t: (None, 1.0 + t, 1.0)  # never satisfies the energy test
    with pytest.raises(earcg.LineSearchError):
        earcg.modified_secant(g, 0.0, -1.0, 1.0, _prm(max_ls=5))


def test_beta_hybrid_fr_prp_clamping():
    assert earcg.beta_fr_prp(2.0, 4.0, 1.0) == pytest.approx(0.25)   # PRP < FR
    assert earcg.beta_fr_prp(2.0, 4.0, -3.0) == pytest.approx(0.5)   # FR < PRP
    assert earcg.beta_fr_prp(2.0, 4.0, 5.0) == 0.0                    # PRP < 0 clamps


def test_oracle_defaults_are_the_paper_constants():
    with open(os.path.join(HERE, "golden", "paper_constants.json")) as fh:
        c = json.load(fh)
    prm = earcg.Params()
    for key in ("delta", "sigma", "gamma", "eps", "mu", "fom_rtol"):
        assert getattr(prm, key) == c[key]["value"], key
    assert min(prm.sigma, 1 - 2 * prm.delta) == c["wolfe_curvature_factor"]["value"]


def test_tpa_shift_of_a_plane_wave_orbital_is_its_kinetic_energy():
    """alpha_i (orbital-wise mean kinetic energy, the TPA shift of Sec. 5.2) of an orbital that
    is one plane wave e^{i(k+G)r} equals 1/2 |k+G|^2."""
    m = Model(small(nb=2, kgrid=(2, 1, 1)))
    for k in range(m.K):
        n = m.nk[k]
        j1, j2 = 3, n - 5
        Phi = np.zeros((n, 2), complex)
        Phi[j1, 0] = 1.0
        Phi[j2, 1] = 1j
        kf = m.kfrac[k]
        want = [0.5 * m.b ** 2 * float(((m.basis[k][j] + kf) ** 2).sum()) for j in (j1, j2)]
        np.testing.assert_allclose(earcg.kinetic_alpha(m, [Phi if q == k else np.eye(m.nk[q], 2)
                                                           for q in range(m.K)])[k], want, rtol=1e-14)


def test_preconditioned_direction_is_tangent_and_a_descent_direction():
    """g = Z - Phi herm(Phi^* Z), Z = P^-1 R: Phi^* g is skew-Hermitian (tangent) and
    <R, g> = <R, P^-1 R> > 0 because Phi^* R = 0 and P^-1 is positive; with P^-1 of unit gain
    at |k+G| = 0 the direction shrinks every plane-wave component of R."""
    m = Model(small(nproj=4, nb=3, kgrid=(2, 1, 1)))
    Phi = earcg.lowdin(start(m))
    pt = earcg.evaluate(m, Phi)
    g = earcg.precond_gradient(m, pt)
    for k in range(m.K):
        M = Phi[k].conj().T @ g[k]
        assert np.abs(M + M.conj().T).max() < 1e-12
    from oracle.model import pairing
    rg = pairing(m, pt.R, g)
    assert rg > 0
    alpha = earcg.kinetic_alpha(m, Phi)
    for k in range(m.K):
        Z = fom.tpa_inverse(m.kin[k], alpha[k])(pt.R[k]) * alpha[k][None, :]
        assert np.all(np.abs(Z) <= np.abs(pt.R[k]) * (1 + 1e-15))
