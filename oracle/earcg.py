"""Energy-adaptive Riemannian CG (Algorithm 3) with the modified secant step size
(Algorithm 2) and hybrid FR-PRP parameter (Sec. 3.4), FP64, on the product of
Stiefel manifolds over k-points (Eq. (5.1)).

TEST INFRASTRUCTURE ONLY (see oracle/model.py).

Readings where the paper is silent, ambiguous or inconsistent:
  * Hamiltonian H = -1/2 Laplacian + V with occupation f = 2, shift mu = 0.01 on H;
    f'(t) = 2 f <r(t), T_{t eta}(eta)> (Eq. (2.5) with DE = 2 f <H Phi, .>);
  * energy test of the approximate Wolfe conditions (Eq. (3.7)) and of the
    "too big" branch of Algorithm 2 read as f(t) <= f(0) + eps |f(0)| (the printed
    (1 + eps) f(0) is stricter than monotone for negative energies);
  * Algorithm 2's bracket update inside [a, b] keeps [a, tau] when f' changes
    sign in [a, tau], i.e. when f'(tau) >= 0, and [tau, b] otherwise (the printed
    condition "f'(tau) < 0" contradicts the comment beside it and Hager-Zhang);
  * a degenerate secant (|f'(b) - f'(a)| < 1e-300 or non-finite tau) is treated
    as "too big": tau = gamma b; more than max_ls trials ends with status "linesearch";
  * the "too small" branch (secant tau < a) is tested first, from the secant value
    alone: Algorithm 2 lists it after the "too big" test, which would evaluate f
    left of a, find it above f(0) with f' < 0 and shrink forever on concave stretches;
  * the initial guess is the polar factor of seeded random coefficients, improved
    by a warm-up phase of the same CG with the TPA-preconditioned projected residual
    g = Z - Phi herm(Phi^* Z), Z = P^{-1} R, until ||R||_F <= warm_res (the paper
    starts from an SCF guess, Sec. 5.2);
  * if <r, g_EA> <= 0 at some point, the preconditioned direction replaces the
    energy-adaptive gradient for that iteration; if <r_new, eta_new> >= 0 the
    direction restarts from -g_new;
  * per-k FOM solves stop independently; transport scaling is omitted (Sec. 5.2).

EARGD (the paper's comparison method, Sec. 5.2 list of methods, which points to another
paper for its details) is read as: the same warm-up, then eta = -g_EA with the alternating
Barzilai-Borwein step (odd energy-adaptive steps <s,s>/|<s,y>|, even ones |<s,y>|/<y,y>,
s = tau T(eta), y = g_new - T(g), clamped to [1e-10, 1e10], 1 at the first step) and
Zhang-Hager non-monotone backtracking: tau <- gamma tau until
f(tau) <= C + nm_delta tau f'(0), with C_0 = E_0, Q_0 = 1,
Q_{k+1} = nm_rho Q_k + 1, C_{k+1} = (nm_rho Q_k C_k + E_{k+1}) / Q_{k+1}
(nm_rho = 0.85, nm_delta = 1e-4).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import fom as fom_mod
from .manifold import herm, outer, polar, sf_inv_from, lyapunov
from .model import Model, pairing, residual_norm


@dataclass
class Params:
    mu: float = 0.01
    res_tol: float = 1e-8
    fom_rtol: float = 2.5e-2
    delta: float = 0.05
    sigma: float = 0.1
    gamma: float = 0.5
    eps: float = 1e-12
    warm_res: float = 1e-2
    max_outer: int = 200
    max_warm: int = 100
    max_fom: int = 50
    max_ls: int = 30
    method: int = 0          # 0: EARCG (Algorithm 3); 1: EARGD (gradient descent, BB step)
    nm_rho: float = 0.85     # EARGD non-monotone averaging
    nm_delta: float = 1e-4   # EARGD sufficient decrease against the reference value


@dataclass
class Point:
    """Everything evaluated at one Phi (one density + one H application)."""
    Phi: list
    rho: np.ndarray
    vtot: np.ndarray
    HPhi: list
    Lam: list
    R: list
    E: float
    terms: dict
    rnorm: float


def evaluate(model: Model, Phi) -> Point:
    """Density, potentials, H Phi, Lambda = herm(Phi^* H Phi) (Eq. (2.6)), residual
    R = H Phi - Phi Lambda and energy at Phi."""
    rho = model.density(Phi)
    vtot, _, _ = model.potentials(rho)
    HPhi = [model.apply_H(k, Phi[k], vtot) for k in range(model.K)]
    Lam = [herm(outer(Phi[k], HPhi[k])) for k in range(model.K)]
    R = [HPhi[k] - Phi[k] @ Lam[k] for k in range(model.K)]
    terms = model.energy_terms(Phi, rho)
    return Point(Phi, rho, vtot, HPhi, Lam, R, float(sum(terms.values())), terms, residual_norm(R))


def lowdin(Psi):
    return [polar(P)[0] for P in Psi]


def kinetic_alpha(model: Model, Phi):
    """alpha_i = <phi_i | -1/2 Laplacian | phi_i> per k (orbital-wise kinetic energy)."""
    return [(model.kin[k][:, None] * np.abs(Phi[k]) ** 2).sum(0) for k in range(model.K)]


def precond_gradient(model: Model, pt: Point):
    """Warm-up direction: Z = P^{-1} R with the TPA scaling alpha_i / (1/2|k+G|^2 + alpha_i)
    (unit gain at G = 0), g = Z - Phi herm(Phi^* Z) (tangent at Phi)."""
    alpha = kinetic_alpha(model, pt.Phi)
    g = []
    for k in range(model.K):
        Z = fom_mod.tpa_inverse(model.kin[k], alpha[k])(pt.R[k]) * alpha[k][None, :]
        g.append(Z - pt.Phi[k] @ herm(outer(pt.Phi[k], Z)))
    return g


def ea_gradient(model: Model, pt: Point, prm: Params, stats=None, fixed_iters=None):
    """G_k = Phi_k - X_k (Phi_k^* X_k)^{-1} with H X - X Sigma = Phi, Sigma = Lambda - mu I
    (Sec. 5.2, Eq. (5.2)), X by Algorithm 4 per k.  fixed_iters (one count per k, optional)
    replaces the stopping test of block k by exactly that many FOM iterations (fewer only on
    a rank-0 block), so that another implementation's iterate after the same number of
    iterations can be compared directly."""
    alpha = kinetic_alpha(model, pt.Phi)
    G = []
    p = model.p
    for k in range(model.K):
        Sigma = pt.Lam[k] - prm.mu * np.eye(p)
        rtol, cap = (prm.fom_rtol, prm.max_fom) if fixed_iters is None else (0.0, int(fixed_iters[k]))
        X, it, rel, ncols = fom_mod.fom(
            lambda V, k=k: model.apply_H(k, V, pt.vtot), pt.Phi[k], pt.HPhi[k], Sigma, prm.mu,
            fom_mod.tpa_inverse(model.kin[k], alpha[k]), rtol, cap)
        if stats is not None:
            stats["fom_iters"].append(it)
            stats["h_cols"] += ncols
        M = outer(pt.Phi[k], X)
        G.append(pt.Phi[k] - X @ np.linalg.inv(M))
    return G


class LineSearchError(RuntimeError):
    pass


class Trial:
    """f(t) = E(R_Phi(t eta)) and f'(t) = 2 f <r(t), T_{t eta}(eta)> (Algorithm 2 input)."""

    def __init__(self, model: Model, base: Point, eta, counter):
        self.model, self.base, self.eta, self.counter = model, base, eta, counter

    def __call__(self, t):
        m = self.model
        Phip, T = [], []
        for k in range(m.K):
            Pk, d, V = polar(self.base.Phi[k] + t * self.eta[k])
            ES = self.eta[k] @ sf_inv_from(d, V)
            Phip.append(Pk)
            T.append(ES - t * Pk @ outer(ES, ES))
        pt = evaluate(m, Phip)
        self.counter["evals"] += 1
        return pt, pt.E, 2.0 * m.occ * pairing(m, pt.R, T)


def modified_secant(fdf, f0, df0, tau0, prm: Params):
    """Algorithm 2 on a scalar function.  fdf(t) -> (payload, f(t), f'(t)).

    Stops at the first trial that satisfies the approximate strong Wolfe
    conditions (Eq. (3.7)), f(t) <= f(0) + eps |f(0)| and
    |f'(t)| <= min(sigma, 1 - 2 delta) |f'(0)|.  Returns (tau, payload, trials)."""
    ftol = f0 + prm.eps * abs(f0)
    cmax = min(prm.sigma, 1.0 - 2.0 * prm.delta) * abs(df0)
    trials = 0

    def ev(t):
        nonlocal trials
        if trials >= prm.max_ls:
            raise LineSearchError("line search trial cap reached")
        trials += 1
        return fdf(t)

    a, dfa = 0.0, df0
    b = tau0
    pb, fb, dfb = ev(b)
    cur = (b, pb, fb, dfb)
    while not (cur[2] <= ftol and abs(cur[3]) <= cmax):
        den = dfb - dfa
        tau = (a * dfb - b * dfa) / den if abs(den) >= 1e-300 else float("nan")
        if not math.isfinite(tau):
            # degenerate secant: treated as a too-big step
            b = prm.gamma * b
            a, dfa = 0.0, df0
            pb, fb, dfb = ev(b)
            cur = (b, pb, fb, dfb)
            continue
        if tau < a:
            # step too small: increase the search interval (decided from the secant
            # value alone, before any evaluation at a point left of a)
            b = b / prm.gamma
            a, dfa = 0.0, df0
            pb, fb, dfb = ev(b)
            cur = (b, pb, fb, dfb)
            continue
        pt, ft, dft = ev(tau)
        if ft > ftol and dft < 0:
            # step too big: decrease the search interval
            b = prm.gamma * b
            a, dfa = 0.0, df0
            pb, fb, dfb = ev(b)
            cur = (b, pb, fb, dfb)
        elif tau > b:
            # tau right of the interval: shift it to the right
            a, dfa = b, dfb
            b, pb, fb, dfb = tau, pt, ft, dft
            cur = (tau, pt, ft, dft)
        else:
            if dft >= 0:
                # f' changes sign in [a, tau]
                b, pb, fb, dfb = tau, pt, ft, dft
            else:
                a, dfa = tau, dft
            cur = (tau, pt, ft, dft)
    return cur[0], cur[1], trials


def secant_step(model, base: Point, eta, tau0, prm: Params, counter):
    """Algorithm 2 on f(t) = E(R_Phi(t eta)); returns (tau, point at tau, trials)."""
    f0 = base.E
    df0 = 2.0 * model.occ * pairing(model, base.R, eta)
    return modified_secant(Trial(model, base, eta, counter), f0, df0, tau0, prm)


def nonmonotone_step(model, base: Point, eta, tau0, C, prm: Params, counter):
    """EARGD backtracking: tau0 gamma^j for the first j with f(tau) <= C + nm_delta tau f'(0)."""
    df0 = 2.0 * model.occ * pairing(model, base.R, eta)
    trial = Trial(model, base, eta, counter)
    t = tau0
    for n in range(1, prm.max_ls + 1):
        pt, f, _ = trial(t)
        if f <= C + prm.nm_delta * t * df0:
            return t, pt, n
        t *= prm.gamma
    raise LineSearchError(f"non-monotone backtracking: no acceptable step in {prm.max_ls} trials")


def bb_step(model, s, y, odd: bool) -> float:
    """Alternating Barzilai-Borwein step in the pairing <.,.> (odd: BB1, even: BB2), clamped."""
    ss = pairing(model, s, s)
    sy = abs(pairing(model, s, y))
    yy = pairing(model, y, y)
    t = ss / sy if odd else sy / yy
    if not math.isfinite(t) or t <= 0:
        return 1.0
    return min(max(t, 1e-10), 1e10)


def beta_fr_prp(r_new_g_new: float, r_old_g_old: float, r_new_Tg_old: float) -> float:
    """Hybrid FR-PRP parameter max{0, min{beta_FR, beta_PRP}} in residual pairings (Sec. 3.4)."""
    bfr = r_new_g_new / r_old_g_old
    bprp = (r_new_g_new - r_new_Tg_old) / r_old_g_old
    return max(0.0, min(bfr, bprp))


def transports(base: Point, new: Point, eta, g, tau, model: Model):
    """T_{tau eta}(eta) in closed form and T_{tau eta}(g) via the Lyapunov equation (Sec. 3.2)."""
    Teta, Tg = [], []
    for k in range(model.K):
        Psi = base.Phi[k] + tau * eta[k]
        d, V = np.linalg.eigh(herm(outer(Psi, Psi)))
        Sinv = sf_inv_from(d, V)
        ES = eta[k] @ Sinv
        Teta.append(ES - tau * new.Phi[k] @ outer(ES, ES))
        xi = tau * eta[k]
        X = lyapunov(np.sqrt(d), V, outer(xi, g[k]) + outer(g[k], xi))
        Tg.append((g[k] - new.Phi[k] @ X) @ Sinv)
    return Teta, Tg


@dataclass
class Result:
    Phi: list
    E: float
    rnorm: float
    iterations: int
    warm_iterations: int
    status: str
    history: list = field(default_factory=list)
    point: Point | None = None


def solve(model: Model, Psi0, prm: Params | None = None, warm=True, callback=None) -> Result:
    """Warm-up CG (preconditioned residual) then EARCG (Algorithm 3) until ||R||_F <= res_tol."""
    prm = prm or Params()
    counter = {"evals": 0}
    hist = []
    pt = evaluate(model, lowdin(Psi0))
    counter["evals"] += 1
    phase = "warm" if (warm and pt.rnorm > prm.warm_res) else "ea"
    it = 0
    warm_it = 0
    tau = 1.0
    stats = {"fom_iters": [], "h_cols": 0}

    def direction_g(p: Point):
        if phase == "warm":
            return precond_gradient(model, p), "pc"
        g = ea_gradient(model, p, prm, stats)
        if pairing(model, p.R, g) <= 0:
            return precond_gradient(model, p), "pc"
        return g, "ea"

    g, gkind = direction_g(pt)
    eta = [-x for x in g]
    rg = pairing(model, pt.R, g)
    hist.append(dict(it=0, E=pt.E, rnorm=pt.rnorm, tau=0.0, beta=0.0, phase=phase, gkind=gkind))
    status = "converged" if pt.rnorm <= prm.res_tol else "maxiter"
    gd = prm.method == 1
    C, Q, ea_it = pt.E, 1.0, 0     # EARGD non-monotone reference and energy-adaptive step count
    while pt.rnorm > prm.res_tol:
        if it >= prm.max_outer:
            status = "maxiter"
            break
        try:
            if gd and phase == "ea":
                tau, new, trials = nonmonotone_step(model, pt, eta, tau, C, prm, counter)
                Qn = prm.nm_rho * Q + 1.0
                C = (prm.nm_rho * Q * C + new.E) / Qn
                Q = Qn
                ea_it += 1
            else:
                tau, new, trials = secant_step(model, pt, eta, tau, prm, counter)
        except LineSearchError:
            status = "linesearch"
            break
        it += 1
        if phase == "warm":
            warm_it += 1
        tau_acc = tau  # the accepted step ("tau" in the history is the next step's start)
        Teta, Tg = transports(pt, new, eta, g, tau, model)
        switch = phase == "warm" and (new.rnorm <= prm.warm_res or warm_it >= prm.max_warm)
        if switch:
            phase = "ea"
        pt = new
        if pt.rnorm <= prm.res_tol:
            hist.append(dict(it=it, E=pt.E, rnorm=pt.rnorm, tau=tau, tau_acc=tau_acc, beta=0.0, phase=phase,
                             gkind=gkind, trials=trials))
            status = "converged"
            break
        gn, gkind = direction_g(pt)
        rgn = pairing(model, pt.R, gn)
        if switch:
            beta = 0.0
            tau = 1.0
            C, Q, ea_it = pt.E, 1.0, 0
        elif gd and phase == "ea":
            beta = 0.0
            s_k = [tau * x for x in Teta]
            y_k = [gn[k] - Tg[k] for k in range(model.K)]
            tau = bb_step(model, s_k, y_k, ea_it % 2 == 1)
        else:
            beta = beta_fr_prp(rgn, rg, pairing(model, pt.R, Tg))
        eta = [-gn[k] + beta * Teta[k] for k in range(model.K)]
        if pairing(model, pt.R, eta) >= 0:
            eta = [-x for x in gn]
            beta = 0.0
        g, rg = gn, rgn
        hist.append(dict(it=it, E=pt.E, rnorm=pt.rnorm, tau=tau, tau_acc=tau_acc, beta=beta, phase=phase,
                         gkind=gkind, trials=trials))
        if callback is not None:
            callback(hist[-1])
    res = Result(pt.Phi, pt.E, pt.rnorm, it, warm_it, status, hist, pt)
    res.evals = counter["evals"]
    res.fom_iters = stats["fom_iters"]
    res.h_cols = stats["h_cols"]
    return res
