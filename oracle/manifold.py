"""Stiefel-manifold geometry of the oracle (FP64, one k-point block at a time).

TEST INFRASTRUCTURE ONLY (see oracle/model.py).

Blocks are (n, p) complex arrays; the outer product of Sec. 2.1 becomes
[[V, W]] = V^* W in the orthonormal plane-wave basis (Sec. 5.1).
"""
from __future__ import annotations

import numpy as np


def outer(V, W):
    """[[V, W]] = V^* W (Sec. 2.1, discrete form of Sec. 5.1)."""
    return V.conj().T @ W


def herm(M):
    return 0.5 * (M + M.conj().T)


def polar(Psi):
    """Polar decomposition Psi = pf(Psi) Sf(Psi) (Eq. (3.1)) from the eigenvalue
    decomposition [[Psi, Psi]] = V D V^*: pf = Psi V D^{-1/2} V^*, Sf = V D^{1/2} V^*.
    Returns (pf, d, V) with d the eigenvalues of the Gram matrix."""
    d, V = np.linalg.eigh(herm(outer(Psi, Psi)))
    if d.min() <= 0:
        raise FloatingPointError("polar factor of a rank-deficient frame")
    pf = Psi @ (V * d ** -0.5) @ V.conj().T
    return pf, d, V


def sf_from(d, V):
    return (V * np.sqrt(d)) @ V.conj().T


def sf_inv_from(d, V):
    return (V / np.sqrt(d)) @ V.conj().T


def retract(Phi, xi):
    """Polar retraction R_Phi(xi) = pf(Phi + xi) (Eq. (3.2))."""
    return polar(Phi + xi)


def lyapunov(d_s, V, M):
    """Solve S X + X S = M with S = V diag(d_s) V^* Hermitian positive definite
    (Eq. (3.4)): X = V [ (V^* M V)_ij / (d_i + d_j) ] V^*."""
    Mt = V.conj().T @ M @ V
    return V @ (Mt / (d_s[:, None] + d_s[None, :])) @ V.conj().T


def transport_general(Phi, xi, eta):
    """Differentiated polar-retraction transport T_xi(eta) = (eta - R(xi) X) S^{-1},
    S = Sf(Phi + xi), S X + X S = [[xi, eta]] + [[eta, xi]] (Prop. 1, Sec. 3.2)."""
    Phip, d, V = polar(Phi + xi)
    ds = np.sqrt(d)
    X = lyapunov(ds, V, outer(xi, eta) + outer(eta, xi))
    return (eta - Phip @ X) @ sf_inv_from(d, V)


def transport_self(Phi, tau, eta):
    """Closed form for xi = tau eta (Sec. 3.2):
    T_{tau eta}(eta) = eta S^{-1} - tau R(tau eta) [[eta S^{-1}, eta S^{-1}]]."""
    Phip, d, V = polar(Phi + tau * eta)
    ES = eta @ sf_inv_from(d, V)
    return ES - tau * Phip @ outer(ES, ES)


def tangent_defect(Phi, eta):
    """|| [[Phi, eta]] + [[eta, Phi]] ||_F, zero on the tangent space (Eq. (2.3))."""
    M = outer(Phi, eta)
    return float(np.linalg.norm(M + M.conj().T))
