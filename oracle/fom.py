"""Preconditioned block FOM for the Sylvester equation H X - X Sigma = Phi (App. A,
Algorithm 4; stopping rule and X_0 of Sec. 5.2), FP64, one k-point block.

TEST INFRASTRUCTURE ONLY (see oracle/model.py).

Readings where the paper is silent or garbled:
  * the new rows of C_{j+1} are V~_{j+1}^* C (the newly added block), which keeps
    C_j = V_j^* C consistent with A_j = V_j^* H V_j;
  * the rank-revealing QR projects out V_j twice, then orthonormalises by a
    Cholesky factorisation of the block Gram matrix with diagonal pivoting, which
    is QR with column pivoting (largest remaining column norm first) written on
    the Gram matrix; it stops when the largest remaining squared column norm is
    below 1e-12 times the largest squared column norm of the block before the
    projection, and repeats the pivoted Cholesky step once on the kept block to
    restore orthonormality; rank 0 ends the iteration;
  * the projected Sylvester equation A_j Y - Y Sigma = C_j is solved by
    diagonalising A_j and Sigma;
  * the TPA preconditioner scales column i by 1 / (1/2 |k+G|^2 + alpha_i),
    alpha_i the kinetic energy of orbital i of the current Phi (Sec. 5.1, 5.2).
"""
from __future__ import annotations

import numpy as np

from .manifold import herm

RANK_TOL = 1e-12


def pivoted_cholesky(G, ref, tol):
    """Diagonally pivoted Cholesky of the Hermitian PSD matrix G: returns (piv, L) with
    G[piv][:, piv] ~ L L^* on the r selected columns (L lower r x r).  Step j takes the
    largest remaining Schur-complement diagonal (first one on ties) and stops when it is
    not above tol * ref.  On a Gram matrix R^* R this is QR with column pivoting of R."""
    S = np.array(G, dtype=np.complex128)
    n = S.shape[0]
    piv = list(range(n))
    L = np.zeros((n, n), dtype=np.complex128)
    r = 0
    for j in range(n):
        d = S.diagonal().real[j:]
        m = j + int(np.argmax(d))
        if not d[m - j] > tol * ref:
            break
        # symmetric swap of positions j and m
        S[[j, m], :] = S[[m, j], :]
        S[:, [j, m]] = S[:, [m, j]]
        L[[j, m], :] = L[[m, j], :]
        piv[j], piv[m] = piv[m], piv[j]
        ljj = np.sqrt(S[j, j].real)
        L[j, j] = ljj
        L[j + 1:, j] = S[j + 1:, j] / ljj
        S[j + 1:, j + 1:] -= np.outer(L[j + 1:, j], L[j + 1:, j].conj())
        r += 1
    return piv[:r], L[:r, :r]


def orthonormalise(R, V=None, tol=RANK_TOL):
    """Orthonormal basis of range((I - V V^*) R), rank-revealing; returns (n, q~) block."""
    R = R.copy()
    ref = float((np.abs(R) ** 2).sum(axis=0).max()) if R.shape[1] else 0.0
    if V is not None and V.shape[1]:
        for _ in range(2):
            R = R - V @ (V.conj().T @ R)
    if not ref > 0:
        return R[:, :0]
    Q = R
    for pass_ref in (ref, None):
        if Q.shape[1] == 0:
            break
        G = herm(Q.conj().T @ Q)
        piv, L = pivoted_cholesky(G, pass_ref if pass_ref is not None else G.diagonal().real.max(), tol)
        # Q_sel = Q_new L^*  =>  Q_new = Q_sel L^{-*}
        Q = np.linalg.solve(L, Q[:, piv].conj().T).conj().T if piv else Q[:, :0]
    return Q


def sylvester_projected(A, Sigma, C):
    """Y with A Y - Y Sigma = C, A and Sigma Hermitian, by diagonalising both."""
    a, U = np.linalg.eigh(herm(A))
    s, Q = np.linalg.eigh(herm(Sigma))
    Ct = U.conj().T @ C @ Q
    Yt = Ct / (a[:, None] - s[None, :])
    return U @ Yt @ Q.conj().T


def tpa_inverse(kin, alpha):
    """Column-wise TPA preconditioner P^{-1}: R[:, i] / (kin + alpha_i)."""
    den = kin[:, None] + alpha[None, :]
    return lambda R: R / den


def fom(apply_H, Phi, HPhi, Sigma, mu, Pinv, rtol=2.5e-2, max_iter=100):
    """Algorithm 4 with X_0 = Phi / mu (Sec. 5.2).  H X_0 = H Phi / mu by linearity.

    Returns (X, iterations, relative residual, number of H-applied columns)."""
    X0 = Phi / mu
    C = Phi - (HPhi / mu - X0 @ Sigma)
    cnorm = np.linalg.norm(C)
    if cnorm == 0:
        return X0, 0, 0.0, 0
    V = orthonormalise(Pinv(C))
    W = apply_H(V)
    ncols = V.shape[1]
    A = herm(V.conj().T @ W)
    Cj = V.conj().T @ C
    it = 0
    while True:
        it += 1
        Y = sylvester_projected(A, Sigma, Cj)
        Res = C - (W @ Y - V @ Y @ Sigma)
        rel = np.linalg.norm(Res) / cnorm
        if rel <= rtol or it >= max_iter:
            break
        Vt = orthonormalise(Pinv(Res), V)
        if Vt.shape[1] == 0:
            break
        Wt = apply_H(Vt)
        ncols += Vt.shape[1]
        H12 = V.conj().T @ Wt
        H22 = herm(Vt.conj().T @ Wt)
        A = np.block([[A, H12], [H12.conj().T, H22]])
        Cj = np.vstack([Cj, Vt.conj().T @ C])
        V = np.hstack([V, Vt])
        W = np.hstack([W, Wt])
    return X0 + V @ Y, it, rel, ncols
