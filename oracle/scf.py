"""Initial guess of the experiments (Sec. 5.2): self-consistent field iterations until the
density difference of two successive iterates is below a tolerance (0.1 in the paper),
FP64, on the discrete model of oracle/model.py.

TEST INFRASTRUCTURE ONLY (see oracle/model.py).

Readings (the paper names the stopping test only):
  * the first input density is the density of the Lowdin-orthonormalised start Phi0;
  * one SCF step: V = V_loc + V_H(rho_in) + V_xc(rho_in); Phi = the p lowest eigenvectors of
    the linear Hamiltonian H[V] at every k-point (here by dense diagonalisation of the
    explicit matrix, so the step is exact); rho_out = rho(Phi);
  * the density difference is the L2 norm over the cell,
    ||rho_out - rho_in||_2 = (Omega / N^3 sum_j (rho_out - rho_in)_j^2)^{1/2};
  * stop when it is below tol (Phi of that step is the guess); otherwise simple (linear)
    mixing rho_in <- rho_in + alpha (rho_out - rho_in) with the damping alpha = 0.5 (the
    paper names only the stopping test; DFTK's damping 0.8 belongs with its LDOS-preconditioned
    mixing, and with plain linear mixing 0.8 oscillates on the small projector models while
    0.5 converges, so 0.5 is the default on both sides).
"""
from __future__ import annotations

import math

import numpy as np

from .earcg import lowdin
from .model import Model


def density_difference(model: Model, a, b) -> float:
    """(integral over the cell of (a - b)^2)^{1/2} on the grid."""
    return math.sqrt(model.omega / model.N ** 3 * float(((a - b) ** 2).sum()))


def lowest_eigenvectors(model: Model, vtot):
    """The p lowest eigenvectors of H[V] per k-point (dense diagonalisation)."""
    out = []
    for k in range(model.K):
        w, U = np.linalg.eigh(model.dense_H(k, vtot))
        out.append(U[:, :model.p])
    return out


def scf_guess(model: Model, Phi0, tol=0.1, alpha=0.5, max_scf=100):
    """Returns (Phi, steps, history of ||rho_out - rho_in||_2, final input density)."""
    Phi = lowdin(Phi0)
    rho_in = model.density(Phi)
    history = []
    for step in range(1, max_scf + 1):
        vtot = model.potentials(rho_in)[0]
        Phi = lowest_eigenvectors(model, vtot)
        rho_out = model.density(Phi)
        d = density_difference(model, rho_out, rho_in)
        history.append(d)
        if d < tol:
            return Phi, step, history, rho_in
        rho_in = rho_in + alpha * (rho_out - rho_in)
    raise RuntimeError(f"SCF did not reach {tol} in {max_scf} steps")
