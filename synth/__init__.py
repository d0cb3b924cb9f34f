"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds no arithmetic of the method: it only draws atoms, coupling
constants, k-point fractions and raw random coefficient blocks from explicit
seeds.  Everything the method computes from them (basis, potentials,
orthonormalisation, ...) is done separately by the oracle and by the library.

Seed recipe (every config carries its own ``seed`` s):
  * default_rng(s)   : atom positions when they are random (uniform in the cell)
  * default_rng(s+1) : nonlocal couplings D_s, D_p per atom, uniform in [0.5, 2] Ha
  * default_rng(s+2) : position jitter N(0, 0.05 bohr) of supercells
  * default_rng(s+3) : raw initial coefficients, complex normal, k-major then band
"""
from __future__ import annotations

import math

import numpy as np

DIAMOND_FRAC = np.array(
    [[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0],
     [0.25, 0.25, 0.25], [0.25, 0.75, 0.75], [0.75, 0.25, 0.75], [0.75, 0.75, 0.25]])


def mp_grid(n1: int, n2: int, n3: int):
    """Unshifted Monkhorst-Pack fractions j/n folded to [-1/2, 1/2), equal weights."""
    def fold(j, n):
        f = j / n
        return f - 1.0 if f >= 0.5 else f
    ks = [[fold(i, n1), fold(j, n2), fold(l, n3)]
          for i in range(n1) for j in range(n2) for l in range(n3)]
    kf = np.array(ks, dtype=np.float64).reshape(-1, 3)
    return kf, np.full(len(kf), 1.0 / len(kf))


def _config(name, a, pos, Z, rc, nproj, width, D, ecut, N, nbands, kgrid, seed,
            hartree=1, xc=1, occ=2.0):
    kf, kw = mp_grid(*kgrid)
    return dict(name=name, a=float(a), pos=np.asarray(pos, np.float64).reshape(-1, 3),
                Z=np.asarray(Z, np.int32), rc=np.asarray(rc, np.float64),
                nproj_per_atom=int(nproj), proj_width=float(width),
                D=np.asarray(D, np.float64).reshape(-1, 2), ecut=float(ecut), N=int(N),
                nbands=int(nbands), kfrac=kf, kweight=kw, hartree=int(hartree), xc=int(xc),
                occ=float(occ), seed=int(seed))


def config_two_atom(seed: int = 1):
    """Simple-cubic a=10 bohr, 2 atoms Z=2 at uniform seeded positions, rc=1.0,
    Ecut 10 Ha, 32^3 grid, 2 bands, Gamma only, Hartree + Slater exchange."""
    rng = np.random.default_rng(seed)
    a = 10.0
    pos = rng.uniform(0.0, a, size=(2, 3))
    return _config("two_atom_sc_a10_N32", a, pos, [2, 2], [1.0, 1.0], 0, 0.7,
                   np.zeros((2, 2)), 10.0, 32, 2, (1, 1, 1), seed)


def _diamond_supercell(reps: int, seed: int, jitter: float):
    a0 = 10.26
    frac = np.concatenate([(DIAMOND_FRAC + np.array([i, j, l])) / reps
                           for i in range(reps) for j in range(reps) for l in range(reps)])
    a = a0 * reps
    pos = frac * a
    if jitter > 0:
        pos = pos + np.random.default_rng(seed + 2).normal(0.0, jitter, size=pos.shape)
    nat = len(pos)
    D = np.random.default_rng(seed + 1).uniform(0.5, 2.0, size=(nat, 2))
    return a, pos, nat, D


def config_diamond(seed: int = 2, kgrid=(4, 4, 4), ecut: float = 15.0, N: int = 48):
    """Diamond-structure cubic cell a=10.26, 8 atoms Z=4 (rc 0.8), 4 Gaussian s/p
    projectors per atom (width 0.7), Ecut 15 Ha, 48^3 grid, 16 bands, 4x4x4 k."""
    a, pos, nat, D = _diamond_supercell(1, seed, 0.0)
    return _config(f"diamond8_k{'x'.join(map(str, kgrid))}_ec{ecut:g}_N{N}", a, pos, [4] * nat,
                   [0.8] * nat, 4, 0.7, D, ecut, N, 16, kgrid, seed)


def config_diamond_supercell(reps: int, seed: int = 3, kgrid=(1, 1, 1), ecut: float = 15.0,
                             N: int | None = None):
    """reps^3 diamond supercell (64 atoms for reps=2, 216 for reps=3), positions
    jittered N(0, 0.05 bohr), Ecut 15 Ha, bands = 2 * atoms."""
    a, pos, nat, D = _diamond_supercell(reps, seed, 0.05)
    if N is None:
        N = {2: 96, 3: 128}[reps]
    return _config(f"diamond{nat}_k{'x'.join(map(str, kgrid))}_N{N}", a, pos, [4] * nat,
                   [0.8] * nat, 4, 0.7, D, ecut, N, 2 * nat, kgrid, seed)


GRID_SIZES = (16, 20, 24, 32, 36, 40, 48, 64, 72, 80, 96)


def smooth_grid_size(nmin: int) -> int:
    """Smallest FFT grid edge n >= nmin from GRID_SIZES (edges built from radices 2, 3, 4 or
    2, 4, 5 that the transforms support)."""
    for n in GRID_SIZES:
        if n >= nmin:
            return n
    raise ValueError(f"no supported grid size >= {nmin}")


def config_serving_request(i: int):
    """Request i of the serving stream: cubic a~U[6,14], 1-16 atoms of Z in {1..4},
    rc~U[0.6,1.2], 0/1/4 projectors per atom, Ecut~U[8,20], bands = sum(Z)/2,
    k-grid n^3 with n in {1,2,3}.  Seed 1000+i."""
    seed = 1000 + i
    rng = np.random.default_rng(seed)
    a = rng.uniform(6.0, 14.0)
    nat = int(rng.integers(1, 17))
    Z = rng.integers(1, 5, size=nat)
    while int(Z.sum()) % 2:
        Z[-1] = rng.integers(1, 5)
    rc = rng.uniform(0.6, 1.2, size=nat)
    nproj = int(rng.choice([0, 1, 4]))
    ecut = rng.uniform(8.0, 20.0)
    nk = int(rng.integers(1, 4))
    pos = rng.uniform(0.0, a, size=(nat, 3))
    D = np.random.default_rng(seed + 1).uniform(0.5, 2.0, size=(nat, 2))
    b = 2.0 * math.pi / a
    mmax = math.sqrt(2.0 * ecut) / b + 0.5
    N = smooth_grid_size(int(math.ceil(4.0 * mmax + 1.0)))
    return _config(f"serve{i}", a, pos, Z, rc, nproj, 0.7, D, ecut, N, int(Z.sum()) // 2,
                   (nk, nk, nk), seed)


def raw_coefficients(seed: int, n_per_k, nbands: int, n_max: int | None = None):
    """Raw (not orthonormal) initial coefficients, complex normal with unit variance.

    Returns an array [K, nbands, n_max] (band-major, coefficient index fastest),
    zero-padded beyond n_k.  Values are drawn k by k, band by band, coefficient by
    coefficient in canonical basis order, real then imaginary part per draw pair.
    """
    rng = np.random.default_rng(seed + 3)
    n_per_k = [int(n) for n in n_per_k]
    if n_max is None:
        n_max = max(n_per_k)
    out = np.zeros((len(n_per_k), nbands, n_max), np.complex128)
    for k, n in enumerate(n_per_k):
        x = rng.standard_normal((nbands, n, 2))
        out[k, :, :n] = (x[..., 0] + 1j * x[..., 1]) / math.sqrt(2.0)
    return out


CONFIGS = {
    "two_atom": config_two_atom,
    "diamond": config_diamond,
}
