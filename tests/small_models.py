"""Small synthetic crystals for the CPU pins (seconds of oracle time)."""
import numpy as np

import synth


def small(a=8.0, N=16, ecut=3.0, nb=2, pos=((1.0, 2.0, 3.0), (5.0, 4.5, 2.5)), Z=(2, 2),
          rc=(1.0, 0.8), nproj=0, width=0.7, D=None, kgrid=(1, 1, 1), hartree=1, xc=1, seed=5):
    pos = np.asarray(pos, np.float64).reshape(-1, 3)
    nat = len(pos)
    if D is None:
        D = np.random.default_rng(seed + 1).uniform(0.5, 2.0, size=(nat, 2))
    return synth._config("small", a, pos, list(Z), list(rc), nproj, width, D, ecut, N, nb, kgrid,
                         seed, hartree=hartree, xc=xc)


def free_electron(a=6.0, N=16, ecut=4.0, nb=7, kgrid=(1, 1, 1)):
    return synth._config("free", a, np.zeros((0, 3)), [], [], 0, 0.7, np.zeros((0, 2)), ecut, N,
                         nb, kgrid, 9, hartree=0, xc=0)


def start(model, seed=11):
    raw = synth.raw_coefficients(seed, model.nk, model.p)
    return [raw[k, :, :model.nk[k]].T.copy() for k in range(model.K)]
