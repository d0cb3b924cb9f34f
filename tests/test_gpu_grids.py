"""Every grid size and line-FFT plan variant with compiled kernels, against the FP64 CPU oracle.

Each supported N gets a small two-atom crystal (two bands, s/p projectors, a shifted
k-point) whose cutoff sphere reaches about a quarter of the grid, so that every
transform phase (x columns, z rows, y lines, the potential multiply, the density) runs
on several lines with a partial disk.  Density and potential (FP64-accurate transforms,
including the full 3D FFT of the Hartree term) to relative 1e-11; H psi to 1e-11 with
FP64-accurate transforms and 5e-6 with FP32 transforms (the tolerances of the main parity
suite).  The FP64-accurate transforms run both ways: in double-float arithmetic (pairs of
FP32 numbers, the default) and in plain FP64."""
import math

import numpy as np
import pytest

from oracle.model import Model
from tests.conftest import ensure_library
from tests.small_models import small

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
ensure_library()
import paper_2503_16225_gb300 as E  # noqa: E402

GRID_N = (8, 12, 16, 20, 24, 32, 36, 40, 48, 64, 72, 80, 96)
PLAN1_N = (16, 32, 36, 48, 64, 72)   # sizes with a second line plan
CASES = [(n, 0, 1) for n in GRID_N] + [(n, 1, 1) for n in PLAN1_N] + [(n, 0, 0) for n in GRID_N]


def grid_model(N):
    a = 8.0
    b = 2.0 * math.pi / a
    mmax = 0.23 * N                      # sphere radius in grid units
    ecut = 0.5 * (b * mmax) ** 2
    return small(a=a, N=N, ecut=ecut, nb=2, nproj=4, kgrid=(2, 1, 1), seed=40 + N)


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


@pytest.mark.parametrize("N,plan,df", CASES)
def test_grid_size(N, plan, df):
    cfg = grid_model(N)
    model = Model(cfg)
    s = E.System(cfg, E.eacg_default_params(fft_plan=plan, df_transforms=df))
    try:
        assert E.eacg_get_plans(s.h) == (plan, plan)
        assert s.nk == model.nk
        rng = np.random.default_rng(N)
        Phi = [np.linalg.qr(rng.standard_normal((n, 2)) + 1j * rng.standard_normal((n, 2)))[0] for n in model.nk]
        t = torch.zeros((s.K, s.p, s.n_max), dtype=torch.complex128)
        for k, P in enumerate(Phi):
            t[k, :, :P.shape[0]] = torch.from_numpy(np.ascontiguousarray(P.T))
        phi = t.cuda()
        rho = s.grid()
        E.eacg_density(s.h, phi, rho, 0)
        rho_o = model.density(Phi)
        assert rel(rho.cpu().numpy(), rho_o) < 1e-11
        v = s.grid()
        E.eacg_get_potential(s.h, v)
        vtot = model.potentials(rho_o)[0]
        assert rel(v.cpu().numpy(), vtot) < 1e-11
        C = [rng.standard_normal(P.shape) + 1j * rng.standard_normal(P.shape) for P in Phi]
        t.zero_()
        for k, Ck in enumerate(C):
            t[k, :, :Ck.shape[0]] = torch.from_numpy(np.ascontiguousarray(Ck.T))
        c = t.cuda()
        for prec, tol in ((0, 1e-11), (1, 5e-6)):
            out = s.block()
            E.eacg_apply_H(s.h, c, out, prec)
            h = out.cpu().numpy()
            for k in range(model.K):
                got = h[k, :, :model.nk[k]].T
                assert rel(got, model.apply_H(k, C[k], vtot)) < tol, (N, prec, k)
                assert np.all(h[k, :, model.nk[k]:] == 0)
    finally:
        s.close()


@pytest.mark.parametrize("N", [24, 48])
def test_autotune_picks_a_compiled_plan(N):
    """fft_plan = -1 (default) times the plans at set-up: the choice is a compiled variant (0 where
    the size has one plan), and a second system of the same shape reuses the cached choice."""
    cfg = grid_model(N)
    a = E.System(cfg)
    b = E.System(cfg)
    try:
        pa, pb = E.eacg_get_plans(a.h), E.eacg_get_plans(b.h)
        assert pa == pb
        assert all(x in ((0, 1) if N in PLAN1_N else (0,)) for x in pa)
    finally:
        a.close()
        b.close()


def test_grid_128_fp32_transforms():
    """N = 128 (the 216-atom supercell's grid): the FP32 transforms (one in-place plane of
    128 x 129 complex64 values per CTA) give the oracle's density, potential and H psi to the
    FP32 bound 5e-6; the FP64-accurate transforms, whose plane would not fit a CTA's shared
    memory, are refused with EACG_EUNSUPPORTED before any launch."""
    N = 128
    cfg = grid_model(N)
    model = Model(cfg)
    s = E.System(cfg)
    try:
        assert s.nk == model.nk
        rng = np.random.default_rng(N)
        Phi = [np.linalg.qr(rng.standard_normal((n, 2)) + 1j * rng.standard_normal((n, 2)))[0] for n in model.nk]
        t = torch.zeros((s.K, s.p, s.n_max), dtype=torch.complex128)
        for k, P in enumerate(Phi):
            t[k, :, :P.shape[0]] = torch.from_numpy(np.ascontiguousarray(P.T))
        phi = t.cuda()
        with pytest.raises(E.EacgError) as err:
            E.eacg_density(s.h, phi, None, 0)
        assert err.value.code == 9
        rho = s.grid()
        E.eacg_density(s.h, phi, rho, 1)
        rho_o = model.density(Phi)
        assert rel(rho.cpu().numpy(), rho_o) < 5e-6
        v = s.grid()
        E.eacg_get_potential(s.h, v)
        vtot = model.potentials(rho_o)[0]
        assert rel(v.cpu().numpy(), vtot) < 5e-6
        C = [rng.standard_normal(P.shape) + 1j * rng.standard_normal(P.shape) for P in Phi]
        t.zero_()
        for k, Ck in enumerate(C):
            t[k, :, :Ck.shape[0]] = torch.from_numpy(np.ascontiguousarray(Ck.T))
        out = s.block()
        E.eacg_apply_H(s.h, t.cuda(), out, 1)
        h = out.cpu().numpy()
        for k in range(model.K):
            got = h[k, :, :model.nk[k]].T
            assert rel(got, model.apply_H(k, C[k], vtot)) < 5e-6, k
            assert np.all(h[k, :, model.nk[k]:] == 0)
        with pytest.raises(E.EacgError):
            E.eacg_apply_H(s.h, t.cuda(), out, 0)
    finally:
        s.close()
