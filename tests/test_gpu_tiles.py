"""Tile autotune of the block-overlap kernel A^H B: the variant recorded for a system's shapes
is one of the compiled ones, and every variant computes bitwise the same product (every
variant adds the same products in the same order), so the timing-based choice cannot change
a result: FP64 overlaps equal across variants and within 1e-12 of numpy; the FP32 H
application, whose projector overlaps use the kernel, equal across variants bit for bit."""
import numpy as np
import pytest

import synth
from tests.conftest import ensure_library

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
ensure_library()
import paper_2503_16225_gb300 as E  # noqa: E402


def test_tuned_tiles_and_every_variant_agree():
    cfg = synth.config_diamond(2, kgrid=(2, 2, 2))
    s = E.System(cfg)  # set-up times the variants for this system's shapes
    try:
        for prec in (0, 1):
            for m in (s.p, 4 * s.p, 32):
                assert E.eacg_gemm_tile(m, s.p, s.n_max, prec) in (1, 2, 4)
        rng = np.random.default_rng(3)
        K, p, n = 8, s.p, s.n_max
        a = rng.standard_normal((K, p, n)) + 1j * rng.standard_normal((K, p, n))
        b = rng.standard_normal((K, p, n)) + 1j * rng.standard_normal((K, p, n))
        ref = np.einsum("kin,kjn->kji", a.conj(), b)  # column-major p x p: [k][j][i] = (a^* b)_ij
        raw = synth.raw_coefficients(cfg["seed"], s.nk, s.p, s.n_max)
        E.eacg_set_psi(s.h, torch.from_numpy(raw).cuda())
        phi = s.block()
        E.eacg_get_psi(s.h, phi)
        E.eacg_density(s.h, phi, None, 0)
        hs, cs = [], []
        for G in (1, 2, 4):
            E.eacg_force_gemm_tile(G)
            assert E.eacg_gemm_tile(p, p, n, 0) == G
            c = torch.zeros((K, p, p), dtype=torch.complex128, device="cuda")
            assert E.eacg_overlap_noalloc(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), c) == 0
            got = c.cpu().numpy()
            assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-12
            cs.append(got)
            out = s.block()
            E.eacg_apply_H(s.h, phi, out, 1)
            hs.append(out.cpu().numpy())
        for c, h in zip(cs[1:], hs[1:]):
            assert np.array_equal(c, cs[0])
            assert np.array_equal(h, hs[0])
    finally:
        E.eacg_force_gemm_tile(0)
        s.close()


def test_force_rejects_other_values():
    with pytest.raises(E.EacgError):
        E.eacg_force_gemm_tile(3)
