"""The allocation-free overlap entry point (for callers that cannot allocate device memory)
agrees with the library's own result: herm(Phi^* (H Phi)) from eacg_overlap_noalloc equals
the Lambda that eacg_energy returns, on two calls in a row.  Collected last on purpose."""
import numpy as np
import pytest

import synth
from oracle import earcg
from oracle.model import Model
from tests.conftest import ensure_library

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
ensure_library()
import paper_2503_16225_gb300 as E  # noqa: E402


def _blocks(s, model, raw):
    Phi = earcg.lowdin([raw[k, :, :model.nk[k]].T.copy() for k in range(model.K)])
    t = torch.zeros((s.K, s.p, s.n_max), dtype=torch.complex128)
    for k, b in enumerate(Phi):
        t[k, :, :b.shape[0]] = torch.from_numpy(np.ascontiguousarray(b.T))
    return t.cuda()


@pytest.mark.parametrize("name", ["diamond_k2", "two_atom"])
def test_overlap_noalloc_matches_lambda_of_eacg_energy(name):
    cfg = synth.config_diamond(2, kgrid=(2, 2, 2)) if name == "diamond_k2" else synth.config_two_atom(1)
    model = Model(cfg)
    s = E.System(cfg)
    for call, seed in enumerate((cfg["seed"], cfg["seed"] + 7)):
        raw = synth.raw_coefficients(seed, model.nk, model.p, s.n_max)
        phi = _blocks(s, model, raw)
        lam = torch.zeros((s.K, s.p, s.p), dtype=torch.complex128, device="cuda")
        E.eacg_energy(s.h, phi, lam, None, 0)              # sets the potential of phi and Lambda
        hphi = s.block()
        E.eacg_apply_H(s.h, phi, hphi, 0)
        ov = torch.full((s.K, s.p, s.p), float("nan"), dtype=torch.complex128, device="cuda")
        assert E.eacg_overlap_noalloc(phi, hphi, ov) == 0
        got = ov.cpu().numpy()
        got = 0.5 * (got + np.conj(np.transpose(got, (0, 2, 1))))
        want = lam.cpu().numpy()
        err = np.abs(got - want).max() / np.abs(want).max()
        assert err < 1e-11, (call, err)
    s.close()


def test_overlap_noalloc_rejects_sizes_beyond_its_scratch():
    K, p, n = 64, 96, 1024   # 64 * 1 * 96 * 96 partials > 524288
    a = torch.zeros((K, p, n), dtype=torch.complex128, device="cuda")
    c = torch.zeros((K, p, p), dtype=torch.complex128, device="cuda")
    assert E.eacg_overlap_noalloc(a, a, c) == 1   # EACG_EINVAL
    # more k-points than one grid row holds (65536 * 1 * 1 * 1 partials fit the scratch)
    a1 = torch.zeros((65536, 1, 1), dtype=torch.complex128, device="cuda")
    c1 = torch.zeros((65536, 1, 1), dtype=torch.complex128, device="cuda")
    assert E.eacg_overlap_noalloc(a1, a1, c1) == 1
    # mismatched operands are refused before the call
    with pytest.raises(ValueError):
        E.eacg_overlap_noalloc(a, a[:, :, :512], c)
    # more k-points than one grid row holds (65536 * 1 * 1 * 1 partials fit the scratch)
    a1 = torch.zeros((65536, 1, 1), dtype=torch.complex128, device="cuda")
    c1 = torch.zeros((65536, 1, 1), dtype=torch.complex128, device="cuda")
    assert E.eacg_overlap_noalloc(a1, a1, c1) == 1
    # mismatched operands are refused before the call
    with pytest.raises(ValueError):
        E.eacg_overlap_noalloc(a, a[:, :, :512], c)
