"""Block overlaps of complex64 blocks on the tensor cores (tcgen05, 3 x TF32 split) and on the
SIMT FP32 path, against FP64 products of the same FP32 inputs.

Shapes span several 128-row tiles of C (with a ragged last tile), one and two column tiles
(128 + 16), several 1024-row chunks with a ragged tail, a single row, and an empty reduction.
The bound 2e-6 of max |error| / max |C| is the FP32 accumulation over a 1024-row chunk of
random data; plain TF32 products (10-bit mantissa) would miss it by two orders."""
import numpy as np
import pytest

from tests.conftest import ensure_library

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
ensure_library()
import paper_2503_16225_gb300 as E  # noqa: E402

SHAPES = [(1, 23847, 256, 128), (3, 1000, 130, 16), (2, 2049, 128, 144), (1, 1, 128, 16), (2, 3000, 384, 48)]


def blocks(K, L, m, n, seed):
    rng = np.random.default_rng(seed)
    a = (rng.standard_normal((K, m, L)) + 1j * rng.standard_normal((K, m, L))).astype(np.complex64)
    b = (rng.standard_normal((K, n, L)) + 1j * rng.standard_normal((K, n, L))).astype(np.complex64)
    return a, b


def reference(a, b):
    a64, b64 = a.astype(np.complex128), b.astype(np.complex128)
    # C_k[i, j] = sum_l conj(a_k[i, l]) b_k[j, l]
    return np.einsum("kil,kjl->kij", a64.conj(), b64)


@pytest.mark.parametrize("K,L,m,n", SHAPES)
@pytest.mark.parametrize("method", [1, 0])
def test_overlap_matches_fp64(K, L, m, n, method):
    a, b = blocks(K, L, m, n, seed=L + m + n)
    want = reference(a, b)
    c = torch.full((K, n, m), float("nan"), dtype=torch.complex128, device="cuda")
    assert E.eacg_overlap_c64(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), c, method) == 0
    got = c.cpu().numpy().transpose(0, 2, 1)   # column-major m x n per k
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err < 2e-6, (method, err)


def test_empty_reduction_and_ineligible_shape():
    a, b = blocks(2, 4, 128, 16, seed=1)
    c = torch.full((2, 16, 128), 7.0, dtype=torch.complex128, device="cuda")
    ad, bd = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    # L = 0: nothing to sum, C = 0
    assert int(E.lib.eacg_overlap_c64(2, 0, 128, 16, E._ptr(ad), E._ptr(bd), E._ptr(c), 1, None)) == 0
    assert torch.count_nonzero(c).item() == 0
    # fewer than 128 rows of C, or n not a multiple of 16: not on the tensor cores
    a2, b2 = blocks(1, 64, 64, 16, seed=2)
    c2 = torch.zeros((1, 16, 64), dtype=torch.complex128, device="cuda")
    assert E.eacg_overlap_c64(torch.from_numpy(a2).cuda(), torch.from_numpy(b2).cuda(), c2, 1) == 9
    a3, b3 = blocks(1, 64, 128, 20, seed=3)
    c3 = torch.zeros((1, 20, 128), dtype=torch.complex128, device="cuda")
    assert E.eacg_overlap_c64(torch.from_numpy(a3).cuda(), torch.from_numpy(b3).cuda(), c3, 1) == 9


def test_tensor_core_and_simt_paths_agree_on_the_supercell_H():
    """The supercell's FP32-phase H application with the projector overlaps on the tensor cores
    and on the SIMT path: same result to FP32 rounding."""
    import synth
    cfg = synth.config_diamond_supercell(2)
    outs = []
    for tc in (1, 0):
        s = E.System(cfg, E.eacg_default_params(tensor_cores=tc))
        try:
            rng = np.random.default_rng(5)
            t = torch.zeros((s.K, s.p, s.n_max), dtype=torch.complex128)
            n = s.nk[0]
            t[0, :, :n] = torch.from_numpy(rng.standard_normal((s.p, n)) + 1j * rng.standard_normal((s.p, n)))
            out = s.block()
            E.eacg_apply_H(s.h, t.cuda(), out, 1)
            outs.append(out.cpu().numpy())
        finally:
            s.close()
    assert np.abs(outs[0] - outs[1]).max() / np.abs(outs[1]).max() < 5e-6


BP_SHAPES = [(1, 23847, 256, 128), (3, 1000, 130, 16), (2, 65, 5, 256), (1, 1, 16, 32)]


@pytest.mark.parametrize("K,L,m,n", BP_SHAPES)
@pytest.mark.parametrize("method", [1, 0])
def test_backprojection_matches_fp64(K, L, m, n, method):
    """c_k += a_k q_k (the nonlocal back-projection B (D P)): ragged 64-row tiles of C, ragged
    16-index reduction stages, the largest column count (256), one row; c keeps what it held."""
    rng = np.random.default_rng(L + 7 * m + n)
    a = (rng.standard_normal((K, m, L)) + 1j * rng.standard_normal((K, m, L))).astype(np.complex64)
    q = rng.standard_normal((K, n, m)) + 1j * rng.standard_normal((K, n, m))
    c0 = rng.standard_normal((K, n, L)) + 1j * rng.standard_normal((K, n, L))
    # column-major: C_k[l, j] = sum_i A_k[l, i] Q_k[i, j], A_k[l, i] = a[k, i, l], Q_k[i, j] = q[k, j, i]
    prod = np.einsum("kil,kji->kjl", a.astype(np.complex128), q)
    c = torch.from_numpy(c0.copy()).cuda()
    assert E.eacg_backproject_c64(torch.from_numpy(a).cuda(), torch.from_numpy(q).cuda(), c, method) == 0
    got = c.cpu().numpy() - c0
    err = np.abs(got - prod).max() / np.abs(prod).max()
    assert err < 2e-6, (method, err)


def test_backprojection_ineligible_shapes():
    a = torch.zeros((1, 16, 64), dtype=torch.complex64, device="cuda")
    for n in (20, 272):
        q = torch.zeros((1, n, 16), dtype=torch.complex128, device="cuda")
        c = torch.zeros((1, n, 64), dtype=torch.complex128, device="cuda")
        assert E.eacg_backproject_c64(a, q, c, 1) == 9


def test_fom_projector_overlaps_on_tensor_cores_inside_graphs():
    """32 atoms with 4 projectors each (nproj = 128) and 32 bands: the FP32 FOM's projector
    overlaps take the tensor-core kernel, captured in the FOM's CUDA graph and replayed.  At a
    point eight warm-up iterations in (Sec. 5.2's setting: the shifted operator is near its
    coercive regime, Prop. 4) the gradient of both overlap kernels equals, element by element,
    the oracle's gradient after the same number of FOM iterations per k (Algorithm 4), within
    the FP32 bound of the mixed-mode FOM (5e-3 of max |G|, derived with the FP32-Krylov
    gradient test of the parity suite: FP32 rounding amplified by |A| / mu in the projected
    shifted solves)."""
    import synth
    from oracle import earcg
    from oracle.model import Model
    rng = np.random.default_rng(31)
    pos = rng.uniform(0.0, 12.0, size=(32, 3))
    cfg = synth._config("tc_fom", 12.0, pos, [2] * 32, [1.0] * 32, 4, 0.7,
                        rng.uniform(0.5, 2.0, size=(32, 2)), 3.0, 16, 32, (1, 1, 1), 31)
    model = Model(cfg)
    raw = synth.raw_coefficients(cfg["seed"], model.nk, model.p)
    Psi0 = [raw[k, :, :model.nk[k]].T.copy() for k in range(model.K)]
    Phi = earcg.solve(model, Psi0, earcg.Params(max_outer=8), warm=True).Phi
    pt = earcg.evaluate(model, Phi)
    stats = {"fom_iters": [], "h_cols": 0}
    earcg.ea_gradient(model, pt, earcg.Params(), stats)
    n = model.nk[0]
    errs = {}
    for tc in (1, 0):
        st = torch.cuda.Stream()
        s = E.System(cfg, E.eacg_default_params(precision=1, tensor_cores=tc), stream=st.cuda_stream)
        try:
            assert s.nk == model.nk
            t = torch.zeros((1, s.p, s.n_max), dtype=torch.complex128)
            t[0, :, :n] = torch.from_numpy(np.ascontiguousarray(Phi[0].T))
            phi, g = t.cuda(), s.block()
            torch.cuda.synchronize()
            iters = E.eacg_ea_gradient(s.h, phi, g, 1, 1)
            got = g.cpu().numpy()[0, :, :n].T
            replays = E.eacg_graph_launches(s.h)
        finally:
            s.close()
        assert iters[0] >= 3 and replays > 0, (iters, replays)
        assert abs(iters[0] - stats["fom_iters"][0]) <= 1, (iters, stats["fom_iters"])
        want = earcg.ea_gradient(model, pt, earcg.Params(), fixed_iters=iters)[0]
        errs[tc] = (iters[0], np.abs(got - want).max() / np.abs(want).max())
    assert max(e for _, e in errs.values()) < 5e-3, errs
