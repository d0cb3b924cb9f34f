"""CUDA-graph replay of the FOM's block H application: results, per-slot profile counts (with
profiling on, so the captured event records are read back) and the launch counter must be the
same as with direct launches (the kernels and their order are identical; every reduction has a
fixed order, so the comparison is bitwise).  Graphs need a stream of the system's own, so each
system here gets one."""
import numpy as np
import pytest

import synth
from tests.conftest import ensure_library
from tests.small_models import small

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)
ensure_library()
import paper_2503_16225_gb300 as E  # noqa: E402


def _gradient(cfg, precision, graphs):
    st = torch.cuda.Stream()
    s = E.System(cfg, E.eacg_default_params(precision=precision, graphs=graphs), stream=st.cuda_stream)
    torch.cuda.synchronize()
    try:
        raw = synth.raw_coefficients(cfg["seed"], s.nk, s.p, s.n_max)
        psi = torch.from_numpy(raw).cuda()
        phi = s.block()
        torch.cuda.synchronize()  # tensors made on torch's stream, used on the system's
        E.eacg_set_psi(s.h, psi)
        E.eacg_get_psi(s.h, phi)
        E.eacg_density(s.h, phi, None, 0)
        outs, its, profs = [], [], []
        for _ in range(2):  # the second call replays graphs captured during the first
            g = s.block()
            torch.cuda.synchronize()
            E.eacg_profile_enable(s.h, 1)
            n0 = E.eacg_launch_count()
            its.append(E.eacg_ea_gradient(s.h, phi, g, s.K, precision))
            st.synchronize()
            profs.append((E.eacg_launch_count() - n0,
                          {k: v["launches"] for k, v in E.eacg_profile_read(s.h).items()}))
            st.synchronize()
            outs.append(g.cpu().numpy())
        replays = E.eacg_graph_launches(s.h)
        assert (replays > 0) if graphs else (replays == 0)
        return outs, its, profs
    finally:
        s.close()


@pytest.mark.parametrize("name,cfg", [("small_nl", small(nproj=4, kgrid=(2, 1, 1), nb=3)),
                                      ("diamond_k2", synth.config_diamond(2, kgrid=(2, 2, 2)))])
@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_equals_direct_launches(name, cfg, precision):
    g_out, g_its, g_prof = _gradient(cfg, precision, 1)
    d_out, d_its, d_prof = _gradient(cfg, precision, 0)
    assert max(max(i) for i in g_its) >= 3, "the FOM must run long enough to capture and replay"
    for a, b in zip(g_out, d_out):
        assert np.array_equal(a, b)
    assert g_its == d_its
    assert g_prof == d_prof
