"""eacg_step_many: several systems stepped together, their transforms launched together over a
table of (system, band) work items, give bit for bit the results of stepping each system
alone (Algorithm 3 is per system; batching only changes which launch carries a band).  Also
the process-wide batching of concurrent eacg_step calls in the serving loop."""
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
from paper_2503_16225_gb300 import serve  # noqa: E402


def _configs():
    # two systems on a 24^3 grid (batched together), one on 16^3, one on 32^3 with projectors
    return [small(nproj=0, kgrid=(3, 1, 1), nb=4, ecut=4.0, N=24, seed=23),
            small(nproj=4, kgrid=(2, 1, 1), nb=3, ecut=4.0, N=24, seed=24),
            small(nproj=1, kgrid=(1, 1, 1), nb=2, N=16, seed=22),
            synth.config_two_atom(1)]


def _start(cfg, prec, stream):
    s = E.System(cfg, E.eacg_default_params(precision=prec), stream=stream)
    raw = synth.raw_coefficients(cfg["seed"], s.nk, s.p, s.n_max)
    E.eacg_set_psi(s.h, torch.from_numpy(raw).cuda())
    return s


@pytest.mark.parametrize("precision", [0, 1])
def test_step_many_equals_steps_alone(precision):
    cfgs = _configs()
    steps = 6
    alone = []
    for cfg in cfgs:
        st = E.eacg_stream_create()
        s = _start(cfg, precision, st)
        hist = [(i.E, i.rnorm, i.tau) for i in (E.eacg_step(s.h) for _ in range(steps))]
        phi = s.block()
        E.eacg_get_psi(s.h, phi)
        alone.append((hist, phi.cpu()))
        s.close()
        E.eacg_stream_destroy(st)
    streams = [E.eacg_stream_create() for _ in cfgs]
    systems = [_start(cfg, precision, st) for cfg, st in zip(cfgs, streams)]
    g0, m0 = E.eacg_batch_counts()
    hist = [[] for _ in cfgs]
    for _ in range(steps):
        infos, sts = E.eacg_step_many([s.h for s in systems], window_us=2000)
        assert sts == [0] * len(cfgs)
        for i, info in enumerate(infos):
            hist[i].append((info.E, info.rnorm, info.tau))
    g1, m1 = E.eacg_batch_counts()
    # the two 24^3 systems shared launches: more requests than groups
    assert g1 > g0 and (m1 - m0) > (g1 - g0)
    for i, s in enumerate(systems):
        assert hist[i] == alone[i][0]
        phi = s.block()
        E.eacg_get_psi(s.h, phi)
        assert torch.equal(phi.cpu(), alone[i][1])
        s.close()
    for st in streams:
        E.eacg_stream_destroy(st)


def test_step_many_rejects_repeated_systems():
    st = E.eacg_stream_create()
    s = _start(_configs()[2], 1, st)
    try:
        with pytest.raises(E.EacgError):
            E.eacg_step_many([s.h, s.h])
        infos, sts = E.eacg_step_many([s.h])
        assert sts == [0] and np.isfinite(infos[0].E)
    finally:
        s.close()
        E.eacg_stream_destroy(st)


def test_served_with_batching_equals_alone():
    """Resident requests of the serving loop stepping with process-wide batching on reach
    bitwise the results they reach alone (the served energies of the stream's batched mode)."""
    cfgs = _configs()

    def reqs():
        out = []
        for i, cfg in enumerate(cfgs):
            def raw(nk, n_max, cfg=cfg):
                return torch.from_numpy(synth.raw_coefficients(cfg["seed"], nk, cfg["nbands"], n_max))
            out.append(serve.Request(rid=i, cfg=cfg, raw=raw, arrival=0.0))
        return out
    alone = {}
    for r in reqs():
        o = serve.Server(hbm_budget=1 << 40, max_resident=1, precision=1, keep_psi=True).run([r])[0]
        assert o.converged
        alone[o.rid] = o
    g0, m0 = E.eacg_batch_counts()
    E.eacg_batching(500)
    try:
        mix = serve.Server(hbm_budget=1 << 40, max_resident=4, precision=1, keep_psi=True).run(reqs())
    finally:
        E.eacg_batching(-1)
    g1, m1 = E.eacg_batch_counts()
    assert m1 - m0 > g1 - g0 > 0
    for o in mix:
        a = alone[o.rid]
        assert o.converged and o.E == a.E and o.iterations == a.iterations
        assert torch.equal(o.psi, a.psi)
