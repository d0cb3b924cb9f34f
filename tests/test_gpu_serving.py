"""Serving loop on the GPU: requests of uneven size resident together on their own streams
give exactly the result each request gets when served alone."""
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
from paper_2503_16225_gb300 import serve  # noqa: E402


def _requests(arrival_gap=0.0):
    cfgs = [synth.config_two_atom(1),
            small(nproj=4, kgrid=(2, 1, 1), nb=3, seed=21),
            small(nproj=1, kgrid=(1, 1, 1), nb=2, N=16, seed=22),
            small(nproj=0, kgrid=(3, 1, 1), nb=4, ecut=4.0, N=24, seed=23)]
    reqs = []
    for i, cfg in enumerate(cfgs):
        def raw(nk, n_max, cfg=cfg):
            return torch.from_numpy(synth.raw_coefficients(cfg["seed"], nk, cfg["nbands"], n_max))
        reqs.append(serve.Request(rid=i, cfg=cfg, raw=raw, arrival=arrival_gap * i))
    return reqs


@pytest.mark.parametrize("precision", [0, 1])
def test_alone_and_in_the_mix_agree_bitwise(precision):
    alone = {}
    for r in _requests():
        o = serve.Server(hbm_budget=1 << 40, max_resident=1, precision=precision, keep_psi=True).run([r])[0]
        assert o.converged, o.status
        alone[r.rid] = o
    mix = serve.Server(hbm_budget=1 << 40, max_resident=4, precision=precision, keep_psi=True).run(
        _requests(arrival_gap=0.01))
    for o in mix:
        a = alone[o.rid]
        assert o.converged and o.rnorm <= 1e-8
        assert o.E == a.E
        assert o.iterations == a.iterations
        assert torch.equal(o.psi, a.psi)
    st = serve.latency_stats(mix)
    assert st["converged"] == 4 and st["solves_per_s"] > 0


def test_budget_limits_residency():
    reqs = _requests()
    srv = serve.Server(hbm_budget=1, max_resident=4, precision=1)   # every request is oversize
    outs = srv.run(reqs)
    assert all(o.converged for o in outs)
    # each admitted only when the previous one left
    spans = sorted((o.admit, o.done) for o in outs)
    for (a0, d0), (a1, d1) in zip(spans, spans[1:]):
        assert a1 >= d0 - 1e-3


def _golden_serving():
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_serving.json")
    with open(path) as fh:
        return json.load(fh)


@pytest.mark.parametrize("precision,tol", [(1, 1e-6), (0, 1e-8)])
def test_served_stream_requests_match_the_oracle(precision, tol):
    """Requests of the 256-crystal serving stream, served together (continuous batching, own
    streams), reach the energies of the oracle's own converged solves (written to
    tests/golden/oracle_serving.json by tests/golden/make_golden.py): within 1e-6 Ha per atom in
    mixed precision and 1e-8 Ha per atom in FP64."""
    g = _golden_serving()
    rows = sorted(g["solves"].values(), key=lambda r: r["oracle_seconds"])[:6]
    reqs = []
    for j, row in enumerate(rows):
        cfg = synth.config_serving_request(row["request"])

        def raw(nk, n_max, cfg=cfg):
            return torch.from_numpy(synth.raw_coefficients(cfg["seed"], nk, cfg["nbands"], n_max))
        reqs.append(serve.Request(rid=j, cfg=cfg, raw=raw, arrival=0.0))
    outs = serve.Server(hbm_budget=1 << 40, max_resident=6, precision=precision).run(reqs)
    for o, row in zip(outs, rows):
        assert row["status"] == "converged"
        assert o.converged and o.rnorm <= 1e-8, (row["request"], o.status)
        assert abs(o.E - row["E"]) <= tol * row["natoms"], (row["request"], o.E, row["E"])
