"""Host logic of the serving loop (admission by HBM budget and slot count, latency
statistics) with fake systems: no GPU work."""
import threading
import time
from types import SimpleNamespace

import pytest

from tests.conftest import ensure_library

ensure_library()
from paper_2503_16225_gb300 import serve  # noqa: E402


class Tracker:
    def __init__(self):
        self.lock = threading.Lock()
        self.bytes = 0
        self.count = 0
        self.max_bytes = 0
        self.max_count = 0
        self.order = []


def install_fakes(monkeypatch, tr, steps_for):
    class FakeSystem:
        def __init__(self, cfg, prm, stream=None):
            self.cfg = cfg
            self.h = SimpleNamespace(cfg=cfg, n=0)
            self.nk, self.n_max = [1], 1
            with tr.lock:
                tr.bytes += cfg["bytes"]
                tr.count += 1
                tr.max_bytes = max(tr.max_bytes, tr.bytes)
                tr.max_count = max(tr.max_count, tr.count)
                tr.order.append(cfg["rid"])

        def close(self):
            with tr.lock:
                tr.bytes -= self.cfg["bytes"]
                tr.count -= 1

    def fake_step(h):
        h.n += 1
        time.sleep(0.005)
        conv = h.n >= steps_for(h.cfg["rid"])
        return SimpleNamespace(E=-1.0 * h.cfg["rid"], rnorm=1e-9 if conv else 1.0, converged=conv)

    monkeypatch.setattr(serve, "System", FakeSystem)
    monkeypatch.setattr(serve, "eacg_set_psi", lambda h, psi: None)
    monkeypatch.setattr(serve, "eacg_step", fake_step)
    monkeypatch.setattr(serve, "eacg_bytes_required", lambda cfg, prm: (cfg["bytes"], 0))


def test_admission_respects_budget_and_slots(monkeypatch):
    tr = Tracker()
    install_fakes(monkeypatch, tr, lambda rid: 3 + rid % 4)
    sizes = [4, 4, 4, 8, 2, 3, 5, 1]
    reqs = [serve.Request(rid=i, cfg={"rid": i, "bytes": b}, raw=None, arrival=0.002 * i)
            for i, b in enumerate(sizes)]
    srv = serve.Server(hbm_budget=10, max_resident=3, use_cuda=False)
    outs = srv.run(reqs)
    assert all(o.converged for o in outs)
    assert tr.max_bytes <= 10
    assert tr.max_count <= 3
    admits = [o.admit for o in outs]           # outcomes are in request (arrival) order
    assert admits == sorted(admits)            # admitted in arrival order
    for o, r in zip(outs, reqs):
        assert o.admit >= o.arrival - 1e-9 and o.done >= o.admit
        assert o.E == -1.0 * r.rid
    st = serve.latency_stats(outs)
    assert st["converged"] == len(sizes) and st["p50_s"] <= st["p99_s"]


def test_oversize_request_runs_alone(monkeypatch):
    tr = Tracker()
    install_fakes(monkeypatch, tr, lambda rid: 2)
    reqs = [serve.Request(rid=0, cfg={"rid": 0, "bytes": 50}, raw=None, arrival=0.0),
            serve.Request(rid=1, cfg={"rid": 1, "bytes": 5}, raw=None, arrival=0.0)]
    outs = serve.Server(hbm_budget=10, max_resident=4, use_cuda=False).run(reqs)
    assert all(o.converged for o in outs)
    assert tr.max_count == 1   # the oversize request is admitted only when nothing else is resident


def test_failed_request_does_not_stop_the_server(monkeypatch):
    tr = Tracker()
    install_fakes(monkeypatch, tr, lambda rid: 2)

    def bad_step(h):
        if h.cfg["rid"] == 1:
            raise RuntimeError("injected failure")
        h.n += 1
        return SimpleNamespace(E=0.0, rnorm=1e-9, converged=h.n >= 2)

    monkeypatch.setattr(serve, "eacg_step", bad_step)
    reqs = [serve.Request(rid=i, cfg={"rid": i, "bytes": 1}, raw=None, arrival=0.0) for i in range(3)]
    outs = serve.Server(hbm_budget=10, max_resident=2, use_cuda=False).run(reqs)
    assert outs[1].status.startswith("failed") and not outs[1].converged
    assert outs[0].converged and outs[2].converged
    assert tr.count == 0   # every system was closed


def test_serving_stream_requests_are_valid_models():
    """The 256 seeded requests of the serving stream: an even electron count (bands = sum Z / 2),
    1-16 atoms, 1-27 k-points, a grid that holds the cutoff sphere with the margin of the
    potential's frequencies (N >= 4 m_max + 1), and a model the library accepts (positive HBM
    estimate, computed on the host)."""
    import math
    import numpy as np
    import synth
    ensure_library()
    import paper_2503_16225_gb300 as E
    for i in range(256):
        cfg = synth.config_serving_request(i)
        Z = np.asarray(cfg["Z"])
        assert int(Z.sum()) % 2 == 0 and cfg["nbands"] == int(Z.sum()) // 2
        assert 1 <= len(Z) <= 16 and len(cfg["kweight"]) in (1, 8, 27)
        mmax = math.sqrt(2.0 * cfg["ecut"]) / (2.0 * math.pi / cfg["a"])
        assert cfg["N"] >= 4 * mmax + 1
        assert E.eacg_bytes_required(cfg)[0] > 0, i
