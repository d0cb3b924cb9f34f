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
