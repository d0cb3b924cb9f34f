"""Continuous-batching serving loop for Kohn-Sham problems on one GPU.

Requests (synthetic crystals of uneven size) arrive at given times.  A dispatcher admits
waiting requests while the resident set fits an HBM budget (eacg_bytes_required plus the
FOM's Krylov growth) and a slot limit; each admitted request gets its own system, CUDA
stream and worker thread that runs eacg_step until ||R||_F <= res_tol (or the iteration
cap), then frees its device state so the next request can be admitted.  The workers'
kernels interleave on the GPU; every system keeps its own buffers and fixed-order
reductions, so a request's result does not depend on what else is resident.
"""
from __future__ import annotations

import queue
import threading
import time
from dataclasses import dataclass, field

import torch

from . import (System, eacg_bytes_required, eacg_default_params, eacg_get_psi, eacg_profile_enable,
               eacg_profile_read, eacg_set_psi, eacg_solve_host, eacg_step, eacg_stream_create,
               eacg_stream_destroy)


@dataclass
class Request:
    rid: int
    cfg: dict
    raw: object            # complex128 tensor [K, p, n_max] (device, or pinned host for host-buffer
                           # serving) or a callable(n_k list, n_max) -> tensor
    arrival: float         # seconds after the start of the run
    max_outer: int = 300
    out: object = None     # host-buffer serving: pinned host tensor that receives the result


@dataclass
class Outcome:
    rid: int
    arrival: float
    admit: float = 0.0
    done: float = 0.0
    E: float = float("nan")
    rnorm: float = float("nan")
    iterations: int = 0
    converged: bool = False
    status: str = ""
    bytes: int = 0
    psi: object = None
    steps: list = field(default_factory=list)
    h_band_apps: int = 0
    end_event: object = None   # CUDA event recorded on the request's stream after its last call


class Server:
    """Admits requests by HBM budget and slot count; one worker thread per resident system."""

    def __init__(self, hbm_budget: int, max_resident: int = 8, precision: int = 1, keep_psi: bool = False,
                 device: int = 0, use_cuda: bool = True, start_event=None, profile: bool = False,
                 host_buffers: bool = False, params: dict | None = None):
        """start_event: a CUDA event every request stream waits on before its first call (device
        timing from one event); profile: live kernel timing of every system, summed into
        self.profile; host_buffers: requests carry pinned host input and output tensors and are
        solved through eacg_solve_host (copies inside the request); params: eacg_params fields
        that replace the defaults for every request."""
        self.params = dict(params or {})
        self.use_cuda = use_cuda
        self.budget = int(hbm_budget)
        self.max_resident = int(max_resident)
        self.precision = precision
        self.keep_psi = keep_psi
        self.device = device
        self.start_event = start_event
        self.profile_on = profile
        self.host_buffers = host_buffers
        self.profile: dict = {}
        self._lock = threading.Lock()
        self._resident_bytes = 0
        self._resident = 0
        self._done = queue.Queue()

    def need_bytes(self, cfg, max_outer) -> int:
        prm = eacg_default_params(precision=self.precision, max_outer=max_outer)
        base, per_iter = eacg_bytes_required(cfg, prm)
        return base + 16 * per_iter   # room for 16 FOM iterations of Krylov storage

    def _work(self, req: Request, out: Outcome, t0: float, slot):
        s = None
        stream = None
        try:
            if self.use_cuda:
                # a stream of the resident slot's own: no two resident systems share a stream
                # (the FOM captures its H application from the system's stream into a graph)
                torch.cuda.set_device(self.device)
                stream = torch.cuda.ExternalStream(slot, device=torch.device("cuda", self.device))
                ctx = torch.cuda.stream(stream)
                handle = slot
            else:
                import contextlib
                ctx, handle = contextlib.nullcontext(), 0
            with ctx:
                if self.start_event is not None and stream is not None:
                    stream.wait_event(self.start_event)
                prm = eacg_default_params(precision=self.precision, max_outer=req.max_outer, **self.params)
                s = System(req.cfg, prm, stream=handle)
                if self.profile_on:
                    eacg_profile_enable(s.h, 1)
                raw = req.raw(s.nk, s.n_max) if callable(req.raw) else req.raw
                if self.host_buffers:
                    r = eacg_solve_host(s.h, raw, req.out, check=False)
                    out.E, out.rnorm, out.iterations = r.E, r.rnorm, r.iterations
                    out.h_band_apps = r.h_band_apps
                    out.converged = r.status == 0 and r.rnorm <= prm.res_tol
                    out.status = "converged" if out.converged else f"status {r.status}"
                else:
                    psi = raw if (not self.use_cuda or raw.is_cuda) else raw.to("cuda", non_blocking=False)
                    eacg_set_psi(s.h, psi)
                    while True:
                        info = eacg_step(s.h)
                        out.steps.append((info.E, info.rnorm))
                        if info.converged:
                            out.converged = True
                            break
                    out.E, out.rnorm = info.E, info.rnorm
                    out.iterations = len(out.steps)
                    out.h_band_apps = getattr(info, "h_band_apps", 0)
                    out.status = "converged"
                if self.keep_psi:
                    phi = s.block()
                    eacg_get_psi(s.h, phi)
                    if stream is not None:
                        stream.synchronize()
                    out.psi = phi.cpu()
        except Exception as exc:  # the request fails, the server goes on
            out.status = f"failed: {exc}"
            if out.steps:
                out.E, out.rnorm = out.steps[-1]
                out.iterations = len(out.steps)
        finally:
            # the request leaves whatever happened: its slot and budget are always returned
            try:
                if s is not None and self.profile_on:
                    prof = eacg_profile_read(s.h)
                    with self._lock:
                        for name, st in prof.items():
                            acc = self.profile.setdefault(name, dict.fromkeys(st, 0))
                            for key, v in st.items():
                                acc[key] += v
                if stream is not None:
                    out.end_event = torch.cuda.Event(enable_timing=True)
                    out.end_event.record(stream)
            except Exception as exc:
                out.status = out.status or f"failed: {exc}"
                out.end_event = None
            finally:
                if s is not None:
                    s.close()
            out.done = time.perf_counter() - t0
            with self._lock:
                self._resident_bytes -= out.bytes
                self._resident -= 1
            self._slots.put(slot)
            self._done.put(out)

    def run(self, requests: list[Request]) -> list[Outcome]:
        """Serve the requests (sorted by arrival); returns one Outcome per request."""
        self._slots = queue.Queue()
        streams = []
        if self.use_cuda:
            torch.cuda.set_device(self.device)
            for _ in range(self.max_resident):
                streams.append(eacg_stream_create())
        for i in range(self.max_resident):
            self._slots.put(streams[i] if streams else i)
        try:
            return self._run(requests)
        finally:
            for h in streams:
                eacg_stream_destroy(h)

    def _run(self, requests: list[Request]) -> list[Outcome]:
        pending = sorted(requests, key=lambda r: r.arrival)
        waiting: list[tuple[Request, Outcome, int]] = []
        outs: dict[int, Outcome] = {}
        threads = []
        t0 = time.perf_counter()
        finished = 0
        i = 0
        while finished < len(pending):
            now = time.perf_counter() - t0
            while i < len(pending) and pending[i].arrival <= now:
                r = pending[i]
                o = Outcome(rid=r.rid, arrival=r.arrival)
                outs[r.rid] = o
                waiting.append((r, o, self.need_bytes(r.cfg, r.max_outer)))
                i += 1
            # admit in arrival order while the budget and slots allow
            while waiting:
                r, o, need = waiting[0]
                with self._lock:
                    fits = (self._resident < self.max_resident and
                            (self._resident_bytes + need <= self.budget or self._resident == 0))
                    if fits:
                        self._resident += 1
                        self._resident_bytes += need
                if not fits:
                    break
                waiting.pop(0)
                o.admit = time.perf_counter() - t0
                o.bytes = need
                th = threading.Thread(target=self._work, args=(r, o, t0, self._slots.get()), daemon=True)
                th.start()
                threads.append(th)
            try:
                self._done.get(timeout=0.002)
                finished += 1
            except queue.Empty:
                pass
            if not waiting and i < len(pending):
                wait = pending[i].arrival - (time.perf_counter() - t0)
                if wait > 0:
                    try:
                        self._done.get(timeout=min(wait, 0.05))
                        finished += 1
                    except queue.Empty:
                        pass
        for th in threads:
            th.join()
        return [outs[r.rid] for r in requests]


def percentile(values, q):
    """Nearest-rank percentile of a list (None when empty)."""
    v = sorted(values)
    if not v:
        return None
    k = min(len(v) - 1, max(0, int(round(q * (len(v) - 1)))))
    return v[k]


def latency_stats(outs: list[Outcome]):
    """solves/s over the whole run, p50/p99 of arrival-to-converged latency and of the solve
    time from admission (converged requests only)."""
    ok = [o for o in outs if o.converged]
    lat = [o.done - o.arrival for o in ok]
    svc = [o.done - o.admit for o in ok]
    span = max(o.done for o in outs) - min(o.arrival for o in outs) if outs else 0.0
    return {"converged": len(ok), "requests": len(outs), "solves_per_s": len(ok) / span if span > 0 else None,
            "p50_s": percentile(lat, 0.5), "p99_s": percentile(lat, 0.99),
            "solve_p50_s": percentile(svc, 0.5), "solve_p99_s": percentile(svc, 0.99)}
