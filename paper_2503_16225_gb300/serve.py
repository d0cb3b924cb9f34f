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

from . import System, eacg_bytes_required, eacg_default_params, eacg_get_psi, eacg_set_psi, eacg_step


@dataclass
class Request:
    rid: int
    cfg: dict
    raw: object            # host complex128 tensor [K, p, n_max] or a callable(n_k list, n_max) -> tensor
    arrival: float         # seconds after the start of the run
    max_outer: int = 300


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


class Server:
    """Admits requests by HBM budget and slot count; one worker thread per resident system."""

    def __init__(self, hbm_budget: int, max_resident: int = 8, precision: int = 1, keep_psi: bool = False,
                 device: int = 0, use_cuda: bool = True):
        self.use_cuda = use_cuda
        self.budget = int(hbm_budget)
        self.max_resident = int(max_resident)
        self.precision = precision
        self.keep_psi = keep_psi
        self.device = device
        self._lock = threading.Lock()
        self._resident_bytes = 0
        self._resident = 0
        self._done = queue.Queue()

    def need_bytes(self, cfg, max_outer) -> int:
        prm = eacg_default_params(precision=self.precision, max_outer=max_outer)
        base, per_iter = eacg_bytes_required(cfg, prm)
        return base + 16 * per_iter   # room for 16 FOM iterations of Krylov storage

    def _work(self, req: Request, out: Outcome, t0: float):
        s = None
        try:
            if self.use_cuda:
                torch.cuda.set_device(self.device)
                stream = torch.cuda.Stream()
                ctx = torch.cuda.stream(stream)
                handle = stream.cuda_stream
            else:
                import contextlib
                stream, ctx, handle = None, contextlib.nullcontext(), 0
            with ctx:
                prm = eacg_default_params(precision=self.precision, max_outer=req.max_outer)
                s = System(req.cfg, prm, stream=handle)
                raw = req.raw(s.nk, s.n_max) if callable(req.raw) else req.raw
                psi = raw.to("cuda", non_blocking=False) if self.use_cuda else raw
                eacg_set_psi(s.h, psi)
                while True:
                    info = eacg_step(s.h)
                    out.steps.append((info.E, info.rnorm))
                    if info.converged:
                        out.converged = True
                        break
                out.E, out.rnorm = info.E, info.rnorm
                out.iterations = len(out.steps)
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
            if s is not None:
                s.close()
            out.done = time.perf_counter() - t0
            with self._lock:
                self._resident_bytes -= out.bytes
                self._resident -= 1
            self._done.put(out)

    def run(self, requests: list[Request]) -> list[Outcome]:
        """Serve the requests (sorted by arrival); returns one Outcome per request."""
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
                th = threading.Thread(target=self._work, args=(r, o, t0), daemon=True)
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


def latency_stats(outs: list[Outcome]):
    """solves/s over the whole run and p50/p99 of arrival-to-converged latency (converged only)."""
    ok = [o for o in outs if o.converged]
    lat = sorted(o.done - o.arrival for o in ok)
    span = max(o.done for o in outs) - min(o.arrival for o in outs) if outs else 0.0

    def pct(q):
        if not lat:
            return None
        k = min(len(lat) - 1, max(0, int(round(q * (len(lat) - 1)))))
        return lat[k]

    return {"converged": len(ok), "requests": len(outs), "solves_per_s": len(ok) / span if span > 0 else None,
            "p50_s": pct(0.5), "p99_s": pct(0.99)}
