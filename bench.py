#!/usr/bin/env python
"""Benchmark: converged eARCG solves per second of the 8-atom diamond crystal
(4x4x4 k-points, 48^3 grid, 16 bands, Ecut 15 Ha) on one GB300, from the seeded
random start to ||R||_F <= 1e-8, with the Hamiltonian-application bandwidth and the
roofline of the dominant kernel.  One step = one complete solve.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
  python bench.py --impl reference ...   # the FP64 CPU oracle on a bounded sample

Multi-GPU: replicas only (each rank solves its own copy; no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_BYTES = 129 * 2 ** 20
# FP64 FMA throughput of a GB300 from unit counts and the maximum SM clock:
# 152 SMs x 2 FP64 FMA per clock x 2 FLOP x 2.07 GHz (a probe measured 1.196 TFLOP/s at ~2.0 GHz)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12    # 152 SMs x 2 FP64 FMA/clk x 2 FLOP x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # 152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz
# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of single-kernel
# slots, from the ncu captures summarised in profiles/ (diamond 4x4x4 workload, 1024 bands per
# launch); a kernel changed since its capture must be removed from this table.
NCU_TRAFFIC_BYTES = {"plane_h_f64": 393.6e6, "plane_h_f32": 170.0e6}
# profile slots that time exactly one kernel (the roofline is reported for the top one)
SINGLE_KERNEL_SLOTS = ("plane_h", "plane_rho", "xpass_inv", "xpass_fwd", "xpass_rho", "fom_solve")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="diamond_k444",
                    choices=["diamond_k444", "diamond_k222", "two_atom", "diamond64_gamma", "diamond64_k222"],
                    help="diamond64_*: the 64-atom supercell (96^3 grid, 128 bands, 256 projectors), "
                         "--op runs only (its p x p dense steps exceed the 64-band limit)")
    ap.add_argument("--serve", type=int, default=0,
                    help="serve a stream of this many synthetic crystals instead (Poisson arrivals)")
    ap.add_argument("--rate", type=float, default=2.0, help="arrival rate of the serving stream (requests/s)")
    ap.add_argument("--resident", type=int, default=8, help="maximum resident requests while serving")
    ap.add_argument("--op", default="solve", choices=["solve", "apply_h", "density", "ea_gradient"],
                    help="apply_h / density / ea_gradient: time a few calls of one operation on the "
                         "workload's start point instead of solves (short runs under a profiler)")
    ap.add_argument("--method", default="earcg", choices=["earcg", "eargd"],
                    help="eargd: the paper's gradient-descent comparator (BB step, non-monotone backtracking)")
    ap.add_argument("--concurrent", type=int, default=4,
                    help="resident systems solved concurrently (own stream and host thread each); "
                         "value = whole-job served solves/s")
    ap.add_argument("--no-fp64-ref", action="store_true",
                    help="skip the plain FP64 one-system solve that the served number is compared with")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the host-buffer (e2e) solves and the CPU baseline (short runs under a profiler)")
    return ap.parse_args()


def run_serve(args):
    """Continuous-batching stream: requests i = 0..n-1 of the serving generator arrive as a
    seeded Poisson process; reports converged solves/s and p50/p99 arrival-to-converged latency."""
    import numpy as np
    import torch
    import synth
    from paper_2503_16225_gb300 import serve
    torch.cuda.set_device(0)
    rng = np.random.default_rng(7)
    t = 0.0
    reqs = []
    for i in range(args.serve):
        cfg = synth.config_serving_request(i)

        def raw(nk, n_max, cfg=cfg):
            return torch.from_numpy(synth.raw_coefficients(cfg["seed"], nk, cfg["nbands"], n_max))
        reqs.append(serve.Request(rid=i, cfg=cfg, raw=raw, arrival=t))
        t += rng.exponential(1.0 / args.rate)
    free, total = torch.cuda.mem_get_info()
    prec = 1 if args.precision == "mixed" else 0
    srv = serve.Server(hbm_budget=int(0.8 * free), max_resident=args.resident, precision=prec)
    t0 = time.perf_counter()
    outs = srv.run(reqs)
    wall = time.perf_counter() - t0
    st = serve.latency_stats(outs)
    line = {"metric": "served eARCG solves/s (synthetic crystal stream, to ||R||<=1e-8)",
            "value": st["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": args.serve, "warmup": 0,
            "ms_per_step": wall * 1e3 / max(1, args.serve), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32/f64" if prec else "f64", "data": "synthetic",
            "config": {"workload": "serving_stream", "requests": args.serve, "rate_per_s": args.rate,
                       "max_resident": args.resident, "precision": args.precision},
            "latency_s": {"p50": st["p50_s"], "p99": st["p99_s"]}, "converged": st["converged"],
            "failed": [o.status for o in outs if not o.converged]}
    print(json.dumps(line))


def rank_env():
    """(world size, rank, local rank) of this process, from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x, world, device=None):
    """The largest of a per-rank value over all ranks (the job's time is its slowest rank's)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, ms):
    """Units of all ranks per second over the slowest rank's time (replicas: weak scaling)."""
    return world * units_per_rank / (ms / 1e3)


WORKLOAD_LABEL = {"diamond_k444": "diamond8 4x4x4k 48^3 p16"}


def metric_name(args, cfg):
    """The headline metric, shared by this arm and the reference arm."""
    label = WORKLOAD_LABEL.get(args.workload, cfg["name"])
    return f"served {'EARGD' if args.method == 'eargd' else 'eARCG'} solves/s ({label}, to ||R||<=1e-8)"


def config_of(args, cfg, world):
    """The workload description, shared by this arm and the reference arm."""
    return {"workload": cfg["name"], "kpoints": len(cfg["kweight"]), "bands": cfg["nbands"], "grid": cfg["N"],
            "ecut": cfg["ecut"], "precision": args.precision, "method": args.method,
            "parallelism": f"replicas{world}", "concurrent_systems": max(1, args.concurrent),
            "l2": "flushed between rounds of concurrent solves (256 MiB write)"}


def workload(name):
    import synth
    return {"diamond_k444": lambda: synth.config_diamond(2, kgrid=(4, 4, 4)),
            "diamond_k222": lambda: synth.config_diamond(2, kgrid=(2, 2, 2)),
            "two_atom": lambda: synth.config_two_atom(1),
            "diamond64_gamma": lambda: synth.config_diamond_supercell(2),
            "diamond64_k222": lambda: synth.config_diamond_supercell(2, kgrid=(2, 2, 2))}[name]()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------ reference arm
def oracle_sample(cfg, nk_sample=4):
    """One oracle evaluation (density of all k, potential, H applied at nk_sample k-points)
    timed on the host cores; returns seconds per band application of H and the cores."""
    import numpy as np
    import synth
    from oracle.model import Model
    from oracle import earcg
    model = Model(cfg)
    raw = synth.raw_coefficients(cfg["seed"], model.nk, model.p)
    Phi = earcg.lowdin([raw[k, :, :model.nk[k]].T.copy() for k in range(model.K)])
    t0 = time.perf_counter()
    rho = model.density(Phi)
    v = model.potentials(rho)[0]
    t_dens = time.perf_counter() - t0
    t1 = time.perf_counter()
    ks = list(range(0, model.K, max(1, model.K // nk_sample)))[:nk_sample]
    for k in ks:
        model.apply_H(k, Phi[k], v)
    t_h = (time.perf_counter() - t1) / (len(ks) * model.p)
    # density pass ~ half an H application per band
    per_band = t_h + t_dens / (model.K * model.p)
    return per_band, os.cpu_count(), f"oracle density of all {model.K} k-points + H at {len(ks)} k-points"


def oracle_band_apps(name):
    path = os.path.join(ROOT, "tests", "golden", f"oracle_{name}.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d["band_applications"], "oracle's own converged solve (tests/golden)"
    return None, None


def run_reference(args):
    _, rank, _ = rank_env()
    if rank != 0:
        return
    cfg = workload(args.workload)
    apps, src = oracle_band_apps(args.workload)
    times = []
    for i in range(args.warmup + args.steps):
        per_band, cores, sample = oracle_sample(cfg)
        if i >= args.warmup:
            times.append(per_band)
    per_band = statistics.median(times)
    if apps is None:
        apps, src = 15000 * len(cfg["kweight"]) * cfg["nbands"] // 1024, "estimate"
    solve_s = per_band * apps
    value = 1.0 / solve_s
    line = {"impl": "reference", "metric": metric_name(args, cfg),
            "value": value, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": solve_s * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": config_of(args, cfg, args.gpus),
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{sample}; scaled by {apps} band applications per solve ({src})"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    import synth
    import paper_2503_16225_gb300 as E

    world, rank, local = rank_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    cfg = workload(args.workload)
    prec = 1 if args.precision == "mixed" else 0
    method = 1 if args.method == "eargd" else 0
    params = E.eacg_default_params(precision=prec, method=method)
    C = max(1, args.concurrent)
    # C resident systems of the workload, each with its own stream and host thread (served)
    systems = []
    for _ in range(C):
        st_i = torch.cuda.Stream(device=dev)
        systems.append((E.System(cfg, params, stream=st_i.cuda_stream), st_i))
    sysm = systems[0][0]
    raw = synth.raw_coefficients(cfg["seed"], sysm.nk, sysm.p, sysm.n_max)
    host = torch.from_numpy(raw).pin_memory()
    psi0 = host.to(dev)
    out_hosts = [torch.empty_like(host).pin_memory() for _ in range(C)]
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()

    def solve_on(i, res, ends):
        sy, st_i = systems[i]
        try:
            E.eacg_set_psi(sy.h, psi0)
            res[i] = E.eacg_solve(sy.h)
        except Exception as exc:  # reported by the caller
            res[i] = exc
        ends[i].record(st_i)

    def one_round():
        """C concurrent solves from the same start; device time from one event that every
        system stream waits on to an event that waits on every stream's end."""
        start = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for _, st_i in systems:
            st_i.wait_event(start)
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(C)]
        res = [None] * C
        ths = [threading.Thread(target=solve_on, args=(i, res, ends)) for i in range(C)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        for e in ends:
            stream.wait_event(e)
        stop = torch.cuda.Event(enable_timing=True)
        stop.record(stream)
        stop.synchronize()
        for r in res:
            if isinstance(r, Exception):
                raise r
            if r.status != 0 or not (r.rnorm <= params.res_tol):
                raise RuntimeError(f"solve did not converge: status {r.status} rnorm {r.rnorm}")
        return start.elapsed_time(stop), [start.elapsed_time(e) for e in ends], res

    for _ in range(args.warmup):
        one_round()
    torch.cuda.synchronize()

    # ---- timed region: K rounds of C concurrent solves, L2 flushed between them (outside the events)
    clocks = Clocks(local)
    for sy, _ in systems:
        E.eacg_profile_enable(sy.h, 1)
    launches0 = E.eacg_launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    per = []
    latencies = []
    results = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        ms, lat, res = one_round()
        per.append(ms)
        latencies += lat
        results += res
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = E.eacg_launch_count() - launches0
    clk = clocks.stop()
    prof = {}
    for sy, _ in systems:  # summed over the resident systems
        for name, st in E.eacg_profile_read(sy.h).items():
            acc = prof.setdefault(name, {"launches": 0, "ms": 0.0, "bytes": 0.0, "flops": 0.0, "units": 0.0})
            for key in acc:
                acc[key] += st[key]
        E.eacg_profile_enable(sy.h, 0)
    total_ms = max_over_ranks(sum(per), world, dev)
    value = whole_job_rate(world, C * args.steps, total_ms)

    # ---- end to end through the host-buffer entry point (copies inside the timed region)
    e2e_ms = []

    def solve_host_on(i, res):
        try:
            res[i] = E.eacg_solve_host(systems[i][0].h, host, out_hosts[i])
        except Exception as exc:
            res[i] = exc

    for _ in range(0 if args.no_extras else max(1, min(args.steps, 2))):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = [None] * C
        ths = [threading.Thread(target=solve_host_on, args=(i, res)) for i in range(C)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        for r in res:
            if isinstance(r, Exception) or r.status != 0:
                raise RuntimeError("host-buffer solve failed")
    e2e_value = (whole_job_rate(world, C, max_over_ranks(statistics.mean(e2e_ms), world, dev))
                 if e2e_ms else None)

    # ---- plain FP64, one system at a time (the comparison the served number is quoted against)
    fp64_ref = None
    if prec == 1 and not args.no_extras and not args.no_fp64_ref:
        p64 = E.eacg_default_params(precision=0, method=method)
        s64 = E.System(cfg, p64)
        for it in range(2):  # one untimed solve, then one timed
            E.eacg_set_psi(s64.h, psi0)
            torch.cuda.synchronize()
            flush.fill_(1.0)
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            r64 = E.eacg_solve(s64.h)
            a1.record(stream)
            a1.synchronize()
        s64.close()
        fp64_ms = a0.elapsed_time(a1)
        fp64_ref = {"solves_per_s": 1e3 / fp64_ms, "ms_per_solve": fp64_ms, "E": r64.E, "rnorm": r64.rnorm,
                    "iterations": r64.iterations, "served_over_fp64": value / (1e3 / fp64_ms)}

    # ---- roofline of the dominant kernel from the live profile
    hbm, peak_kind = measured_peaks()
    bytes_per_band = hpsi_bytes_per_band(sysm, prec_bytes=8)
    roof = None
    kernels = {}
    for name, st in (prof or {}).items():
        if st["ms"] <= 0:
            continue
        sec = st["ms"] / 1e3
        kernels[name] = {"launches": st["launches"], "ms": round(st["ms"], 3),
                         "avg_ms": st["ms"] / st["launches"], "GBps": st["bytes"] / sec / 1e9,
                         "TFLOPs": st["flops"] / sec / 1e12}
    single = {k: v for k, v in (prof or {}).items() if k.rsplit("_", 1)[0] in SINGLE_KERNEL_SLOTS}
    top = max(single, key=lambda k: single[k]["ms"]) if single else None
    if top is not None:
        st = prof[top]
        n = max(1, st["launches"])
        avg_ms = st["ms"] / n
        achieved = (st["flops"] / n) / (avg_ms / 1e3) / 1e12
        if top.endswith("_f64"):
            peak, pk = FP64_PEAK_TFLOPS, "derived: 152 SMs x 2 FP64 FMA/clk x 2 FLOP x 2.07 GHz"
        else:
            peak, pk = FP32_PEAK_TFLOPS, "derived: 152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz"
        roof = {"bound": "alu", "kernel": top, "achieved": achieved, "peak": peak, "peak_kind": pk,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": NCU_TRAFFIC_BYTES.get(top) if args.workload == "diamond_k444" else None,
                "traffic_unit": "bytes per launch (ncu)", "avg_launch_ms": avg_ms,
                "launches": n, "hbm_GBps_algorithmic": (st["bytes"] / n) / (avg_ms / 1e3) / 1e9,
                "hbm_peak_GBps": hbm, "hbm_peak_kind": peak_kind}
    apps = sum(r.h_band_apps for r in results)
    hpsi_gbs = (apps * bytes_per_band) / (total_ms / 1e3) / 1e9

    line = {
        "metric": metric_name(args, cfg),
        "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32/f64" if prec else "f64", "data": "synthetic",
        "config": config_of(args, cfg, world),
        "time_to_1e8_ms": {"p50": statistics.median(latencies), "p99": max(latencies), "all": latencies},
        "vs_fp64_one_at_a_time": fp64_ref,
        "solve": {"E": results[-1].E, "rnorm": results[-1].rnorm, "iterations": results[-1].iterations,
                  "warm_iterations": results[-1].warm_iterations, "h_band_apps": results[-1].h_band_apps,
                  "ls_trials": results[-1].ls_trials},
        "hpsi_gbs": hpsi_gbs,
        "roofline": roof,
        "profile": kernels,
        "gpu_launches": launches,
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": C * host.numel() * 16,
                "d2h_bytes_per_step": C * host.numel() * 16},
    }
    if rank == 0 and world == 1 and not args.no_extras:
        try:
            per_band, cores, sample = oracle_sample(cfg)
            apps_solve = results[-1].h_band_apps
            cpu_v = 1.0 / (per_band * apps_solve)
            line["cpu_baseline"] = {"value": cpu_v, "unit": "solves/s", "cores": cores, "kind": "oracle",
                                    "sample": f"{sample}, scaled by this solve's {apps_solve} band applications"}
        except Exception as exc:  # the baseline is a report, not the measurement
            line["cpu_baseline"] = {"value": None, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                                    "sample": f"failed: {exc}"}
    if rank == 0:
        print(json.dumps(line))
    for sy, _ in systems:
        sy.close()
    if world > 1:
        dist.destroy_process_group()


def hpsi_bytes_per_band(sysm, prec_bytes=8):
    """Algorithmic HBM bytes of one band application of H with the pruned transforms:
    coefficients in + out (complex double) and the x-pass intermediate written, read and
    written back by the plane kernel, then read (4 passes of N * ncols complex values)."""
    return 2 * sysm.n_max * 16 + 4 * sysm.N * sysm.ncols * 2 * prec_bytes


def run_op(args):
    """A few calls of one hot-path operation (H application, density or energy-adaptive
    gradient) on the workload's start point, timed with CUDA events: a short program for
    profiler captures."""
    import numpy as np
    import torch
    import synth
    import paper_2503_16225_gb300 as E

    cfg = workload(args.workload)
    prec = 1 if args.precision == "mixed" else 0
    sysm = E.System(cfg, E.eacg_default_params(precision=prec))
    raw = synth.raw_coefficients(cfg["seed"], sysm.nk, sysm.p, sysm.n_max)
    phi = sysm.block()
    if sysm.p <= E.EACG_MAX_BANDS_DENSE:
        E.eacg_set_psi(sysm.h, torch.from_numpy(raw).cuda())
        E.eacg_get_psi(sysm.h, phi)
    else:  # orthonormal start by host QR (the library's polar factor needs p <= 64)
        for k, n in enumerate(sysm.nk):
            q = np.linalg.qr(raw[k, :, :n].T)[0]
            phi[k, :, :n] = torch.from_numpy(np.ascontiguousarray(q.T))
    E.eacg_density(sysm.h, phi, None, 0)
    out = sysm.block()
    if args.op == "apply_h":
        call = lambda: E.eacg_apply_H(sysm.h, phi, out, prec)  # noqa: E731
    elif args.op == "density":
        call = lambda: E.eacg_density(sysm.h, phi, None, prec)  # noqa: E731
    else:
        call = lambda: E.eacg_ea_gradient(sysm.h, phi, out, sysm.K, prec)  # noqa: E731
    for _ in range(args.warmup):
        call()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        call()
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / max(1, args.steps)
    line = {"op": args.op, "workload": cfg["name"], "precision": args.precision, "calls": args.steps,
            "ms_per_call": ms, "bands": sysm.K * sysm.p}
    if args.op == "apply_h":
        # band applications per second and algorithmic H-psi bytes (pruned transforms) per second
        line["band_apps_per_s"] = sysm.K * sysm.p / (ms / 1e3)
        line["hpsi_gbs"] = sysm.K * sysm.p * hpsi_bytes_per_band(sysm, 8 if prec else 16) / (ms / 1e3) / 1e9
    print(json.dumps(line))
    sysm.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.serve > 0:
        run_serve(args)
    elif args.op != "solve":
        run_op(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
