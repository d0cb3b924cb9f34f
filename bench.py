#!/usr/bin/env python
"""Benchmark: served eARCG solves per second on one GB300.

Default workload: the serving stream of 256 seeded synthetic crystals
(synth.config_serving_request: cubic cells a 6-14 bohr with 1-16 atoms of Z 1-4, 0/1/4 Gaussian
projectors per atom, Ecut 8-20 Ha, 1-23 bands, 1, 8 or 27 k-points, grids 20^3-64^3), each
solved from its seeded random start to ||R||_F <= 1e-8 in mixed precision, admitted by HBM
budget and slot count and served with continuous batching (one system, CUDA stream and host
thread per resident request).  One step = ceil(256 / K) consecutive requests of the stream;
the timed region queues the K steps' requests at t = 0 (saturating load) and serves them
continuously, so that it covers the whole stream once.

Beside the headline: the same stream through host buffers (e2e), the plain FP64
one-system-at-a-time solve rate on a sample of the stream (the denominator of the served
speed-up), p50/p99 arrival-to-converged latency of Poisson streams at 0.5x and 2x that FP64
rate, the energy error per atom against stored oracle solves, the roofline of the dominant
kernel (timed on the sample solved one at a time, no overlapping kernels) and the CPU oracle
timed on sampled requests.

  python bench.py [--gpus N] [--steps K] [--warmup W]
  python bench.py --impl reference ...          # the FP64 CPU oracle on sampled requests
  python bench.py --workload diamond_k444|two_atom|...   # one-workload solve benches
  python bench.py --op apply_h --workload diamond64_gamma # a few calls of one operation

Multi-GPU: replicas only (each rank serves its own copy of the stream; no collective on the
data path).
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
STREAM = 256                 # requests of the serving stream
FP64_SAMPLE_STRIDE = 16      # the FP64 one-at-a-time sample: every 16th request of the stream
# FMA throughput of a GB300 from unit counts and the maximum SM clock (a probe measured
# 1.196 TFLOP/s FP64 and 69.7 TFLOP/s FP32 at ~2.0 GHz)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12    # 152 SMs x 2 FP64 FMA/clk x 2 FLOP x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # 152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz
# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of single-kernel
# slots, from the ncu captures summarised in profiles/ (diamond 4x4x4 workload, 1024 bands per
# launch); a kernel changed since its capture must be removed from this table.  The FP64-accurate
# slots (_f64) run in double-float arithmetic by default.
NCU_TRAFFIC_BYTES = {"plane_h_f64": 395.6e6, "plane_rho_f64": 240.2e6, "plane_h_f32": 170.0e6}
# FP32 instructions (FADD + FMUL + FFMA, thread level) per algorithmic FLOP (5 N log2 N per line)
# of the double-float kernels, from the same captures: their roofline is the FP32 pipe's
# instruction rate (152 SMs x 128 lanes x clock) divided by this ratio.
NCU_DF_INSTR_PER_FLOP = {"plane_h_f64": 11.54, "plane_rho_f64": 12.99}
FP32_INSTR_PEAK = 152 * 128 * 2.07e9
# profile slots that time exactly one kernel (the roofline is reported for the top one)
SINGLE_KERNEL_SLOTS = ("plane_h", "plane_rho", "xpass_inv", "xpass_fwd", "xpass_rho", "fom_solve")
# profile slots of the H application and density (algorithmic H-psi bytes)
HPSI_SLOTS = ("xpass_inv", "plane_h", "xpass_fwd", "nonlocal", "xpass_rho", "plane_rho", "nonlocal_eval")
GOLDEN_SERVING = os.path.join(ROOT, "tests", "golden", "oracle_serving.json")
SERVE_PARAMS: dict = {}   # eacg_params overrides of the served requests (set from the flags)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="serving_stream",
                    choices=["serving_stream", "diamond_k444", "diamond_k222", "two_atom", "diamond64_gamma",
                             "diamond64_k222", "diamond64_ec5", "diamond216_gamma"],
                    help="serving_stream: the 256-request stream (headline); the others: concurrent solves "
                         "of one workload; diamond64_*: the 64-atom supercell (128 bands, 256 projectors; "
                         "96^3 grid at Ecut 15, or 48^3 at Ecut 5 for diamond64_ec5, whose oracle solve is "
                         "stored); diamond216_gamma (N = 128): --op runs with FP32 transforms only")
    ap.add_argument("--resident", type=int, default=16, help="maximum resident requests while serving")
    ap.add_argument("--op", default="solve", choices=["solve", "apply_h", "density", "ea_gradient"],
                    help="apply_h / density / ea_gradient: time a few calls of one operation on the "
                         "workload's start point instead of solves (short runs under a profiler)")
    ap.add_argument("--method", default="earcg", choices=["earcg", "eargd"],
                    help="eargd: the paper's gradient-descent comparator (BB step, non-monotone backtracking)")
    ap.add_argument("--concurrent", type=int, default=4,
                    help="one-workload solves: resident systems solved concurrently (own stream and host "
                         "thread each)")
    ap.add_argument("--batch-window", type=int, default=-1,
                    help="serving: batch the transforms of concurrently stepping systems, each waiting at most "
                         "this many microseconds (eacg_batching); -1: off")
    ap.add_argument("--step-many", action="store_true",
                    help="one-workload solves: step the concurrent systems together with eacg_step_many "
                         "(batched transform launches) instead of one host thread per system")
    ap.add_argument("--switch-res", type=float, default=None,
                    help="mixed precision: residual below which the evaluations switch to FP64-accurate "
                         "transforms (library default if not given)")
    ap.add_argument("--stream-start", type=int, default=0,
                    help="serving: first request of the timed stream (0; another value only for short profiler runs)")
    ap.add_argument("--stream-len", type=int, default=256,
                    help="serving: requests of the stream that the K steps cover (256; fewer only for short "
                         "profiler runs)")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the timed region (short runs under a profiler): no e2e, FP64 sample, Poisson "
                         "latency runs or CPU baseline")
    return ap.parse_args()


# ------------------------------------------------------------------------ shared helpers
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


def per_step(steps, length=STREAM):
    """Requests per step: the K steps cover the stream (256 requests) once."""
    return int(math.ceil(length / max(1, steps)))


def stream_ids(start, count):
    return [(start + j) % STREAM for j in range(count)]


def fp64_sample_ids():
    return list(range(0, STREAM, FP64_SAMPLE_STRIDE))


WORKLOAD_LABEL = {"diamond_k444": "diamond8 4x4x4k 48^3 p16"}


def metric_name(args, cfg=None):
    """The headline metric, shared by this arm and the reference arm."""
    meth = "EARGD" if args.method == "eargd" else "eARCG"
    if args.workload == "serving_stream":
        return f"served {meth} solves/s (stream of {STREAM} synthetic crystals, to ||R||<=1e-8)"
    label = WORKLOAD_LABEL.get(args.workload, cfg["name"])
    return f"served {meth} solves/s ({label}, to ||R||<=1e-8)"


def config_of(args, cfg, world):
    """The workload description, shared by this arm and the reference arm."""
    if args.workload == "serving_stream":
        return {"workload": f"serving_stream_{STREAM}" if args.stream_len == STREAM else
                f"serving_stream_requests_{args.stream_start}_to_{args.stream_start + args.stream_len - 1}",
                "requests_per_step": per_step(args.steps, args.stream_len),
                "requests": "synth.config_serving_request(i), i < 256: a 6-14, 1-16 atoms, Z 1-4, Ecut 8-20, "
                            "1/8/27 k, N 20-64, p 1-23",
                "arrivals": "all queued at t=0 (saturating load)", "precision": args.precision,
                "method": args.method, "parallelism": f"replicas{world}", "max_resident": args.resident,
                "batch_window_us": args.batch_window, "l2": "inputs of the stream (GBs) exceed L2; no flush"}
    return {"workload": cfg["name"], "kpoints": len(cfg["kweight"]), "bands": cfg["nbands"], "grid": cfg["N"],
            "ecut": cfg["ecut"], "precision": args.precision, "method": args.method,
            "parallelism": f"replicas{world}", "concurrent_systems": max(1, args.concurrent),
            "stepping": "eacg_step_many" if args.step_many else "one host thread per system",
            "l2": "flushed between rounds of concurrent solves (256 MiB write)"}


def workload(name):
    import synth
    return {"diamond_k444": lambda: synth.config_diamond(2, kgrid=(4, 4, 4)),
            "diamond_k222": lambda: synth.config_diamond(2, kgrid=(2, 2, 2)),
            "two_atom": lambda: synth.config_two_atom(1),
            "diamond64_gamma": lambda: synth.config_diamond_supercell(2),
            "diamond64_k222": lambda: synth.config_diamond_supercell(2, kgrid=(2, 2, 2)),
            "diamond64_ec5": lambda: synth.config_diamond_supercell(2, ecut=5.0, N=48),
            "diamond216_gamma": lambda: synth.config_diamond_supercell(3)}[name]()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def golden_serving():
    try:
        with open(GOLDEN_SERVING) as fh:
            return json.load(fh)
    except OSError:
        return None


def r4(x):
    return None if x is None else float(f"{x:.4g}")


class Clocks:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")
        import resource
        self.ru0 = resource.getrusage(resource.RUSAGE_SELF)
        self.t0 = time.perf_counter()
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
        sm, mx, reasons, util = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
                util.append(float(r[9]))
            except (ValueError, IndexError):
                continue
        import resource
        ru = resource.getrusage(resource.RUSAGE_SELF)
        wall = time.perf_counter() - self.t0
        cpu = (ru.ru_utime - self.ru0.ru_utime) + (ru.ru_stime - self.ru0.ru_stime)
        # kernel-active share of the samples and the host cores kept busy (context for the number)
        self.busy = {"gpu_util_pct_median": statistics.median(util) if util else None,
                     "host_cores_busy": round(cpu / wall, 2) if wall > 0 else None}
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def profile_summary(prof, total_ms=None):
    """Per-slot launches, ms, average ms, algorithmic GB/s and TFLOP/s (for stderr)."""
    out = {}
    for name, st in (prof or {}).items():
        if st["ms"] <= 0:
            continue
        sec = st["ms"] / 1e3
        out[name] = {"launches": st["launches"], "ms": round(st["ms"], 3), "avg_ms": st["ms"] / st["launches"],
                     "GBps": st["bytes"] / sec / 1e9, "TFLOPs": st["flops"] / sec / 1e12}
        if total_ms:
            out[name]["share"] = st["ms"] / total_ms
    return out


def roofline_of(prof, traffic_table=None, df=True, slot=None):
    """Roofline of one single-kernel profile slot (default: the one with the largest summed
    time): achieved algorithmic FLOP/s per launch against the derived FP64 / FP32 ALU peak, or
    for the double-float kernels against the FP32 instruction peak over their measured
    instructions per FLOP."""
    single = {k: v for k, v in (prof or {}).items()
              if k.rsplit("_", 1)[0] in SINGLE_KERNEL_SLOTS and v["ms"] > 0 and v["launches"] > 0}
    if not single or (slot is not None and slot not in single):
        return None
    top = slot if slot is not None else max(single, key=lambda k: single[k]["ms"])
    st = prof[top]
    n = st["launches"]
    avg_ms = st["ms"] / n
    achieved = (st["flops"] / n) / (avg_ms / 1e3) / 1e12
    if top.endswith("_f64") and df and top in NCU_DF_INSTR_PER_FLOP:
        ratio = NCU_DF_INSTR_PER_FLOP[top]
        peak = FP32_INSTR_PEAK / ratio / 1e12
        pk = (f"double-float on the FP32 pipe: 152 SMs x 128 lanes x 2.07 GHz FP32 instructions / {ratio} "
              f"instructions per FLOP (ncu)")
    elif top.endswith("_f64"):
        peak, pk = FP64_PEAK_TFLOPS, "derived: 152 SMs x 2 FP64 FMA/clk x 2 FLOP x 2.07 GHz"
    else:
        peak, pk = FP32_PEAK_TFLOPS, "derived: 152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz"
    hbm, hk = measured_peaks()
    return {"bound": "alu", "kernel": top, "achieved": r4(achieved), "peak": r4(peak), "peak_kind": pk,
            "unit": "TFLOP/s", "frac": r4(achieved / peak),
            "traffic": (traffic_table or {}).get(top), "avg_launch_ms": r4(avg_ms), "launches": n,
            "hbm_GBps_algorithmic": r4((st["bytes"] / n) / (avg_ms / 1e3) / 1e9), "hbm_peak_GBps": hbm,
            "hbm_peak_kind": hk}


# ------------------------------------------------------------------------ reference arm
def oracle_serving_solves(ids):
    """Full FP64 oracle solves of the given stream requests on the host cores: seconds each."""
    import synth
    from oracle import earcg
    from oracle.model import Model
    times = []
    for i in ids:
        cfg = synth.config_serving_request(i)
        model = Model(cfg)
        raw = synth.raw_coefficients(cfg["seed"], model.nk, model.p)
        t0 = time.perf_counter()
        res = earcg.solve(model, [raw[k, :, :model.nk[k]].T.copy() for k in range(model.K)])
        times.append(time.perf_counter() - t0)
        if res.status != "converged":
            raise RuntimeError(f"oracle solve of request {i}: {res.status}")
    return times


def oracle_cpu_sample():
    """The cheapest requests of the stored oracle sample (about 10-30 s of host work)."""
    g = golden_serving()
    if not g:
        return []
    rows = sorted(g["solves"].values(), key=lambda r: r["oracle_seconds"])
    pick, tot = [], 0.0
    for r in rows:
        if tot > 12.0 and len(pick) >= 3:
            break
        pick.append(r["request"])
        tot += r["oracle_seconds"]
    return pick


def oracle_sample(cfg, nk_sample=4):
    """One oracle evaluation (density of all k, potential, H applied at nk_sample k-points)
    timed on the host cores; returns seconds per band application of H and the cores."""
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
    per_band = t_h + t_dens / (model.K * model.p)
    return per_band, os.cpu_count(), f"oracle density of all {model.K} k-points + H at {len(ks)} k-points"


def run_reference(args):
    _, rank, _ = rank_env()
    if rank != 0:
        return
    if args.workload == "serving_stream":
        ids = oracle_cpu_sample()
        if not ids:
            print(json.dumps({"impl": "reference", "unavailable": "tests/golden/oracle_serving.json missing"}))
            return
        times = []
        for j in range(args.warmup + args.steps):
            t = oracle_serving_solves([ids[j % len(ids)]])[0]
            if j >= args.warmup:
                times.append(t)
        value = len(times) / sum(times)
        sample = (f"full FP64 oracle solves (warm-up + EARCG to ||R||<=1e-8) of stream requests {ids}, "
                  f"cycled, one per step")
        line = {"impl": "reference", "metric": metric_name(args), "value": value, "unit": "solves/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic", "config": config_of(args, None, args.gpus),
                "cpu_baseline": {"value": value, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    cfg = workload(args.workload)
    if args.workload == "two_atom":
        times = []
        for j in range(args.warmup + args.steps):
            t = oracle_solve_seconds(cfg)
            if j >= args.warmup:
                times.append(t)
        value, sample, kind = len(times) / sum(times), "full oracle solves of the workload, one per step", "oracle"
    else:
        apps, src = oracle_band_apps(args.workload)
        times = []
        for i in range(args.warmup + args.steps):
            per_band, cores, smp = oracle_sample(cfg)
            if i >= args.warmup:
                times.append(per_band)
        if apps is None:
            apps, src = 15000 * len(cfg["kweight"]) * cfg["nbands"] // 1024, "estimate"
        value = 1.0 / (statistics.median(times) * apps)
        sample = f"{smp}; scaled by {apps} band applications per solve ({src})"
        kind = "oracle (extrapolated from a timed sample)"
    line = {"impl": "reference", "metric": metric_name(args, cfg),
            "value": value, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": config_of(args, cfg, args.gpus),
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": os.cpu_count(), "kind": kind,
                             "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def oracle_solve_seconds(cfg):
    import synth
    from oracle import earcg
    from oracle.model import Model
    model = Model(cfg)
    raw = synth.raw_coefficients(cfg["seed"], model.nk, model.p)
    t0 = time.perf_counter()
    res = earcg.solve(model, [raw[k, :, :model.nk[k]].T.copy() for k in range(model.K)])
    if res.status != "converged":
        raise RuntimeError(f"oracle solve: {res.status}")
    return time.perf_counter() - t0


def oracle_band_apps(name):
    path = os.path.join(ROOT, "tests", "golden", f"oracle_{name}.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d["band_applications"], "oracle's own converged solve (tests/golden)"
    return None, None


# ------------------------------------------------------------------------ GPU arm: serving stream
class StreamInputs:
    """Seeded initial coefficients of stream requests: resident on the device (headline) and in
    pinned host memory (end-to-end run), with pinned host result buffers."""

    def __init__(self, ids, dev):
        import torch
        import synth
        import paper_2503_16225_gb300 as E
        self.cfg, self.dev, self.host, self.out = {}, {}, {}, {}
        for i in sorted(set(ids)):
            cfg = synth.config_serving_request(i)
            s = E.System(cfg, E.eacg_default_params(precision=1))   # basis sizes of the request
            raw = torch.from_numpy(synth.raw_coefficients(cfg["seed"], s.nk, s.p, s.n_max))
            s.close()
            self.cfg[i] = cfg
            self.host[i] = raw.pin_memory()
            self.dev[i] = self.host[i].to(dev)
            self.out[i] = torch.empty_like(raw).pin_memory()
        torch.cuda.synchronize()

    def requests(self, ids, arrivals=None, host=False):
        from paper_2503_16225_gb300 import serve
        reqs = []
        for j, i in enumerate(ids):
            reqs.append(serve.Request(rid=j, cfg=self.cfg[i], raw=self.host[i] if host else self.dev[i],
                                      arrival=0.0 if arrivals is None else arrivals[j],
                                      out=self.out[i] if host else None))
        return reqs


def serve_run(inputs, ids, precision, resident, profile=False, host=False, arrivals=None):
    """Serves the requests; returns (device ms from one start event to the end of every request
    stream, wall seconds, outcomes, summed kernel profile)."""
    import torch
    from paper_2503_16225_gb300 import serve
    main = torch.cuda.current_stream()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    free, _ = torch.cuda.mem_get_info()
    srv = serve.Server(hbm_budget=int(0.8 * free), max_resident=resident, precision=precision,
                       start_event=start, profile=profile, host_buffers=host, params=SERVE_PARAMS)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    start.record(main)
    outs = srv.run(inputs.requests(ids, arrivals=arrivals, host=host))
    for o in outs:
        if o.end_event is not None:
            main.wait_event(o.end_event)
    stop.record(main)
    stop.synchronize()
    wall = time.perf_counter() - t0
    return start.elapsed_time(stop), wall, outs, srv.profile


def one_at_a_time(inputs, ids, precision, profile=False):
    """Each request solved alone on a stream of its own (plain one-system-at-a-time solving):
    CUDA-event ms per request, results, summed profile."""
    import torch
    import paper_2503_16225_gb300 as E
    ms, res, prof = [], [], {}
    for i in ids:
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            s = E.System(inputs.cfg[i], E.eacg_default_params(precision=precision, **SERVE_PARAMS),
                     stream=st.cuda_stream)
            if profile:
                E.eacg_profile_enable(s.h, 1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(st)
            E.eacg_set_psi(s.h, inputs.dev[i])
            r = E.eacg_solve(s.h, check=False)
            b.record(st)
            b.synchronize()
            ms.append(a.elapsed_time(b))
            res.append(r)
            if profile:
                for name, v in E.eacg_profile_read(s.h).items():
                    acc = prof.setdefault(name, dict.fromkeys(v, 0))
                    for key, x in v.items():
                        acc[key] += x
            s.close()
    return ms, res, prof


def accuracy_vs_oracle(outs, ids):
    """|E - E_oracle| per atom for the stream requests that have a stored oracle solve."""
    g = golden_serving()
    if not g:
        return None
    errs = []
    for o in outs:
        i = ids[o.rid]
        ref = g["solves"].get(str(i))
        if ref is None or not o.converged:
            continue
        errs.append(abs(o.E - ref["E"]) / max(1, ref["natoms"]))
    return {"max_dE_per_atom_Ha": r4(max(errs)) if errs else None, "requests": len(errs),
            "tolerance": 1e-6, "oracle": "tests/golden/oracle_serving.json"}


def run_serving(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    import paper_2503_16225_gb300 as E
    from paper_2503_16225_gb300.serve import latency_stats

    world, rank, local = rank_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = 1 if args.precision == "mixed" else 0
    E.eacg_batching(args.batch_window)
    if args.switch_res is not None:
        SERVE_PARAMS["switch_res"] = args.switch_res
    M = per_step(args.steps, args.stream_len)
    timed = stream_ids(args.stream_start, args.steps * M)
    warm = stream_ids(0, args.warmup * M)
    sample = fp64_sample_ids()
    inputs = StreamInputs(timed + warm + ([] if args.no_extras else sample), dev)
    log = {}

    # ---- warm-up: W steps of the stream (set-up caches: FFT plans, GEMM tiles per shape)
    if warm:
        serve_run(inputs, warm, prec, args.resident)

    # ---- timed region: K steps (the whole stream), all queued at t = 0
    clocks = Clocks(local)
    launches0 = E.eacg_launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ms, wall, outs, prof = serve_run(inputs, timed, prec, args.resident, profile=True)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = E.eacg_launch_count() - launches0
    clk = clocks.stop()
    log["busy"] = getattr(clocks, "busy", None)
    conv = sum(1 for o in outs if o.converged)
    total_ms = max_over_ranks(ms, world, dev)
    value = whole_job_rate(world, conv, total_ms)
    st = latency_stats(outs)
    hpsi_bytes = sum(v["bytes"] for k, v in prof.items() if k.rsplit("_", 1)[0] in HPSI_SLOTS)
    failed = [f"{timed[o.rid]}: {o.status}" for o in outs if not o.converged]
    log["served_profile_overlapped"] = profile_summary(prof, ms)

    line = {
        "metric": metric_name(args), "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32/f64" if prec else "f64", "data": "synthetic", "config": config_of(args, None, world),
        "converged": conv, "requests": len(outs), "failed": failed[:4],
        "latency_s": {"saturated": {"solve_p50": r4(st["solve_p50_s"]), "solve_p99": r4(st["solve_p99_s"])}},
        "hpsi_gbs": r4(hpsi_bytes / (ms / 1e3) / 1e9),
        "gpu_launches": launches, "clocks": clk, "busy": log["busy"],
    }
    acc = accuracy_vs_oracle(outs, timed)
    if acc:
        line["accuracy"] = acc

    if not args.no_extras:
        # ---- end to end: the same stream through eacg_solve_host (pinned host input and output,
        # copies inside each request), wall clock with a synchronize on both sides
        torch.cuda.synchronize()
        _, e2e_wall, e_outs, _ = serve_run(inputs, timed, prec, args.resident, host=True)
        e2e_conv = sum(1 for o in e_outs if o.converged)
        e2e_s = max_over_ranks(e2e_wall, world, dev)
        nbytes = sum(inputs.host[i].numel() * 16 for i in timed)
        line["e2e"] = {"value": whole_job_rate(world, e2e_conv, e2e_s * 1e3), "unit": "solves/s",
                       "h2d_bytes_per_step": nbytes // args.steps, "d2h_bytes_per_step": nbytes // args.steps}

        # ---- plain FP64, one system at a time, on the sample (the served speed-up's denominator),
        # and the mixed mode alone on the same requests (profiled: no overlapping kernels)
        f_ms, f_res, _ = one_at_a_time(inputs, sample, 0)
        m_ms, m_res, m_prof = one_at_a_time(inputs, sample, prec, profile=True)
        fp64_rate = len(sample) / (sum(f_ms) / 1e3)
        line["fp64_one_at_a_time"] = {
            "solves_per_s": r4(fp64_rate), "sample": f"stream requests i % {FP64_SAMPLE_STRIDE} == 0 "
            f"({len(sample)})", "converged": sum(1 for r in f_res if r.status == 0),
            "mixed_alone_solves_per_s": r4(len(sample) / (sum(m_ms) / 1e3))}
        line["served_over_fp64"] = r4(value / world / fp64_rate)
        line["roofline"] = roofline_of(m_prof)
        if line["roofline"]:
            line["roofline"]["timed"] = "sample requests solved one at a time in mixed precision"
        # the transform kernels of the H application (FP64-accurate and FP32) on the same sample
        line["roofline_transforms"] = {}
        for slot in ("plane_h_f64", "plane_h_f32"):
            r = roofline_of(m_prof, slot=slot)
            if r:
                line["roofline_transforms"][slot] = {k: r[k] for k in ("achieved", "peak", "unit", "frac",
                                                                        "avg_launch_ms", "launches")}
        log["mixed_alone_profile"] = profile_summary(m_prof, sum(m_ms))

        # ---- Poisson streams at 0.5x and 2x the FP64 one-at-a-time rate (arrival -> converged)
        rng = np.random.default_rng(7)
        for tag, mult, count in (("poisson_2x_fp64", 2.0, 32), ("poisson_0.5x_fp64", 0.5, 12)):
            rate = mult * fp64_rate
            gaps = rng.exponential(1.0 / rate, size=count)
            arrivals = list(np.concatenate([[0.0], np.cumsum(gaps[:-1])]))
            ids = stream_ids(0, count)
            _, _, p_outs, _ = serve_run(inputs, ids, prec, args.resident, arrivals=arrivals)
            pst = latency_stats(p_outs)
            line["latency_s"][tag] = {"rate_per_s": r4(rate), "requests": count, "p50": r4(pst["p50_s"]),
                                      "p99": r4(pst["p99_s"]), "converged": pst["converged"]}

        # ---- CPU baseline: the oracle as it stands, full solves of sampled requests (rank 0)
        if rank == 0 and world == 1:
            ids = oracle_cpu_sample()
            try:
                times = oracle_serving_solves(ids)
                line["cpu_baseline"] = {
                    "value": r4(len(ids) / sum(times)), "unit": "solves/s", "cores": os.cpu_count(),
                    "kind": "oracle", "sample": f"full FP64 oracle solves of stream requests {ids} "
                    f"({sum(times):.1f} s of host time)"}
            except Exception as exc:  # the baseline is a report, not the measurement
                line["cpu_baseline"] = {"value": None, "unit": "solves/s", "cores": os.cpu_count(),
                                        "kind": "oracle", "sample": f"failed: {exc}"}
    if rank == 0:
        sys.stderr.write(json.dumps(log) + "\n")
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------------------ GPU arm: one workload
def run_solve(args):
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

    def many_on(res, ends):
        """All systems stepped together by eacg_step_many until every one has converged."""
        for sy, _ in systems:
            E.eacg_set_psi(sy.h, psi0)
        live = list(range(C))
        iters = [0] * C
        apps = [0] * C
        while live:
            infos, sts = E.eacg_step_many([systems[i][0].h for i in live], window_us=2000)
            nxt = []
            for j, i in enumerate(live):
                iters[i] += 1
                apps[i] = infos[j].h_band_apps
                if infos[j].converged:
                    res[i] = E.EacgResult(E=infos[j].E, rnorm=infos[j].rnorm, iterations=iters[i] - 1,
                                          warm_iterations=0, status=0, ls_trials=0, h_band_apps=apps[i])
                    ends[i].record(systems[i][1])
                elif iters[i] > params.max_outer + 1:
                    res[i] = RuntimeError("step_many: iteration cap")
                    ends[i].record(systems[i][1])
                else:
                    nxt.append(i)
            live = nxt

    def one_round():
        start = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for _, st_i in systems:
            st_i.wait_event(start)
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(C)]
        res = [None] * C
        if args.step_many:
            ths = [threading.Thread(target=many_on, args=(res, ends))]
        else:
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

    clocks = Clocks(local)
    for sy, _ in systems:
        E.eacg_profile_enable(sy.h, 1)
    launches0 = E.eacg_launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    per, latencies, results = [], [], []
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
    for sy, _ in systems:
        for name, st in E.eacg_profile_read(sy.h).items():
            acc = prof.setdefault(name, dict.fromkeys(st, 0))
            for key in acc:
                acc[key] += st[key]
        E.eacg_profile_enable(sy.h, 0)
    total_ms = max_over_ranks(sum(per), world, dev)
    value = whole_job_rate(world, C * args.steps, total_ms)

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

    fp64_ref = None
    if prec == 1 and not args.no_extras:
        s64 = E.System(cfg, E.eacg_default_params(precision=0, method=method))
        for _ in range(2):  # one untimed solve, then one timed
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
        fp64_ref = {"solves_per_s": r4(1e3 / fp64_ms), "iterations": r64.iterations}

    roof = roofline_of(prof, NCU_TRAFFIC_BYTES if args.workload == "diamond_k444" else None)
    if roof:
        roof["timed"] = f"{C} concurrent systems (kernels of other systems may overlap)"
    apps = sum(r.h_band_apps for r in results)
    hpsi_gbs = sum(v["bytes"] for k, v in prof.items() if k.rsplit("_", 1)[0] in HPSI_SLOTS) / (total_ms / 1e3) / 1e9

    line = {
        "metric": metric_name(args, cfg),
        "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32/f64" if prec else "f64", "data": "synthetic",
        "config": config_of(args, cfg, world),
        "time_to_1e8_ms": {"p50": r4(statistics.median(latencies)), "p99": r4(max(latencies))},
        "fp64_one_at_a_time": fp64_ref,
        "served_over_fp64": r4(value / world / fp64_ref["solves_per_s"]) if fp64_ref else None,
        "solve": {"E": results[-1].E, "rnorm": results[-1].rnorm, "iterations": results[-1].iterations,
                  "h_band_apps": results[-1].h_band_apps, "band_apps_total": apps},
        "hpsi_gbs": r4(hpsi_gbs), "roofline": roof, "gpu_launches": launches, "clocks": clk,
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": C * host.numel() * 16,
                "d2h_bytes_per_step": C * host.numel() * 16},
    }
    gpath = os.path.join(ROOT, "tests", "golden", f"oracle_{args.workload}.json")
    if os.path.exists(gpath):  # the oracle's own converged solve of this workload
        with open(gpath) as fh:
            gd = json.load(fh)
        line["accuracy"] = {"dE_per_atom_Ha": r4(abs(results[-1].E - gd["E"]) / max(1, gd["natoms"])),
                            "tolerance": 1e-6 if prec else 1e-8, "oracle": os.path.relpath(gpath, ROOT)}
    if rank == 0 and world == 1 and not args.no_extras:
        try:
            if args.workload == "two_atom":
                t = oracle_solve_seconds(cfg)
                line["cpu_baseline"] = {"value": r4(1.0 / t), "unit": "solves/s", "cores": os.cpu_count(),
                                        "kind": "oracle", "sample": "one full oracle solve of the workload"}
            else:
                per_band, cores, sample = oracle_sample(cfg)
                apps_solve = results[-1].h_band_apps
                line["cpu_baseline"] = {"value": r4(1.0 / (per_band * apps_solve)), "unit": "solves/s",
                                        "cores": cores, "kind": "oracle (extrapolated from a timed sample)",
                                        "sample": f"{sample}, scaled by this solve's {apps_solve} band applications"}
        except Exception as exc:
            line["cpu_baseline"] = {"value": None, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                                    "sample": f"failed: {exc}"}
    if rank == 0:
        sys.stderr.write(json.dumps({"profile": profile_summary(prof, total_ms)}) + "\n")
        print(json.dumps(line))
    for sy, _ in systems:
        sy.close()
    if world > 1:
        dist.destroy_process_group()


def hpsi_bytes_per_band(sysm, prec_bytes):
    """Algorithmic HBM bytes of one band application of H with the pruned transforms:
    coefficients in + out (complex double) and the x-pass intermediate written, read and
    written back by the plane kernel, then read (4 passes of N * ncols complex values of
    2 * prec_bytes bytes: 8 for FP32 transforms, 16 for FP64)."""
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
    else:  # orthonormal start by host QR (p above the library's dense-kernel limit)
        for k, n in enumerate(sysm.nk):
            q = np.linalg.qr(raw[k, :, :n].T)[0]
            phi[k, :, :n] = torch.from_numpy(np.ascontiguousarray(q.T))
    E.eacg_density(sysm.h, phi, None, 0 if sysm.N <= 96 else 1)   # N = 128: FP32 transforms only
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
        line["band_apps_per_s"] = sysm.K * sysm.p / (ms / 1e3)
        line["hpsi_gbs"] = sysm.K * sysm.p * hpsi_bytes_per_band(sysm, 4 if prec else 8) / (ms / 1e3) / 1e9
    print(json.dumps(line))
    sysm.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.op != "solve":
        run_op(args)
    elif args.workload == "serving_stream":
        run_serving(args)
    else:
        run_solve(args)


if __name__ == "__main__":
    main()
