"""Writes tests/golden/oracle_<name>.json: the FP64 CPU oracle's converged eARCG solve of a
synthetic workload (energy, residual, iteration and Hamiltonian-application counts).

Calls only oracle/ (and the seeded input generators in synth/).  Usage:
    python tests/golden/make_golden.py diamond_k444     # 8-atom diamond, 4x4x4 k, 48^3, 16 bands
    python tests/golden/make_golden.py two_atom
    python tests/golden/make_golden.py diamond64_ec5    # 64-atom supercell, Ecut 5, 48^3, 128 bands
    python tests/golden/make_golden.py diamond64_gamma  # 64-atom supercell, Ecut 15, 96^3 (hours)
    python tests/golden/make_golden.py serving          # sampled requests of the serving stream

The serving target writes tests/golden/oracle_serving.json: converged oracle solves of
SERVING_SAMPLE requests of the 256-request stream (synth.config_serving_request), drawn with
numpy default_rng(256) among the requests of oracle cost K p N^3 <= 8 * 3 * 32^3 (the
oracle finishes each in seconds), so that the served energies can be checked per atom.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import earcg  # noqa: E402
from oracle.model import Model  # noqa: E402

WORKLOADS = {
    "two_atom": lambda: synth.config_two_atom(1),
    "diamond_k111": lambda: synth.config_diamond(2, kgrid=(1, 1, 1)),
    "diamond_k222": lambda: synth.config_diamond(2, kgrid=(2, 2, 2)),
    "diamond_k444": lambda: synth.config_diamond(2, kgrid=(4, 4, 4)),
    # 128 bands (64-atom supercell) at a low cutoff: the many-band dense path at oracle cost
    "diamond64_ec5": lambda: synth.config_diamond_supercell(2, ecut=5.0, N=48),
    # the full-size 64-atom supercell at Gamma (Ecut 15, 96^3, 128 bands): hours of oracle time
    "diamond64_gamma": lambda: synth.config_diamond_supercell(2),
}


def main(name):
    cfg = WORKLOADS[name]()
    model = Model(cfg)
    raw = synth.raw_coefficients(cfg["seed"], model.nk, model.p)
    psi0 = [raw[k, :, :model.nk[k]].T.copy() for k in range(model.K)]
    t0 = time.time()
    log = []

    def cb(h):
        log.append({k: h[k] for k in ("it", "E", "rnorm", "tau", "beta", "phase", "trials")})
        print(json.dumps(log[-1]), f"{time.time() - t0:.1f}s", flush=True)

    res = earcg.solve(model, psi0, callback=cb)
    out = {
        "workload": cfg["name"], "status": res.status, "E": res.E, "rnorm": res.rnorm,
        "iterations": res.iterations, "warm_iterations": res.warm_iterations,
        "trial_evaluations": res.evals, "fom_h_columns": res.h_cols,
        "band_applications": res.evals * model.K * model.p + res.h_cols,
        "natoms": int(len(cfg["Z"])), "nk": model.nk, "terms": res.point.terms,
        "oracle_seconds": time.time() - t0, "history": log,
        "note": "band_applications counts one band at one k-point as one H application",
    }
    with open(os.path.join(HERE, f"oracle_{name}.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(res.status, res.E, res.rnorm, res.iterations)


SERVING_STREAM = 256
SERVING_SAMPLE = 16
SERVING_COST_MAX = 8 * 3 * 32 ** 3


def serving_sample():
    """Request indices of the serving stream whose oracle solves are stored (seeded choice)."""
    import numpy as np
    cheap = []
    for i in range(SERVING_STREAM):
        c = synth.config_serving_request(i)
        if len(c["kweight"]) * c["nbands"] * c["N"] ** 3 <= SERVING_COST_MAX:
            cheap.append(i)
    pick = np.random.default_rng(256).choice(len(cheap), SERVING_SAMPLE, replace=False)
    return sorted(int(cheap[j]) for j in pick)


def solve_request(i):
    cfg = synth.config_serving_request(i)
    model = Model(cfg)
    raw = synth.raw_coefficients(cfg["seed"], model.nk, model.p)
    t0 = time.time()
    res = earcg.solve(model, [raw[k, :, :model.nk[k]].T.copy() for k in range(model.K)])
    return {"request": i, "status": res.status, "E": res.E, "rnorm": res.rnorm, "iterations": res.iterations,
            "natoms": int(len(cfg["Z"])), "nk": len(cfg["kweight"]), "nbands": model.p, "N": model.N,
            "band_applications": res.evals * model.K * model.p + res.h_cols,
            "oracle_seconds": time.time() - t0}


def main_serving():
    from concurrent.futures import ProcessPoolExecutor
    import multiprocessing as mp
    ids = serving_sample()
    with ProcessPoolExecutor(max_workers=1, mp_context=mp.get_context("spawn")) as ex:
        rows = list(ex.map(solve_request, ids))
    for r in rows:
        print(json.dumps(r), flush=True)
    out = {"stream": "synth.config_serving_request(i), i < 256", "sample": ids,
           "selection": f"default_rng(256) choice of {SERVING_SAMPLE} among requests with K p N^3 <= "
                        f"{SERVING_COST_MAX}", "solves": {str(r["request"]): r for r in rows}}
    with open(os.path.join(HERE, "oracle_serving.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    if sys.argv[1] == "serving":
        main_serving()
    else:
        main(sys.argv[1])
