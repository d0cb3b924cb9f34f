"""Writes tests/golden/oracle_<name>.json: the FP64 CPU oracle's converged eARCG solve of a
synthetic workload (energy, residual, iteration and Hamiltonian-application counts).

Calls only oracle/ (and the seeded input generators in synth/).  Usage:
    python tests/golden/make_golden.py diamond_k444     # 8-atom diamond, 4x4x4 k, 48^3, 16 bands
    python tests/golden/make_golden.py two_atom
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


if __name__ == "__main__":
    main(sys.argv[1])
