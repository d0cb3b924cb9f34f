"""k-point sharding of the evaluation across ranks (the design of a multi-GPU
variant), checked as two gloo ranks on the CPU over the oracle.  H is block-diagonal in k
(Sec. 5.1, Eq. (5.1)): a rank holding the k-points r, r + 2, ... with their global weights
computes its partial density, one all-reduce makes the full density (so every rank builds the
same potential), and the k-sums of the kinetic and nonlocal energies, ||R||^2 and the pairings
<R, G> are all-reduces of scalars.  The FOM and the energy-adaptive gradient are per k and need
no exchange.  The sharded results equal the one-rank evaluation."""
import copy
import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from oracle import earcg  # noqa: E402
from oracle.manifold import herm, outer  # noqa: E402
from oracle.model import Model  # noqa: E402
from tests.small_models import small, start  # noqa: E402


def _cfg():
    return small(nproj=4, kgrid=(2, 2, 1), nb=3, ecut=3.0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _allreduce(x):
    t = torch.as_tensor(np.asarray(x, dtype=np.float64).copy())
    dist.all_reduce(t)
    return t.numpy()


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cfg = _cfg()
        full = Model(cfg)
        Phi_all = earcg.lowdin(start(full))
        ks = list(range(rank, full.K, world))
        sub_cfg = copy.deepcopy(cfg)
        sub_cfg["kfrac"] = cfg["kfrac"][ks]
        sub_cfg["kweight"] = cfg["kweight"][ks]          # global weights of this rank's k-points
        sub = Model(sub_cfg)
        Phi = [Phi_all[k] for k in ks]
        # density: partial sums, one all-reduce of the N^3 grid
        rho = _allreduce(sub.density(Phi))
        vtot = sub.potentials(rho)[0]
        HPhi = [sub.apply_H(k, Phi[k], vtot) for k in range(sub.K)]
        Lam = [herm(outer(Phi[k], HPhi[k])) for k in range(sub.K)]
        R = [HPhi[k] - Phi[k] @ Lam[k] for k in range(sub.K)]
        terms = sub.energy_terms(Phi, rho)
        kin, nl = _allreduce([terms["kin"], terms["nl"]])
        r2 = float(_allreduce([sum(float(np.vdot(r, r).real) for r in R)])[0])
        E = kin + nl + terms["loc"] + terms["hartree"] + terms["xc"]
        # energy-adaptive gradient per k (no exchange) and the pairing <R, G> as one all-reduce
        pt = earcg.Point(Phi, rho, vtot, HPhi, Lam, R, E, terms, np.sqrt(r2))
        G = earcg.ea_gradient(sub, pt, earcg.Params())
        rg = float(_allreduce([sum(sub.kw[k] * np.vdot(R[k], G[k]).real for k in range(sub.K))])[0])
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
            json.dump({"E": E, "kin": float(kin), "nl": float(nl), "rnorm": float(np.sqrt(r2)), "rg": rg,
                       "rho_sum": float(rho.sum()), "ks": ks}, fh)
        np.save(os.path.join(out_dir, f"rho{rank}.npy"), rho)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_the_k_points_and_match_one_rank(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    cfg = _cfg()
    model = Model(cfg)
    Phi = earcg.lowdin(start(model))
    pt = earcg.evaluate(model, Phi)
    G = earcg.ea_gradient(model, pt, earcg.Params())
    from oracle.model import pairing
    rg = pairing(model, pt.R, G)
    ranks = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    assert sorted(ranks[0]["ks"] + ranks[1]["ks"]) == list(range(model.K)) and model.K == 4
    for d in ranks:
        assert abs(d["E"] - pt.E) <= 1e-12 * abs(pt.E)
        assert abs(d["kin"] - pt.terms["kin"]) <= 1e-12 * abs(pt.terms["kin"])
        assert abs(d["nl"] - pt.terms["nl"]) <= 1e-12 * abs(pt.terms["nl"])
        assert abs(d["rnorm"] - pt.rnorm) <= 1e-12 * pt.rnorm
        # the density's k-sum runs in another order (partial sums + all-reduce): last-bit
        # differences, which the FOM at this random (not yet coercive) point amplifies ~1e8 times
        assert abs(d["rg"] - rg) <= 1e-7 * abs(rg)
    for r in range(world):
        np.testing.assert_allclose(np.load(tmp_path / f"rho{r}.npy"), pt.rho, rtol=0, atol=1e-13 * np.abs(pt.rho).max())
