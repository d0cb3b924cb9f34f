"""The multi-rank host logic of bench.py (replicas: no collective on the data path, the job's
time is the slowest rank's, the value counts the units of all ranks), run as two gloo ranks on
the CPU, and the reference arm's rank handling."""
import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.rank_env()
        local_ms = 10.0 * (rank + 1)          # rank 1 is the slow one
        ms = bench.max_over_ranks(local_ms, w)
        rate = bench.whole_job_rate(w, 4, ms)  # 4 solves per rank
        dist.barrier()
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
            json.dump({"env": [w, r, local], "ms": ms, "rate": rate}, fh)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_all_units(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for rank in range(world):
        d = json.load(open(tmp_path / f"rank{rank}.json"))
        assert d["env"] == [world, rank, rank]
        assert d["ms"] == 20.0
        assert d["rate"] == pytest.approx(2 * 4 / 0.020)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.whole_job_rate(1, 3, 1500.0) == pytest.approx(2.0)


def test_reference_arm_prints_only_on_rank_zero(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    bench.run_reference(bench.parse())
    assert capsys.readouterr().out == ""


def test_both_arms_share_metric_and_config():
    """Both arms build the metric name and the config from the same helpers: the default is the
    256-request serving stream, split into K steps that cover the stream once."""
    import synth
    import sys
    old = sys.argv
    try:
        sys.argv = ["bench.py", "--steps", "20"]
        args = bench.parse()
        sys.argv = ["bench.py", "--workload", "diamond_k444"]
        args_d = bench.parse()
    finally:
        sys.argv = old
    assert args.workload == "serving_stream"
    assert bench.metric_name(args) == "served eARCG solves/s (stream of 256 synthetic crystals, to ||R||<=1e-8)"
    c = bench.config_of(args, None, 1)
    assert c["workload"] == "serving_stream_256" and c["parallelism"] == "replicas1"
    assert c["requests_per_step"] == 13 and 13 * 20 >= 256
    assert bench.stream_ids(250, 8) == [250, 251, 252, 253, 254, 255, 0, 1]
    assert bench.fp64_sample_ids() == list(range(0, 256, 16))
    cfg = synth.config_diamond(2, kgrid=(4, 4, 4))
    assert bench.metric_name(args_d, cfg) == "served eARCG solves/s (diamond8 4x4x4k 48^3 p16, to ||R||<=1e-8)"
    c = bench.config_of(args_d, cfg, 1)
    assert c["workload"] == cfg["name"] and c["parallelism"] == "replicas1" and c["concurrent_systems"] == 4
