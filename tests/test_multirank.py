"""The benchmark's multi-rank path on the CPU: two processes in a gloo process group (the
same collectives the NCCL run makes). Replicas only: every rank advances its own
realisation and the job's throughput is the work of all ranks over the slowest rank's time;
the reference arm runs on rank 0 alone."""
import json
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (1 + r) seconds for 10 (r + 1) units of work
        value, t, w = bench.replica_totals(1.0 + rank, 10.0 * (rank + 1), world, "cpu")
        mx = bench.reduce_over_ranks(3.0 - rank, "max", world, "cpu")
        sm = bench.reduce_over_ranks(0.5, "sum", world, "cpu")
        with open(os.path.join(outdir, f"rank{rank}.json"), "w") as fh:
            json.dump({"value": value, "t": t, "w": w, "max": mx, "sum": sm}, fh)
    finally:
        dist.destroy_process_group()


def test_replica_totals_over_two_gloo_ranks(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:  # every rank sees the same job totals
        assert r["t"] == 2.0 and r["w"] == 30.0 and r["value"] == pytest.approx(15.0)
        assert r["max"] == 3.0 and r["sum"] == 1.0


def test_single_rank_reductions_are_the_identity():
    assert bench.replica_totals(2.0, 8.0, 1, "cpu") == (4.0, 2.0, 8.0)
    assert bench.reduce_over_ranks(5.0, "max", 1, "cpu") == 5.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import argparse

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(gpus=2, steps=1, warmup=0)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""  # the other ranks exit without work or output
