"""Host logic of bench.py for more than one rank, on CPU with gloo.

bench.py runs one independent replica per GPU (the path has no exchange
step: scenarios of one system are not split across GPUs), so the only
multi-rank logic is the max-over-ranks timing, the whole-job throughput,
the per-rank instance draw and the rank-0-only reference arm. These run
here as two gloo ranks on CPU.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import bmgen


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 95.5][rank]                     # rank 0 is the slow one
        slowest = bench.max_over_ranks(local_ms, dist)
        value = bench.whole_job_gflops(world, 4.7e7, 10, slowest)
        w = bmgen.WORKLOADS["plain-s4-n16-nb4"]
        d = bmgen.generate(w, instance=rank)
        dist.barrier()
        out[rank] = (slowest, value, float(d["r"][:4].sum()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 120.0
    assert res[0][1] == res[1][1] == pytest.approx(2 * 4.7e7 * 10 / 0.120 / 1e9)
    assert res[0][2] != res[1][2]            # each replica draws its own system


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_gflops(1, 1e9, 2, 1000.0) == pytest.approx(2.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = bench.argparse.Namespace(workload="plain-s4-n16-nb4", steps=1, warmup=0, ref_budget=0.01, gpus=2)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_rank_zero(monkeypatch, capsys):
    import json
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    args = bench.argparse.Namespace(workload="plain-s4-n16-nb4", steps=2, warmup=1, ref_budget=0.02, gpus=1)
    assert bench.run_reference(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "GFLOP/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
