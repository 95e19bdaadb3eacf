"""The multi-GPU path is N independent replicas (the method's hot path has no
exchange step on one GPU); what crosses ranks is host logic, tested here with
two gloo ranks on the CPU: the job time is the slowest rank's, each rank runs
its own seeded replica, and the reference arm prints from rank 0 only."""
import argparse
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # per-rank times: the job's is the largest
        out[rank] = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    world = 2
    port = _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert dict(out) == {0: 15.0, 1: 15.0}


def test_max_over_ranks_without_a_process_group():
    import bench
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25


def test_each_rank_runs_its_own_replica():
    import bench
    a, b = bench.make_scene("ring50", 0), bench.make_scene("ring50", 1)
    assert a.n_cams == b.n_cams and not np.allclose(a.obs_uv[:10], b.obs_uv[:10])


def test_reference_arm_prints_from_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(argparse.Namespace(workload="ring50", steps=1, warmup=0))
    assert capsys.readouterr().out == ""


def test_reference_arm_line_keeps_the_contract(monkeypatch, capsys):
    """Rank 0 of the reference arm (the oracle on the host) prints one JSON
    line with the contract's keys."""
    import json
    import bench
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setenv("RANK", "0")
    bench.run_reference(argparse.Namespace(workload="ring50", steps=1, warmup=0))
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
