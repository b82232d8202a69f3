"""The multi-GPU path of bench.py runs independent replicas: each rank times its
own work, the job time is the slowest rank's, the value counts every rank's
units.  Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.reduce_max([1.0 + rank, 10.0 - rank, 3.0])
        q.put((rank, got, bench.job_value(world, 100.0, got[0])))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    [p.start() for p in procs]
    [p.join(120) for p in procs]
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=5) for _ in range(2))
    for rank, got, value in res:
        assert got == [2.0, 10.0, 3.0]           # the slowest rank's time, element-wise
        assert value == pytest.approx(2 * 100.0 / 2.0)


def test_single_process_is_identity():
    import bench
    assert bench.reduce_max([4.0, 5.0]) == [4.0, 5.0]
    assert bench.job_value(1, 10.0, 2.0) == 5.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun the reference arm (the CPU oracle) runs on rank 0 alone;
    the other ranks exit without work or output."""
    import argparse
    import bench
    calls = []
    monkeypatch.setattr(bench, "oracle_step", lambda d: calls.append(d) or (10, 0.5, None))
    args = argparse.Namespace(steps=2, warmup=1)
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(args)
    assert calls == [] and capsys.readouterr().out == ""
    monkeypatch.setenv("RANK", "0")
    bench.run_reference(args)
    out = capsys.readouterr().out
    import json
    line = json.loads(out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and len(calls) == 3
    assert line["value"] == 10 / 0.5 and line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["config"]["workload"] == bench.WORKLOAD
