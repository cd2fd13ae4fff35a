"""The multi-process path of bench.py on the CPU: two gloo ranks.

Across GPUs the solve runs as replicas (one independent copy of the workload per rank, no
collective on the data path), so what needs checking is the host logic around it: every rank
synchronises on the barrier, the step time reported is the maximum over ranks, and the value is
all particles of all ranks divided by that time.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        per_rank_ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        t = bench.max_over_ranks(per_rank_ms, world)
        n = 1000
        value = world * n / (t / 1e3)
        out[rank] = (t, value)
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_ranks_barrier_and_max_time():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1]
    t, value = out[0]
    assert t == pytest.approx(15.0)
    assert value == pytest.approx(2 * 1000 / 0.015)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun the CPU reference arm runs and prints on rank 0 only; other ranks exit
    without work."""
    import argparse

    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "1")  # no rendezvous needed for this check
    args = argparse.Namespace(impl="reference", config="c2", n=0, steps=1, warmup=0, cpu_sample=0,
                              kernel="m4")
    bench.run_reference(args)
    assert capsys.readouterr().out == ""
