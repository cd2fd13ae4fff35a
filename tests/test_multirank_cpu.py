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


@pytest.mark.parametrize("config,n,knn,sample", [("c2", 16384, 0, 256), ("c4", 0, 0, 40),
                                                 ("c5", 65536, 0, 32), ("c2", 16384, 16, 64)])
def test_reference_arm_json_line(monkeypatch, capsys, config, n, knn, sample):
    """The reference arm (the oracle on a bounded sample) prints one line with the keys of the
    bench contract, its own value repeated as cpu_baseline and e2e, and no host copies."""
    import argparse
    import json

    import bench

    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    args = argparse.Namespace(impl="reference", config=config, n=n, steps=2, warmup=1,
                              cpu_sample=sample, kernel="m4", knn=knn)
    bench.run_reference(args)
    lines = [x for x in capsys.readouterr().out.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1
    assert d["metric"] == (bench.KNN_METRIC if knn else bench.METRIC) and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["value"] > 0
    assert d["config"]["workload"].startswith(config + ":")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
