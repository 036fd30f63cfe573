"""Multi-rank bench logic on CPU (gloo, world size 2): each rank runs its own copy of the
independent-instance workload, and the only collective is the max over ranks of the timed
region; the reference arm runs on rank 0 alone."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    got = bench.max_over_ranks([10.0 * (rank + 1), 3.0 - rank], dist, "cpu")
    rate = bench.aggregate_rate(world, 1000, 10, got[0] * 1e-3)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got, rate))


def test_max_over_ranks_and_weak_scaling_rate():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, rate in res:
        assert got == [20.0, 3.0]
        # 2 ranks x 1000 cells x 10 steps in 20 ms
        assert rate == pytest.approx(2 * 1000 * 10 / 0.020 / 1e6)


def test_reference_arm_is_rank0_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup = 1, 0
    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""
