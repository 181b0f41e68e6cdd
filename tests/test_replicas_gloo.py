"""The multi-rank path of the benchmark on CPU: two gloo ranks, each timing its own replica.

On one GPU per rank the solver does not shard (one problem per GPU, no data-path collective);
the only collective is the max-over-ranks reduction of the per-step time.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, queue):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    v = bench.reduce_over_ranks(10.0 + 3.0 * rank, world, torch.device("cpu"))
    dist.barrier()
    dist.destroy_process_group()
    queue.put((rank, v))


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: 13.0, 1: 13.0}


def test_single_rank_is_identity():
    import bench
    import torch

    assert bench.reduce_over_ranks(7.5, 1, torch.device("cpu")) == 7.5


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    import bench

    monkeypatch.setenv("RANK", "1")

    class A:
        n, s, sweeps, algo, form, steps, warmup, gpus = 256, 4, 3, "literal", "stencil", 1, 1, 2

    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""
