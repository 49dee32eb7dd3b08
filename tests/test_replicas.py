"""Host logic of the multi-GPU replicas, on CPU: the batch sharding and the timing summary over
two gloo ranks (the same code aggregates over NCCL on GPUs)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1210_2258_b300 import replicas


def test_shard_covers_every_problem_once_and_balances():
    sizes = [1024 ** 2, 128 ** 2, 512 ** 2, 768 ** 2, 256 ** 2, 1024 ** 2, 384 ** 2, 128 ** 2, 512 ** 2]
    for world in (1, 2, 3, 4):
        parts = [replicas.shard(sizes, r, world) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)
    with pytest.raises(ValueError):
        replicas.shard(sizes, 2, 2)


def test_aggregate_single_process():
    assert replicas.aggregate(12.5, 33) == (12.5, 33)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, it = replicas.aggregate(10.0 + 5.0 * rank, 30 + rank)
        out[rank] = (ms, it)
    finally:
        dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    # slowest rank's time, total iterations, identical on both ranks
    assert res[0] == res[1] == (15.0, 61)
