"""The multi-rank (replica) host logic on CPU: world_size 2 over gloo."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2408_12894_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = replicas.world()
    views = list(range(10))
    mine = replicas.shard(views, r, w)
    times = replicas.max_over_ranks([1.0 + r, 5.0 - r])
    replicas.barrier(device_sync=False)
    q.put((r, w, lr, mine, times))
    dist.destroy_process_group()


def test_two_replicas_shard_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, m0, t0), (r1, w1, l1, m1, t1) = out
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert sorted(m0 + m1) == list(range(10)) and not set(m0) & set(m1)
    assert t0 == t1 == [2.0, 5.0]


def test_single_process_defaults():
    assert replicas.shard([1, 2, 3], 0, 1) == [1, 2, 3]
    assert replicas.max_over_ranks([3.5]) == [3.5]
