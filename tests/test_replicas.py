"""Host side of `bench.py --gpus N` (replicas only, no data-path
collective): two gloo ranks on the CPU check the per-replica camera batches
and the max-over-ranks timing reduction."""
import os
import socket
import sys

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = bench.replica_batches(rank, world, 16, 8)
        worst = bench.max_over_ranks(10.0 + rank, world)
        everyone = [None] * world
        dist.all_gather_object(everyone, mine)
        out.put((rank, mine, worst, everyone))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_disjoint_batches_and_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res.sort()
    for rank, mine, worst, everyone in res:
        assert worst == 10.0 + world - 1
        assert mine == [(rank + 2 * i) % 16 for i in range(8)]
        assert not set(everyone[0]) & set(everyone[1])


def test_single_process_needs_no_process_group():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.replica_batches(0, 1, 4, 6) == [0, 1, 2, 3, 0, 1]

