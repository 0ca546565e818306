"""The benchmark's multi-rank logic on CPU with gloo, world size 2 (no GPU).

Samples are independent (the paper's G x B x T parallelism, Sec. 5.2), so
ranks shard the pointing stream with no data-path collective; the only
collectives are the barrier and the max of the timed region over ranks.
"""

import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        a, b = bench.shard(n, rank, world)
        sizes = [None] * world
        dist.all_gather_object(sizes, (a, b))
        slowest = bench.max_over_ranks(10.0 + rank, "cpu")
        dist.barrier()
        out.put((rank, sizes, slowest))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("n", [10, 1_000_003])
def test_two_gloo_ranks_shard_and_take_the_slowest_time(n):
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, out)) for r in range(world)]
    for p in procs:
        p.start()
    results = [out.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, sizes, slowest in results:
        # contiguous, disjoint, covering [0, n)
        assert sizes[0][0] == 0 and sizes[-1][1] == n
        assert all(sizes[k][1] == sizes[k + 1][0] for k in range(world - 1))
        assert slowest == 11.0


def test_single_process_needs_no_process_group():
    assert bench.shard(7, 0, 1) == (0, 7)
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
