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


class _FakePlan:
    """Stands in for a plan on CPU: its 'transposes' are fixed linear maps of the samples,
    so the sum over ranks' shards must equal the map of the whole stream."""

    def adjoint(self, theta, phi, psi, tod, det=0):
        import torch
        w = torch.stack([torch.cos(theta), torch.sin(phi), psi])       # (3, n)
        return (w * tod[None, :]).reshape(3, -1).sum(dim=1, keepdim=True) * torch.arange(1.0, 5.0)[None, :]

    def beam_grid_adjoint(self, theta, phi, psi, y, det=0):
        import torch
        return torch.outer(torch.stack([theta @ y, phi @ y]), torch.arange(1.0, 4.0)).reshape(6)[:, None, None] \
            * torch.ones(6, 2, 2, dtype=theta.dtype)

    def omega_adjoint(self, tod, y, grad, det=0):
        grad[0] -= float(tod @ y)
        return grad


def _transpose_worker(rank, world, port, out):
    import torch
    from paper_1908_05662_gb300 import distributed as pd
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = torch.Generator().manual_seed(0)
        n = 101
        th, ph, ps, y, d = (torch.randn(n, dtype=torch.float64, generator=g) for _ in range(5))
        a, b = pd.shard_range(n, rank, world)
        plan = _FakePlan()
        maps = pd.sharded_adjoint(plan, th[a:b], ph[a:b], ps[a:b], y[a:b])
        grad = pd.sharded_beam_grid_adjoint(plan, th[a:b], ph[a:b], ps[a:b], y[a:b], tod=d[a:b])
        full_maps = plan.adjoint(th, ph, ps, y)
        full_grad = plan.omega_adjoint(d, y, plan.beam_grid_adjoint(th, ph, ps, y))
        out.put((rank, float((maps - full_maps).abs().max()), float((grad - full_grad).abs().max())))
    finally:
        dist.destroy_process_group()


def test_sharded_transposes_sum_over_two_gloo_ranks():
    """The transposes of a sharded scan: each rank's partial sky maps and beam-grid gradient
    (with its share of the Omega~ term), summed by one all-reduce, equal the whole stream's."""
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_transpose_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    results = [out.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, dm, dg in results:
        assert dm < 1e-12 and dg < 1e-12, (rank, dm, dg)
