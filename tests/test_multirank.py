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


class _OracleTransposes:
    """The transposes of the FP64 oracle for one sky, beam and detector, behind the calls
    paper_1908_05662_gb300.distributed makes on a plan (torch tensors in and out, CPU)."""

    def __init__(self, nside, radius, sky, grids, det):
        from oracle import beam as ob
        self.nside, self.radius, self.sky, self.grids, self.det = nside, radius, sky, grids, det
        self.omega = ob.omega_tilde(grids[0], radius)

    def adjoint(self, theta, phi, psi, tod, det=0):
        import torch
        from oracle import convolve as oc
        return torch.as_tensor(oc.adjoint(self.nside, self.radius, self.grids, self.det, self.omega, theta.numpy(),
                                          phi.numpy(), psi.numpy(), tod.numpy()))

    def beam_grid_adjoint(self, theta, phi, psi, y, det=0):
        import torch
        from oracle import convolve as oc
        return torch.as_tensor(oc.beam_grid_adjoint(self.nside, self.radius, self.sky, self.grids, self.det,
                                                    self.omega, theta.numpy(), phi.numpy(), psi.numpy(), y.numpy()))

    def adjoint_sky_beam(self, theta, phi, psi, tod, det=0):
        return self.adjoint(theta, phi, psi, tod), self.beam_grid_adjoint(theta, phi, psi, tod)

    def omega_adjoint(self, tod, y, grad, det=0):
        # Omega~ is linear in B_TT: its gradient is Omega~ of the unit map of each node
        import numpy as np
        import torch
        from oracle import beam as ob
        n = self.grids.shape[-1]
        dom = np.zeros((n, n))
        for j in range(n):
            for i in range(n):
                e = np.zeros((n, n))
                e[j, i] = 1.0
                dom[j, i] = ob.omega_tilde(e, self.radius)
        grad[0] -= float((tod * y).sum()) / self.omega * torch.as_tensor(dom)
        return grad


def _oracle_transpose_worker(rank, world, port, out):
    import math
    import numpy as np
    import torch
    from oracle import convolve as oc
    from paper_1908_05662_gb300 import distributed as pd
    from paper_1908_05662_gb300 import synthetic as sy
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nside, r = 8, math.radians(20.0)
        sky = sy.white_sky(nside, 3).numpy()
        grids = sy.random_beam_maps(11, 4).astype(np.float64)
        det = (0.3, 0.05, 1.1)
        th, ph, ps = sy.raster_scan(24, center=(1.2, 2.0), half_size=math.radians(8.0), rows=3)
        y = np.random.default_rng(5).standard_normal(24)
        plan = _OracleTransposes(nside, r, sky, grids, det)
        d = oc.tod(nside, r, sky, grids, det, plan.omega, th, ph, ps)
        T = [torch.as_tensor(np.ascontiguousarray(a)) for a in (th, ph, ps, y, d)]
        a, b = pd.shard_range(24, rank, world)
        maps, grad = pd.sharded_adjoint_sky_beam(plan, *(t[a:b] for t in T[:3]), T[3][a:b])
        grad_om = pd.sharded_beam_grid_adjoint(plan, *(t[a:b] for t in T[:3]), T[3][a:b], tod=T[4][a:b])
        full_maps = plan.adjoint(*T[:4])
        full_grad = plan.beam_grid_adjoint(*T[:4])
        full_om = plan.omega_adjoint(T[4], T[3], full_grad.clone())
        scale = float(full_maps.abs().max()), float(full_grad.abs().max())
        out.put((rank, float((maps - full_maps).abs().max()) / scale[0], float((grad - full_grad).abs().max()) / scale[1],
                 float((grad_om - full_om).abs().max()) / scale[1], b - a))
    finally:
        dist.destroy_process_group()


def test_oracle_transposes_of_two_gloo_shards_sum_to_the_whole_stream():
    """Each rank runs the oracle's sky and beam-grid transposes on its own contiguous shard of
    the scan (with its share of the Omega~ term); one all-reduce per result through the
    library's sharded helpers gives the transposes of the whole stream to rounding."""
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_oracle_transpose_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    results = [out.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(r[4] for r in results) == [12, 12]
    for rank, dm, dg, do, _ in results:
        assert dm < 1e-12 and dg < 1e-12 and do < 1e-12, (rank, dm, dg, do)
