"""Sample sharding of the transposes on one GPU: the shards of a scan, run one after the other
(as ranks would run them on their own GPUs) and summed, give the transposes of the whole scan.

The sums are FP32 atomic adds in another order.  The sky maps agree to 1e-6 of the largest
entry; a beam-grid node sums contributions of both signs from many samples (the TOD weights y
are random), so its rounding is relative to the sum of their magnitudes, not to the result:
the gradients are allowed 3e-5 of the largest entry.  Across GPUs the sum is the one all-reduce of `paper_1908_05662_gb300.distributed`,
whose reduction logic the gloo tests cover on CPU.
"""

import math

import numpy as np
import pytest
import torch

from paper_1908_05662_gb300 import distributed as pd
from paper_1908_05662_gb300 import pisco
from paper_1908_05662_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def test_sharded_transposes_sum_to_the_whole_scan():
    nside, r = 64, math.radians(6.0)
    sky = sy.gaussian_sky(nside, 2, device=DEV)
    g = torch.as_tensor(sy.gaussian_beam_maps(121, r, 2.0, ellipticity=0.05, xpol=0.01), device=DEV)[None]
    th, ph, ps = (a.contiguous() for a in sy.ces_scan(50000, device=DEV))
    y = torch.randn(len(th), device=DEV, generator=torch.Generator(device=DEV).manual_seed(3))
    world = 3
    with pisco.Plan(nside, r, sky, [(0.3, 0.01, 1.0)], g) as plan:
        d = plan.convolve(th, ph, ps)
        full_maps = plan.adjoint(th, ph, ps, y)
        full_grad = plan.beam_grid_adjoint(th, ph, ps, y)
        plan.omega_adjoint(d, y, full_grad)
        full_m2, full_g2 = plan.adjoint_sky_beam(th, ph, ps, y)
        maps = torch.zeros_like(full_maps)
        grad = torch.zeros_like(full_grad)
        m2 = torch.zeros_like(full_m2)
        g2 = torch.zeros_like(full_g2)
        for rank in range(world):
            a, b = pd.shard_range(len(th), rank, world)
            sl = slice(a, b)
            maps += pd.sharded_adjoint(plan, th[sl], ph[sl], ps[sl], y[sl])
            grad += pd.sharded_beam_grid_adjoint(plan, th[sl], ph[sl], ps[sl], y[sl], tod=d[sl])
            pm, pg = pd.sharded_adjoint_sky_beam(plan, th[sl], ph[sl], ps[sl], y[sl])
            m2 += pm
            g2 += pg
        plan.sync_status()
    for got, want, tol in ((maps, full_maps, 1e-6), (grad, full_grad, 3e-5), (m2, full_m2, 1e-6),
                           (g2, full_g2, 3e-5)):
        scale = want.abs().max().item()
        assert (got - want).abs().max().item() <= tol * scale
