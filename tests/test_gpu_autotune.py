"""The tile-shape autotuner (pisco_plan_autotune) through the C ABI.

It must pick one of the shapes the kernel is built for, leave the plan using
that shape (the FP32 forward pass is deterministic, so a fresh plan created
with the chosen shape gives bit-identical TOD), keep results within the FP32
path's bound of the oracle, and refuse plans it cannot tune.
"""

import math

import numpy as np
import pytest
import torch

from oracle import beam as ob
from oracle import convolve as oc
from paper_1908_05662_gb300 import pisco
from paper_1908_05662_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def test_autotune_picks_a_built_shape_and_the_plan_uses_it():
    nside, r = 64, math.radians(6.0)
    sky = sy.gaussian_sky(nside, 4).numpy()
    grids = sy.gaussian_beam_maps(121, r, 2.0, ellipticity=0.05, xpol=0.01)
    det = (0.2, 0.01, 1.0)
    th, ph, ps = (a.numpy() for a in sy.ces_scan(30000))
    g = torch.as_tensor(grids, device=DEV)[None]
    with pisco.Plan(nside, r, _t(sky), [det], g) as plan:
        tile, npx, ms = plan.autotune(_t(th), _t(ph), _t(ps), reps=2)
        assert tile in (8, 16, 32) and npx in (1, 2) and ms > 0
        tuned = plan.convolve(_t(th), _t(ph), _t(ps))
        plan.sync_status()
    with pisco.Plan(nside, r, _t(sky), [det], g, tile_samples=tile, pixels_per_thread=npx) as fresh:
        ref_shape = fresh.convolve(_t(th), _t(ph), _t(ps))
    torch.testing.assert_close(tuned, ref_shape, rtol=0, atol=0)
    idx = np.arange(0, 30000, 1500)
    g64 = grids.astype(np.float64)
    omega = ob.omega_tilde(g64[0], r)
    ref = oc.tod(nside, r, sky, g64, det, omega, th[idx], ph[idx], ps[idx])
    out = tuned.double().cpu().numpy()[idx]
    assert np.max(np.abs(out - ref)) <= 1e-6 * np.max(np.abs(ref))


def test_autotune_refuses_plain_plans_and_bad_arguments():
    nside, r = 16, math.radians(10.0)
    sky = _t(sy.white_sky(nside, 1).numpy())
    g = torch.as_tensor(sy.random_beam_maps(31, 2), device=DEV)[None]
    th, ph, ps = (_t(a) for a in sy.raster_scan(64, center=(1.0, 1.0), half_size=0.05, rows=2))
    with pisco.Plan(nside, r, sky, [(0.0, 0.0, 1.0)], g, precision=pisco.PISCO_FP64_PLAIN) as plan:
        with pytest.raises(pisco.PiscoError) as e:
            plan.autotune(th, ph, ps)
        assert e.value.status == pisco.PISCO_EUNSUPPORTED
    with pisco.Plan(nside, r, sky, [(0.0, 0.0, 1.0)], g, tile_samples=32) as plan:
        with pytest.raises(pisco.PiscoError) as e:
            plan.autotune(th, ph, ps, reps=0)
        assert e.value.status == pisco.PISCO_EINVAL
        with pytest.raises(pisco.PiscoError):
            plan.autotune(th, ph, ps, det=3)


def test_batched_autotune_tunes_every_detector_and_the_plan_uses_the_shape():
    """A focal plane tuned on slices of all detectors' scans: the shape is one the kernel is built
    for, the batched launch afterwards equals a fresh plan created with that shape (bit for bit),
    and the detectors' TODs stay within the FP32 bound of the oracle."""
    nside, r, n_det = 32, math.radians(8.0), 3
    sky = sy.gaussian_sky(nside, 6).numpy()
    grids = np.stack([sy.random_beam_maps(41, 60 + d) for d in range(n_det)])
    dets = [(0.1 * d, 0.01 * d, 1.0) for d in range(n_det)]
    lengths = [700, 1100, 400]
    parts = [sy.ces_scan(m, offset=(0.03 * d, -0.02 * d)) for d, m in enumerate(lengths)]
    th, ph, ps = (torch.cat([p[k] for p in parts]).numpy() for k in range(3))
    offsets = [0] + list(np.cumsum(lengths))
    sl = [np.arange(offsets[d], offsets[d] + 200) for d in range(n_det)]
    sl_off = [0, 200, 400, 600]
    ts, ps_, ss = (_t(np.concatenate([a[i] for i in sl])) for a in (th, ph, ps))
    g = torch.as_tensor(grids, device=DEV).contiguous()
    with pisco.Plan(nside, r, _t(sky), dets, g) as plan:
        tile, npx, ms = plan.autotune_batched(sl_off, ts, ps_, ss, reps=2)
        assert tile in (8, 16, 32) and npx in (1, 2) and ms > 0
        tuned = plan.convolve_batched(offsets, _t(th), _t(ph), _t(ps))
        plan.sync_status()
        with pytest.raises(pisco.PiscoError) as e:
            plan.autotune_batched([0, 5, 3], ts, ps_, ss)
        assert e.value.status == pisco.PISCO_EINVAL
    with pisco.Plan(nside, r, _t(sky), dets, g, tile_samples=tile, pixels_per_thread=npx) as fresh:
        ref_shape = fresh.convolve_batched(offsets, _t(th), _t(ph), _t(ps))
    torch.testing.assert_close(tuned, ref_shape, rtol=0, atol=0)
    out = tuned.double().cpu().numpy()
    for d in range(n_det):
        idx = offsets[d] + np.array([0, lengths[d] // 2, lengths[d] - 1])
        g64 = grids[d].astype(np.float64)
        omega = ob.omega_tilde(g64[0], r)
        ref = oc.tod(nside, r, sky, g64, dets[d], omega, th[idx], ph[idx], ps[idx])
        for k, t in enumerate(idx):
            pix, w = oc.sample_weights(nside, r, g64, dets[d], omega, th[t], ph[t], ps[t])
            assert abs(out[t] - ref[k]) <= 2e-6 * np.sum(np.abs(w * sky[:, pix].T))
