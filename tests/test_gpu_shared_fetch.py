"""FP32 path with the folded node grid staged in shared memory (PISCO_FETCH_SHARED).

Same arithmetic as the 64-byte cells up to FP32 rounding (bilinear from the
four nodes instead of the cell's coefficients), so the FP32 path's bounds hold:
2e-6 of sum_k |w_k . S_k| per sample and 1e-6 of ||d||_inf normwise on
CMB-like inputs.  Also checked: a batched focal plane whose blocks change
detector (the node grid is restaged), the transposes and the shared-geometry
pass on this fetch, and the size limit.
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
SHARED = pisco.PISCO_FETCH_SHARED


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _oracle(nside, radius, sky, grids, det, theta, phi, psi):
    g64 = np.asarray(grids, np.float64)
    omega = ob.omega_tilde(g64[0], radius)
    d = oc.tod(nside, radius, sky, g64, det, omega, theta, phi, psi)
    mag = np.array([np.sum(np.abs(w * sky[:, pix].T)) for pix, w in
                    (oc.sample_weights(nside, radius, g64, det, omega, a, b, c) for a, b, c in zip(theta, phi, psi))])
    return d, mag


@pytest.mark.parametrize("nside,radius_deg,n_grid,tile", [(32, 8.0, 61, 16), (64, 4.0, 30, 8), (16, 20.0, 108, 32)])
def test_shared_fetch_forward_matches_oracle(nside, radius_deg, n_grid, tile):
    r = math.radians(radius_deg)
    sky = sy.white_sky(nside, 3).numpy()
    grids = sy.random_beam_maps(n_grid, 7 + nside)
    det = (0.5, 0.04, 1.1)
    th, ph, ps = sy.raster_scan(260, center=(1.1, 2.5), half_size=math.radians(5.0), rows=4)
    ref, mag = _oracle(nside, r, sky, grids, det, th, ph, ps)
    with pisco.Plan(nside, r, _t(sky), [det], torch.as_tensor(grids, device=DEV)[None], beam_fetch=SHARED,
                    tile_samples=tile) as plan:
        out = plan.convolve(_t(th), _t(ph), _t(ps)).double().cpu().numpy()
        counts = plan.disc_count(_t(th), _t(ph)).cpu().numpy()
        plan.sync_status()
    np.testing.assert_array_less(np.abs(out - ref), 2e-6 * mag)
    np.testing.assert_array_equal(counts, oc.disc_count(nside, r, th, ph))


def test_shared_fetch_c1_configuration_normwise_and_equal_to_cells():
    """The plain-FP64 baseline configuration's resolution (nside 128, 101^2 grid over 5 deg,
    elliptical 1.5 deg beam, CMB-like sky, raster scan)."""
    nside, r = 128, math.radians(5.0)
    sky = sy.gaussian_sky(nside, 1).numpy()
    grids = sy.gaussian_beam_maps(101, r, 1.5, ellipticity=0.05)
    det = (0.0, 0.0, 1.0)
    th, ph, ps = sy.raster_scan(2000, rows=20)
    idx = np.arange(0, 2000, 25)
    ref, _ = _oracle(nside, r, sky, grids, det, th[idx], ph[idx], ps[idx])
    g = torch.as_tensor(grids, device=DEV)[None]
    with pisco.Plan(nside, r, _t(sky), [det], g, beam_fetch=SHARED) as plan:
        out = plan.convolve(_t(th), _t(ph), _t(ps)).double().cpu().numpy()
    with pisco.Plan(nside, r, _t(sky), [det], g) as cells:
        ref_cells = cells.convolve(_t(th), _t(ph), _t(ps)).double().cpu().numpy()
    assert np.max(np.abs(out[idx] - ref)) <= 1e-6 * np.max(np.abs(ref))
    assert np.max(np.abs(out - ref_cells)) <= 1e-6 * np.max(np.abs(ref_cells))


def test_shared_fetch_batched_detectors_restage_the_grid():
    nside, r = 32, math.radians(8.0)
    sky = sy.gaussian_sky(nside, 9).numpy()
    n_det = 4
    grids = np.stack([sy.random_beam_maps(41, 80 + d) for d in range(n_det)])
    dets = [(0.3 * d, 0.02, 1.0) for d in range(n_det)]
    lengths = [150, 40, 300, 90]
    offsets = [0] + list(np.cumsum(lengths))
    parts = [sy.raster_scan(m, center=(0.8 + 0.2 * d, 1.0 + d), half_size=0.05, rows=3) for d, m in enumerate(lengths)]
    th, ph, ps = (np.concatenate([p[k] for p in parts]) for k in range(3))
    g = torch.as_tensor(grids, device=DEV).contiguous()
    with pisco.Plan(nside, r, _t(sky), dets, g, beam_fetch=SHARED) as plan:
        out = plan.convolve_batched(offsets, _t(th), _t(ph), _t(ps)).double().cpu().numpy()
        plan.sync_status()
    for d in range(n_det):
        a = offsets[d]
        idx = a + np.array([0, lengths[d] // 2, lengths[d] - 1])
        ref, mag = _oracle(nside, r, sky, grids[d], dets[d], th[idx], ph[idx], ps[idx])
        np.testing.assert_array_less(np.abs(out[idx] - ref), 2e-6 * mag)


def test_shared_fetch_transposes_and_psb_match_oracle():
    nside, r = 32, math.radians(8.0)
    sky = sy.gaussian_sky(nside, 5).numpy()
    grids = sy.random_beam_maps(61, 15)
    det = (0.25, 0.03, 1.0)
    th, ph, ps = sy.raster_scan(200, center=(1.2, 2.0), half_size=math.radians(3.0), rows=4)
    y = np.random.default_rng(3).standard_normal(len(th))
    g64 = grids.astype(np.float64)
    omega = ob.omega_tilde(g64[0], r)
    ref_adj = oc.adjoint(nside, r, g64, det, omega, th, ph, ps, y)
    with pisco.Plan(nside, r, _t(sky), [det], torch.as_tensor(grids, device=DEV)[None], beam_fetch=SHARED) as plan:
        adj = plan.adjoint(_t(th), _t(ph), _t(ps), _t(y).float()).double().cpu().numpy()
        pair = plan.convolve_psb(_t(th), _t(ph), _t(ps), [0.25, 0.25 - 0.5 * math.pi]).double().cpu().numpy()
        plan.sync_status()
    np.testing.assert_allclose(adj, ref_adj, rtol=0, atol=1e-5 * np.max(np.abs(ref_adj)))
    for k, z in enumerate([0.25, 0.25 - 0.5 * math.pi]):
        ref, mag = _oracle(nside, r, sky, grids, (z, det[1], det[2]), th, ph, ps)
        np.testing.assert_array_less(np.abs(pair[k] - ref), 2e-6 * mag)


def test_shared_fetch_rejects_grids_beyond_its_limit():
    nside, r = 8, math.radians(10.0)
    g = torch.zeros(1, 6, 109, 109, device=DEV)
    g[0, 0] = 1.0
    with pytest.raises(pisco.PiscoError) as e:
        pisco.Plan(nside, r, _t(np.zeros((3, 12 * nside * nside))), [(0, 0, 1)], g, beam_fetch=SHARED)
    assert e.value.status == pisco.PISCO_EINVAL
