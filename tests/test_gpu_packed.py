"""FP32 path with packed 32-byte beam cells (PISCO_FETCH_PACKED) against the FP64 oracle.

Tolerance from the format: per cell and map the value at the first node is
FP32 and the three bilinear slopes are int16 on a power-of-two scale, each
within 2^-15 of the largest slope of its cell and map, so an interpolated
beam value is off by at most 1.5 * 2^-15 of that slope (~5e-5 of it) on top
of the FP32 path's rounding.  Slopes are a fraction (grid spacing / beam
scale) of the values, and the errors of different cells are independent, so
per sample the tests allow 2e-5 of sum_k |w_k . S_k| and normwise the FP32
path's 1e-6 of ||d||_inf on CMB-like inputs.
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
PACKED = pisco.PISCO_FETCH_PACKED


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _oracle(nside, radius, sky, grids, det, theta, phi, psi, omega=None):
    g64 = np.asarray(grids, np.float64)
    omega = ob.omega_tilde(g64[0], radius) if omega is None else omega
    d = oc.tod(nside, radius, sky, g64, det, omega, theta, phi, psi)
    mag = np.zeros(len(theta))
    for t in range(len(theta)):
        if np.isfinite(d[t]):
            pix, w = oc.sample_weights(nside, radius, g64, det, omega, theta[t], phi[t], psi[t])
            mag[t] = np.sum(np.abs(w * sky[:, pix].T))
    return d, mag


def _plan(nside, r, sky, grids, det, **kw):
    g = torch.as_tensor(np.asarray(grids, np.float32), device=DEV)[None].contiguous()
    return pisco.Plan(nside, r, sky if torch.is_tensor(sky) else _t(sky), [det], g, beam_fetch=PACKED, **kw)


@pytest.mark.parametrize("nside,radius_deg,n_grid", [(16, 20.0, 41), (32, 8.0, 61), (64, 4.0, 30)])
def test_packed_forward_random_beams(nside, radius_deg, n_grid):
    r = math.radians(radius_deg)
    sky = sy.white_sky(nside, 5).numpy()
    grids = sy.random_beam_maps(n_grid, nside + n_grid)
    det = (0.7, 0.08, 1.3)
    th, ph, ps = sy.random_pointings(70, 3 * nside)
    ref, mag = _oracle(nside, r, sky, grids, det, th, ph, ps)
    with _plan(nside, r, sky, grids, det) as plan:
        out = plan.convolve(_t(th), _t(ph), _t(ps)).double().cpu().numpy()
        plan.sync_status()
    np.testing.assert_array_less(np.abs(out - ref), 2e-5 * mag + 1e-300)


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_packed_scan_tiles_normwise(tile):
    nside, r = 128, math.radians(5.0)
    sky = sy.gaussian_sky(nside, 1).numpy()
    grids = sy.gaussian_beam_maps(101, r, 1.5, ellipticity=0.05, xpol=0.01)
    grids[2] = 0.02 * grids[0]
    det = (0.3, 0.01, 1.0)
    th, ph, ps = sy.raster_scan(600, rows=6)
    ref, mag = _oracle(nside, r, sky, grids, det, th, ph, ps)
    with _plan(nside, r, sky, grids, det, tile_samples=tile) as plan:
        out = plan.convolve(_t(th), _t(ph), _t(ps)).double().cpu().numpy()
    np.testing.assert_array_less(np.abs(out - ref), 2e-5 * mag)
    assert np.max(np.abs(out - ref)) <= 1e-6 * np.max(np.abs(ref))


def test_packed_single_detector_workload_sampled():
    """The benchmark workload (nside 512, 501^2 grid over 10 deg, sidelobe ring, cross-polar
    leakage, azimuth scan), 2e5 samples, every 1000th against the oracle."""
    nside, r = 512, math.radians(10.0)
    sky = sy.gaussian_sky(nside, 1, device=DEV)
    grids = sy.gaussian_beam_maps(501, r, 1.5, ellipticity=0.0, xpol=0.005, sidelobe=(0.01, 7.0, 0.5))
    det = (0.0, 0.0, 1.0)
    th, ph, ps = sy.ces_scan(200000, device=DEV)
    with _plan(nside, r, sky, grids, det) as plan:
        out = plan.convolve(th, ph, ps).double().cpu().numpy()
        plan_omega = plan.omega(0)[0]
    omega = ob.omega_tilde(grids[0].astype(np.float64), r)
    assert abs(plan_omega / omega - 1.0) < 1e-12
    idx = np.arange(0, 200000, 1000)
    ref, mag = _oracle(nside, r, sky.cpu().numpy(), grids, det, th.cpu().numpy()[idx], ph.cpu().numpy()[idx],
                       ps.cpu().numpy()[idx], omega)
    np.testing.assert_array_less(np.abs(out[idx] - ref), 2e-5 * mag)
    assert np.max(np.abs(out[idx] - ref)) <= 1e-6 * np.max(np.abs(ref))


def test_packed_adjoint_and_psb_match_oracle():
    nside, r = 32, math.radians(8.0)
    sky = sy.gaussian_sky(nside, 9).numpy()
    grids = sy.random_beam_maps(61, 12)
    det = (0.25, 0.03, 1.0)
    th, ph, ps = sy.raster_scan(200, center=(1.2, 2.0), half_size=math.radians(3.0), rows=4)
    y = np.random.default_rng(3).standard_normal(len(th))
    omega = ob.omega_tilde(grids[0].astype(np.float64), r)
    ref_adj = oc.adjoint(nside, r, grids.astype(np.float64), det, omega, th, ph, ps, y)
    with _plan(nside, r, sky, grids, det) as plan:
        adj = plan.adjoint(_t(th), _t(ph), _t(ps), _t(y).float()).double().cpu().numpy()
        pair = plan.convolve_psb(_t(th), _t(ph), _t(ps), [0.25, 0.25 - 0.5 * math.pi]).double().cpu().numpy()
    np.testing.assert_allclose(adj, ref_adj, rtol=0, atol=2e-5 * np.max(np.abs(ref_adj)))
    for k, z in enumerate([0.25, 0.25 - 0.5 * math.pi]):
        ref, mag = _oracle(nside, r, sky, grids, (z, det[1], det[2]), th, ph, ps)
        np.testing.assert_array_less(np.abs(pair[k] - ref), 2e-5 * mag)


def test_packed_update_beams_and_range_check():
    nside, r = 16, math.radians(10.0)
    sky = _t(sy.white_sky(nside, 2).numpy())
    g1 = torch.as_tensor(sy.random_beam_maps(31, 1), device=DEV)[None]
    g2 = torch.as_tensor(sy.random_beam_maps(31, 2), device=DEV)[None]
    th, ph, ps = (_t(a) for a in sy.raster_scan(64, center=(1.0, 1.0), half_size=0.05, rows=4))
    with pisco.Plan(nside, r, sky, [(0.1, 0.0, 1.0)], g1, beam_fetch=PACKED) as a, \
            pisco.Plan(nside, r, sky, [(0.1, 0.0, 1.0)], g2, beam_fetch=PACKED) as b:
        a.update_beams(g2)
        torch.testing.assert_close(a.convolve(th, ph, ps), b.convolve(th, ph, ps), rtol=0, atol=0)
    with pytest.raises(pisco.PiscoError) as e:
        pisco.Plan(nside, r, sky, [(0.1, 0.0, 1.0)], g1 * 1e-28, omega_tilde=[1.0], beam_fetch=PACKED)
    assert e.value.status == pisco.PISCO_EINVAL
