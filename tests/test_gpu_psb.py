"""Shared-geometry pass for detectors that differ only in polarisation angle
(PSB pairs, Sec. 3 eq. copol_bolo), through pisco_convolve_psb.

Each output row is compared with the FP64 oracle for a detector whose zeta is
that row's angle, element by element: the pass runs the FP32 kernel with the
intensity and the complex polarised sums accumulated separately, so the
per-sample bound is the FP32 path's 2e-6 of sum_k |w_k . S_k|.  Against
separate pisco_convolve calls it agrees to FP32 rounding (1e-6 of ||d||_inf).
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


def _oracle(nside, radius, sky, grids, det, theta, phi, psi):
    g64 = np.asarray(grids, np.float64)
    omega = ob.omega_tilde(g64[0], radius)
    d = oc.tod(nside, radius, sky, g64, det, omega, theta, phi, psi)
    mag = np.zeros(len(theta))
    for t in range(len(theta)):
        if np.isfinite(d[t]):
            pix, w = oc.sample_weights(nside, radius, g64, det, omega, theta[t], phi[t], psi[t])
            mag[t] = np.sum(np.abs(w * sky[:, pix].T))
    return d, mag


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_psb_pair_and_extra_angles_match_oracle(tile):
    nside, r = 32, math.radians(8.0)
    sky = sy.gaussian_sky(nside, 21).numpy()
    grids = sy.random_beam_maps(61, 22)
    eps, s = 0.04, 1.1
    zeta0 = 0.35
    zetas = [zeta0, zeta0 - 0.5 * math.pi, zeta0 + 0.25 * math.pi, -1.2]
    th, ph, ps = sy.raster_scan(230, center=(1.3, 2.2), half_size=math.radians(4.0), rows=5)
    g = torch.as_tensor(grids, device=DEV)[None]
    with pisco.Plan(nside, r, _t(sky), [(zeta0, eps, s)], g, tile_samples=tile) as plan:
        out = plan.convolve_psb(_t(th), _t(ph), _t(ps), zetas).double().cpu().numpy()
        plan.sync_status()
    assert out.shape == (len(zetas), len(th))
    for k, z in enumerate(zetas):
        ref, mag = _oracle(nside, r, sky, grids, (z, eps, s), th, ph, ps)
        np.testing.assert_array_less(np.abs(out[k] - ref), 2e-6 * mag + 1e-30)


def test_psb_agrees_with_separate_convolutions_and_pair_sum_is_intensity():
    nside, r = 64, math.radians(5.0)
    sky = sy.gaussian_sky(nside, 5).numpy()
    grids = sy.gaussian_beam_maps(101, r, 1.5, ellipticity=0.05, xpol=0.01)
    th, ph, ps = (_t(a) for a in sy.ces_scan(3000))
    zeta = 0.7
    g = torch.as_tensor(grids, device=DEV)[None]
    with pisco.Plan(nside, r, _t(sky), [(zeta, 0.0, 1.0)], g) as plan:
        pair = plan.convolve_psb(th, ph, ps, [zeta, zeta - 0.5 * math.pi]).double()
        a = plan.convolve(th, ph, ps).double()
    with pisco.Plan(nside, r, _t(sky), [(zeta - 0.5 * math.pi, 0.0, 1.0)], g) as plan:
        b = plan.convolve(th, ph, ps).double()
    scale = torch.max(torch.abs(a)).item()
    assert torch.max(torch.abs(pair[0] - a)).item() <= 1e-6 * scale
    assert torch.max(torch.abs(pair[1] - b)).item() <= 1e-6 * scale
    # the pair's sum sees the intensity only: cos 2(zeta - 90 deg) = -cos 2 zeta
    sky_i = sky.copy()
    sky_i[1:] = 0.0
    with pisco.Plan(nside, r, _t(sky_i), [(zeta, 0.0, 1.0)], g) as plan:
        i_only = plan.convolve(th, ph, ps).double()
    assert torch.max(torch.abs(pair[0] + pair[1] - 2.0 * i_only)).item() <= 2e-6 * scale


def test_psb_invalid_pointings_empty_and_errors():
    nside, r = 16, math.radians(10.0)
    sky = _t(sy.white_sky(nside, 2).numpy())
    g = torch.as_tensor(sy.random_beam_maps(31, 4), device=DEV)[None]
    th, ph, ps = sy.raster_scan(40, center=(1.0, 1.0), half_size=0.05, rows=2)
    th = th.copy()
    th[7] = np.nan
    with pisco.Plan(nside, r, sky, [(0.1, 0.0, 1.0)], g) as plan:
        out = plan.convolve_psb(_t(th), _t(ph), _t(ps), [0.0, 1.0, 2.0]).cpu().numpy()
        assert np.all(np.isnan(out[:, 7])) and np.all(np.isfinite(np.delete(out, 7, axis=1)))
        empty = torch.empty(0, dtype=torch.float64, device=DEV)
        assert plan.convolve_psb(empty, empty, empty, [0.0]).shape == (1, 0)
        for bad in ([], [0.0] * 9, [float("nan")]):
            with pytest.raises(pisco.PiscoError) as e:
                plan.convolve_psb(_t(th), _t(ph), _t(ps), bad, out=torch.empty(max(len(bad), 1), 40, device=DEV))
            assert e.value.status == pisco.PISCO_EINVAL
    for kw in ({"precision": pisco.PISCO_FP64_PLAIN}, {"beam_fetch": pisco.PISCO_FETCH_TEXTURE}):
        with pisco.Plan(nside, r, sky, [(0.1, 0.0, 1.0)], g, **kw) as plan:
            with pytest.raises(pisco.PiscoError) as e:
                plan.convolve_psb(_t(th), _t(ph), _t(ps), [0.0, 1.0])
            assert e.value.status == pisco.PISCO_EUNSUPPORTED
