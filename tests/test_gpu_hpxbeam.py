"""HEALPix beam input on the GPU (pisco_beam_grids_from_healpix) against the oracle.

The kernel evaluates the same ring-wise interpolation in FP64 and stores
float32, so node values agree with the oracle (fed the same float32 maps) to
the float32 rounding of the result: 2e-7 of max |map| allowed.  The TOD of a
plan built from resampled HEALPix beams is then compared with the oracle's TOD
on the oracle's own resampled grids, per sample, at the FP32 path's bound
(2e-6 of sum_k |w_k . S_k|).
"""

import math

import numpy as np
import pytest
import torch

from oracle import beam as ob
from oracle import convolve as oc
from oracle import healpix as hp
from paper_1908_05662_gb300 import beams
from paper_1908_05662_gb300 import pisco
from paper_1908_05662_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


@pytest.mark.parametrize("nside_b,radius_deg,n", [(1, 60.0, 9), (2, 30.0, 17), (8, 10.0, 33), (16, 50.0, 41),
                                                  (64, 5.0, 64)])
def test_resampling_matches_oracle(nside_b, radius_deg, n):
    r = math.radians(radius_deg)
    rng = np.random.default_rng(nside_b)
    maps = rng.standard_normal((6, hp.npix(nside_b))).astype(np.float32)
    maps[0] += 3.0
    got = pisco.pisco_beam_grids_from_healpix(torch.as_tensor(maps, device=DEV), nside_b, r, n)
    torch.cuda.synchronize()
    ref = ob.grid_from_healpix(maps.astype(np.float64), nside_b, r, n)
    np.testing.assert_allclose(got.double().cpu().numpy(), ref, rtol=0, atol=2e-7 * np.max(np.abs(maps)))


def test_resampling_of_the_paper_like_beam_and_batch_shape():
    """nside_b 512 (the beam resolution of Sec. 5.3), two detectors' maps in one call."""
    r, n = math.radians(4.0), 161
    m = torch.stack([beams.gaussian_beam_healpix(512, 1.5, 0.05),
                     beams.gaussian_beam_healpix(512, 1.2, 0.0, xpol=0.01)]).float()
    got = pisco.pisco_beam_grids_from_healpix(m.to(DEV), 512, r, n)
    assert got.shape == (2, 6, n, n)
    ref = ob.grid_from_healpix(m[1, [0, 4]].double().numpy(), 512, r, n)
    np.testing.assert_allclose(got[1, [0, 4]].double().cpu().numpy(), ref, rtol=0, atol=2e-7)
    analytic = beams.gaussian_beam_grids(n, r, 1.5, 0.05).numpy()[0]
    assert np.max(np.abs(got[0, 0].double().cpu().numpy() - analytic)) < 4e-3  # interpolation error at nside 512


def test_tod_from_healpix_beams_matches_oracle():
    nside, r = 32, math.radians(8.0)
    nside_b = 4 * nside
    sky = sy.gaussian_sky(nside, 31).numpy()
    maps = beams.gaussian_beam_healpix(nside_b, 3.0, 0.08, xpol=0.02).float()
    maps[2] = 0.01 * maps[0]  # a U_T leakage term so every folded map is non-zero
    n = 65
    grids = pisco.pisco_beam_grids_from_healpix(maps.to(DEV), nside_b, r, n)
    ref_grids = ob.grid_from_healpix(maps.double().numpy(), nside_b, r, n)
    det = (0.4, 0.03, 1.0)
    th, ph, ps = sy.raster_scan(150, center=(1.0, 2.5), half_size=math.radians(3.0), rows=5)
    with pisco.Plan(nside, r, _t(sky), [det], grids[None].contiguous()) as plan:
        d = plan.convolve(_t(th), _t(ph), _t(ps)).double().cpu().numpy()
        plan.sync_status()
    omega = ob.omega_tilde(ref_grids[0], r)
    ref = oc.tod(nside, r, sky, ref_grids, det, omega, th, ph, ps)
    mag = np.empty(len(th))
    for t in range(len(th)):
        pix, w = oc.sample_weights(nside, r, ref_grids, det, omega, th[t], ph[t], ps[t])
        mag[t] = np.sum(np.abs(w * sky[:, pix].T))
    np.testing.assert_array_less(np.abs(d - ref), 2e-6 * mag)


def test_resampling_rejects_host_pointers():
    maps = torch.zeros(6, hp.npix(4), dtype=torch.float32)
    with pytest.raises(ValueError):
        pisco.pisco_beam_grids_from_healpix(maps, 4, 0.1, 11)
    out = torch.empty(6, 11, 11)
    with pytest.raises(pisco.PiscoError) as e:
        pisco.pisco_beam_grids_from_healpix(maps.to(DEV), 4, 0.1, 11, grids=out)
    assert e.value.status == pisco.PISCO_EINVAL
