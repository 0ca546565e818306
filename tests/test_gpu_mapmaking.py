"""Map-making on the GPU (pisco_ang2pix, pisco_map_accumulate, pisco_map_solve) against the oracle.

Pixel indices are integer work: bit-exact.  The normal equations are FP64
sums accumulated with atomics (order varies), so the maps agree with the
oracle to rounding amplified by the pixel's condition number: 1e-9 relative
to the map's scale for rcond >= 1e-3.  Which pixels are solved is decided in
FP64 on both sides from the same counts; pixels whose reciprocal condition
number lies within 10 % of the threshold are left out of that comparison.
"""

import math

import numpy as np
import pytest
import torch

from oracle import beam as ob
from oracle import convolve as oc
from oracle import healpix as hp
from oracle import mapmaking as mm
from paper_1908_05662_gb300 import pisco
from paper_1908_05662_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


@pytest.mark.parametrize("nside", [1, 8, 512, 8192])
def test_ang2pix_bit_exact(nside):
    rng = np.random.default_rng(nside)
    th = np.arccos(rng.uniform(-1, 1, 20000))
    ph = rng.uniform(-10.0, 10.0, 20000)
    ct, cp = hp.pix2ang(nside, rng.integers(0, hp.npix(nside), 2000))
    th = np.concatenate([th, ct, [0.0, math.pi, math.acos(2 / 3), math.acos(-2 / 3), 1.0, np.nan, -0.1]])
    ph = np.concatenate([ph, cp, [0.0, 0.0, 1.0, 2.0, -1e-300, 0.0, 0.0]])
    got = pisco.pisco_ang2pix(nside, _t(th), _t(ph)).cpu().numpy()
    ok = np.isfinite(th) & (th >= 0) & (th <= math.pi)
    np.testing.assert_array_equal(got[ok], mm.ang2pix(nside, th[ok], ph[ok]))
    assert np.all(got[~ok] == -1)


def _compare(nside, maps, acc, ref_maps, ata, hits, rcond_min):
    acc = acc.cpu().numpy()
    np.testing.assert_array_equal(acc[9].round().astype(np.int64), hits)
    lam = np.linalg.eigvalsh(ata)
    with np.errstate(divide="ignore", invalid="ignore"):
        rc = np.where(lam[:, -1] > 0, lam[:, 0] / lam[:, -1], 0.0)
    clear = (hits < 3) | (np.abs(rc - rcond_min) > 0.1 * rcond_min)
    maps = maps.cpu().numpy()
    np.testing.assert_array_equal(np.isnan(maps[0])[clear], np.isnan(ref_maps[0])[clear])
    solved = clear & np.isfinite(ref_maps[0])
    scale = np.max(np.abs(ref_maps[:, solved]))
    np.testing.assert_allclose(maps[:, solved], ref_maps[:, solved], rtol=0, atol=1e-9 * scale)
    return solved


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_binned_map_of_a_scan_matches_oracle(dtype):
    """A patch hit at random angles (about 170 hits per pixel) plus a stretch of the azimuth
    scan (few angles per pixel: mostly unsolved pixels)."""
    nside = 64
    rng = np.random.default_rng(5)
    n = 60000
    th = np.arccos(rng.uniform(math.cos(1.2), math.cos(1.0), n))
    ph = rng.uniform(0.0, 0.5, n)
    ps = rng.uniform(0.0, math.pi, n)
    st, sp, ss = (a.numpy() for a in sy.ces_scan(20000))
    th, ph, ps = np.r_[th, st], np.r_[ph, sp], np.r_[ps, ss]
    det = (0.3, 0.02, 1.1)
    d = rng.standard_normal(len(th))
    d_dev = _t(d, dtype)
    d_ref = d_dev.double().cpu().numpy()  # the same rounded values on both sides
    acc = pisco.pisco_map_accumulate(nside, _t(th), _t(ph), _t(ps), det, d_dev)
    maps = pisco.pisco_map_solve(nside, acc, 1e-3)
    ata, atd, hits = mm.normal_equations(nside, th, ph, ps, det, d_ref)
    ref = mm.solve(ata, atd, hits, 1e-3)
    solved = _compare(nside, maps, acc, ref, ata, hits, 1e-3)
    assert solved.sum() > 100


def test_focal_plane_accumulation_and_invalid_samples():
    nside = 16
    rng = np.random.default_rng(6)
    dets = [(0.0, 0.0, 1.0), (0.5 * math.pi, 0.01, 0.9), (0.25 * math.pi, 0.0, 1.0)]
    acc = None
    ata = np.zeros((hp.npix(nside), 3, 3))
    atd = np.zeros((hp.npix(nside), 3))
    hits = np.zeros(hp.npix(nside), np.int64)
    for k, det in enumerate(dets):
        n = 5000
        th = np.arccos(rng.uniform(-1, 1, n))
        ph = rng.uniform(0, 2 * math.pi, n)
        ps = rng.uniform(0, math.pi, n)
        d = rng.standard_normal(n)
        th[:3] = [np.nan, -0.5, 4.0]
        d[5] = np.inf
        acc = pisco.pisco_map_accumulate(nside, _t(th), _t(ph), _t(ps), det, _t(d), acc=acc, accumulate=k > 0)
        a, b, h = mm.normal_equations(nside, th, ph, ps, det, d)
        ata, atd, hits = ata + a, atd + b, hits + h
    maps = pisco.pisco_map_solve(nside, acc, 1e-4)
    _compare(nside, maps, acc, mm.solve(ata, atd, hits, 1e-4), ata, hits, 1e-4)


def test_convolve_then_map_pixel_centres_at_three_angles():
    """Sec. 6.1's observation pattern: every pixel centre at psi = 0, 45, 90 deg, one detector
    (zeta 0, s 1, eps 0), TOD from the FP32 path binned on the GPU, against the oracle's TOD
    binned by the oracle.  Three hits per pixel determine I, Q, U exactly, so the maps carry the
    FP32 TOD error amplified by the 3 x 3 solve: 1e-5 of the map scale."""
    nside, r = 8, math.radians(12.0)
    sky = sy.gaussian_sky(nside, 41).numpy()
    grids = sy.gaussian_beam_maps(61, r, 5.0, ideal=True)
    th_c, ph_c = hp.pix2ang(nside, np.arange(hp.npix(nside)))
    a = np.radians([0.0, 45.0, 90.0])
    th, ph, ps = np.repeat(th_c, 3), np.repeat(ph_c, 3), np.tile(a, len(th_c))
    det = (0.0, 0.0, 1.0)
    with pisco.Plan(nside, r, _t(sky), [det], torch.as_tensor(grids, device=DEV)[None]) as plan:
        tod = plan.convolve(_t(th), _t(ph), _t(ps))
    maps, hits = pisco.binned_map(nside, _t(th), _t(ph), _t(ps), det, tod)
    assert torch.all(hits == 3)
    g64 = grids.astype(np.float64)
    d_ref = oc.tod(nside, r, sky, g64, det, ob.omega_tilde(g64[0], r), th, ph, ps)
    ref, ref_hits = mm.binned_map(nside, th, ph, ps, det, d_ref)
    np.testing.assert_allclose(maps.cpu().numpy(), ref, rtol=0, atol=1e-5 * np.max(np.abs(ref)))


def test_map_calls_reject_bad_arguments():
    th = _t(np.array([1.0]))
    with pytest.raises(pisco.PiscoError):
        pisco.pisco_ang2pix(0, th, th)
    with pytest.raises(pisco.PiscoError):
        pisco.pisco_map_accumulate(8, th, th, th, (float("nan"), 0.0, 1.0), _t(np.array([1.0])))
    acc = torch.zeros(10, 12 * 64, dtype=torch.float64, device=DEV)
    with pytest.raises(pisco.PiscoError):
        pisco.pisco_map_solve(8, acc, 2.0)
    with pytest.raises(pisco.PiscoError):
        pisco.pisco_map_solve(8, acc.cpu(), 1e-6)
