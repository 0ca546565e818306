"""GPU path versus the FP64 oracle, element by element, through the C ABI.

Tolerances (derived from the arithmetic, stated per test):
* disc membership and counts are index work: bit-exact;
* the plain FP64 path evaluates the same sum as the oracle in another order
  and by the vector route: 1e-11 relative to the per-sample magnitude
  sum_k |w_k . S_k|;
* the FP32 path: the in-frame offsets are formed from O(1e-1)-sized FP32
  terms (relative rounding ~1e-7 of the offset) and the sum is accumulated in
  FP32 per thread, so the error is a few 1e-7 of sum_k |w_k . S_k|; the tests
  allow 2e-6 of that magnitude per sample and 1e-6 of ||d||_inf normwise on
  CMB-like inputs (the target for the FP32 path).
"""

import math

import numpy as np
import pytest
import torch

from oracle import beam as ob
from oracle import convolve as oc
from oracle import healpix as hp
from paper_1908_05662_gb300 import pisco
from paper_1908_05662_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _oracle(nside, radius, sky, grids, det, theta, phi, psi, omega=None):
    g64 = np.asarray(grids, np.float64)
    omega = ob.omega_tilde(g64[0], radius) if omega is None else omega
    d = oc.tod(nside, radius, sky, g64, det, omega, theta, phi, psi)
    mag = np.empty(len(theta))
    for t in range(len(theta)):
        if not np.isfinite(d[t]):
            mag[t] = np.nan
            continue
        pix, w = oc.sample_weights(nside, radius, g64, det, omega, theta[t], phi[t], psi[t])
        mag[t] = np.sum(np.abs(w * sky[:, pix].T))
    return d, mag


def _gpu(nside, radius, sky, grids, dets, theta, phi, psi, precision, tile=0, det=0, np_=0):
    g = torch.as_tensor(np.asarray(grids, np.float32), device=DEV)
    if g.dim() == 3:
        g = g[None]
    with pisco.Plan(nside, radius, _t(sky), dets, g.contiguous(), precision=precision, tile_samples=tile,
                    pixels_per_thread=np_) as plan:
        out = plan.convolve(_t(theta), _t(phi), _t(psi), det=det)
        torch.cuda.synchronize()
        plan.sync_status()
        return out.double().cpu().numpy()


def _mixed_pointings(n, seed, nside):
    """Random pointings, including poles, the longitude wrap and exact pixel centres of the
    nside sky (rho = 0, as in Table 1 and Sec. 6)."""
    th, ph, ps = sy.random_pointings(n, seed)
    th[:4] = [0.0, math.pi, 1e-7, math.pi - 1e-7]
    ph[4:6] = [-1e-13, 2 * math.pi - 1e-13]
    tc, pc, _, _ = sy.pixel_centre_pointings(nside, 6, seed)
    th[6:12], ph[6:12] = tc, pc
    return th, ph, ps


# --------------------------------------------------------------------------- disc


@pytest.mark.parametrize("precision", [pisco.PISCO_FP32, pisco.PISCO_FP64_PLAIN])
@pytest.mark.parametrize("nside,radius_deg", [(8, 30.0), (32, 10.0), (64, 5.0)])
def test_disc_counts_bit_exact(precision, nside, radius_deg):
    r = math.radians(radius_deg)
    th, ph, ps = _mixed_pointings(150, nside, nside)
    # add a scan so the FP32 path traverses grouped discs as well
    st, sp, _ = sy.raster_scan(100, center=(1.2, 0.5), half_size=math.radians(2.0), rows=5)
    th, ph = np.concatenate([th, st]), np.concatenate([ph, sp])
    sky = np.zeros((3, hp.npix(nside)))
    grids = sy.random_beam_maps(11, 1)
    with pisco.Plan(nside, r, _t(sky), [(0, 0, 1)], torch.as_tensor(grids, device=DEV)[None],
                    precision=precision) as plan:
        c = plan.disc_count(_t(th), _t(ph)).cpu().numpy()
    np.testing.assert_array_equal(c, oc.disc_count(nside, r, th, ph))


# --------------------------------------------------------------------------- forward


@pytest.mark.parametrize("precision,rel", [(pisco.PISCO_FP64_PLAIN, 1e-11), (pisco.PISCO_FP32, 2e-6)])
@pytest.mark.parametrize("nside,radius_deg,n_grid", [(16, 20.0, 41), (32, 8.0, 61), (64, 4.0, 30)])
def test_forward_random_beams_random_pointings(precision, rel, nside, radius_deg, n_grid):
    r = math.radians(radius_deg)
    sky = sy.white_sky(nside, 5).numpy()
    grids = sy.random_beam_maps(n_grid, nside + n_grid)
    det = (0.7, 0.08, 1.3)
    th, ph, ps = _mixed_pointings(70, 3 * nside, nside)
    ref, mag = _oracle(nside, r, sky, grids, det, th, ph, ps)
    out = _gpu(nside, r, sky, grids, [det], th, ph, ps, precision)
    np.testing.assert_array_less(np.abs(out - ref), rel * mag + 1e-300)


@pytest.mark.parametrize("tile", [8, 16, 32])
@pytest.mark.parametrize("np_", [1, 2])
def test_fp32_scan_tiles_and_ragged_tail(tile, np_):
    """Consecutive scan samples share disc traversals; n is not a multiple of the tile."""
    nside, r = 64, math.radians(6.0)
    sky = sy.gaussian_sky(nside, 7).numpy()
    grids = sy.gaussian_beam_maps(121, r, 2.0, ellipticity=0.05, xpol=0.01)
    grids[3] = 0.05 * grids[0]
    grids[2] = 0.02 * grids[0]
    det = (0.4, 0.02, 1.0)
    th, ph, ps = sy.raster_scan(301, center=(0.9, 4.0), half_size=math.radians(4.0), rows=6)
    ref, mag = _oracle(nside, r, sky, grids, det, th, ph, ps)
    out = _gpu(nside, r, sky, grids, [det], th, ph, ps, pisco.PISCO_FP32, tile=tile, np_=np_)
    np.testing.assert_array_less(np.abs(out - ref), 2e-6 * mag)
    assert np.max(np.abs(out - ref)) <= 1e-6 * np.max(np.abs(ref))


def test_fp32_c1_like_workload_normwise():
    """nside 128, 101 x 101 grid over 5 deg, elliptical 1.5 deg beam, CMB-like sky, raster scan."""
    nside, r = 128, math.radians(5.0)
    sky = sy.gaussian_sky(nside, 1).numpy()
    grids = sy.gaussian_beam_maps(101, r, 1.5, ellipticity=0.05)
    det = (0.0, 0.0, 1.0)
    th, ph, ps = sy.raster_scan(1000, rows=10)
    ref, mag = _oracle(nside, r, sky, grids, det, th, ph, ps)
    for precision, tol in ((pisco.PISCO_FP32, 1e-6), (pisco.PISCO_FP64_PLAIN, 1e-12)):
        out = _gpu(nside, r, sky, grids, [det], th, ph, ps, precision)
        assert np.max(np.abs(out - ref)) <= tol * np.max(np.abs(ref)), precision


def test_invalid_samples_give_nan_and_others_unaffected():
    nside, r = 16, math.radians(15.0)
    sky = sy.white_sky(nside, 2).numpy()
    grids = sy.random_beam_maps(31, 4)
    th, ph, ps = sy.raster_scan(40, center=(1.0, 1.0), half_size=math.radians(3.0), rows=4)
    th, ph, ps = th.copy(), ph.copy(), ps.copy()
    th[3], ph[7], ps[11], th[20], th[21] = np.nan, np.inf, np.nan, -0.1, math.pi + 0.1
    bad = np.zeros(40, bool)
    bad[[3, 7, 11, 20, 21]] = True
    ref, mag = _oracle(nside, r, sky, grids, (0, 0, 1), np.where(bad, 1.0, th), ph, ps)
    for precision, rel in ((pisco.PISCO_FP32, 2e-6), (pisco.PISCO_FP64_PLAIN, 1e-11)):
        out = _gpu(nside, r, sky, grids, [(0, 0, 1)], th, ph, ps, precision)
        assert np.all(np.isnan(out[bad]))
        np.testing.assert_array_less(np.abs(out[~bad] - ref[~bad]), rel * mag[~bad])


def test_empty_input_is_a_no_op():
    nside, r = 8, math.radians(10.0)
    sky = np.ones((3, hp.npix(nside)))
    grids = torch.as_tensor(sy.random_beam_maps(11, 1), device=DEV)[None]
    with pisco.Plan(nside, r, _t(sky), [(0, 0, 1)], grids) as plan:
        e = torch.empty(0, dtype=torch.float64, device=DEV)
        out = plan.convolve(e, e, e)
        assert out.numel() == 0
        plan.sync_status()


# --------------------------------------------------------------------------- batched, host, splits


def test_batched_focal_plane_equals_single_detector_calls():
    nside, r = 32, math.radians(8.0)
    sky = sy.gaussian_sky(nside, 9).numpy()
    n_det = 5
    rng = np.random.default_rng(0)
    grids = np.stack([sy.random_beam_maps(41, 50 + d) for d in range(n_det)])
    dets = [(rng.uniform(0, 3), rng.uniform(0, 0.1), rng.uniform(0.8, 1.2)) for _ in range(n_det)]
    lengths = [37, 0, 120, 5, 64]
    offsets = np.concatenate([[0], np.cumsum(lengths)])
    pts = [sy.raster_scan(max(m, 1), center=(0.5 + 0.3 * d, 1.0 + d), half_size=0.04, rows=3)
           for d, m in enumerate(lengths)]
    th = np.concatenate([p[0][:m] for p, m in zip(pts, lengths)])
    ph = np.concatenate([p[1][:m] for p, m in zip(pts, lengths)])
    ps = np.concatenate([p[2][:m] for p, m in zip(pts, lengths)])
    for precision in (pisco.PISCO_FP32, pisco.PISCO_FP64_PLAIN):
        with pisco.Plan(nside, r, _t(sky), dets, torch.as_tensor(grids, device=DEV), precision=precision) as plan:
            batched = plan.convolve_batched(list(offsets), _t(th), _t(ph), _t(ps)).cpu().numpy()
            for d in range(n_det):
                a, b = offsets[d], offsets[d + 1]
                if b == a:
                    continue
                single = plan.convolve(_t(th[a:b]), _t(ph[a:b]), _t(ps[a:b]), det=d).cpu().numpy()
                np.testing.assert_array_equal(batched[a:b], single)
                omega = ob.omega_tilde(grids[d][0].astype(np.float64), r)
                assert abs(plan.omega(d)[0] / omega - 1.0) < 1e-12, d
                ref, mag = _oracle(nside, r, sky, grids[d], dets[d], th[a:b], ph[a:b], ps[a:b], omega)
                rel = 2e-6 if precision == pisco.PISCO_FP32 else 1e-11
                np.testing.assert_array_less(np.abs(single - ref), rel * mag)


def test_host_buffer_entry_point_matches_device_call():
    nside, r = 32, math.radians(8.0)
    sky = sy.gaussian_sky(nside, 3).numpy()
    grids = torch.as_tensor(sy.random_beam_maps(41, 3), device=DEV)[None]
    th, ph, ps = sy.raster_scan(3000, center=(1.4, 2.0), half_size=math.radians(5.0), rows=20)
    with pisco.Plan(nside, r, _t(sky), [(0.1, 0.0, 1.0)], grids) as plan:
        dev_out = plan.convolve(_t(th), _t(ph), _t(ps)).cpu()
        host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (th, ph, ps)]
        host_out = plan.convolve_host(*host)
    torch.testing.assert_close(host_out, dev_out, rtol=0, atol=0)


def test_split_calls_agree():
    """A scan convolved in two calls equals one call to FP32 rounding (tiles differ)."""
    nside, r = 32, math.radians(8.0)
    sky = sy.gaussian_sky(nside, 4).numpy()
    grids = torch.as_tensor(sy.random_beam_maps(41, 8), device=DEV)[None]
    th, ph, ps = sy.raster_scan(500, center=(1.0, 3.0), half_size=math.radians(4.0), rows=5)
    with pisco.Plan(nside, r, _t(sky), [(0.0, 0.0, 1.0)], grids) as plan:
        whole = plan.convolve(_t(th), _t(ph), _t(ps)).cpu().numpy()
        a = plan.convolve(_t(th[:173]), _t(ph[:173]), _t(ps[:173])).cpu().numpy()
        b = plan.convolve(_t(th[173:]), _t(ph[173:]), _t(ps[173:])).cpu().numpy()
    np.testing.assert_allclose(np.concatenate([a, b]), whole, rtol=0, atol=1e-6 * np.max(np.abs(whole)))


# --------------------------------------------------------------------------- adjoint


@pytest.mark.parametrize("precision", [pisco.PISCO_FP32, pisco.PISCO_FP64_PLAIN])
def test_adjoint_matches_oracle_transpose(precision):
    nside, r = 16, math.radians(15.0)
    grids = sy.random_beam_maps(31, 12)
    det = (0.5, 0.03, 1.1)
    th, ph, ps = sy.raster_scan(200, center=(1.1, 0.3), half_size=math.radians(6.0), rows=8)
    y = np.random.default_rng(3).standard_normal(len(th))
    omega = ob.omega_tilde(grids[0].astype(np.float64), r)
    ref = oc.adjoint(nside, r, grids.astype(np.float64), det, omega, th, ph, ps, y)
    sky = np.zeros((3, hp.npix(nside)))
    dt = torch.float32 if precision == pisco.PISCO_FP32 else torch.float64
    with pisco.Plan(nside, r, _t(sky), [det], torch.as_tensor(grids, device=DEV)[None], precision=precision) as plan:
        maps = plan.adjoint(_t(th), _t(ph), _t(ps), torch.as_tensor(y, dtype=dt, device=DEV)).cpu().double().numpy()
    tol = (1e-5 if precision == pisco.PISCO_FP32 else 1e-11) * np.max(np.abs(ref))
    np.testing.assert_allclose(maps, ref, rtol=0, atol=tol)


@pytest.mark.parametrize("precision", [pisco.PISCO_FP32, pisco.PISCO_FP64_PLAIN])
def test_adjoint_dot_product_identity_on_gpu(precision):
    """<A S, y> = <S, A^T y> with both sides computed by the GPU."""
    nside, r = 32, math.radians(8.0)
    sky = sy.white_sky(nside, 21).numpy()
    grids = torch.as_tensor(sy.random_beam_maps(41, 22), device=DEV)[None]
    th, ph, ps = sy.raster_scan(800, center=(2.0, 5.0), half_size=math.radians(5.0), rows=8)
    y = np.random.default_rng(5).standard_normal(len(th))
    dt = torch.float32 if precision == pisco.PISCO_FP32 else torch.float64
    with pisco.Plan(nside, r, _t(sky), [(0.2, 0.1, 0.9)], grids, precision=precision) as plan:
        d = plan.convolve(_t(th), _t(ph), _t(ps)).double().cpu().numpy()
        at = plan.adjoint(_t(th), _t(ph), _t(ps), torch.as_tensor(y, dtype=dt, device=DEV)).double().cpu().numpy()
    lhs, rhs = np.dot(d, y), np.sum(sky * at)
    scale = np.sum(np.abs(d * y))
    assert abs(lhs - rhs) <= (1e-5 if precision == pisco.PISCO_FP32 else 1e-11) * scale


# --------------------------------------------------------------------------- full size, sampled


def test_fp32_single_detector_workload_sampled():
    """The single-detector benchmark workload (nside 512, 501 x 501 grid over 10 deg with a
    sidelobe ring and cross-polar leakage, azimuth scan) in the benchmark's launch
    configuration, on 2e5 samples; every 1000th sample is checked against the oracle."""
    nside, r = 512, math.radians(10.0)
    sky = sy.gaussian_sky(nside, 1, device=DEV)
    grids = sy.gaussian_beam_maps(501, r, 1.5, ellipticity=0.0, xpol=0.005, sidelobe=(0.01, 7.0, 0.5))
    det = (0.0, 0.0, 1.0)
    th, ph, ps = sy.ces_scan(200000, device=DEV)
    with pisco.Plan(nside, r, sky, [det], torch.as_tensor(grids, device=DEV)[None]) as plan:
        out = plan.convolve(th, ph, ps).double().cpu().numpy()
        plan_omega = plan.omega(0)[0]
    idx = np.arange(0, 200000, 1000)
    skyn = sky.cpu().numpy()
    omega = ob.omega_tilde(grids[0].astype(np.float64), r)
    assert abs(plan_omega / omega - 1) < 1e-12
    ref, mag = _oracle(nside, r, skyn, grids, det, th.cpu().numpy()[idx], ph.cpu().numpy()[idx],
                       ps.cpu().numpy()[idx], omega)
    np.testing.assert_array_less(np.abs(out[idx] - ref), 2e-6 * mag)
    assert np.max(np.abs(out[idx] - ref)) <= 1e-6 * np.max(np.abs(ref))


def test_focal_plane_configuration_batched_sampled():
    """The focal-plane configuration (64 detectors with their own offsets, FWHM 1.2-1.8 deg,
    ellipticity 0-0.1 and 201^2 grids of radius 6 deg, nside 256 sky) in the benchmark's launch:
    one pisco_convolve_batched call over uneven scan lengths; three samples of every detector
    checked against the oracle."""
    nside, r, n_det = 256, math.radians(6.0), 64
    sky = sy.gaussian_sky(nside, 1, device=DEV)
    off, fwhm, ell, zeta = sy.focal_plane(n_det, 3)
    grids = np.stack([sy.gaussian_beam_maps(201, r, fwhm[d], ellipticity=ell[d]) for d in range(n_det)])
    dets = [(float(zeta[d]), 0.0, 1.0) for d in range(n_det)]
    lengths = np.random.default_rng(4).integers(200, 3001, n_det)
    parts = [sy.ces_scan(int(lengths[d]), offset=tuple(off[d]), device=DEV) for d in range(n_det)]
    th, ph, ps = (torch.cat([p[k] for p in parts]).contiguous() for k in range(3))
    offsets = [0] + list(np.cumsum(lengths))
    with pisco.Plan(nside, r, sky, dets, torch.as_tensor(grids, device=DEV).contiguous()) as plan:
        out = plan.convolve_batched(offsets, th, ph, ps).double().cpu().numpy()
        plan_omegas = [plan.omega(d)[0] for d in range(n_det)]
        plan.sync_status()
    omegas = [ob.omega_tilde(grids[d][0].astype(np.float64), r) for d in range(n_det)]
    for d in range(n_det):
        assert abs(plan_omegas[d] / omegas[d] - 1.0) < 1e-12, d
    skyn, thn, phn, psn = sky.cpu().numpy(), th.cpu().numpy(), ph.cpu().numpy(), ps.cpu().numpy()
    for d in range(n_det):
        idx = offsets[d] + np.array([0, lengths[d] // 2, lengths[d] - 1])
        ref, mag = _oracle(nside, r, skyn, grids[d], dets[d], thn[idx], phn[idx], psn[idx], omegas[d])
        np.testing.assert_array_less(np.abs(out[idx] - ref), 2e-6 * mag)


def test_differentiation_configuration_transposes_dot_identities():
    """The differentiation configuration (nside 512, parametric beam on a 201^2 grid of radius
    5 deg) at full resolution on 1e6 azimuth-scan samples: the sky and beam-grid transposes
    satisfy <A_S s, y> = <s, A_S^T y> and <A_G G, y> = <G, A_G^T y> (Omega~ held fixed, where
    the TOD is linear in the grids), all sums from the GPU, to FP32 accumulation accuracy."""
    from paper_1908_05662_gb300 import beams
    nside, r, n = 512, math.radians(5.0), 1_000_000
    sky = sy.gaussian_sky(nside, 1, device=DEV)
    g = beams.gaussian_beam_grids(201, r, 1.5, 0.05, 0.005, device=DEV).float()[None].contiguous()
    th, ph, ps = (a.contiguous() for a in sy.ces_scan(n, device=DEV))
    y = torch.randn(n, device=DEV, generator=torch.Generator(device=DEV).manual_seed(5))
    with pisco.Plan(nside, r, sky, [(0.2, 0.01, 1.0)], g, omega_tilde=[0.002]) as plan:
        d = plan.convolve(th, ph, ps).double()
        maps, grad = plan.adjoint_sky_beam(th, ph, ps, y)
        plan.sync_status()
    lhs = torch.dot(d, y.double()).item()
    scale = torch.sum(torch.abs(d * y.double())).item()
    rhs_sky = torch.sum(sky.double() * maps.double()).item()
    rhs_grid = torch.sum(g[0].double() * grad.double()).item()
    assert abs(lhs - rhs_sky) <= 1e-5 * scale, (lhs, rhs_sky)
    assert abs(lhs - rhs_grid) <= 1e-5 * scale, (lhs, rhs_grid)
