"""The paper's own pointings and the disc boundary, element by element against the FP64 oracle.

* Pointings exactly on sky pixel centres (rho = 0 for that pixel: the Table 1 and
  Sec. 6 runs convolve at every pixel centre).  At rho = 0 the antenna azimuth
  sigma is undefined and chi tends to psi0 + zeta (Appendix A); the oracle takes
  that limit, the kernels reach it through their own arithmetic.
* Pointings at distance R -+ 1e-12 rad from a pixel centre (that pixel just inside
  or just outside the disc, Sec. 5.2 / Table 1's rho_max cut).  The margin,
  1e-12 x sin R >= 7e-14 in k . p0, is hundreds of ulps above the FP64 rounding
  of either side's dot product, so every path must take the oracle's decision:
  disc counts are compared bit for bit, TODs with the tolerance of each path
  (FP32 2e-6, plain FP64 1e-11, packed cells 2e-5, tensor cores 1e-5 BF16 /
  2e-6 FP16 of the per-sample magnitude sum_k |w_k . S_k|).

Omega~ comes from the oracle (the plan's own value is checked against it).
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


def _pointings(nside, radius, seed):
    """Pixel-centre pointings (random pixels, then a walk along consecutive pixels of one ring,
    which the FP32 kernel groups into shared traversals) followed by disc-edge pointings."""
    th_c, ph_c, ps_c, _ = sy.pixel_centre_pointings(nside, 24, seed)
    th_all, ph_all = sy.healpix_centres(nside)
    first = 2 * nside * (nside - 1) + 4 * nside * (nside // 2)  # a ring of the equatorial belt, z = 1/3
    walk = first + np.arange(24)
    ps_w = np.random.default_rng(seed + 1).uniform(0.0, 2.0 * math.pi, 24)
    th_e, ph_e, ps_e, _ = sy.disc_edge_pointings(nside, radius, 40, seed + 2)
    th = np.concatenate([th_c, th_all[walk], th_e])
    ph = np.concatenate([ph_c, ph_all[walk], ph_e])
    ps = np.concatenate([ps_c, ps_w, ps_e])
    return th, ph, ps


def _oracle(nside, radius, sky, grids, det, theta, phi, psi):
    g64 = np.asarray(grids, np.float64)
    omega = ob.omega_tilde(g64[0], radius)
    d = oc.tod(nside, radius, sky, g64, det, omega, theta, phi, psi)
    mag = np.empty(len(theta))
    for t in range(len(theta)):
        pix, w = oc.sample_weights(nside, radius, g64, det, omega, theta[t], phi[t], psi[t])
        mag[t] = np.sum(np.abs(w * sky[:, pix].T))
    return d, mag, omega


CASES = [(32, 8.0, 41), (64, 4.0, 61), (32, 20.0, 41)]


@pytest.mark.parametrize("nside,radius_deg,n_grid", CASES)
def test_edge_disc_counts_bit_exact(nside, radius_deg, n_grid):
    r = math.radians(radius_deg)
    th, ph, _ = _pointings(nside, r, nside)
    ref = oc.disc_count(nside, r, th, ph)
    sky = np.zeros((3, hp.npix(nside)))
    g = torch.as_tensor(sy.random_beam_maps(n_grid, 1), device=DEV)[None]
    for precision in (pisco.PISCO_FP32, pisco.PISCO_FP64_PLAIN):
        with pisco.Plan(nside, r, _t(sky), [(0, 0, 1)], g, precision=precision) as plan:
            c = plan.disc_count(_t(th), _t(ph)).cpu().numpy()
        np.testing.assert_array_equal(c, ref, err_msg=f"precision {precision}")


@pytest.mark.parametrize("nside,radius_deg,n_grid", CASES)
@pytest.mark.parametrize("precision,fetch,rel", [(pisco.PISCO_FP32, pisco.PISCO_FETCH_CELLS, 2e-6),
                                                 (pisco.PISCO_FP32, pisco.PISCO_FETCH_PACKED, 2e-5),
                                                 (pisco.PISCO_FP64_PLAIN, 0, 1e-11)])
def test_edge_forward_elementwise(nside, radius_deg, n_grid, precision, fetch, rel):
    r = math.radians(radius_deg)
    sky = sy.white_sky(nside, 7).numpy()
    grids = sy.random_beam_maps(n_grid, 3 + nside)
    det = (0.6, 0.05, 1.2)
    th, ph, ps = _pointings(nside, r, 2 * nside)
    ref, mag, omega = _oracle(nside, r, sky, grids, det, th, ph, ps)
    g = torch.as_tensor(grids, device=DEV)[None]
    with pisco.Plan(nside, r, _t(sky), [det], g, precision=precision, beam_fetch=fetch) as plan:
        out = plan.convolve(_t(th), _t(ph), _t(ps)).double().cpu().numpy()
        plan.sync_status()
        assert abs(plan.omega(0)[0] / omega - 1.0) < 1e-12
    np.testing.assert_array_less(np.abs(out - ref), rel * mag)


@pytest.mark.parametrize("nside,radius_deg,n_grid", CASES)
def test_edge_psb_pair_elementwise(nside, radius_deg, n_grid):
    r = math.radians(radius_deg)
    sky = sy.white_sky(nside, 8).numpy()
    grids = sy.random_beam_maps(n_grid, 5 + nside)
    zeta0, eps, s = 0.4, 0.03, 0.9
    zetas = [zeta0, zeta0 - 0.5 * math.pi]
    th, ph, ps = _pointings(nside, r, 3 * nside)
    with pisco.Plan(nside, r, _t(sky), [(zeta0, eps, s)], torch.as_tensor(grids, device=DEV)[None]) as plan:
        out = plan.convolve_psb(_t(th), _t(ph), _t(ps), zetas).double().cpu().numpy()
        plan.sync_status()
    for k, z in enumerate(zetas):
        ref, mag, _ = _oracle(nside, r, sky, grids, (z, eps, s), th, ph, ps)
        np.testing.assert_array_less(np.abs(out[k] - ref), 2e-6 * mag)


@pytest.mark.parametrize("precision,dtype,bound", [(pisco.PISCO_BF16_MR, torch.bfloat16, 1e-5),
                                                   (pisco.PISCO_FP16_MR, torch.float16, 2e-6)])
def test_edge_multirealization_elementwise(precision, dtype, bound):
    """The tensor-core path on the same pointings, per realization, against the oracle
    evaluated on the realizations as stored."""
    nside, r, n_real = 32, math.radians(8.0), 64
    rng = np.random.default_rng(17)
    base = np.stack([sy.gaussian_sky(nside, 40 + k).numpy() for k in range(3)])  # (3 fields, 3, Npix)
    coef = rng.standard_normal((n_real, 3))
    stack = torch.as_tensor(np.einsum("rk,kmp->pmr", coef, base), device=DEV).to(dtype).contiguous()
    stack64 = stack.double().cpu().numpy()
    grids = sy.random_beam_maps(61, 9)
    det = (0.2, 0.04, 1.1)
    th, ph, ps = _pointings(nside, r, 5)
    g64 = grids.astype(np.float64)
    omega = ob.omega_tilde(g64[0], r)
    ref = np.empty((len(th), n_real))
    mag = np.empty_like(ref)
    for t in range(len(th)):
        pix, w = oc.sample_weights(nside, r, g64, det, omega, th[t], ph[t], ps[t])
        ref[t] = np.einsum("km,kmr->r", w, stack64[pix])
        mag[t] = np.einsum("km,kmr->r", np.abs(w), np.abs(stack64[pix]))
    with pisco.Plan(nside, r, stack, [det], torch.as_tensor(grids, device=DEV)[None], precision=precision) as plan:
        out = plan.convolve(_t(th), _t(ph), _t(ps)).double().cpu().numpy()
        plan.sync_status()
        assert abs(plan.omega(0)[0] / omega - 1.0) < 1e-12
    np.testing.assert_array_less(np.abs(out - ref), bound * mag)
