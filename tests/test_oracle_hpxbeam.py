"""Pins of the oracle's HEALPix beam input: ring-wise interpolation and the
resampling of HEALPix beam maps onto the tangent-plane grid.

Each pin is fixed by something other than the oracle's own formula: exact
reproduction of pixel values, of functions that the scheme must carry exactly
(linear in theta between rings, linear in phi along a ring, quadratic in theta
in the caps), a brute-force stencil search over every pixel of a small map,
convergence on smooth functions, and the analytic Gaussian beam.
"""

import math

import numpy as np
import pytest

from oracle import beam as ob
from oracle import healpix as hp
from paper_1908_05662_gb300 import beams
from paper_1908_05662_gb300 import synthetic as sy


def _points(n, seed):
    rng = np.random.default_rng(seed)
    return np.arccos(rng.uniform(-1.0, 1.0, n)), rng.uniform(0.0, 2.0 * math.pi, n)


@pytest.mark.parametrize("nside", [1, 2, 4, 16])
def test_weights_sum_to_one_with_signs_of_the_reading(nside):
    th, ph = _points(400, nside)
    th = np.concatenate([th, [0.0, 1e-9, math.pi, math.pi - 1e-9]])
    ph = np.concatenate([ph, [0.0, 1.0, 2.0, 6.28]])
    pix, w = hp.interp_weights(nside, th, ph)
    np.testing.assert_allclose(w.sum(axis=0), 1.0, rtol=0, atol=1e-12)
    tr = hp.ring_theta(nside)
    cap = (th < tr[0]) | (th >= tr[-1])
    assert np.all(w[:, ~cap] >= -1e-15)
    north = th < tr[0]
    assert np.all(w[:2, north] >= 0) and np.all(w[2:, north] <= 1e-15)
    south = th >= tr[-1]
    assert np.all(w[2:, south] >= -1e-15) and np.all(w[:2, south] <= 1e-15)
    assert pix.min() >= 0 and pix.max() < hp.npix(nside)


@pytest.mark.parametrize("nside", [1, 4])
def test_pixel_centres_reproduce_the_map(nside):
    m = np.random.default_rng(1).standard_normal(hp.npix(nside))
    th, ph = hp.pix2ang(nside, np.arange(hp.npix(nside)))
    np.testing.assert_allclose(hp.interpolate(nside, m, th, ph), m, rtol=0, atol=1e-12)


def test_linear_in_theta_between_rings():
    nside = 8
    tp, _ = hp.pix2ang(nside, np.arange(hp.npix(nside)))
    tr = hp.ring_theta(nside)
    th, ph = _points(500, 2)
    keep = (th >= tr[0]) & (th < tr[-1])
    np.testing.assert_allclose(hp.interpolate(nside, tp, th[keep], ph[keep]), th[keep], rtol=0, atol=1e-12)


def test_quadratic_in_theta_in_the_caps():
    nside = 8
    tp, _ = hp.pix2ang(nside, np.arange(hp.npix(nside)))
    tr = hp.ring_theta(nside)
    rng = np.random.default_rng(3)
    th_n = rng.uniform(0.0, tr[0], 50)
    th_s = math.pi - rng.uniform(0.0, math.pi - tr[-1], 50)
    ph = rng.uniform(0.0, 2 * math.pi, 50)
    np.testing.assert_allclose(hp.interpolate(nside, tp ** 2, th_n, ph), th_n ** 2, rtol=0, atol=1e-14)
    np.testing.assert_allclose(hp.interpolate(nside, (math.pi - tp) ** 2, th_s, ph), (math.pi - th_s) ** 2,
                               rtol=0, atol=1e-14)
    # a peak at the pole, a + theta^2 (b + c cos 2 phi): the extrapolation recovers a up to the
    # phi-interpolation error of the cos 2 phi term on rings of 4 and 8 pixels, far closer than
    # ring 1's mean (a + b theta_1^2) would be
    a, b, c = 1.0, -3.0, 0.4
    _, pp = hp.pix2ang(nside, np.arange(hp.npix(nside)))
    m = a + tp ** 2 * (b + c * np.cos(2 * pp))
    err = abs(hp.interpolate(nside, m, 0.0, 0.3) - a)
    assert err < 0.3 * abs(c) * tr[1] ** 2 and err < 0.2 * abs(b) * tr[0] ** 2


def test_linear_in_phi_along_a_ring():
    nside = 4
    r, j = hp.pix2ring(nside, np.arange(hp.npix(nside)))
    t = hp.ring_table(nside)
    tr = hp.ring_theta(nside)
    rng = np.random.default_rng(4)
    for ring in (0, 2, nside - 1, 2 * nside, 4 * nside - 2):
        x = rng.uniform(0.0, t["count"][ring] - 1.0, 20)  # stays clear of the wrap
        ph = t["phi0"][ring] + x * t["dphi"][ring]
        val = hp.interpolate(nside, j.astype(float), np.full(20, tr[ring]), ph)
        np.testing.assert_allclose(val, x, rtol=0, atol=1e-11)


def _brute_value(nside, m, theta, phi):
    """Same reading, found by scanning every pixel: bracketing rings from the sorted set of
    pixel colatitudes, bracketing pixels on a ring from their phi distances."""
    tp, pp = hp.pix2ang(nside, np.arange(hp.npix(nside)))
    rings = np.array(sorted({round(float(x), 12): float(x) for x in tp}.values()))  # exact ring colatitudes

    def ring_value(t_ring, phi):
        on = np.where(np.abs(tp - t_ring) < 1e-9)[0]
        d = np.mod(phi - pp[on], 2 * math.pi)
        lo = on[np.argmin(d)]
        step = 2 * math.pi / on.size
        hi = on[np.argmin(np.abs(np.mod(pp[on] - pp[lo] - step + math.pi, 2 * math.pi) - math.pi))]
        f = np.min(d) / step
        return (1 - f) * m[lo] + f * m[hi]

    if theta < rings[0]:
        t1, t2 = rings[0], rings[1]
        w = (theta ** 2 - t1 ** 2) / (t2 ** 2 - t1 ** 2)
    elif theta >= rings[-1]:
        t1, t2 = rings[-2], rings[-1]
        a, b, c = math.pi - theta, math.pi - t2, math.pi - t1
        w = 1.0 - (a * a - b * b) / (c * c - b * b)
    else:
        t1 = rings[rings <= theta].max()
        t2 = rings[rings > theta].min()
        w = (theta - t1) / (t2 - t1)
    return (1 - w) * ring_value(t1, phi) + w * ring_value(t2, phi)


@pytest.mark.parametrize("nside", [1, 2, 4])
def test_matches_brute_force_stencil_search(nside):
    m = np.random.default_rng(nside).standard_normal(hp.npix(nside))
    th, ph = _points(60, 10 + nside)
    th = np.concatenate([th, [0.01, math.pi - 0.01]])
    ph = np.concatenate([ph, [5.0, 0.2]])
    got = hp.interpolate(nside, m, th, ph)
    ref = np.array([_brute_value(nside, m, a, b) for a, b in zip(th, ph)])
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


def test_smooth_function_error_falls_quadratically():
    """Second-order scheme: the rms error on a smooth function falls ~4x per halving of the pixel."""
    rms, worst = [], []
    th, ph = _points(2000, 5)
    exact = np.sin(th) * np.cos(ph) + 0.5 * np.cos(th) ** 2
    for nside in (16, 32, 64):
        tp, pp = hp.pix2ang(nside, np.arange(hp.npix(nside)))
        e = hp.interpolate(nside, np.sin(tp) * np.cos(pp) + 0.5 * np.cos(tp) ** 2, th, ph) - exact
        rms.append(np.sqrt(np.mean(e * e)))
        worst.append(np.max(np.abs(e)))
    assert worst[2] < 2e-3
    assert rms[0] / rms[1] > 3.5 and rms[1] / rms[2] > 3.5


def _gaussian_healpix(nside, fwhm_deg, e):
    th, ph = sy.healpix_centres(nside)
    u, v = np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph)
    s = math.radians(fwhm_deg) * beams.FWHM_TO_SIGMA
    return np.exp(-0.5 * ((u / (s * (1 + e))) ** 2 + (v / (s * (1 - e))) ** 2))


def test_grid_from_healpix_converges_to_the_analytic_beam():
    r, n = math.radians(4.0), 81
    ref = beams.gaussian_beam_grids(n, r, 1.5, 0.05).numpy()[0]
    e256 = np.max(np.abs(ob.grid_from_healpix(_gaussian_healpix(256, 1.5, 0.05), 256, r, n) - ref))
    e512 = np.max(np.abs(ob.grid_from_healpix(_gaussian_healpix(512, 1.5, 0.05), 512, r, n) - ref))
    assert e512 < 3e-3 and e256 / e512 > 3.0


def test_grid_from_healpix_orientation_and_off_hemisphere_nodes():
    nside, r, n = 64, math.radians(50.0), 11
    tp, pp = hp.pix2ang(nside, np.arange(hp.npix(nside)))
    maps = np.stack([np.sin(tp) * np.cos(pp), np.sin(tp) * np.sin(pp), tp])
    g = ob.grid_from_healpix(maps, nside, r, n)
    u = ob.nodes(n, r)
    uu, vv = np.meshgrid(u, u, indexing="xy")
    on = uu ** 2 + vv ** 2 <= 1.0
    assert np.all(g[:, ~on] == 0.0) and np.any(~on)
    rho = np.arcsin(np.sqrt(np.minimum(uu ** 2 + vv ** 2, 1.0)))
    t1 = hp.ring_theta(nside)[0]
    belt = on & (rho >= t1)
    np.testing.assert_allclose(g[0][belt], uu[belt], rtol=0, atol=2e-3)   # u along i (theta'0)
    np.testing.assert_allclose(g[1][belt], vv[belt], rtol=0, atol=2e-3)   # v along j (phi'0)
    np.testing.assert_allclose(g[2][belt], rho[belt], rtol=0, atol=1e-12)
    # a tilt through the pole is odd in theta, so the centre node sees the extrapolation's
    # first-order error: bounded by the ring-1 colatitude
    assert np.all(np.abs(g[:2, n // 2, n // 2]) < t1)
