"""Pins of the oracle's map-making: RING ang2pix and the binned map-maker.

ang2pix is fixed by pixel centres (each lies in its own pixel), the equal
areas of the scheme (Monte Carlo counts), locality against a brute-force
nearest-centre search, the north-south mirror symmetry and periodicity in
phi.  The binned solver is fixed by exact recovery of maps from delta-beam
TOD built with the convolution's own D(chi) (a separate function), by numpy's
least squares per pixel, by the degenerate cases, and by the sign convention
of the forward model: a uniform polarised sky convolved with a narrow beam is
recovered.
"""

import math

import numpy as np
import pytest

from oracle import beam as ob
from oracle import convolve as oc
from oracle import healpix as hp
from oracle import mapmaking as mm
from paper_1908_05662_gb300 import synthetic as sy


@pytest.mark.parametrize("nside", [1, 2, 4, 16, 64])
def test_pixel_centres_lie_in_their_own_pixel(nside):
    p = np.arange(hp.npix(nside))
    th, ph = hp.pix2ang(nside, p)
    np.testing.assert_array_equal(mm.ang2pix(nside, th, ph), p)


def test_equal_area_monte_carlo():
    nside, n = 2, 480_000
    rng = np.random.default_rng(0)
    th = np.arccos(rng.uniform(-1, 1, n))
    ph = rng.uniform(0, 2 * math.pi, n)
    counts = np.bincount(mm.ang2pix(nside, th, ph), minlength=hp.npix(nside))
    expect = n / hp.npix(nside)
    assert np.all(np.abs(counts - expect) < 6 * math.sqrt(expect)), counts


def test_assigned_pixel_is_a_near_centre():
    nside = 16
    rng = np.random.default_rng(1)
    th = np.arccos(rng.uniform(-1, 1, 3000))
    ph = rng.uniform(0, 2 * math.pi, 3000)
    pix = mm.ang2pix(nside, th, ph)
    cv = hp.pix2vec(nside, np.arange(hp.npix(nside)))
    pv = hp.ang2vec(th, ph)
    dots = pv @ cv.T
    rank = np.argsort(-dots, axis=1)[:, :6]
    assert np.all(np.any(rank == pix[:, None], axis=1))
    size = math.sqrt(4 * math.pi / hp.npix(nside))
    assert np.all(np.arccos(np.clip(dots[np.arange(3000), pix], -1, 1)) < 1.2 * size)


def test_mirror_symmetry_and_phi_periodicity():
    nside = 8
    rng = np.random.default_rng(2)
    th = np.arccos(rng.uniform(-1, 1, 2000))
    ph = rng.uniform(0, 2 * math.pi, 2000)
    pix = mm.ang2pix(nside, th, ph)
    r, j = hp.pix2ring(nside, pix)
    rm, jm = hp.pix2ring(nside, mm.ang2pix(nside, math.pi - th, ph))
    nr = 4 * nside - 1
    np.testing.assert_array_equal(rm, nr - 1 - r)
    np.testing.assert_array_equal(jm, j)
    np.testing.assert_array_equal(mm.ang2pix(nside, th, ph + 2 * math.pi), pix)
    np.testing.assert_array_equal(mm.ang2pix(nside, th, ph - 2 * math.pi), pix)


def test_cap_belt_transition_rings():
    nside = 8
    z0 = 2.0 / 3.0
    ph = np.linspace(0.01, 6.2, 50)
    up = mm.ang2pix(nside, np.full(50, math.acos(z0 + 1e-9)), ph)
    dn = mm.ang2pix(nside, np.full(50, math.acos(z0 - 1e-9)), ph)
    assert set(hp.pix2ring(nside, up)[0]) <= {nside - 2, nside - 1}
    assert set(hp.pix2ring(nside, dn)[0]) <= {nside - 1, nside}


def _centre_scan(nside, angles_deg):
    th, ph = hp.pix2ang(nside, np.arange(hp.npix(nside)))
    a = np.radians(angles_deg)
    return np.repeat(th, len(a)), np.repeat(ph, len(a)), np.tile(a, len(th))


def test_exact_recovery_from_delta_beam_tod():
    nside = 8
    det = (0.3, 0.05, 1.2)
    sky = np.random.default_rng(3).standard_normal((3, hp.npix(nside)))
    th, ph, ps = _centre_scan(nside, [0.0, 45.0, 90.0, 130.0])
    pix = np.repeat(np.arange(hp.npix(nside)), 4)
    chi = ps + det[0]
    d = np.einsum("tm,mt->t", oc.detector_row(chi, det[1], det[2])[:, :3], sky[:, pix])
    maps, hits = mm.binned_map(nside, th, ph, ps, det, d)
    assert np.all(hits == 4)
    np.testing.assert_allclose(maps, sky, rtol=0, atol=1e-12)


def test_matches_numpy_least_squares_per_pixel():
    nside = 4
    det = (0.0, 0.0, 1.0)
    rng = np.random.default_rng(4)
    n = 4000
    th = np.arccos(rng.uniform(-1, 1, n))
    ph = rng.uniform(0, 2 * math.pi, n)
    ps = rng.uniform(0, math.pi, n)
    d = rng.standard_normal(n)
    maps, hits = mm.binned_map(nside, th, ph, ps, det, d)
    pix = mm.ang2pix(nside, th, ph)
    rows = oc.detector_row(ps + det[0], det[1], det[2])[:, :3]
    for p in range(hp.npix(nside)):
        sel = pix == p
        assert hits[p] == sel.sum()
        ref = np.linalg.lstsq(rows[sel], d[sel], rcond=None)[0]
        np.testing.assert_allclose(maps[:, p], ref, rtol=1e-10, atol=1e-12)


def test_degenerate_pixels_are_nan():
    nside = 2
    th, ph = hp.pix2ang(nside, np.array([0, 1, 2, 3]))
    # pixel 0: 2 hits; 1: three hits at one angle; 2: angles 0 and 90 deg only (U unconstrained);
    # 3: three well-spread angles; every other pixel: no hit
    T = np.array([th[0], th[0], th[1], th[1], th[1], th[2], th[2], th[2], th[3], th[3], th[3]])
    P = np.array([ph[0], ph[0], ph[1], ph[1], ph[1], ph[2], ph[2], ph[2], ph[3], ph[3], ph[3]])
    a = np.radians([0, 60, 10, 10, 10, 0, 90, 0, 0, 60, 120])
    d = np.ones(len(T))
    maps, hits = mm.binned_map(nside, T, P, a, (0.0, 0.0, 1.0), d)
    assert np.all(np.isnan(maps[:, :3])) and np.all(np.isfinite(maps[:, 3]))
    assert np.all(np.isnan(maps[:, 4:]))
    np.testing.assert_allclose(maps[:, 3], [2.0, 0.0, 0.0], atol=1e-12)
    bad = np.array([np.nan, 0.5, 0.5])
    maps2, hits2 = mm.binned_map(nside, np.r_[T, bad], np.r_[P, 0.1, np.nan, 0.1], np.r_[a, 0, 0, 0],
                                 (0.0, 0.0, 1.0), np.r_[d, 1.0, 1.0, np.inf])
    np.testing.assert_array_equal(hits2, hits)


def test_uniform_polarised_sky_through_the_convolution_is_recovered():
    """The forward model's sign convention: TOD of a uniform (I, Q, U) sky through the
    pixelised convolution with a narrow ideal beam, binned, gives back (I, Q, U)."""
    nside, r = 256, math.radians(3.0)
    grids = sy.gaussian_beam_maps(121, r, 1.0, ideal=True).astype(np.float64)
    omega = ob.omega_tilde(grids[0], r)
    sky = np.empty((3, hp.npix(nside)))
    sky[0], sky[1], sky[2] = 1.0, 0.3, -0.2
    det = (0.4, 0.0, 1.0)
    pix = np.array([100000, 300000, 500000])  # away from the poles, where uniform Q, U is singular
    th, ph = hp.pix2ang(nside, pix)
    T, P, A = np.repeat(th, 3), np.repeat(ph, 3), np.tile(np.radians([0.0, 45.0, 90.0]), 3)
    d = oc.tod(nside, r, sky, grids, det, omega, T, P, A)
    maps, _ = mm.binned_map(nside, T, P, A, det, d)
    np.testing.assert_allclose(maps[:, pix].T, np.tile([1.0, 0.3, -0.2], (3, 1)), rtol=0, atol=2e-3)
