"""Pins of the oracle's HEALPix RING geometry and disc query (CPU only)."""

import math

import numpy as np
import pytest

from oracle import healpix as hp
from conftest import golden_rows


def test_nside1_centres_match_base_layout():
    rows = golden_rows("healpix_nside1_centres.txt")
    pix = np.array([int(r[0]) for r in rows])
    theta, phi = hp.pix2ang(1, pix)
    np.testing.assert_allclose(np.cos(theta), [r[1] for r in rows], atol=1e-15)
    np.testing.assert_allclose(phi / math.pi, [r[2] for r in rows], atol=1e-15)


@pytest.mark.parametrize("nside", [1, 2, 3, 8, 64, 512])
def test_ring_sizes_and_total(nside):
    t = hp.ring_table(nside)
    assert len(t["count"]) == 4 * nside - 1
    assert t["count"].sum() == hp.npix(nside)
    i = np.arange(1, 4 * nside)
    expect = np.where(i < nside, 4 * i, np.where(i > 3 * nside, 4 * (4 * nside - i), 4 * nside))
    np.testing.assert_array_equal(t["count"], expect)


@pytest.mark.parametrize("nside", [1, 2, 5, 16, 128])
def test_equal_area_identity(nside):
    """Pixels above the middle of ring i fill exactly the area above z_i.

    Equal-area pixels placed on iso-latitude rings satisfy
    first(i) + count(i) / 2 = Npix (1 - z_i) / 2 for every ring; a wrong
    ring height or ring size breaks it.
    """
    t = hp.ring_table(nside)
    lhs = t["first"] + t["count"] / 2.0
    rhs = hp.npix(nside) * (1.0 - t["z"]) / 2.0
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-9 * hp.npix(nside))


@pytest.mark.parametrize("nside", [2, 4, 7])
def test_north_south_mirror_and_stagger(nside):
    t = hp.ring_table(nside)
    np.testing.assert_allclose(t["z"], -t["z"][::-1], atol=1e-15)
    np.testing.assert_allclose(t["phi0"], t["phi0"][::-1], atol=1e-15)
    # Belt rings alternate between a half-pixel offset and none, starting
    # with the offset shared by the polar-cap rings (ring i = nside).
    belt = np.arange(nside - 1, 3 * nside)
    off = t["phi0"][belt] / t["dphi"][belt]
    np.testing.assert_allclose(off, 0.5 * ((np.arange(len(belt)) + 1) % 2), atol=1e-15)


def test_unit_vectors_are_unit_and_sorted():
    k = hp.pix2vec(16, np.arange(hp.npix(16)))
    np.testing.assert_allclose(np.linalg.norm(k, axis=-1), 1.0, atol=1e-15)
    assert np.all(np.diff(k[:, 2]) <= 0)  # RING order runs north to south


def _pointings(seed, n):
    rng = np.random.default_rng(seed)
    theta = np.arccos(rng.uniform(-1, 1, n))
    phi = rng.uniform(-2 * math.pi, 4 * math.pi, n)  # includes wrapped longitudes
    special = [(0.0, 0.3), (math.pi, 1.0), (1e-9, 5.0), (math.pi - 1e-9, 2.0),
               (math.pi / 2, 0.0), (math.pi / 2, 2 * math.pi - 1e-12), (0.7, -1e-12)]
    theta = np.concatenate([theta, [s[0] for s in special]])
    phi = np.concatenate([phi, [s[1] for s in special]])
    return theta, phi


@pytest.mark.parametrize("nside,radius_deg", [(1, 40.0), (2, 25.0), (4, 30.0), (16, 10.0),
                                              (32, 5.0), (32, 60.0), (8, 89.0)])
def test_ring_query_equals_brute_force(nside, radius_deg):
    theta, phi = _pointings(nside * 7 + int(radius_deg), 40)
    r = math.radians(radius_deg)
    for a, b in zip(theta, phi):
        np.testing.assert_array_equal(hp.query_disc(nside, a, b, r),
                                      hp.query_disc_brute(nside, a, b, r))


def test_mean_disc_count_matches_cap_area():
    nside, r = 64, math.radians(6.0)
    theta, phi = _pointings(3, 200)
    counts = [len(hp.query_disc(nside, a, b, r)) for a, b in zip(theta, phi)]
    expect = 2 * math.pi * (1 - math.cos(r)) / (4 * math.pi / hp.npix(nside))
    assert abs(np.mean(counts) / expect - 1.0) < 0.01


def test_table1_disc_pixel_counts():
    """Disc sizes at nside 128 agree with the paper's Table 1 within 2.5 %."""
    nside = 128
    pointings = [0, 1000, hp.npix(nside) // 2 + 77, 2 * nside * (nside - 1) + 5]
    for rho_max, pixels in golden_rows("table1_disc_pixels.txt"):
        for p in pointings:
            th, ph = hp.pix2ang(nside, p)
            n = len(hp.query_disc(nside, th, ph, math.radians(rho_max)))
            assert abs(n / pixels - 1.0) < 0.025, (rho_max, p, n, pixels)
