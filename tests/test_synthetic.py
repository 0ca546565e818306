"""The input generators: the sky synthesis against scipy's spherical harmonics (CPU only)."""

import math

import numpy as np
import torch
from scipy.special import sph_harm_y

from oracle import healpix as hp
from paper_1908_05662_gb300 import synthetic as sy


def test_sky_synthesis_reproduces_spherical_harmonics():
    nside = 8
    lmax = 3 * nside - 1
    rng = np.random.default_rng(0)
    alms = []
    terms = []
    for _ in range(2):
        a = torch.zeros(lmax + 1, lmax + 1, dtype=torch.complex128)
        for _ in range(6):
            ell = int(rng.integers(1, lmax + 1))
            m = int(rng.integers(0, ell + 1))
            c = complex(rng.standard_normal(), rng.standard_normal() if m else 0.0)
            a[ell, m] += c
            terms.append((len(alms), ell, m, c))
        alms.append(a)
    maps = sy._synthesise(alms, nside, "cpu").numpy()
    theta, phi = hp.pix2ang(nside, np.arange(hp.npix(nside)))
    for f in range(2):
        ref = np.zeros(hp.npix(nside))
        for ff, ell, m, c in terms:
            if ff != f:
                continue
            y = sph_harm_y(ell, m, theta, phi)
            ref += np.real(c * y) if m == 0 else 2.0 * np.real(c * y)
        np.testing.assert_allclose(maps[f], ref, atol=1e-12)


def test_gaussian_sky_statistics():
    sky = sy.gaussian_sky(16, 3).numpy()
    assert sky.shape == (3, 12 * 16 * 16)
    np.testing.assert_allclose(sky.std(axis=1, ddof=1), [1.0, 0.1, 0.1], rtol=1e-12)
    # independent fields
    assert abs(np.corrcoef(sky[0], sky[1])[0, 1]) < 0.3


def test_scan_generators_are_well_formed():
    th, ph, ps = sy.ces_scan(20000)
    assert torch.all((th > 0) & (th < math.pi))
    steps = torch.arccos(torch.clamp(torch.sin(th[1:]) * torch.sin(th[:-1]) * torch.cos(ph[1:] - ph[:-1])
                                     + torch.cos(th[1:]) * torch.cos(th[:-1]), -1, 1))
    # 1 deg/s in azimuth at 45 deg elevation, 20 Hz: ~0.035 deg per sample
    assert abs(math.degrees(torch.median(steps).item()) - 0.0354) < 0.002
    th, ph, ps = sy.raster_scan(1000, rows=10)
    assert np.all(np.diff(th[:100]) == 0) and np.all(np.diff(ps) > 0)
