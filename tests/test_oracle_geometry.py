"""Pins of the oracle's antenna-frame geometry and beam re-pixelisation (CPU only)."""

import math

import numpy as np
import pytest
from scipy import integrate

from oracle import beam as ob
from oracle import geometry as og
from oracle import healpix as hp


def _configs(seed, n, max_sep_deg=30.0):
    """Random pointings (theta0, phi0, psi0, zeta) and sky directions within max_sep of them."""
    rng = np.random.default_rng(seed)
    theta0 = np.arccos(rng.uniform(-0.98, 0.98, n))
    phi0 = rng.uniform(0, 2 * math.pi, n)
    psi0 = rng.uniform(-math.pi, math.pi, n)
    zeta = rng.uniform(0, math.pi, n)
    rho = np.radians(max_sep_deg * rng.uniform(1e-3, 1.0, n))
    sig = rng.uniform(-math.pi, math.pi, n)
    k = np.empty((n, 3))
    for t in range(n):
        p, th, ph = og.antenna_basis(theta0[t], phi0[t], psi0[t])
        k[t] = np.sin(rho[t]) * (np.cos(sig[t]) * th + np.sin(sig[t]) * ph) + np.cos(rho[t]) * p
    theta = np.arctan2(np.hypot(k[:, 0], k[:, 1]), k[:, 2])
    phi = np.arctan2(k[:, 1], k[:, 0])
    return theta0, phi0, psi0, zeta, k, theta, phi, rho, sig


def test_sky_and_antenna_bases_are_right_handed_orthonormal():
    rng = np.random.default_rng(1)
    for _ in range(50):
        a, b, c = rng.uniform(0, math.pi), rng.uniform(0, 2 * math.pi), rng.uniform(0, 2 * math.pi)
        for p, th, ph in (og.sky_basis(a, b), og.antenna_basis(a, b, c)):
            m = np.stack([th, ph, p])
            np.testing.assert_allclose(m @ m.T, np.eye(3), atol=1e-14)
            np.testing.assert_allclose(np.cross(th, ph), p, atol=1e-14)


def test_appendix_route_equals_vector_route():
    """Appendix A's spherical trigonometry and Sec. 2's vectors give the same (rho, sigma, chi)."""
    theta0, phi0, psi0, zeta, k, theta, phi, rho, sig = _configs(2, 4000)
    r1, s1, c1 = og.appendix_route(theta, phi, theta0, phi0, psi0, zeta)
    r2, s2, c2 = np.empty(len(k)), np.empty(len(k)), np.empty(len(k))
    for t in range(len(k)):
        r2[t], s2[t], c2[t] = og.vector_route(k[t], theta0[t], phi0[t], psi0[t], zeta[t])
    np.testing.assert_allclose(r1, rho, atol=1e-11)
    np.testing.assert_allclose(r2, rho, atol=1e-12)
    np.testing.assert_allclose(og.wrap_angle(s1 - sig), 0.0, atol=1e-11)
    np.testing.assert_allclose(og.wrap_angle(s2 - sig), 0.0, atol=1e-12)
    np.testing.assert_allclose(og.wrap_angle(c1 - c2), 0.0, atol=1e-11)


def test_rho_sigma_hats_are_derivatives_of_k():
    """rho_hat = dk/drho and sigma_hat = dk/dsigma / sin(rho): pins the cos(rho) sin(sigma) reading."""
    rng = np.random.default_rng(3)
    h = 1e-6
    for _ in range(100):
        p, th, ph = og.antenna_basis(rng.uniform(0.1, 3.0), rng.uniform(0, 6.2), rng.uniform(0, 6.2))
        rho, sig = rng.uniform(0.01, 1.0), rng.uniform(-3.1, 3.1)

        def kvec(r, s):
            return np.sin(r) * np.cos(s) * th + np.sin(r) * np.sin(s) * ph + np.cos(r) * p

        rho_hat, sigma_hat = og.antenna_tangents(rho, sig, th, ph, p)
        np.testing.assert_allclose(rho_hat, (kvec(rho + h, sig) - kvec(rho - h, sig)) / (2 * h), atol=1e-9)
        np.testing.assert_allclose(sigma_hat, (kvec(rho, sig + h) - kvec(rho, sig - h)) / (2 * h * math.sin(rho)),
                                   atol=1e-9)


def test_copol_at_beam_centre_is_detector_a():
    """As rho -> 0, Ludwig-3 e_co, e_cx tend to eq. copol_bolo's e_a,co and e_a,cx."""
    rng = np.random.default_rng(4)
    for _ in range(50):
        p, th, ph = og.antenna_basis(rng.uniform(0.1, 3.0), rng.uniform(0, 6.2), rng.uniform(0, 6.2))
        zeta, sig = rng.uniform(0, math.pi), rng.uniform(-3.1, 3.1)
        e_co, e_cx = og.copol_vectors(1e-9, sig, zeta, th, ph, p)
        np.testing.assert_allclose(e_co, math.cos(zeta) * th + math.sin(zeta) * ph, atol=1e-8)
        np.testing.assert_allclose(e_cx, math.sin(zeta) * th - math.cos(zeta) * ph, atol=1e-8)


def test_copol_is_unit_tangent_and_orthogonal():
    theta0, phi0, psi0, zeta, k, theta, phi, rho, sig = _configs(5, 200)
    for t in range(len(k)):
        p, th, ph = og.antenna_basis(theta0[t], phi0[t], psi0[t])
        e_co, e_cx = og.copol_vectors(rho[t], sig[t], zeta[t], th, ph, p)
        assert abs(np.linalg.norm(e_co) - 1) < 1e-14 and abs(np.linalg.norm(e_cx) - 1) < 1e-14
        assert abs(e_co @ k[t]) < 1e-14 and abs(e_cx @ k[t]) < 1e-14 and abs(e_co @ e_cx) < 1e-14


def test_chi_limit_at_beam_centre():
    """chi -> psi0 + zeta (mod pi) as the pixel approaches the pointing."""
    theta0, phi0, psi0, zeta, k, theta, phi, rho, sig = _configs(6, 500, max_sep_deg=1e-6)
    _, _, chi = og.appendix_route(theta, phi, theta0, phi0, psi0, zeta)
    d = np.mod(chi - psi0 - zeta + math.pi / 2, math.pi) - math.pi / 2
    np.testing.assert_allclose(d, 0.0, atol=1e-7)


def test_chi_special_cases():
    """Hand-solved cases on the equator: the co-pol direction of a zeta = 0 detector
    at psi0 = 0 stays along theta_hat (chi = 0) for pixels due east or due north,
    and a pixel due east of a psi0 = 90 deg pointing sees chi = 90 deg."""
    d = math.radians(3.0)
    cases = [(math.pi / 2, d, 0.0, 0.0), (math.pi / 2 - d, 0.0, 0.0, 0.0), (math.pi / 2, d, math.pi / 2, math.pi / 2)]
    for theta, phi, psi0, expect in cases:
        _, _, chi = og.appendix_route(theta, phi, math.pi / 2, 0.0, psi0, 0.0)
        assert abs(og.wrap_angle(chi - expect)) < 1e-12


def test_bilinear_reproduces_bilinear_functions_and_nodes():
    n, r = 21, math.radians(5.0)
    u = ob.nodes(n, r)
    uu, vv = np.meshgrid(u, u, indexing="xy")
    f = lambda a, b: 0.3 + 2.0 * a - 1.5 * b + 40.0 * a * b
    grid = f(uu, vv)
    rng = np.random.default_rng(7)
    pu, pv = rng.uniform(-math.sin(r), math.sin(r), (2, 1000))
    np.testing.assert_allclose(ob.bilinear(grid, pu, pv, r), f(pu, pv), atol=1e-14)
    np.testing.assert_allclose(ob.bilinear(grid, uu.ravel(), vv.ravel(), r), grid.ravel(), atol=1e-15)
    idx, w = ob.bilinear_weights(pu, pv, n, r)
    np.testing.assert_allclose((grid.ravel()[idx] * w).sum(0), f(pu, pv), atol=1e-14)


@pytest.mark.parametrize("fwhm_deg,n,radius_deg", [(1.5, 201, 5.0), (1.5, 501, 10.0), (6.0, 301, 25.0)])
def test_omega_tilde_of_gaussian_matches_1d_quadrature(fwhm_deg, n, radius_deg):
    """Omega~ of exp(-sin^2 rho / 2 s^2) by the grid rule equals 2 pi int b sin rho drho."""
    r = math.radians(radius_deg)
    s = math.radians(fwhm_deg) / math.sqrt(8 * math.log(2))
    u = ob.nodes(n, r)
    uu, vv = np.meshgrid(u, u, indexing="xy")
    grid = np.exp(-(uu * uu + vv * vv) / (2 * s * s))
    exact = 2 * math.pi * integrate.quad(lambda x: math.exp(-math.sin(x) ** 2 / (2 * s * s)) * math.sin(x),
                                         0, math.pi / 2, epsabs=0, epsrel=1e-13, limit=200)[0]
    assert abs(ob.omega_tilde(grid, r) / exact - 1) < 1e-9


def test_pixel_centres_lie_on_sphere_grid_coordinates():
    """u, v of a pixel from the appendix route equal its projections on theta'0, phi'0."""
    nside = 16
    k = hp.pix2vec(nside, np.arange(hp.npix(nside)))
    theta, phi = hp.pix2ang(nside, np.arange(hp.npix(nside)))
    t0, f0, s0 = 1.1, 2.2, 0.4
    p, th, ph = og.antenna_basis(t0, f0, s0)
    near = k @ p > math.cos(math.radians(20))
    rho, sig, _ = og.appendix_route(theta[near], phi[near], t0, f0, s0, 0.0)
    np.testing.assert_allclose(np.sin(rho) * np.cos(sig), k[near] @ th, atol=1e-13)
    np.testing.assert_allclose(np.sin(rho) * np.sin(sig), k[near] @ ph, atol=1e-13)
