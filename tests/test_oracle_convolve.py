"""Pins of the oracle's pixelised convolution and its transposes (CPU only)."""

import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import beam as ob
from oracle import convolve as oc
from oracle import geometry as og
from oracle import healpix as hp
from paper_1908_05662_gb300 import synthetic as sy


def _gauss_grid(n, radius, fwhm_deg, ell=0.0):
    return sy.gaussian_beam_maps(n, radius, fwhm_deg, ellipticity=ell, ideal=True).astype(np.float64)


def test_uniform_sky_closed_form():
    """S = (I0, 0, 0): d = (s/2)(Omega_pix/Omega~) I0 sum_k [(1+eps) B_TT + (1-eps) B_TQ]."""
    nside, r = 16, math.radians(20.0)
    grids = sy.random_beam_maps(41, 11).astype(np.float64)
    det = (0.3, 0.07, 1.3)
    omega = ob.omega_tilde(grids[0], r)
    sky = np.zeros((3, hp.npix(nside)))
    sky[0] = 2.5
    th, ph, ps = sy.random_pointings(12, 5)
    d = oc.tod(nside, r, sky, grids, det, omega, th, ph, ps)
    for t in range(len(th)):
        pix, u, v, chi = oc.disc_geometry(nside, r, th[t], ph[t], ps[t], det[0])
        btt = ob.bilinear(grids[0], u, v, r)
        btq = ob.bilinear(grids[3], u, v, r)
        expect = 0.5 * det[2] * oc.omega_pix(nside) / omega * 2.5 * np.sum((1 + det[1]) * btt + (1 - det[1]) * btq)
        assert abs(d[t] - expect) <= 1e-13 * abs(expect)


def test_uniform_sky_is_normalised():
    """A uniform unpolarised sky seen by a Gaussian beam returns (s/2)(1+eps) I0 (Sec. 3 normalisation)."""
    nside, r = 64, math.radians(12.0)
    grids = _gauss_grid(301, r, 4.0)
    omega = ob.omega_tilde(grids[0], r)
    sky = np.zeros((3, hp.npix(nside)))
    sky[0] = 1.0
    th, ph, ps = sy.random_pointings(6, 9, theta_range=(0.3, 2.8))
    d = oc.tod(nside, r, sky, grids, (0.0, 0.1, 2.0), omega, th, ph, ps)
    np.testing.assert_allclose(d, 0.5 * 2.0 * 1.1, rtol=2e-3)


def test_point_source_on_beam_centre():
    """A single bright pixel observed at its centre: rho = 0, chi = psi0 + zeta, and
    d = (s/2)(Omega_pix/Omega~)[(1+eps)(B_TT I + B_QT Q' + B_UT U') + (1-eps)(B_TQ I + B_QQ Q' + B_UQ U')]
    with Q' = Q cos 2chi + U sin 2chi, U' = -Q sin 2chi + U cos 2chi and B at the grid centre."""
    nside, r, n = 32, math.radians(6.0), 61
    grids = sy.random_beam_maps(n, 21).astype(np.float64)
    omega = ob.omega_tilde(grids[0], r)
    det = (0.4, 0.05, 0.8)
    rng = np.random.default_rng(2)
    for p in rng.integers(0, hp.npix(nside), 8):
        sky = np.zeros((3, hp.npix(nside)))
        iqu = rng.standard_normal(3)
        sky[:, p] = iqu
        th, ph = hp.pix2ang(nside, p)
        for psi0 in (0.0, 0.6, 2.0):
            d = oc.tod(nside, r, sky, grids, det, omega, [th], [ph], [psi0])[0]
            c, s = math.cos(2 * (psi0 + det[0])), math.sin(2 * (psi0 + det[0]))
            qp, up = iqu[1] * c + iqu[2] * s, -iqu[1] * s + iqu[2] * c
            b = grids[:, n // 2, n // 2]
            expect = 0.5 * det[2] * oc.omega_pix(nside) / omega * (
                (1 + det[1]) * (b[0] * iqu[0] + b[1] * qp + b[2] * up)
                + (1 - det[1]) * (b[3] * iqu[0] + b[4] * qp + b[5] * up))
            assert abs(d - expect) < 1e-12 * max(abs(expect), 1e-30)


def test_polarisation_convention():
    """Ideal beam, eps = 0: a zeta = 0 detector at psi0 = 0 sees +Q, at psi0 = 45 deg sees +U
    (Fig. 2's convention: +Q along theta_hat, +U along (theta_hat + phi_hat)/sqrt 2).
    The ratio to the uniform-I response removes the pixelisation error of the beam sum;
    chi varies across the beam by ~1e-3 rad here, so the ratio is exact to ~1e-5."""
    nside, r = 64, math.radians(8.0)
    grids = _gauss_grid(161, r, 2.0)
    omega = ob.omega_tilde(grids[0], r)
    th, ph = math.radians(80.0), 1.0
    ones = np.zeros((3, hp.npix(nside)))
    ones[0] = 1.0
    for q, u, psi0, expect in [(1, 0, 0.0, 1.0), (1, 0, math.pi / 2, -1.0), (0, 1, math.pi / 4, 1.0),
                               (0, 1, -math.pi / 4, -1.0), (1, 0, math.pi / 4, 0.0)]:
        sky = np.zeros((3, hp.npix(nside)))
        sky[1], sky[2] = q, u
        d = oc.tod(nside, r, sky, grids, (0.0, 0.0, 1.0), omega, [th], [ph], [psi0])[0]
        d1 = oc.tod(nside, r, ones, grids, (0.0, 0.0, 1.0), omega, [th], [ph], [psi0])[0]
        assert abs(d / d1 - expect) < 1e-4


def test_no_temperature_to_polarisation_leakage():
    """Axisymmetric ideal beam, I-only sky: the pair difference of orthogonal orientations,
    d(psi0) - d(psi0 + 90 deg), vanishes (Sec. 6.1.1 finds T -> P leakage zero to machine
    precision).  A square grid with axisymmetric node values maps onto itself under a 90 deg
    turn, so the bilinear beam is exactly invariant and the difference is rounding only;
    for other angles psi0 the response changes only by the interpolation error."""
    nside, r = 32, math.radians(10.0)
    grids = _gauss_grid(201, r, 3.0)
    omega = ob.omega_tilde(grids[0], r)
    sky = sy.gaussian_sky(nside, 4).numpy()
    sky[1:] = 0.0
    th, ph, ps = sy.random_pointings(6, 31, theta_range=(0.2, 2.9))
    det = (0.3, 0.0, 1.0)
    d0 = oc.tod(nside, r, sky, grids, det, omega, th, ph, ps)
    d90 = oc.tod(nside, r, sky, grids, det, omega, th, ph, ps + math.pi / 2)
    np.testing.assert_allclose(d0, d90, rtol=0, atol=1e-13 * np.max(np.abs(d0)))
    d30 = oc.tod(nside, r, sky, grids, det, omega, th, ph, ps + math.pi / 6)
    np.testing.assert_allclose(d0, d30, rtol=0, atol=1e-3 * np.max(np.abs(d0)))


def test_point_symmetric_beam_period_pi():
    """An elliptical Gaussian is symmetric under (u, v) -> (-u, -v): d(psi0 + pi) = d(psi0)."""
    nside, r = 16, math.radians(15.0)
    grids = sy.gaussian_beam_maps(101, r, 5.0, ellipticity=0.1, xpol=0.02).astype(np.float64)
    grids[3] = 0.3 * grids[0]
    omega = ob.omega_tilde(grids[0], r)
    sky = sy.gaussian_sky(nside, 6).numpy()
    th, ph, ps = sy.random_pointings(5, 3, theta_range=(0.4, 2.7))
    d1 = oc.tod(nside, r, sky, grids, (0.2, 0.03, 1.0), omega, th, ph, ps)
    d2 = oc.tod(nside, r, sky, grids, (0.2, 0.03, 1.0), omega, th, ph, ps + math.pi)
    np.testing.assert_allclose(d1, d2, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("ell", [1, 2, 3])
def test_funk_hecke_single_harmonic(ell):
    """Axisymmetric beam on I = Y_l0 about an arbitrary axis: d = (s/2) (b_l / Omega~) P_l(p0 . a) * norm,
    with b_l = 2 pi int b(rho) P_l(cos rho) sin rho drho (Funk-Hecke), to pixelisation accuracy."""
    nside, r, fwhm = 64, math.radians(20.0), 6.0
    grids = _gauss_grid(401, r, fwhm)
    omega = ob.omega_tilde(grids[0], r)
    s = math.radians(fwhm) / math.sqrt(8 * math.log(2))
    bl = 2 * math.pi * integrate.quad(lambda x: math.exp(-math.sin(x) ** 2 / (2 * s * s))
                                      * special.eval_legendre(ell, math.cos(x)) * math.sin(x),
                                      0, r, epsabs=0, epsrel=1e-12, limit=200)[0]
    axis = np.array([0.3, -0.5, 0.81])
    axis /= np.linalg.norm(axis)
    k = hp.pix2vec(nside, np.arange(hp.npix(nside)))
    sky = np.zeros((3, hp.npix(nside)))
    sky[0] = special.eval_legendre(ell, k @ axis)
    th, ph, ps = sy.random_pointings(6, 17, theta_range=(0.3, 2.8))
    d = oc.tod(nside, r, sky, grids, (0.0, 0.0, 1.0), omega, th, ph, ps)
    expect = 0.5 * bl / omega * special.eval_legendre(ell, hp.ang2vec(th, ph) @ axis)
    np.testing.assert_allclose(d, expect, atol=2e-3 * 0.5)


def test_uniform_q_sky_follows_two_psi():
    """Small ideal beam away from the poles on uniform (0, Q, U): d ~ (s/2)(Q cos 2(psi0+zeta) + U sin 2(psi0+zeta))."""
    nside, r = 64, math.radians(6.0)
    grids = _gauss_grid(161, r, 2.0)
    omega = ob.omega_tilde(grids[0], r)
    sky = np.zeros((3, hp.npix(nside)))
    sky[1], sky[2] = 0.7, -0.4
    th, ph, ps = sy.random_pointings(8, 23, theta_range=(1.0, 2.1))
    zeta = 0.35
    d = oc.tod(nside, r, sky, grids, (zeta, 0.0, 1.0), omega, th, ph, ps)
    a = 2 * (ps + zeta)
    np.testing.assert_allclose(d, 0.5 * (0.7 * np.cos(a) - 0.4 * np.sin(a)), atol=3e-3)


def test_linearity_and_sky_adjoint():
    nside, r = 8, math.radians(25.0)
    grids = sy.random_beam_maps(31, 5).astype(np.float64)
    omega = ob.omega_tilde(grids[0], r)
    det = (0.2, 0.1, 1.1)
    s1, s2 = sy.white_sky(nside, 1).numpy(), sy.white_sky(nside, 2).numpy()
    th, ph, ps = sy.random_pointings(20, 4)
    d1 = oc.tod(nside, r, s1, grids, det, omega, th, ph, ps)
    d2 = oc.tod(nside, r, s2, grids, det, omega, th, ph, ps)
    d12 = oc.tod(nside, r, 2.0 * s1 - 3.0 * s2, grids, det, omega, th, ph, ps)
    np.testing.assert_allclose(d12, 2.0 * d1 - 3.0 * d2, rtol=1e-12, atol=1e-13)
    y = np.random.default_rng(0).standard_normal(len(th))
    at_y = oc.adjoint(nside, r, grids, det, omega, th, ph, ps, y)
    assert abs(np.dot(d1, y) - np.sum(s1 * at_y)) < 1e-12 * np.sum(np.abs(d1 * y))


def test_beam_grid_adjoint_is_transpose():
    nside, r, n = 8, math.radians(25.0), 21
    grids = sy.random_beam_maps(n, 7).astype(np.float64)
    omega = ob.omega_tilde(grids[0], r)
    det = (0.7, -0.05, 0.9)
    sky = sy.white_sky(nside, 3).numpy()
    th, ph, ps = sy.random_pointings(10, 8)
    y = np.random.default_rng(1).standard_normal(len(th))
    g = oc.beam_grid_adjoint(nside, r, sky, grids, det, omega, th, ph, ps, y)
    # d is linear in the grids at fixed Omega~: <d(G), y> = <G, g>
    d = oc.tod(nside, r, sky, grids, det, omega, th, ph, ps)
    assert abs(np.dot(d, y) - np.sum(grids * g)) < 1e-12 * np.sum(np.abs(d * y))
    # and each map's gradient is the derivative: perturb one node of one map
    e, j, i = 4, n // 2 + 1, n // 2 - 2
    h = 1e-3
    gp = grids.copy(); gp[e, j, i] += h
    gm = grids.copy(); gm[e, j, i] -= h
    fd = (np.dot(oc.tod(nside, r, sky, gp, det, omega, th, ph, ps), y)
          - np.dot(oc.tod(nside, r, sky, gm, det, omega, th, ph, ps), y)) / (2 * h)
    assert abs(fd - g[e, j, i]) < 1e-9 * max(1.0, abs(fd))


def test_brute_force_all_pixel_sum():
    """Every pixel of the sphere, disc by indicator, geometry by the vector route: equals the oracle."""
    nside, r = 4, math.radians(40.0)
    grids = sy.random_beam_maps(25, 9).astype(np.float64)
    omega = ob.omega_tilde(grids[0], r)
    det = (1.1, 0.2, 0.7)
    sky = sy.white_sky(nside, 10).numpy()
    th, ph, ps = sy.random_pointings(15, 12)
    d = oc.tod(nside, r, sky, grids, det, omega, th, ph, ps)
    k = hp.pix2vec(nside, np.arange(hp.npix(nside)))
    for t in range(len(th)):
        acc = 0.0
        p0 = hp.ang2vec(th[t], ph[t])
        for pix in range(hp.npix(nside)):
            if k[pix] @ p0 < math.cos(r):
                continue
            rho, sig, chi = og.vector_route(k[pix], th[t], ph[t], ps[t], det[0])
            u, v = math.sin(rho) * math.cos(sig), math.sin(rho) * math.sin(sig)
            b = [ob.bilinear(grids[e], u, v, r) for e in range(6)]
            c, s = math.cos(2 * chi), math.sin(2 * chi)
            i_, q_, u_ = sky[:, pix]
            qp, up = q_ * c + u_ * s, -q_ * s + u_ * c
            acc += (1 + det[1]) * (b[0] * i_ + b[1] * qp + b[2] * up) + (1 - det[1]) * (b[3] * i_ + b[4] * qp + b[5] * up)
        expect = 0.5 * det[2] * oc.omega_pix(nside) / omega * acc
        assert abs(d[t] - expect) < 1e-11 * max(1.0, abs(expect))


def test_rows_u_and_v_never_reach_the_tod():
    """D Lambda(chi) = s/2 [(1+eps), (1-eps), 0, 0] for every chi (eqs. M_pol, lambda_operator)."""
    chi = np.linspace(-4, 4, 101)
    row = np.einsum("ki,kil->kl", oc.detector_row(chi, 0.2, 1.7), oc.stokes_rotation(chi))
    np.testing.assert_allclose(row, np.tile([0.85 * 1.2, 0.85 * 0.8, 0, 0], (101, 1)), atol=1e-15)


def test_nan_pointing_gives_nan():
    nside, r = 4, math.radians(20.0)
    grids = sy.random_beam_maps(11, 1).astype(np.float64)
    d = oc.tod(nside, r, np.ones((3, hp.npix(nside))), grids, (0, 0, 1), 1.0, [np.nan, 1.0], [0.0, 0.0], [0.0, 0.0])
    assert np.isnan(d[0]) and np.isfinite(d[1])


def test_worker_processes_reproduce_the_oracle():
    """The multi-process harness that times the oracle on all host cores returns exactly what
    one call of the oracle gives for the samples it processed."""
    from oracle import parallel as op
    nside, r = 8, math.radians(20.0)
    grids = sy.random_beam_maps(21, 4).astype(np.float64)
    det = (0.2, 0.05, 1.0)
    omega = ob.omega_tilde(grids[0], r)
    sky = sy.white_sky(nside, 3).numpy()
    th, ph, ps = sy.random_pointings(9, 6)
    idx, d, span, used = op.tod_sampled(nside, r, sky, grids, det, omega, th, ph, ps, processes=3, budget_s=1e9)
    assert used == 3 and span > 0
    np.testing.assert_array_equal(idx, np.arange(9))
    np.testing.assert_array_equal(d, oc.tod(nside, r, sky, grids, det, omega, th, ph, ps))
    idx, d, _, _ = op.tod_sampled(nside, r, sky, grids, det, omega, th, ph, ps, processes=2, max_per_worker=2)
    np.testing.assert_array_equal(idx, [0, 1, 4, 5])
    np.testing.assert_array_equal(d, oc.tod(nside, r, sky, grids, det, omega, th[idx], ph[idx], ps[idx]))
