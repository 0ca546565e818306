"""The pixelised PISCO convolution and its transposes, FP64.  ORACLE: test infrastructure only.

One TOD sample (Sec. 4.2, eq. discrete_beam_conv_tensor):

    d(q0) = sum_k  D_i(chi_k, eps, s) Lambda^i_l(chi_k) B^l_j(rho_k, sigma_k) Lambda^j_m(-chi_k) S^m_k

over the sky pixels k inside the disc of radius R around the pointing q0 =
(theta0, phi0, psi0), with

* D(chi, eps, s) = s/2 [(1 + eps), (1 - eps) cos 2chi, (1 - eps) sin 2chi, 0]
  (eq. M_pol, Sec. 4.1); the argument is chi as in eq. pisco_equation_cont;
* Lambda(chi) the Stokes rotation of eq. lambda_operator;
* B = (1 / Omega~) [B_ij] the beamsor (eq. beamsor, Sec. 3), rows
  l = T, Q, U, V and columns j = T, Q, U, V, so that row T holds
  (B_TT, B_QT, B_UT, B_VT) and row Q holds (B_TQ, B_QQ, B_UQ, B_VQ);
* S = (I, Q, U, V) with V = 0 (Sec. 6.2: the CMB has no V).

Six beam maps are given, in the order TT, QT, UT, TQ, QQ, UQ; every other
element is zero.  Rows U and V of B never reach d because D Lambda(chi) =
s/2 [(1 + eps), (1 - eps), 0, 0] for every chi.

Reading of the measure: the pixel sum replaces the integral of eq.
pisco_equation_cont, whose measure dOmega becomes the (equal) pixel area
Omega_pix = 4 pi / (12 nside^2); the sum is multiplied by Omega_pix.

The oracle evaluates that contraction literally per pixel, 4 x 4 matrices and
all, with (rho, sigma, chi) from the Appendix A route and the beamsor
re-pixelised bilinearly on the tangent-plane grid (``oracle.beam``).
"""

import numpy as np

from . import beam as _beam
from . import geometry as _geo
from . import healpix as _hp

MAP_ORDER = ("TT", "QT", "UT", "TQ", "QQ", "UQ")
_STOKES = "TQUV"


def omega_pix(nside):
    """Area of one HEALPix pixel, 4 pi / (12 nside^2)."""
    return 4.0 * np.pi / _hp.npix(nside)


def stokes_rotation(chi):
    """Lambda(chi) (..., 4, 4), eq. lambda_operator."""
    chi = np.asarray(chi, np.float64)
    c, s = np.cos(2.0 * chi), np.sin(2.0 * chi)
    lam = np.zeros(chi.shape + (4, 4))
    lam[..., 0, 0] = 1.0
    lam[..., 1, 1] = c
    lam[..., 1, 2] = -s
    lam[..., 2, 1] = s
    lam[..., 2, 2] = c
    lam[..., 3, 3] = 1.0
    return lam


def detector_row(chi, eps, s_resp):
    """D(chi, eps, s) (..., 4), eq. M_pol."""
    chi = np.asarray(chi, np.float64)
    d = np.zeros(chi.shape + (4,))
    d[..., 0] = 0.5 * s_resp * (1.0 + eps)
    d[..., 1] = 0.5 * s_resp * (1.0 - eps) * np.cos(2.0 * chi)
    d[..., 2] = 0.5 * s_resp * (1.0 - eps) * np.sin(2.0 * chi)
    return d


def beamsor(grids, u, v, radius):
    """Unnormalised beamsor [B_ij] (..., 4, 4) re-pixelised at (u, v); rows = l, columns = j."""
    b = np.zeros(np.shape(u) + (4, 4))
    for e, name in enumerate(MAP_ORDER):
        col = _STOKES.index(name[0])  # input Stokes (j)
        row = _STOKES.index(name[1])  # output Stokes (l)
        b[..., row, col] = _beam.bilinear(grids[e], u, v, radius)
    return b


def disc_geometry(nside, radius, theta0, phi0, psi0, zeta):
    """Disc pixels of one pointing and their (u, v, chi)."""
    pix = _hp.query_disc(nside, theta0, phi0, radius)
    theta_k, phi_k = _hp.pix2ang(nside, pix)
    rho, sigma, chi = _geo.appendix_route(theta_k, phi_k, theta0, phi0, psi0, zeta)
    u = np.sin(rho) * np.cos(sigma)
    v = np.sin(rho) * np.sin(sigma)
    return pix, u, v, chi


def sample_weights(nside, radius, grids, det, omega, theta0, phi0, psi0):
    """Disc pixels and weights w (m, 3) with d = sum_k w_k . (I_k, Q_k, U_k).

    The weights are the literal contraction D Lambda(chi) (B / Omega~)
    Lambda(-chi) restricted to the I, Q, U columns, times Omega_pix.
    ``det`` = (zeta, eps, s_resp); ``omega`` = Omega~.
    """
    zeta, eps, s_resp = det
    pix, u, v, chi = disc_geometry(nside, radius, theta0, phi0, psi0, zeta)
    b = beamsor(grids, u, v, radius) / omega
    row = np.einsum("ki,kil->kl", detector_row(chi, eps, s_resp), stokes_rotation(chi))
    m = np.einsum("kl,klj,kjm->km", row, b, stokes_rotation(-chi))
    return pix, omega_pix(nside) * m[:, :3]


def tod(nside, radius, sky, grids, det, omega, theta0, phi0, psi0):
    """TOD samples d(q0) for pointings (theta0, phi0, psi0); sky is (3, Npix) I, Q, U."""
    sky = np.asarray(sky, np.float64)
    theta0 = np.atleast_1d(np.asarray(theta0, np.float64))
    phi0 = np.atleast_1d(np.asarray(phi0, np.float64))
    psi0 = np.atleast_1d(np.asarray(psi0, np.float64))
    out = np.empty(theta0.shape[0])
    for t in range(theta0.shape[0]):
        if not (np.isfinite(theta0[t]) and np.isfinite(phi0[t]) and np.isfinite(psi0[t])):
            out[t] = np.nan
            continue
        pix, w = sample_weights(nside, radius, grids, det, omega, theta0[t], phi0[t], psi0[t])
        out[t] = np.sum(w * sky[:, pix].T)
    return out


def adjoint(nside, radius, grids, det, omega, theta0, phi0, psi0, y):
    """Transpose with respect to the sky: maps (3, Npix) = sum_t y_t dd_t / d(I, Q, U)."""
    maps = np.zeros((3, _hp.npix(nside)))
    for t in range(len(y)):
        pix, w = sample_weights(nside, radius, grids, det, omega, theta0[t], phi0[t], psi0[t])
        np.add.at(maps.T, pix, y[t] * w)
    return maps


def beam_grid_adjoint(nside, radius, sky, grids, det, omega, theta0, phi0, psi0, y):
    """Transpose with respect to the six beam grids, Omega~ held fixed.

    Returns g (6, N, N) with g[e] = sum_t y_t dd_t / d grids[e].  Each map
    element enters d through one beamsor entry B^l_j, multiplied by the
    matching components of D Lambda(chi) and Lambda(-chi) S, and reaches the
    grid through the four bilinear weights of its cell.
    """
    zeta, eps, s_resp = det
    sky = np.asarray(sky, np.float64)
    n = np.asarray(grids).shape[-1]
    g = np.zeros((6, n * n))
    for t in range(len(y)):
        pix, u, v, chi = disc_geometry(nside, radius, theta0[t], phi0[t], psi0[t], zeta)
        row = np.einsum("ki,kil->kl", detector_row(chi, eps, s_resp), stokes_rotation(chi))
        s4 = np.zeros((len(pix), 4))
        s4[:, :3] = sky[:, pix].T
        rot = np.einsum("kjm,km->kj", stokes_rotation(-chi), s4)
        idx, wts = _beam.bilinear_weights(u, v, n, radius)
        for e, name in enumerate(MAP_ORDER):
            col = _STOKES.index(name[0])
            rw = _STOKES.index(name[1])
            coef = y[t] * omega_pix(nside) / omega * row[:, rw] * rot[:, col]
            for c in range(4):
                np.add.at(g[e], idx[c], coef * wts[c])
    return g.reshape(6, n, n)


def disc_count(nside, radius, theta0, phi0):
    """Number of disc pixels per pointing."""
    return np.array([len(_hp.query_disc(nside, a, b, radius))
                     for a, b in zip(np.atleast_1d(theta0), np.atleast_1d(phi0))])
