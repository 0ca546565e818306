"""Sky basis, antenna basis, antenna coordinates and chi, FP64.  ORACLE: test infrastructure only.

Two independent routes to the same numbers:

* ``appendix_route`` -- Appendix A: rho by the law of cosines, the angle alpha
  at the pointing, sigma = pi - psi0 - alpha, the angle beta at the pixel and
  chi = beta + zeta - sigma.  The appendix writes alpha and beta as
  arctan(a / b) next to explicit sin and cos expressions; they are read as
  atan2(a, b), which is what those sin/cos expressions define.
* ``vector_route``   -- Sec. 2 and Appendix A in vector form: the antenna basis
  (eq. antenna_base_vectors), k = sin rho cos sigma theta'0 + sin rho sin sigma
  phi'0 + cos rho p'0, the tangent vectors rho_hat and sigma_hat, the Ludwig-3
  co-polarisation vector e_co = cos(sigma - zeta) rho_hat
  - sin(sigma - zeta) sigma_hat, and chi as the signed angle from theta_hat at
  the pixel to e_co, positive towards phi_hat (the sense in which psi grows,
  Sec. 2, Fig. 1).

Reading of a garbled formula: Sec. 2 prints the theta'0 component of rho_hat as
cos(rho) cos(sigma) but its phi'0 component as sin(rho) sin(sigma); rho_hat is
the derivative of k with respect to rho, so that component is cos(rho)
sin(sigma).  ``tests/test_oracle_geometry.py`` checks this reading by finite
differences of k(rho, sigma).
"""

import numpy as np


def sky_basis(theta, phi):
    """p, theta_hat, phi_hat at (theta, phi): eqs. p_sky_basis, tangent_sky_basis (Sec. 2)."""
    theta = np.asarray(theta, np.float64)
    phi = np.asarray(phi, np.float64)
    st, ct = np.sin(theta), np.cos(theta)
    sp, cp = np.sin(phi), np.cos(phi)
    p = np.stack([st * cp, st * sp, ct], -1)
    th = np.stack([ct * cp, ct * sp, -st], -1)
    ph = np.stack([-sp, cp, np.zeros_like(st)], -1)
    return p, th, ph


def antenna_basis(theta0, phi0, psi0):
    """p'0, theta'0, phi'0: eq. antenna_base_vectors (Sec. 2)."""
    p, th, ph = sky_basis(theta0, phi0)
    c = np.cos(psi0)[..., None] if np.ndim(psi0) else np.cos(psi0)
    s = np.sin(psi0)[..., None] if np.ndim(psi0) else np.sin(psi0)
    th_a = c * th + s * ph
    ph_a = -s * th + c * ph
    return p, th_a, ph_a


def appendix_route(theta, phi, theta0, phi0, psi0, zeta):
    """(rho, sigma, chi) of sky direction (theta, phi) for pointing (theta0, phi0, psi0).

    Appendix A: Delta phi = phi - phi0;
    rho from the law of cosines, cos rho = cos t cos t0 + sin t sin t0 cos Dphi;
    alpha = atan2(sin t sin Dphi, cos t sin t0 - sin t cos t0 cos Dphi);
    sigma = pi - psi0 - alpha;
    beta = atan2(sin t0 sin Dphi, cos t0 sin t - sin t0 cos t cos Dphi);
    chi = beta + zeta - sigma.
    Every 1 - cos x inside these expressions is written 2 sin^2(x / 2), the
    same numbers without the cancellation that costs arccos sqrt(eps) of
    precision next to rho = 0: sin^2(rho/2) = sin^2((t - t0)/2)
    + sin t sin t0 sin^2(Dphi/2), and the second atan2 argument of alpha
    (beta) is sin(t0 - t) + 2 sin t cos t0 sin^2(Dphi/2)
    (sin(t - t0) + 2 sin t0 cos t sin^2(Dphi/2)).
    At rho = 0 both atan2 calls see (0, 0) and return 0; chi then equals
    psi0 + zeta - pi, the rho -> 0 limit modulo pi, and sigma is irrelevant.
    """
    dphi = phi - phi0
    st, ct = np.sin(theta), np.cos(theta)
    st0, ct0 = np.sin(theta0), np.cos(theta0)
    sdp = np.sin(dphi)
    hav_dphi = np.sin(0.5 * dphi) ** 2
    hav_rho = np.sin(0.5 * (theta - theta0)) ** 2 + st * st0 * hav_dphi
    rho = 2.0 * np.arcsin(np.sqrt(np.clip(hav_rho, 0.0, 1.0)))
    alpha = np.arctan2(st * sdp, np.sin(theta0 - theta) + 2.0 * st * ct0 * hav_dphi)
    sigma = np.pi - psi0 - alpha
    beta = np.arctan2(st0 * sdp, np.sin(theta - theta0) + 2.0 * st0 * ct * hav_dphi)
    chi = beta + zeta - sigma
    return rho, sigma, chi


def antenna_tangents(rho, sigma, th_a, ph_a, p_a):
    """rho_hat and sigma_hat (Sec. 2), with the cos(rho) sin(sigma) reading."""
    rho = np.asarray(rho)[..., None]
    sigma = np.asarray(sigma)[..., None]
    rho_hat = (np.cos(rho) * np.cos(sigma) * th_a + np.cos(rho) * np.sin(sigma) * ph_a
               - np.sin(rho) * p_a)
    sigma_hat = -np.sin(sigma) * th_a + np.cos(sigma) * ph_a
    return rho_hat, sigma_hat


def copol_vectors(rho, sigma, zeta, th_a, ph_a, p_a):
    """Ludwig-3 co- and cross-polarisation vectors at (rho, sigma) (Appendix A)."""
    rho_hat, sigma_hat = antenna_tangents(rho, sigma, th_a, ph_a, p_a)
    a = np.asarray(sigma - zeta)[..., None]
    e_co = np.cos(a) * rho_hat - np.sin(a) * sigma_hat
    e_cx = -np.sin(a) * rho_hat - np.cos(a) * sigma_hat
    return e_co, e_cx


def vector_route(k, theta0, phi0, psi0, zeta):
    """(rho, sigma, chi) of unit vectors k (..., 3) by the vector definitions.

    x, y, z = k . theta'0, k . phi'0, k . p'0 give rho = atan2(sqrt(x^2 + y^2), z)
    and sigma = atan2(y, x); chi = atan2(e_co . phi_hat_k, e_co . theta_hat_k).
    """
    k = np.asarray(k, np.float64)
    p_a, th_a, ph_a = antenna_basis(theta0, phi0, psi0)
    x, y, z = k @ th_a, k @ ph_a, k @ p_a
    rho = np.arctan2(np.hypot(x, y), z)
    sigma = np.arctan2(y, x)
    e_co, _ = copol_vectors(rho, sigma, zeta, th_a, ph_a, p_a)
    theta_k = np.arctan2(np.hypot(k[..., 0], k[..., 1]), k[..., 2])
    phi_k = np.arctan2(k[..., 1], k[..., 0])
    _, th_k, ph_k = sky_basis(theta_k, phi_k)
    chi = np.arctan2(np.sum(e_co * ph_k, -1), np.sum(e_co * th_k, -1))
    return rho, sigma, chi


def wrap_angle(a):
    """Angle folded into (-pi, pi]."""
    return np.pi - np.mod(np.pi - a, 2.0 * np.pi)
