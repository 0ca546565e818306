"""Parametric beam model on the library's tangent-plane grid, differentiable in torch.

The paper defers the beamsor elements to O'Dea et al. (Sec. 3); this is the
synthetic family used for benchmark inputs and beam-parameter gradients:

    g(u, v) = exp(-1/2 [(u / s_x)^2 + (v / s_y)^2]),  s = FWHM / sqrt(8 ln 2),
    s_x = s (1 + e),  s_y = s (1 - e)   (major axis along theta'0),

cross-polar leakage l gives B_TT = (1 + l) g and B_QQ = (1 - l) g, an optional
sidelobe ring a exp(-1/2 ((rho - c)/w)^2) is added to both, and the other
four maps are zero (``ideal`` gives B_TT = B_QQ = g, the Kronecker beamsor of
Sec. 3).  Nodes sit at orthographic coordinates u_i = sin(R)(2 i/(N-1) - 1),
element [j][i] = (u_i, v_j).  Parameters may be tensors with requires_grad:
the grids are then differentiable and PiscoConvolve chains the beam-grid
adjoint into d(loss)/d(FWHM, e, l).
"""

import math

import torch

FWHM_TO_SIGMA = 1.0 / math.sqrt(8.0 * math.log(2.0))


def gaussian_beam_at(u, v, fwhm_deg, ellipticity=0.0, xpol=0.0, sidelobe=None, ideal=False):
    """(6, ...) maps TT, QT, UT, TQ, QQ, UQ of the parametric beam at orthographic coordinates
    u = sin(rho) cos(sigma), v = sin(rho) sin(sigma) (tensors of one shape)."""
    t = lambda x: torch.as_tensor(x, dtype=u.dtype, device=u.device)
    s = torch.deg2rad(t(fwhm_deg)) * FWHM_TO_SIGMA
    e = t(ellipticity)
    sx, sy = s * (1.0 + e), s * (1.0 - e)
    g = torch.exp(-0.5 * ((u / sx) ** 2 + (v / sy) ** 2))
    if sidelobe is not None:
        amp, c, w = sidelobe
        rho = torch.asin(torch.clamp(torch.sqrt(u * u + v * v), max=1.0))
        g = g + amp * torch.exp(-0.5 * ((rho - math.radians(c)) / math.radians(w)) ** 2)
    zero = torch.zeros_like(g)
    if ideal:
        return torch.stack([g, zero, zero, zero, g, zero])
    xp = t(xpol)
    return torch.stack([(1.0 + xp) * g, zero, zero, zero, (1.0 - xp) * g, zero])


def gaussian_beam_grids(n, radius, fwhm_deg, ellipticity=0.0, xpol=0.0, sidelobe=None, ideal=False,
                        device="cpu", dtype=torch.float64):
    """(6, n, n) maps TT, QT, UT, TQ, QQ, UQ of the parametric beam."""
    u = math.sin(radius) * (2.0 * torch.arange(n, dtype=dtype, device=device) / (n - 1) - 1.0)
    vv, uu = torch.meshgrid(u, u, indexing="ij")  # [j][i] -> (u_i, v_j)
    return gaussian_beam_at(uu, vv, fwhm_deg, ellipticity, xpol, sidelobe, ideal)


def gaussian_beam_healpix(nside_b, fwhm_deg, ellipticity=0.0, xpol=0.0, sidelobe=None, ideal=False,
                          device="cpu", dtype=torch.float64):
    """(6, 12 nside_b^2) HEALPix RING maps of the same beam centred on the north pole, the
    paper's beam representation: pixel (theta, phi) holds the beam at rho = theta, sigma = phi.
    Pixels beyond the equator (rho > 90 deg) are zero."""
    from .synthetic import healpix_centres
    th, ph = (torch.as_tensor(a, dtype=dtype, device=device) for a in healpix_centres(nside_b))
    st = torch.sin(th)
    maps = gaussian_beam_at(st * torch.cos(ph), st * torch.sin(ph), fwhm_deg, ellipticity, xpol, sidelobe, ideal)
    return torch.where(th <= 0.5 * math.pi, maps, torch.zeros_like(maps))
