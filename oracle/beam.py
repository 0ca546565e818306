"""Tangent-plane beam grids, their bilinear re-pixelisation and Omega~, FP64.  ORACLE: test infrastructure only.

The paper re-pixelises the beamsor "via interpolation" at each sky pixel's
antenna coordinates (Sec. 4.2) without naming the scheme.  The beams here are
given as six maps on an N x N grid in the plane tangent to the beam centre.
Readings (each is a choice the paper leaves open):

* grid coordinates are the orthographic (direction-cosine) coordinates
  u = sin(rho) cos(sigma) = k . theta'0 and v = sin(rho) sin(sigma) = k . phi'0;
* the grid of "radius R" spans u, v in [-sin R, sin R] with nodes
  u_i = sin(R) (2 i / (N - 1) - 1), i = 0 .. N - 1; array index [j][i] holds
  the node (u_i, v_j);
* re-pixelisation is bilinear in (u, v) on the cell that contains the point,
  the cell index clamped to [0, N - 2];
* Omega~ = integral of B_TT over the sphere (Sec. 3) is taken as the
  trapezoid rule over the whole grid with the orthographic area element
  dOmega = du dv / sqrt(1 - u^2 - v^2); the beam is zero off the grid.
"""

import numpy as np


def nodes(n, radius):
    """Node coordinates u_i (= v_i) of an n-node grid of angular radius ``radius``."""
    return np.sin(radius) * (2.0 * np.arange(n) / (n - 1) - 1.0)


def cell(u, n, radius):
    """Cell index i (clamped to [0, n - 2]) and fractional offset f of coordinate u."""
    h = 2.0 * np.sin(radius) / (n - 1)
    t = (np.asarray(u, np.float64) + np.sin(radius)) / h
    i = np.clip(np.floor(t), 0, n - 2).astype(np.int64)
    return i, t - i


def bilinear(grid, u, v, radius):
    """Bilinear value of ``grid`` ([N][N], index [j][i] = node (u_i, v_j)) at (u, v)."""
    grid = np.asarray(grid, np.float64)
    n = grid.shape[-1]
    i, fx = cell(u, n, radius)
    j, fy = cell(v, n, radius)
    g00 = grid[..., j, i]
    g10 = grid[..., j, i + 1]
    g01 = grid[..., j + 1, i]
    g11 = grid[..., j + 1, i + 1]
    return ((1 - fx) * (1 - fy) * g00 + fx * (1 - fy) * g10
            + (1 - fx) * fy * g01 + fx * fy * g11)


def bilinear_weights(u, v, n, radius):
    """Flat node indices (4, ...) and weights (4, ...) of the bilinear stencil."""
    i, fx = cell(u, n, radius)
    j, fy = cell(v, n, radius)
    idx = np.stack([j * n + i, j * n + i + 1, (j + 1) * n + i, (j + 1) * n + i + 1])
    w = np.stack([(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy])
    return idx, w


def omega_tilde(b_tt, radius):
    """Omega~ = integral of B_TT dOmega (Sec. 3), trapezoid on the orthographic grid."""
    b_tt = np.asarray(b_tt, np.float64)
    n = b_tt.shape[-1]
    u = nodes(n, radius)
    h = u[1] - u[0]
    w = np.ones(n)
    w[0] = w[-1] = 0.5
    uu, vv = np.meshgrid(u, u, indexing="xy")  # [j][i] -> (u_i, v_j)
    jac = 1.0 / np.sqrt(1.0 - uu * uu - vv * vv)
    return float(h * h * np.sum(w[:, None] * w[None, :] * b_tt * jac))


def grid_from_healpix(maps, nside_b, radius, n):
    """Tangent-plane grids (..., n, n) of beam maps given as HEALPix RING maps (..., 12 nside_b^2).

    The paper stores each beamsor element as a HEALPix map (Sec. 5.1, beam
    NSIDE 4x the sky's in Sec. 5.3 and Sec. 6).  Reading: the beam centre is
    the map's north pole and the antenna coordinates are its spherical
    coordinates, rho = theta and sigma = phi, so sigma = 0 lies along theta'0
    (u = sin rho cos sigma).  Node (u_i, v_j) takes the ring-wise bilinear
    value (``healpix.interp_weights``) at rho = arcsin(sqrt(u^2 + v^2)),
    sigma = atan2(v, u); nodes with u^2 + v^2 > 1 lie off the hemisphere and
    are zero.
    """
    from . import healpix as hp
    maps = np.asarray(maps, np.float64)
    u = nodes(n, radius)
    uu, vv = np.meshgrid(u, u, indexing="xy")  # [j][i] -> (u_i, v_j)
    r2 = uu * uu + vv * vv
    on = r2 <= 1.0
    rho = np.arcsin(np.sqrt(np.where(on, r2, 0.0)))
    sigma = np.arctan2(vv, uu)
    vals = hp.interpolate(nside_b, maps, rho, sigma)
    return np.where(on, vals, 0.0)
