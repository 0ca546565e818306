"""HEALPix RING pixel centres and the disc query, FP64.  ORACLE: test infrastructure only.

The paper stores sky and beamsor as HEALPix maps (Sec. 5.1, citing Gorski et
al. 2005).  The convolution needs only the pixel centres in RING order:

* rings i = 1 .. 4 nside - 1, ordered north to south;
* north polar cap (i < nside): z_i = 1 - i^2 / (3 nside^2), 4 i pixels,
  phi_j = (j + 1/2) * pi / (2 i);
* equatorial belt (nside <= i <= 3 nside): z_i = 4/3 - 2 i / (3 nside),
  4 nside pixels, phi_j = (j + s/2) * pi / (2 nside) with
  s = (i - nside + 1) mod 2 (neighbouring rings are staggered by half a pixel);
* south polar cap: mirror image of the north cap (z -> -z, same phi layout);
* pixel numbers run ring by ring, j = 0 .. n_i - 1 inside a ring.

The disc query follows Sec. 5.2 (the list of sky pixels "inside" the
beamsor extension) cut at rho_max (Sec. 5.3, Table 1): a pixel belongs to the
disc of pointing p0 when its centre k satisfies  k . p0 >= cos(rho_max)
(centre-in-disc, inclusive).  ``query_disc_brute`` applies that test to every
pixel of the sphere; ``query_disc`` visits only the rings that can intersect
the disc and applies the same test to a superset of candidates per ring.
"""

import numpy as np


def npix(nside):
    """Number of pixels of a HEALPix map, 12 nside^2."""
    return 12 * nside * nside


def ring_table(nside):
    """Per-ring geometry for rings i = 1 .. 4 nside - 1 (array index i - 1).

    Returns a dict of arrays: ``z`` (cos theta of the ring), ``sin_theta``,
    ``count`` (pixels in the ring), ``first`` (pixel number of j = 0),
    ``phi0`` (phi of j = 0) and ``dphi`` (phi step).
    """
    n = int(nside)
    i = np.arange(1, 4 * n, dtype=np.int64)
    z = np.empty(i.shape, np.float64)
    one_minus_z = np.empty(i.shape, np.float64)
    count = np.empty(i.shape, np.int64)
    phi0 = np.empty(i.shape, np.float64)
    dphi = np.empty(i.shape, np.float64)

    north = i < n
    south = i > 3 * n
    belt = ~north & ~south

    ic = i[north].astype(np.float64)
    one_minus_z[north] = ic * ic / (3.0 * n * n)
    z[north] = 1.0 - one_minus_z[north]
    count[north] = 4 * i[north]
    dphi[north] = np.pi / (2.0 * ic)
    phi0[north] = 0.5 * dphi[north]

    ib = i[belt]
    z[belt] = 4.0 / 3.0 - 2.0 * ib / (3.0 * n)
    one_minus_z[belt] = 1.0 - z[belt]
    count[belt] = 4 * n
    dphi[belt] = np.pi / (2.0 * n)
    shift = (ib - n + 1) % 2
    phi0[belt] = 0.5 * shift * dphi[belt]

    im = (4 * n - i[south]).astype(np.float64)  # mirrored ring number
    z[south] = -(1.0 - im * im / (3.0 * n * n))
    one_minus_z[south] = 1.0 - z[south]
    count[south] = 4 * (4 * n - i[south])
    dphi[south] = np.pi / (2.0 * im)
    phi0[south] = 0.5 * dphi[south]

    # sin(theta) from (1 - z)(1 + z) keeps full precision next to the poles.
    sin_theta = np.sqrt(one_minus_z * (1.0 + z))
    first = np.concatenate([[0], np.cumsum(count)[:-1]]).astype(np.int64)
    return dict(z=z, sin_theta=sin_theta, count=count, first=first,
                phi0=phi0, dphi=dphi)


def pix2ring(nside, pix):
    """Ring array index (0-based) and in-ring position j of RING pixels."""
    t = ring_table(nside)
    pix = np.asarray(pix, dtype=np.int64)
    r = np.searchsorted(t["first"], pix, side="right") - 1
    return r, pix - t["first"][r]


def pix2ang(nside, pix):
    """Colatitude theta and longitude phi of RING pixel centres."""
    t = ring_table(nside)
    r, j = pix2ring(nside, pix)
    theta = np.arctan2(t["sin_theta"][r], t["z"][r])
    phi = t["phi0"][r] + j * t["dphi"][r]
    return theta, phi


def pix2vec(nside, pix):
    """Unit vectors (..., 3) of RING pixel centres (sky basis x, y, z)."""
    t = ring_table(nside)
    r, j = pix2ring(nside, pix)
    phi = t["phi0"][r] + j * t["dphi"][r]
    s = t["sin_theta"][r]
    return np.stack([s * np.cos(phi), s * np.sin(phi), t["z"][r]], axis=-1)


def ang2vec(theta, phi):
    """Unit vector of (theta, phi), eq. p_sky_basis (Sec. 2)."""
    st = np.sin(theta)
    return np.stack([st * np.cos(phi), st * np.sin(phi), np.cos(theta)], axis=-1)


def in_disc(k, p0, cos_r):
    """Membership test k . p0 >= cos(radius), evaluated in one fixed order."""
    return k[..., 0] * p0[0] + k[..., 1] * p0[1] + k[..., 2] * p0[2] >= cos_r


def query_disc_brute(nside, theta0, phi0, radius):
    """All RING pixels whose centre k satisfies k . p0 >= cos(radius), sorted."""
    k = pix2vec(nside, np.arange(npix(nside)))
    p0 = ang2vec(theta0, phi0)
    return np.nonzero(in_disc(k, p0, np.cos(radius)))[0]


def query_disc(nside, theta0, phi0, radius):
    """Same set as ``query_disc_brute``, visiting only the rings that can meet the disc.

    For each ring whose colatitude lies within ``radius`` of theta0, the
    candidates are the pixels whose phi lies within the largest possible
    half-width of the disc on that ring plus one pixel of margin; every
    candidate then takes the same k . p0 >= cos(radius) test.
    """
    t = ring_table(nside)
    p0 = ang2vec(theta0, phi0)
    cos_r = np.cos(radius)
    theta_r = np.arctan2(t["sin_theta"], t["z"])
    near = np.abs(theta_r - theta0) <= radius + 1e-9
    out = []
    s0 = np.sin(theta0)
    z0 = np.cos(theta0)
    for r in np.nonzero(near)[0]:
        z, s, cnt = t["z"][r], t["sin_theta"][r], int(t["count"][r])
        denom = s * s0
        if denom <= 1e-9:
            js = np.arange(cnt)
        else:
            c = (cos_r - z * z0) / denom
            if c <= -1.0:
                js = np.arange(cnt)
            elif c > 1.0 + 1e-9:
                continue
            else:
                half = np.arccos(min(c, 1.0))
                lo = int(np.floor((phi0 - half - t["phi0"][r]) / t["dphi"][r])) - 1
                hi = int(np.ceil((phi0 + half - t["phi0"][r]) / t["dphi"][r])) + 1
                if hi - lo + 1 >= cnt:
                    js = np.arange(cnt)
                else:
                    js = np.unique(np.mod(np.arange(lo, hi + 1), cnt))
        pix = t["first"][r] + js
        phi = t["phi0"][r] + js * t["dphi"][r]
        k = np.stack([s * np.cos(phi), s * np.sin(phi), np.full(phi.shape, z)], -1)
        out.append(pix[in_disc(k, p0, cos_r)])
    if not out:
        return np.zeros(0, np.int64)
    return np.sort(np.concatenate(out))


def ring_theta(nside):
    """Colatitudes theta_i of rings i = 1 .. 4 nside - 1 (array index i - 1), increasing."""
    t = ring_table(nside)
    return np.arctan2(t["sin_theta"], t["z"])


def interp_weights(nside, theta, phi):
    """Four RING pixels and weights of the ring-wise bilinear interpolation at (theta, phi).

    The paper re-pixelises HEALPix beam maps "via interpolation" (Sec. 4.2,
    Sec. 5.1) without naming the scheme; this is the reading used here:

    * on a ring, linear in phi between the two pixel centres that bracket phi
      (the ring is periodic, so the pair may straddle phi = 0);
    * between the rings i and i + 1 that bracket theta (theta_i <= theta <
      theta_{i+1}), linear in theta between the two on-ring values;
    * above the first ring (theta < theta_1) the value is extrapolated from
      rings 1 and 2, quadratic in theta: with w = (theta^2 - theta_1^2) /
      (theta_2^2 - theta_1^2) <= 0 it is (1 - w) ring_1 + w ring_2 (a smooth
      map is even in theta near the pole, and a beam has its peak there: the
      pole value is extrapolated, not averaged from ring 1); the south cap is
      the mirror image with the last two rings and pi - theta.

    Returns (pix, w), each of shape (4,) + shape(theta): two pixels on each
    of two rings.  The weights sum to one; they are non-negative except in
    the polar caps, where the farther ring's are <= 0.
    """
    theta = np.asarray(theta, np.float64)
    phi = np.asarray(phi, np.float64)
    shape = np.broadcast(theta, phi).shape
    theta = np.broadcast_to(theta, shape).ravel()
    phi = np.broadcast_to(phi, shape).ravel()
    t = ring_table(nside)
    th_r = ring_theta(nside)
    nr = th_r.shape[0]
    pix = np.zeros((4, theta.size), np.int64)
    w = np.zeros((4, theta.size), np.float64)

    def on_ring(r, ph):
        """Two bracketing pixels of ring index r and their phi weights."""
        cnt, dphi = t["count"][r], t["dphi"][r]
        x = (ph - t["phi0"][r]) / dphi
        j0 = np.floor(x)
        f = x - j0
        j0 = np.mod(j0.astype(np.int64), cnt)
        j1 = np.mod(j0 + 1, cnt)
        return t["first"][r] + j0, t["first"][r] + j1, 1.0 - f, f

    for k in range(theta.size):
        th, ph = theta[k], phi[k]
        if th < th_r[0]:  # north cap: rings 1, 2
            r, wt = 0, (th * th - th_r[0] ** 2) / (th_r[1] ** 2 - th_r[0] ** 2)
        elif th >= th_r[-1]:  # south cap: the last two rings, mirrored
            r, a, b, c = nr - 2, np.pi - th, np.pi - th_r[-1], np.pi - th_r[-2]
            wt = 1.0 - (a * a - b * b) / (c * c - b * b)
        else:
            r = int(np.searchsorted(th_r, th, side="right")) - 1  # th_r[r] <= th < th_r[r + 1]
            wt = (th - th_r[r]) / (th_r[r + 1] - th_r[r])
        p0, p1, a0, a1 = on_ring(r, ph)
        q0, q1, b0, b1 = on_ring(r + 1, ph)
        pix[:, k] = [p0, p1, q0, q1]
        w[:, k] = [(1 - wt) * a0, (1 - wt) * a1, wt * b0, wt * b1]
    return pix.reshape((4,) + shape), w.reshape((4,) + shape)


def interpolate(nside, m, theta, phi):
    """Ring-wise bilinear value of map(s) m (..., Npix) at (theta, phi) (``interp_weights``)."""
    pix, w = interp_weights(nside, theta, phi)
    return np.sum(np.asarray(m, np.float64)[..., pix] * w, axis=-pix.ndim)
