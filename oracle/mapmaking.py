"""Binned map-making from TOD and the HEALPix RING pixel of a direction, FP64.
ORACLE: test infrastructure only.

The paper sends PISCO's TOD to "a map-making code" (Sec. 5.1, Fig. 3) and in
Sec. 6 makes maps from TOD in which every pixel is observed at its centre at
three position angles; it names no map-maker.  Reading: the binned (naive)
map-maker, i.e. per-pixel least squares with the pointing matrix of a delta
beam at the boresight,

    a_t = D(chi_t, eps, s)[I, Q, U]
        = s/2 [(1 + eps), (1 - eps) cos 2 chi_t, (1 - eps) sin 2 chi_t]   (eq. M_pol)

with chi_t = psi_t + zeta the co-polarisation angle at the beam centre
(Appendix A at rho = 0), and per pixel p the 3 x 3 normal equations

    (sum_{t in p} a_t a_t^T) m_p = sum_{t in p} a_t d_t .

A pixel is solved when it has at least 3 hits and the reciprocal condition
number lambda_min / lambda_max of its matrix is at least ``rcond_min``;
otherwise its I, Q, U are NaN.  Samples with non-finite angles or data, or
theta outside [0, pi], are skipped.

``ang2pix`` is the RING-scheme pixel index of Gorski et al. (2005, ApJ 622,
759, Sec. 4 and the scheme's published pixel boundaries): polar caps
(|z| > 2/3) are indexed by the two families of boundary lines through
t = nside sqrt(3 (1 - |z|)), the equatorial belt by the lines
nside (1/2 + phi / (pi/2)) -+ 3/4 nside z.
"""

import numpy as np

from . import healpix as _hp


def ang2pix(nside, theta, phi):
    """RING pixel containing direction (theta, phi), Gorski et al. (2005)."""
    theta = np.asarray(theta, np.float64)
    phi = np.asarray(phi, np.float64)
    n = int(nside)
    z = np.cos(theta)
    za = np.abs(z)
    tt = np.mod(phi, 2.0 * np.pi) / (0.5 * np.pi)  # in [0, 4)
    tt = np.where(tt >= 4.0, 0.0, tt)
    pix = np.empty(np.broadcast(theta, phi).shape, np.int64)
    pix = np.atleast_1d(pix)
    z, za, tt = (np.atleast_1d(np.broadcast_to(a, pix.shape)) for a in (z, za, tt))

    belt = za <= 2.0 / 3.0
    # equatorial belt: boundary-line indices of the ascending and descending families
    t1 = n * (0.5 + tt[belt])
    t2 = 0.75 * n * z[belt]
    jp = np.floor(t1 - t2).astype(np.int64)
    jm = np.floor(t1 + t2).astype(np.int64)
    ir = n + 1 + jp - jm                      # ring counted from z = 2/3, 1 .. 2 nside + 1
    kshift = 1 - (ir & 1)
    ip = (jp + jm - n + kshift + 1) // 2
    ip = np.mod(ip, 4 * n)
    pix[belt] = 2 * n * (n - 1) + 4 * n * (ir - 1) + ip

    cap = ~belt
    tp = tt[cap] - np.floor(tt[cap])
    tmp = n * np.sqrt(3.0 * (1.0 - za[cap]))
    jp = np.floor(tp * tmp).astype(np.int64)
    jm = np.floor((1.0 - tp) * tmp).astype(np.int64)
    ir = jp + jm + 1                          # ring counted from the nearer pole
    ip = np.floor(tt[cap] * ir).astype(np.int64)
    ip = np.mod(ip, 4 * ir)
    north = z[cap] > 0
    pix[cap] = np.where(north, 2 * ir * (ir - 1) + ip, 12 * n * n - 2 * ir * (ir + 1) + ip)
    return pix.reshape(np.broadcast(theta, phi).shape)


def pointing_rows(psi, zeta, eps, s_resp):
    """Delta-beam pointing rows a_t (n, 3) for I, Q, U (eq. M_pol at chi = psi + zeta)."""
    chi = np.asarray(psi, np.float64) + zeta
    a = np.empty(chi.shape + (3,))
    a[..., 0] = 0.5 * s_resp * (1.0 + eps)
    a[..., 1] = 0.5 * s_resp * (1.0 - eps) * np.cos(2.0 * chi)
    a[..., 2] = 0.5 * s_resp * (1.0 - eps) * np.sin(2.0 * chi)
    return a


def binned_map(nside, theta, phi, psi, det, d, rcond_min=1e-6):
    """Binned maps (3, Npix) I, Q, U and hit counts (Npix,) from one detector's TOD.

    ``det`` = (zeta, eps, s_resp); several detectors: concatenate per-detector
    normal equations with ``normal_equations`` and call ``solve``.
    """
    ata, atd, hits = normal_equations(nside, theta, phi, psi, det, d)
    return solve(ata, atd, hits, rcond_min), hits


def normal_equations(nside, theta, phi, psi, det, d):
    """Per-pixel sum a a^T (Npix, 3, 3), sum a d (Npix, 3) and hits (Npix,)."""
    theta, phi, psi, d = (np.asarray(x, np.float64) for x in (theta, phi, psi, d))
    ok = np.isfinite(theta) & np.isfinite(phi) & np.isfinite(psi) & np.isfinite(d)
    ok &= (theta >= 0.0) & (theta <= np.pi)
    npix = _hp.npix(nside)
    ata = np.zeros((npix, 3, 3))
    atd = np.zeros((npix, 3))
    hits = np.zeros(npix, np.int64)
    if not np.any(ok):
        return ata, atd, hits
    pix = ang2pix(nside, theta[ok], phi[ok])
    a = pointing_rows(psi[ok], det[0], det[1], det[2])
    np.add.at(ata, pix, a[:, :, None] * a[:, None, :])
    np.add.at(atd, pix, a * d[ok][:, None])
    np.add.at(hits, pix, 1)
    return ata, atd, hits


def solve(ata, atd, hits, rcond_min=1e-6):
    """m_p = (sum a a^T)^-1 sum a d where hits >= 3 and lambda_min / lambda_max >= rcond_min."""
    maps = np.full((3, ata.shape[0]), np.nan)
    for p in np.nonzero(hits >= 3)[0]:
        lam = np.linalg.eigvalsh(ata[p])
        if lam[-1] > 0 and lam[0] / lam[-1] >= rcond_min:
            maps[:, p] = np.linalg.solve(ata[p], atd[p])
    return maps
