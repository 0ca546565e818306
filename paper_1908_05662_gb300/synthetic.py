"""Seeded synthetic inputs: CMB-like skies, scans and beam grids.

This module only *makes inputs*; it holds none of the convolution's
arithmetic (no disc query, no antenna frame, no interpolation, no Stokes
rotation).  Tests feed the same arrays to the CUDA library and to the FP64
oracle, and ``bench.py`` uses it to build the benchmark workloads.

* ``gaussian_sky``  -- a Gaussian random field with angular power spectrum
  C_l ~ l^slope (l >= 2, C_0 = C_1 = 0), synthesised from random a_lm on the
  pixel centres of a HEALPix RING map (the data format of the paper's sky
  maps, Sec. 5.1).  Q and U are independent fields of the same spectrum
  scaled to ``pol_frac`` of the I rms.  It stands in for the CAMB + synfast
  maps of Sec. 6.2, which need tools and parameters this project does not
  have.
* scans -- a constant-elevation raster, a constant-elevation azimuth scan
  with sidereal drift and daily boresight rotation (the CLASS-like strategy
  of Sec. 7.1, with synthetic site and timing), focal-plane offsets, and
  uniformly random pointings.
* beams -- six tangent-plane maps (TT, QT, UT, TQ, QQ, UQ) of an elliptical
  Gaussian main beam with optional sidelobe ring and cross-polar leakage (the
  parametric model of ``beams``), or random smooth maps for parity tests.  Grid nodes sit at orthographic
  coordinates u_i = sin(R) (2 i / (N - 1) - 1), the library's grid format.
"""

import math

import numpy as np
import torch

FWHM_TO_SIGMA = 1.0 / math.sqrt(8.0 * math.log(2.0))


# --------------------------------------------------------------------------
# sky
# --------------------------------------------------------------------------

def _ring_layout(nside):
    """z, phi of pixel 0, and pixel count of every RING ring (the map format)."""
    n = nside
    out = []
    for i in range(1, 4 * n):
        if i < n:
            out.append((1.0 - i * i / (3.0 * n * n), math.pi / (4 * i), 4 * i))
        elif i <= 3 * n:
            s = (i - n + 1) % 2
            out.append((4.0 / 3.0 - 2.0 * i / (3.0 * n), 0.5 * s * math.pi / (2 * n), 4 * n))
        else:
            m = 4 * n - i
            out.append((-(1.0 - m * m / (3.0 * n * n)), math.pi / (4 * m), 4 * m))
    return out


def _alm(lmax, slope, gen):
    """Random a_lm (complex, [l][m], m <= l) with C_l = l^slope for l >= 2."""
    ell = torch.arange(lmax + 1, dtype=torch.float64)
    cl = torch.zeros(lmax + 1, dtype=torch.float64)
    cl[2:] = ell[2:] ** slope
    re = torch.randn(lmax + 1, lmax + 1, generator=gen, dtype=torch.float64)
    im = torch.randn(lmax + 1, lmax + 1, generator=gen, dtype=torch.float64)
    m = torch.arange(lmax + 1)
    scale = torch.sqrt(cl)[:, None] * torch.where(m[None, :] == 0, 1.0, math.sqrt(0.5))
    a = torch.complex(re * scale, torch.where(m[None, :] == 0, 0.0, im * scale))
    mask = m[None, :] <= torch.arange(lmax + 1)[:, None]
    return a * mask


def _synthesise(alms, nside, device):
    """Maps (len(alms), Npix) of real fields with the given a_lm, on RING pixel centres."""
    layout = _ring_layout(nside)
    lmax = alms[0].shape[0] - 1
    # North rings and the equator; the south follows from P_lm(-z) = (-1)^(l+m) P_lm(z).
    nr = 2 * nside
    z = torch.tensor([layout[r][0] for r in range(nr)], dtype=torch.float64, device=device)
    st = torch.sqrt((1.0 - z) * (1.0 + z))
    nf = len(alms)
    a = torch.stack([x.to(device) for x in alms])                 # (F, L, M)
    m = torch.arange(lmax + 1, device=device, dtype=torch.float64)
    even = torch.zeros(nf, lmax + 1, nr, dtype=torch.complex128, device=device)
    odd = torch.zeros_like(even)
    # Normalised associated Legendre functions by the standard three-term recursion in l.
    lam_mm = torch.zeros(lmax + 1, nr, dtype=torch.float64, device=device)
    lam_mm[0] = 1.0 / math.sqrt(4.0 * math.pi)
    for mm in range(1, lmax + 1):
        lam_mm[mm] = -math.sqrt((2 * mm + 1) / (2.0 * mm)) * st * lam_mm[mm - 1]
    prev2 = torch.zeros(lmax + 1, nr, dtype=torch.float64, device=device)
    prev1 = torch.zeros(lmax + 1, nr, dtype=torch.float64, device=device)
    for ell in range(lmax + 1):
        cur = torch.zeros(lmax + 1, nr, dtype=torch.float64, device=device)
        cur[ell] = lam_mm[ell]
        if ell >= 1:
            cur[ell - 1] = math.sqrt(2 * ell + 1) * z * prev1[ell - 1]
        if ell >= 2:
            mv = m[: ell - 1]
            a1 = torch.sqrt((4.0 * ell * ell - 1.0) / (ell * ell - mv * mv))
            a2 = torch.sqrt(((ell - 1.0) ** 2 - mv * mv) / (4.0 * (ell - 1.0) ** 2 - 1.0))
            cur[: ell - 1] = a1[:, None] * (z[None, :] * prev1[: ell - 1] - a2[:, None] * prev2[: ell - 1])
        contrib = a[:, ell, :, None] * cur[None, :, :]             # (F, M, R)
        sign_even = ((ell + torch.arange(lmax + 1, device=device)) % 2 == 0)
        even += torch.where(sign_even[None, :, None], contrib, torch.zeros_like(contrib))
        odd += torch.where(sign_even[None, :, None], torch.zeros_like(contrib), contrib)
        prev2, prev1 = prev1, cur
    # Each ring is a real Fourier series in phi: fold m into the ring's bins and
    # inverse-FFT.  The 2 nside + 1 belt rings share one length and go in one batch.
    cm = torch.where(m == 0, 1.0, 2.0).to(torch.complex128)
    midx = torch.arange(lmax + 1, device=device)

    def ring_coeffs(f, rows):
        north = torch.tensor([r if r < nr else 4 * nside - 2 - r for r in rows], device=device)
        sgn = torch.tensor([1.0 if r < nr else -1.0 for r in rows], dtype=torch.float64, device=device)
        fm = even[f][:, north].T + sgn[:, None] * odd[f][:, north].T          # (rows, M)
        phi0 = torch.tensor([layout[r][1] for r in rows], dtype=torch.float64, device=device)
        return cm[None, :] * fm * torch.exp(1j * m[None, :] * phi0[:, None])

    belt = list(range(nside - 1, 3 * nside))
    maps = []
    for f in range(nf):
        out = torch.empty(12 * nside * nside, dtype=torch.float64, device=device)
        coef = ring_coeffs(f, belt)
        folded = torch.zeros(len(belt), 4 * nside, dtype=torch.complex128, device=device)
        folded.index_add_(1, midx % (4 * nside), coef)
        vals = torch.real(torch.fft.ifft(folded, dim=1) * (4 * nside))
        start = 2 * nside * (nside - 1)
        out[start:start + vals.numel()] = vals.reshape(-1)
        first = 0
        for r in range(4 * nside - 1):
            cnt = layout[r][2]
            if not (nside - 1 <= r < 3 * nside):
                c = ring_coeffs(f, [r])[0]
                folded = torch.zeros(cnt, dtype=torch.complex128, device=device)
                folded.index_add_(0, midx % cnt, c)
                out[first:first + cnt] = torch.real(torch.fft.ifft(folded) * cnt)
            first += cnt
        maps.append(out)
    return torch.stack(maps)


def gaussian_sky(nside, seed, slope=-2.0, pol_frac=0.1, lmax=None, device="cpu"):
    """(3, 12 nside^2) float64 I, Q, U maps in RING order, I with unit rms."""
    lmax = 3 * nside - 1 if lmax is None else lmax
    gen = torch.Generator().manual_seed(int(seed))
    alms = [_alm(lmax, slope, gen) for _ in range(3)]
    maps = _synthesise(alms, nside, device)
    maps = maps / maps.std(dim=1, keepdim=True)
    maps[1:] *= pol_frac
    return maps


def uniform_sky(nside, i=1.0, q=0.0, u=0.0, device="cpu"):
    """Constant I, Q, U maps."""
    npix = 12 * nside * nside
    return torch.tensor([i, q, u], dtype=torch.float64, device=device)[:, None].expand(3, npix).clone()


def white_sky(nside, seed, device="cpu"):
    """Independent N(0, 1) values for I, Q, U in every pixel."""
    gen = torch.Generator().manual_seed(int(seed))
    return torch.randn(3, 12 * nside * nside, generator=gen, dtype=torch.float64).to(device)


# --------------------------------------------------------------------------
# scans
# --------------------------------------------------------------------------

def random_pointings(n, seed, theta_range=(0.0, math.pi)):
    """Uniform directions (theta restricted to ``theta_range``) and uniform psi, float64 numpy."""
    rng = np.random.default_rng(seed)
    zlo, zhi = math.cos(theta_range[1]), math.cos(theta_range[0])
    theta = np.arccos(rng.uniform(zlo, zhi, n))
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    psi = rng.uniform(0.0, 2.0 * math.pi, n)
    return theta, phi, psi


def raster_scan(n, center=(math.radians(60.0), math.radians(45.0)), half_size=math.radians(5.0),
                rows=100):
    """Constant-colatitude raster over a square field; psi steps uniformly over [0, 2 pi).

    ``rows`` rows of constant theta0 from center - half_size to center + half_size,
    each sweeping phi0 across the field (width 2 half_size / sin theta0).
    """
    t = np.arange(n)
    per_row = int(math.ceil(n / rows))
    row = t // per_row
    frac = (t % per_row) / max(per_row - 1, 1)
    theta = center[0] - half_size + 2.0 * half_size * row / max(rows - 1, 1)
    phi = center[1] + (2.0 * frac - 1.0) * half_size / np.sin(theta)
    psi = 2.0 * math.pi * t / n
    return theta, phi, psi


def ces_scan(n, rate_hz=20.0, latitude_deg=-23.0, elevation_deg=45.0, az_speed_deg=1.0,
             az_span_deg=720.0, boresight_deg=(-45.0, -30.0, -15.0, 0.0, 15.0, 30.0, 45.0),
             lst0=0.0, offset=None, device="cpu", start=0):
    """Constant-elevation azimuth scan, float64 (theta, phi, psi) torch tensors: samples
    start .. start + n - 1 of the scan.

    The azimuth sweeps a triangle wave over ``az_span_deg`` at ``az_speed_deg``
    per second; the sky turns at the sidereal rate; the boresight angle
    steps daily through ``boresight_deg``.  psi is the parallactic angle plus
    the boresight angle.  ``offset`` = (dx, dy) radians places a detector off
    the boresight in the focal plane (dx along the elevation axis).
    """
    f64 = torch.float64
    t = torch.arange(start, start + n, dtype=f64, device=device) / rate_hz
    period = 2.0 * az_span_deg / az_speed_deg
    ph = torch.remainder(t, period) / period
    az = torch.deg2rad(az_span_deg * torch.where(ph < 0.5, 2.0 * ph, 2.0 - 2.0 * ph))
    el = torch.full_like(t, math.radians(elevation_deg))
    day = torch.floor(t / 86400.0).long() % len(boresight_deg)
    bore = torch.deg2rad(torch.tensor(boresight_deg, dtype=f64, device=device))[day]
    if offset is not None:
        dx, dy = offset
        # Rotate the focal-plane offset by the boresight angle and apply it on the
        # horizon sphere (small-angle placement is enough for synthetic detectors).
        cb, sb = torch.cos(bore), torch.sin(bore)
        de = dx * cb - dy * sb
        da = dx * sb + dy * cb
        el = el + de
        az = az + da / torch.cos(el)
    lat = math.radians(latitude_deg)
    sin_dec = math.sin(lat) * torch.sin(el) + math.cos(lat) * torch.cos(el) * torch.cos(az)
    dec = torch.asin(torch.clamp(sin_dec, -1.0, 1.0))
    ha = torch.atan2(-torch.sin(az) * torch.cos(el),
                     math.cos(lat) * torch.sin(el) - math.sin(lat) * torch.cos(el) * torch.cos(az))
    lst = lst0 + 2.0 * math.pi * t / 86164.0905
    ra = torch.remainder(lst - ha, 2.0 * math.pi)
    par = torch.atan2(torch.sin(ha), math.tan(lat) * torch.cos(dec) - torch.sin(dec) * torch.cos(ha))
    theta = 0.5 * math.pi - dec
    psi = torch.remainder(par + bore, 2.0 * math.pi)
    return theta, ra, psi


def healpix_centres(nside):
    """(theta, phi) float64 of every RING pixel centre (pointings on pixel centres)."""
    th, ph = [], []
    for z, phi0, cnt in _ring_layout(nside):
        th.append(np.full(cnt, math.atan2(math.sqrt((1.0 - z) * (1.0 + z)), z)))
        ph.append(phi0 + np.arange(cnt) * (2.0 * math.pi / cnt))
    return np.concatenate(th), np.concatenate(ph)


def pixel_centre_pointings(nside, n, seed):
    """Pointings exactly on ``n`` seeded RING pixel centres (rho = 0 for that pixel, as in the
    paper's Table 1 and Sec. 6 runs), with uniform psi; float64 numpy (theta, phi, psi, pix)."""
    rng = np.random.default_rng(seed)
    th, ph = healpix_centres(nside)
    pix = rng.choice(len(th), n, replace=False)
    return th[pix], ph[pix], rng.uniform(0.0, 2.0 * math.pi, n), pix


def disc_edge_pointings(nside, radius, n, seed, delta=1e-12):
    """Pointings at angular distance radius - delta (even entries) or radius + delta (odd
    entries) from a seeded RING pixel centre, in a seeded direction: that pixel lies just
    inside or just outside the pointing's disc.  Pixels are drawn with theta in
    [radius + 0.05, pi - radius - 0.05] so no pointing reaches a pole.  float64 numpy
    (theta, phi, psi, pix)."""
    rng = np.random.default_rng(seed)
    th, ph = healpix_centres(nside)
    ok = np.nonzero((th > radius + 0.05) & (th < math.pi - radius - 0.05))[0]
    pix = rng.choice(ok, n, replace=False)
    a = rng.uniform(0.0, 2.0 * math.pi, n)
    dist = radius + np.where(np.arange(n) % 2 == 0, -delta, delta)
    t, p = th[pix], ph[pix]
    k = np.stack([np.sin(t) * np.cos(p), np.sin(t) * np.sin(p), np.cos(t)], -1)
    e_t = np.stack([np.cos(t) * np.cos(p), np.cos(t) * np.sin(p), -np.sin(t)], -1)
    e_p = np.stack([-np.sin(p), np.cos(p), np.zeros(n)], -1)
    d = np.cos(a)[:, None] * e_t + np.sin(a)[:, None] * e_p
    v = np.cos(dist)[:, None] * k + np.sin(dist)[:, None] * d
    theta0 = np.arctan2(np.hypot(v[:, 0], v[:, 1]), v[:, 2])
    phi0 = np.mod(np.arctan2(v[:, 1], v[:, 0]), 2.0 * math.pi)
    return theta0, phi0, rng.uniform(0.0, 2.0 * math.pi, n), pix


def focal_plane(n_det, seed, max_offset_deg=10.0):
    """Seeded focal-plane offsets (radians) and beam parameters for ``n_det`` detectors."""
    rng = np.random.default_rng(seed)
    off = np.radians(rng.uniform(-max_offset_deg, max_offset_deg, (n_det, 2)))
    fwhm = rng.uniform(1.2, 1.8, n_det)
    ell = rng.uniform(0.0, 0.1, n_det)
    zeta = rng.uniform(0.0, math.pi, n_det)
    return off, fwhm, ell, zeta


# --------------------------------------------------------------------------
# beams
# --------------------------------------------------------------------------

def grid_nodes(n, radius):
    """Orthographic node coordinates u_i = sin(R) (2 i / (N - 1) - 1)."""
    return np.sin(radius) * (2.0 * np.arange(n) / (n - 1) - 1.0)


def gaussian_beam_maps(n, radius, fwhm_deg, ellipticity=0.0, xpol=0.0, sidelobe=None,
                       ideal=False):
    """Six float32 maps (TT, QT, UT, TQ, QQ, UQ) of an elliptical Gaussian beam
    (the parametric family of ``beams.gaussian_beam_grids``) as a numpy array.

    ``sidelobe`` = (amplitude, centre_deg, width_deg) adds a ring to B_TT and B_QQ;
    ``ideal`` gives B_TT = B_QQ = g (the Kronecker beamsor of Sec. 3).
    """
    from .beams import gaussian_beam_grids
    g = gaussian_beam_grids(n, radius, fwhm_deg, ellipticity, xpol, sidelobe, ideal)
    return np.ascontiguousarray(g.numpy(), dtype=np.float32)


def random_beam_maps(n, seed, smooth=True):
    """Six float32 maps with every element non-zero, for parity tests.

    B_TT is positive (a Gaussian bump times a random positive field); the
    other five maps are smaller signed random fields.
    """
    rng = np.random.default_rng(seed)
    x = np.linspace(-1.0, 1.0, n)
    xx, yy = np.meshgrid(x, x, indexing="xy")
    bump = np.exp(-2.0 * (xx * xx + yy * yy))
    maps = rng.standard_normal((6, n, n))
    if smooth:
        k = np.array([0.25, 0.5, 0.25])
        for _ in range(3):
            maps = (np.apply_along_axis(lambda a: np.convolve(a, k, "same"), -1, maps))
            maps = (np.apply_along_axis(lambda a: np.convolve(a, k, "same"), -2, maps))
    maps[0] = bump * (1.0 + 0.3 * np.tanh(maps[0]))
    maps[1:] = 0.2 * bump * maps[1:]
    return np.ascontiguousarray(maps, dtype=np.float32)
