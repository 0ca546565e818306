"""Multi-realization (tensor-core) path versus the FP64 oracle, per realization.

The plan stores R realizations in BF16 or FP16; the FP32 pair weights enter
the tensor cores as two 16-bit parts (rounded value + rounded remainder), so
a weight is off by at most u = 2^-17 (BF16: 8 + 8 significant bits) or
2^-23 (FP16: 11 + 11) relative, and products accumulate in FP32.  Against the
oracle evaluated on the realizations exactly as stored, every sample obeys
|d - d_ref| <= (u + FP32 accumulation ~1e-6) sum_k |w_k . S_k|; the tests allow
1e-5 (BF16) and 2e-6 (FP16) of that sum.  Against the unrounded realizations the storage rounding
(2^-9 BF16, 2^-12 FP16 per value, averaged over the beam) adds to that; the
per-realization normwise error of the configuration-like case stays below
1e-3 (BF16) and 2e-4 (FP16) even so.
"""

import math

import numpy as np
import pytest
import torch

from oracle import beam as ob
from oracle import convolve as oc
from oracle import healpix as hp
from paper_1908_05662_gb300 import pisco
from paper_1908_05662_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _stack(nside, n_real, dtype, seed):
    """(Npix, 3, R) realization stack: smooth CMB-like skies, half of them plus white noise."""
    rng = np.random.default_rng(seed)
    base = [sy.gaussian_sky(nside, seed + k).numpy() for k in range(4)]
    out = np.empty((hp.npix(nside), 3, n_real))
    for r in range(n_real):
        c = rng.standard_normal(4)
        s = sum(c[k] * base[k] for k in range(4)) / 2.0
        if r % 2:
            s = s + 0.3 * rng.standard_normal(s.shape)
        out[:, :, r] = s.T
    t = torch.as_tensor(out, device=DEV).to(dtype)
    return t, t.double().cpu().numpy()


def _oracle_mr(nside, radius, stack64, grids, det, theta, phi, psi):
    """Reference TOD [t][r] and the per-(sample, realization) magnitude sum_k |w_k . S_k|."""
    g64 = np.asarray(grids, np.float64)
    omega = ob.omega_tilde(g64[0], radius)
    ref = np.empty((len(theta), stack64.shape[2]))
    mag = np.empty_like(ref)
    for t in range(len(theta)):
        pix, w = oc.sample_weights(nside, radius, g64, det, omega, theta[t], phi[t], psi[t])
        ref[t] = np.einsum("km,kmr->r", w, stack64[pix])
        mag[t] = np.einsum("km,kmr->r", np.abs(w), np.abs(stack64[pix]))
    return ref, mag


@pytest.mark.parametrize("precision,dtype,bound", [(pisco.PISCO_BF16_MR, torch.bfloat16, 1e-5),
                                                   (pisco.PISCO_FP16_MR, torch.float16, 2e-6)])
@pytest.mark.parametrize("n_real", [64, 96, 160, 256])
def test_multirealization_matches_oracle_per_realization(precision, dtype, bound, n_real):
    nside, r = 32, math.radians(8.0)
    stack, stack64 = _stack(nside, n_real, dtype, 100)
    grids = sy.gaussian_beam_maps(81, r, 2.5, ellipticity=0.05, xpol=0.01)
    grids[2] = 0.02 * grids[0]
    grids[3] = 0.03 * grids[0]
    det = (0.3, 0.02, 1.0)
    th, ph, ps = sy.raster_scan(200, center=(1.1, 2.0), half_size=math.radians(4.0), rows=5)
    ref, mag = _oracle_mr(nside, r, stack64, grids, det, th, ph, ps)
    with pisco.Plan(nside, r, stack, [det], torch.as_tensor(grids, device=DEV)[None], precision=precision) as plan:
        out = plan.convolve(_t(th), _t(ph), _t(ps)).double().cpu().numpy()
        plan.sync_status()
    assert out.shape == (200, n_real)
    np.testing.assert_array_less(np.abs(out - ref), bound * mag)


@pytest.mark.parametrize("precision,dtype,tol", [(pisco.PISCO_BF16_MR, torch.bfloat16, 1e-3),
                                                 (pisco.PISCO_FP16_MR, torch.float16, 2e-4)])
def test_multirealization_configuration_normwise(precision, dtype, tol):
    """The multi-realization configuration's resolution: nside 256, 256 realizations, a 1.5 deg
    Gaussian beam of radius 4 deg on a 161^2 grid, azimuth-scan samples.  The reference uses
    the realizations before their 16-bit storage, so the storage rounding is part of the error."""
    nside, r, n_real = 256, math.radians(4.0), 256
    gen = torch.Generator().manual_seed(11)
    coef = torch.randn(n_real, 4, generator=gen, dtype=torch.float64).to(DEV) / 2.0
    base = torch.stack([sy.gaussian_sky(nside, 11 + k, device=DEV) for k in range(4)])  # (4, 3, Npix)
    exact = torch.einsum("rk,kmp->pmr", coef, base).contiguous()                          # (Npix, 3, R)
    stack = exact.to(dtype)
    grids = sy.gaussian_beam_maps(161, r, 1.5)
    det = (0.0, 0.0, 1.0)
    th, ph, ps = (a.numpy() for a in sy.ces_scan(4000))
    th, ph, ps = th[::25], ph[::25], ps[::25]
    g64 = grids.astype(np.float64)
    omega = ob.omega_tilde(g64[0], r)
    ref = np.empty((len(th), n_real))
    for t in range(len(th)):
        pix, w = oc.sample_weights(nside, r, g64, det, omega, th[t], ph[t], ps[t])
        ref[t] = np.einsum("km,kmr->r", w, exact[torch.as_tensor(pix, device=DEV)].cpu().numpy())
    with pisco.Plan(nside, r, stack, [det], torch.as_tensor(grids, device=DEV)[None], precision=precision) as plan:
        out = plan.convolve(_t(th), _t(ph), _t(ps)).double().cpu().numpy()
    err = np.max(np.abs(out - ref), axis=0) / np.max(np.abs(ref), axis=0)
    assert np.all(err <= tol), (err.max(), err.argmax())


def test_multirealization_agrees_with_the_fp32_path_per_realization():
    nside, r, n_real = 32, math.radians(6.0), 32
    stack, stack64 = _stack(nside, n_real, torch.float16, 7)
    grids = sy.random_beam_maps(61, 3)
    det = (0.9, 0.05, 1.2)
    th, ph, ps = sy.raster_scan(100, center=(2.0, 4.0), half_size=math.radians(3.0), rows=4)
    g = torch.as_tensor(grids, device=DEV)[None]
    with pisco.Plan(nside, r, stack, [det], g, precision=pisco.PISCO_FP16_MR) as plan:
        mr = plan.convolve(_t(th), _t(ph), _t(ps)).double().cpu().numpy()
    for k in (0, 5, 31):
        with pisco.Plan(nside, r, _t(stack64[:, :, k].T), [det], g) as plan:
            one = plan.convolve(_t(th), _t(ph), _t(ps)).double().cpu().numpy()
        assert np.max(np.abs(mr[:, k] - one)) <= 2e-5 * np.max(np.abs(one))


def test_multirealization_invalid_samples_and_unsupported_calls():
    nside, r, n_real = 16, math.radians(10.0), 32
    stack, _ = _stack(nside, n_real, torch.bfloat16, 3)
    grids = torch.as_tensor(sy.random_beam_maps(31, 5), device=DEV)[None]
    th, ph, ps = sy.raster_scan(20, center=(1.0, 1.0), half_size=0.05, rows=2)
    th = th.copy()
    th[4] = np.nan
    with pisco.Plan(nside, r, stack, [(0, 0, 1)], grids, precision=pisco.PISCO_BF16_MR) as plan:
        out = plan.convolve(_t(th), _t(ph), _t(ps)).cpu().numpy()
        assert np.all(np.isnan(out[4])) and np.all(np.isfinite(np.delete(out, 4, axis=0)))
        with pytest.raises(pisco.PiscoError) as e:
            plan.adjoint(_t(th), _t(ph), _t(ps), torch.zeros(20, device=DEV))
        assert e.value.status == pisco.PISCO_EUNSUPPORTED
    with pytest.raises(pisco.PiscoError):
        bad = torch.zeros(hp.npix(nside), 3, 48, dtype=torch.bfloat16, device=DEV)
        pisco.Plan(nside, r, bad, [(0, 0, 1)], grids, precision=pisco.PISCO_BF16_MR)


def test_multirealization_batched_detectors_equal_single_calls_and_empty_input():
    """Two detectors with their own beams in one pisco_convolve_batched launch (128-sample tiles
    of each detector's range, uneven lengths) give the same TOD as one call per detector, and an
    empty input is a no-op."""
    nside, r, n_real = 32, math.radians(8.0), 64
    stack, _ = _stack(nside, n_real, torch.bfloat16, 21)
    grids = torch.as_tensor(np.stack([sy.random_beam_maps(41, 31), sy.random_beam_maps(41, 32)]), device=DEV)
    dets = [(0.2, 0.01, 1.0), (1.3, 0.03, 0.9)]
    th, ph, ps = sy.raster_scan(330, center=(1.1, 2.0), half_size=math.radians(4.0), rows=5)
    offsets = [0, 130, 330]
    with pisco.Plan(nside, r, stack, dets, grids, precision=pisco.PISCO_BF16_MR) as plan:
        both = plan.convolve_batched(offsets, _t(th), _t(ph), _t(ps)).cpu()
        for d in range(2):
            a, b = offsets[d], offsets[d + 1]
            one = plan.convolve(_t(th[a:b]), _t(ph[a:b]), _t(ps[a:b]), det=d).cpu()
            torch.testing.assert_close(both[a:b], one, rtol=0, atol=0)
        empty = torch.empty(0, dtype=torch.float64, device=DEV)
        assert plan.convolve(empty, empty, empty).shape == (0, n_real)
        plan.sync_status()
