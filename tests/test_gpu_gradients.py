"""Beam-grid adjoint, Omega~ term and beam-parameter gradients through the C ABI.

Checked against the oracle's explicit transpose (oracle.convolve.beam_grid_adjoint),
dot-product identities, and central finite differences of the FP64 oracle
(h = 1e-4 in natural units: FWHM in degrees, ellipticity and leakage
dimensionless), to 1e-4 relative.
"""

import math

import numpy as np
import pytest
import torch

from oracle import beam as ob
from oracle import convolve as oc
from paper_1908_05662_gb300 import autograd as pag
from paper_1908_05662_gb300 import beams
from paper_1908_05662_gb300 import pisco
from paper_1908_05662_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
PATHS = [(pisco.PISCO_FP32, torch.float32, 2e-5), (pisco.PISCO_FP64_PLAIN, torch.float64, 1e-10)]


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


@pytest.mark.parametrize("precision,dt,tol", PATHS)
def test_beam_grid_adjoint_matches_oracle_transpose(precision, dt, tol):
    nside, r, n = 16, math.radians(15.0), 31
    grids = sy.random_beam_maps(n, 33)
    det = (0.6, 0.07, 1.2)
    sky = sy.white_sky(nside, 4).numpy()
    th, ph, ps = sy.raster_scan(120, center=(1.2, 2.5), half_size=math.radians(5.0), rows=6)
    y = np.random.default_rng(9).standard_normal(len(th))
    omega = ob.omega_tilde(grids[0].astype(np.float64), r)
    ref = oc.beam_grid_adjoint(nside, r, sky, grids.astype(np.float64), det, omega, th, ph, ps, y)
    with pisco.Plan(nside, r, _t(sky), [det], torch.as_tensor(grids, device=DEV)[None], precision=precision) as plan:
        g = plan.beam_grid_adjoint(_t(th), _t(ph), _t(ps), _t(y, dt)).double().cpu().numpy()
    np.testing.assert_allclose(g, ref, rtol=0, atol=tol * np.max(np.abs(ref)))


@pytest.mark.parametrize("precision,dt,tol", PATHS)
def test_beam_grid_adjoint_dot_identity(precision, dt, tol):
    """At fixed Omega~ the TOD is linear in the grids: <d(G), y> = <G, A_G^T y>, both from the GPU."""
    nside, r, n = 32, math.radians(8.0), 41
    grids = sy.random_beam_maps(n, 44)
    sky = sy.gaussian_sky(nside, 2).numpy()
    th, ph, ps = sy.raster_scan(600, center=(2.0, 1.0), half_size=math.radians(4.0), rows=6)
    y = np.random.default_rng(1).standard_normal(len(th))
    with pisco.Plan(nside, r, _t(sky), [(0.3, 0.05, 1.0)], torch.as_tensor(grids, device=DEV)[None],
                    omega_tilde=[0.01], precision=precision) as plan:
        d = plan.convolve(_t(th), _t(ph), _t(ps)).double().cpu().numpy()
        g = plan.beam_grid_adjoint(_t(th), _t(ph), _t(ps), _t(y, dt)).double().cpu().numpy()
    lhs, rhs = np.dot(d, y), np.sum(grids.astype(np.float64) * g)
    assert abs(lhs - rhs) <= max(tol, 1e-6) * np.sum(np.abs(d * y))


@pytest.mark.parametrize("precision,dt,tol", PATHS)
def test_full_grid_gradient_with_omega_term_vs_finite_differences(precision, dt, tol):
    """Omega~ computed from B_TT: the beam gradient includes the Omega~ term (pisco_omega_adjoint)."""
    nside, r, n = 16, math.radians(15.0), 21
    grids = sy.random_beam_maps(n, 55).astype(np.float64)
    det = (0.2, 0.03, 1.0)
    sky = sy.white_sky(nside, 6).numpy()
    th, ph, ps = sy.raster_scan(60, center=(1.0, 4.0), half_size=math.radians(4.0), rows=4)
    y = np.random.default_rng(2).standard_normal(len(th))
    sky_t = _t(sky)
    gt = torch.tensor(grids, dtype=torch.float64, device=DEV, requires_grad=True)
    tod = pag.convolve(sky_t, gt, _t(th), _t(ph), _t(ps), nside, r, det, precision)
    (tod.double() * _t(y)).sum().backward()
    grad = gt.grad.cpu().numpy()

    def loss(gr):
        om = ob.omega_tilde(gr[0], r)
        return np.dot(oc.tod(nside, r, sky, gr, det, om, th, ph, ps), y)

    h = 1e-4
    rng = np.random.default_rng(3)
    for e in (0, 0, 3, 4, 1):  # TT twice (it carries the Omega~ term)
        j, i = rng.integers(2, n - 2, 2)
        gp, gm = grids.copy(), grids.copy()
        gp[e, j, i] += h
        gm[e, j, i] -= h
        fd = (loss(gp) - loss(gm)) / (2 * h)
        assert abs(grad[e, j, i] - fd) <= 1e-4 * max(abs(fd), 1e-3 * np.max(np.abs(grad))), (e, j, i)


@pytest.mark.parametrize("precision,dt,tol", PATHS)
def test_beam_parameter_gradients_vs_finite_differences(precision, dt, tol):
    """chi^2 between the TOD of beam parameters p and a target from perturbed parameters;
    d chi^2 / d(FWHM, e, l) by autograd through the library versus central differences of
    the FP64 oracle with h = 1e-4."""
    nside, r, n = 64, math.radians(5.0), 101
    sky = sy.gaussian_sky(nside, 8).numpy()
    th, ph, ps = sy.raster_scan(300, center=(1.1, 0.7), half_size=math.radians(2.0), rows=6)
    det = (0.1, 0.02, 1.0)
    p0 = np.array([1.5, 0.05, 0.005])
    pt = np.array([1.52, 0.06, 0.004])

    def oracle_tod(p):
        g = beams.gaussian_beam_grids(n, r, p[0], p[1], p[2]).numpy()
        return oc.tod(nside, r, sky, g, det, ob.omega_tilde(g[0], r), th, ph, ps)

    target = oracle_tod(pt)

    def chi2(p):
        return np.sum((oracle_tod(p) - target) ** 2)

    params = torch.tensor(p0, dtype=torch.float64, device=DEV, requires_grad=True)
    g = beams.gaussian_beam_grids(n, r, params[0], params[1], params[2], device=DEV)
    tod = pag.convolve(_t(sky), g, _t(th), _t(ph), _t(ps), nside, r, det, precision)
    loss = ((tod.double() - _t(target)) ** 2).sum()
    loss.backward()
    grad = params.grad.cpu().numpy()
    h = 1e-4
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd = (chi2(p0 + e) - chi2(p0 - e)) / (2 * h)
        assert abs(grad[k] - fd) <= 1e-4 * abs(fd), (k, grad[k], fd)


def test_sky_gradient_is_the_adjoint():
    nside, r = 16, math.radians(12.0)
    grids = sy.random_beam_maps(31, 66)
    det = (0.4, 0.0, 1.0)
    th, ph, ps = sy.raster_scan(80, center=(1.3, 3.0), half_size=math.radians(4.0), rows=4)
    y = np.random.default_rng(4).standard_normal(len(th))
    sky = torch.tensor(sy.white_sky(nside, 7).numpy(), device=DEV, requires_grad=True)
    tod = pag.convolve(sky, _t(grids, torch.float32), _t(th), _t(ph), _t(ps), nside, r, det,
                       pisco.PISCO_FP64_PLAIN)
    (tod * _t(y)).sum().backward()
    omega = ob.omega_tilde(grids[0].astype(np.float64), r)
    ref = oc.adjoint(nside, r, grids.astype(np.float64), det, omega, th, ph, ps, y)
    np.testing.assert_allclose(sky.grad.cpu().numpy(), ref, rtol=0, atol=1e-11 * np.max(np.abs(ref)))


def test_update_beams_equals_new_plan():
    nside, r, n = 32, math.radians(8.0), 41
    sky = _t(sy.gaussian_sky(nside, 3).numpy())
    g1 = torch.as_tensor(sy.random_beam_maps(n, 1), device=DEV)[None]
    g2 = torch.as_tensor(sy.random_beam_maps(n, 2), device=DEV)[None]
    th, ph, ps = (_t(a) for a in sy.raster_scan(200, center=(1.0, 1.0), half_size=0.05, rows=4))
    for precision in (pisco.PISCO_FP32, pisco.PISCO_FP64_PLAIN):
        for fetch in (pisco.PISCO_FETCH_CELLS, pisco.PISCO_FETCH_TEXTURE):
            with pisco.Plan(nside, r, sky, [(0.1, 0.0, 1.0)], g1, precision=precision, beam_fetch=fetch) as a, \
                    pisco.Plan(nside, r, sky, [(0.1, 0.0, 1.0)], g2, precision=precision, beam_fetch=fetch) as b:
                a.update_beams(g2)
                assert a.omega() == b.omega()
                torch.testing.assert_close(a.convolve(th, ph, ps), b.convolve(th, ph, ps), rtol=0, atol=0)


def test_fused_sky_and_beam_transposes_match_the_separate_ones_and_the_oracle():
    """pisco_adjoint_sky_beam runs both transposes in one traversal: the same sums as
    pisco_adjoint and pisco_beam_grid_adjoint (atomic-add order aside) and the oracle's."""
    nside, r, n = 16, math.radians(15.0), 31
    grids = sy.random_beam_maps(n, 77)
    det = (0.6, 0.07, 1.2)
    sky = sy.white_sky(nside, 8).numpy()
    th, ph, ps = sy.raster_scan(150, center=(1.2, 2.5), half_size=math.radians(5.0), rows=6)
    y = np.random.default_rng(12).standard_normal(len(th))
    omega = ob.omega_tilde(grids[0].astype(np.float64), r)
    ref_maps = oc.adjoint(nside, r, grids.astype(np.float64), det, omega, th, ph, ps, y)
    ref_grid = oc.beam_grid_adjoint(nside, r, sky, grids.astype(np.float64), det, omega, th, ph, ps, y)
    yt = _t(y, torch.float32)
    with pisco.Plan(nside, r, _t(sky), [det], torch.as_tensor(grids, device=DEV)[None]) as plan:
        maps, grad = plan.adjoint_sky_beam(_t(th), _t(ph), _t(ps), yt)
        maps1 = plan.adjoint(_t(th), _t(ph), _t(ps), yt)
        grad1 = plan.beam_grid_adjoint(_t(th), _t(ph), _t(ps), yt)
        maps2, grad2 = plan.adjoint_sky_beam(_t(th), _t(ph), _t(ps), yt, maps=maps.clone(), grad=grad.clone(),
                                             accumulate=True)
        plan.sync_status()
    m, g = maps.double().cpu().numpy(), grad.double().cpu().numpy()
    np.testing.assert_allclose(m, maps1.double().cpu().numpy(), rtol=0, atol=1e-6 * np.max(np.abs(ref_maps)))
    np.testing.assert_allclose(g, grad1.double().cpu().numpy(), rtol=0, atol=1e-6 * np.max(np.abs(ref_grid)))
    np.testing.assert_allclose(m, ref_maps, rtol=0, atol=2e-5 * np.max(np.abs(ref_maps)))
    np.testing.assert_allclose(g, ref_grid, rtol=0, atol=2e-5 * np.max(np.abs(ref_grid)))
    np.testing.assert_allclose(maps2.double().cpu().numpy(), 2 * m, rtol=0, atol=2e-6 * np.max(np.abs(ref_maps)))
    np.testing.assert_allclose(grad2.double().cpu().numpy(), 2 * g, rtol=0, atol=2e-6 * np.max(np.abs(ref_grid)))
    with pisco.Plan(nside, r, _t(sky), [det], torch.as_tensor(grids, device=DEV)[None],
                    precision=pisco.PISCO_FP64_PLAIN) as plain:
        with pytest.raises(pisco.PiscoError) as e:
            plain.adjoint_sky_beam(_t(th), _t(ph), _t(ps), _t(y))
        assert e.value.status == pisco.PISCO_EUNSUPPORTED
