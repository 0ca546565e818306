"""Differentiable TOD: torch.autograd.Function over the C-ABI library.

``PiscoConvolve.apply(sky, beam_grids, theta, phi, psi, nside, radius, det)``
returns the TOD of one detector (pisco_convolve).  Its backward pass runs
the library's transposes: pisco_adjoint for the sky (TOD -> I, Q, U maps) and
pisco_beam_grid_adjoint + pisco_omega_adjoint for the six beam grids (the
Omega~ term only when Omega~ is computed from B_TT); when both gradients are
wanted from an FP32 plan, pisco_adjoint_sky_beam runs the two transposes in
one traversal.  Gradients with respect
to beam parameters (FWHM, ellipticity, cross-polar leakage) follow by
building ``beam_grids`` from them with ``beams.gaussian_beam_grids``.
"""

import torch

from . import pisco


class PiscoConvolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sky, beam_grids, theta, phi, psi, nside, radius, det, precision=pisco.PISCO_FP32,
                omega_tilde=None):
        plan = pisco.Plan(nside, radius, sky.detach(), [tuple(det)],
                          beam_grids.detach().to(torch.float32)[None].contiguous(),
                          omega_tilde=None if omega_tilde is None else [omega_tilde], precision=precision)
        tod = plan.convolve(theta, phi, psi)
        ctx.plan = plan
        ctx.omega_given = omega_tilde is not None
        ctx.sky_dtype, ctx.beam_dtype = sky.dtype, beam_grids.dtype
        ctx.save_for_backward(theta, phi, psi, tod)
        return tod

    @staticmethod
    def backward(ctx, grad_tod):
        theta, phi, psi, tod = ctx.saved_tensors
        plan = ctx.plan
        g = grad_tod.contiguous().to(plan.out_dtype)
        grad_sky = grad_beam = None
        both = ctx.needs_input_grad[0] and ctx.needs_input_grad[1]
        if both and plan.precision == pisco.PISCO_FP32:
            maps, gb = plan.adjoint_sky_beam(theta, phi, psi, g)  # one traversal for both transposes
            grad_sky = maps.to(ctx.sky_dtype)
        else:
            if ctx.needs_input_grad[0]:
                grad_sky = plan.adjoint(theta, phi, psi, g).to(ctx.sky_dtype)
            gb = plan.beam_grid_adjoint(theta, phi, psi, g) if ctx.needs_input_grad[1] else None
        if gb is not None:
            if not ctx.omega_given:
                plan.omega_adjoint(tod, g, gb)
            grad_beam = gb.to(ctx.beam_dtype)
        plan.close()
        ctx.plan = None
        return grad_sky, grad_beam, None, None, None, None, None, None, None, None


def convolve(sky, beam_grids, theta, phi, psi, nside, radius, det=(0.0, 0.0, 1.0), precision=pisco.PISCO_FP32,
             omega_tilde=None):
    """TOD of one detector, differentiable in ``sky`` (3, Npix) and ``beam_grids`` (6, N, N)."""
    return PiscoConvolve.apply(sky, beam_grids, theta, phi, psi, nside, radius, det, precision, omega_tilde)
