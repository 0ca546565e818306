"""Failure detection of the tensor-core kernel: a bounded wait that runs out.

pisco_inject_mr_stall makes the next multi-realization launch wait, before it
issues any copy or MMA, on an mbarrier that nothing arrives on, with a short
limit (1e5 SM clocks).  The wait gives up, every block records error bit 2
and returns with its tensor memory released; the host sees PISCO_ETIMEOUT from
pisco_sync_status, the flag is cleared, and the next launch on the same plan
gives the TOD it gave before (the kernel is deterministic), which matches the
oracle.  No GPU fault is involved.

Host-side fault injection of an allocation failure: a plan whose realization
stack cannot fit in device memory fails its allocation before anything is read
from the caller's buffers (PISCO_ENOMEM), and the device serves the next plan.
"""

import ctypes
import math

import numpy as np
import pytest
import torch

from oracle import beam as ob
from oracle import convolve as oc
from paper_1908_05662_gb300 import pisco
from paper_1908_05662_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


@pytest.mark.parametrize("precision,dtype", [(pisco.PISCO_BF16_MR, torch.bfloat16),
                                             (pisco.PISCO_FP16_MR, torch.float16)])
def test_bounded_wait_times_out_and_plan_recovers(precision, dtype):
    nside, r, n_real = 16, math.radians(10.0), 32
    sky = sy.gaussian_sky(nside, 4).numpy()                        # (3, Npix)
    fac = np.random.default_rng(6).uniform(0.5, 1.5, n_real)
    stack = torch.as_tensor(sky.T[:, :, None] * fac[None, None, :], device=DEV).to(dtype).contiguous()
    grids = sy.random_beam_maps(41, 7)
    det = (0.2, 0.03, 1.0)
    th, ph, ps = sy.raster_scan(300, center=(1.0, 2.0), half_size=math.radians(3.0), rows=3)
    t = [_t(a) for a in (th, ph, ps)]
    with pisco.Plan(nside, r, stack, [det], torch.as_tensor(grids, device=DEV)[None], precision=precision) as plan:
        good = plan.convolve(*t).clone()
        plan.sync_status()
        plan.inject_mr_stall(100_000)
        out = torch.full_like(good, 7.0)
        plan.convolve(*t, out=out)
        with pytest.raises(pisco.PiscoError) as e:
            plan.sync_status()
        assert e.value.status == pisco.PISCO_ETIMEOUT
        assert torch.all(out == 7.0)  # the blocks stopped before writing any TOD
        plan.sync_status()            # the flag was cleared
        again = plan.convolve(*t)
        plan.sync_status()
    torch.testing.assert_close(again, good, rtol=0, atol=0)
    # the recovered launch against the oracle on the stored realizations (every 30th sample)
    stack64 = stack.double().cpu().numpy()
    g64 = grids.astype(np.float64)
    omega = ob.omega_tilde(g64[0], r)
    got = again.double().cpu().numpy()
    for k in range(0, len(th), 30):
        pix, w = oc.sample_weights(nside, r, g64, det, omega, th[k], ph[k], ps[k])
        ref = np.einsum("km,kmr->r", w, stack64[pix])
        mag = np.einsum("km,kmr->r", np.abs(w), np.abs(stack64[pix]))
        np.testing.assert_array_less(np.abs(got[k] - ref), 1e-5 * mag)


def test_stall_hook_rejects_other_plans_and_bad_lengths():
    nside, r = 8, math.radians(10.0)
    g = torch.as_tensor(sy.random_beam_maps(21, 1), device=DEV)[None]
    with pisco.Plan(nside, r, _t(np.zeros((3, 12 * nside * nside))), [(0, 0, 1)], g) as plan:
        with pytest.raises(pisco.PiscoError) as e:
            plan.inject_mr_stall(1000)
        assert e.value.status == pisco.PISCO_EUNSUPPORTED
    stack = torch.zeros(12 * nside * nside, 3, 32, dtype=torch.bfloat16, device=DEV)
    with pisco.Plan(nside, r, stack, [(0, 0, 1)], g, precision=pisco.PISCO_BF16_MR) as plan:
        for bad in (0, -5, 10**11):
            with pytest.raises(pisco.PiscoError) as e:
                plan.inject_mr_stall(bad)
            assert e.value.status == pisco.PISCO_EINVAL


def test_allocation_failure_reports_enomem_and_the_device_serves_the_next_plan():
    """256 BF16 realizations at nside 7723 ask for a 1.1 TB stack, several times the device
    memory: the stack's allocation fails before anything is read from `sky` (a small buffer
    here), so the call returns PISCO_ENOMEM with a message and no plan."""
    lib = pisco.load_library()
    nside, n_real = 7723, 256
    need = 12 * nside * nside * 3 * n_real * 2
    if need <= 2 * torch.cuda.get_device_properties(0).total_memory:
        pytest.skip("the device could hold the stack")
    small = torch.zeros(64, dtype=torch.bfloat16, device=DEV)
    grids = torch.zeros(1, 6, 11, 11, device=DEV)
    handle = ctypes.c_void_p()
    det = (pisco.pisco_detector * 1)(pisco.pisco_detector(0.0, 0.0, 1.0))
    opt = pisco.pisco_options(pisco.PISCO_BF16_MR, 0, 0, 0, n_real)
    st = lib.pisco_plan_create(ctypes.byref(handle), nside, 0.1, ctypes.c_void_p(small.data_ptr()),
                               pisco.PISCO_DTYPE_BF16, 1, det, 11, ctypes.c_void_p(grids.data_ptr()), None,
                               ctypes.byref(opt), None)
    assert st == pisco.PISCO_ENOMEM
    assert handle.value is None
    assert b"allocation" in lib.pisco_last_error(None)
    torch.cuda.synchronize()

    # the next plan works and matches the oracle
    nside, r, n = 16, math.radians(10.0), 40
    sky = sy.gaussian_sky(nside, 5)
    g = sy.random_beam_maps(31, 6)
    det = (0.2, 0.02, 1.0)
    th, ph, ps = sy.random_pointings(n, 9)
    ref = oc.tod(nside, r, sky.numpy(), g.astype(np.float64), det, ob.omega_tilde(g[0].astype(np.float64), r),
                 th, ph, ps)
    with pisco.Plan(nside, r, sky.to(DEV), [det], torch.as_tensor(g, device=DEV)[None]) as plan:
        out = plan.convolve(_t(th), _t(ph), _t(ps)).double().cpu().numpy()
        plan.sync_status()
    assert np.max(np.abs(out - ref)) <= 2e-6 * np.max(np.abs(ref))
