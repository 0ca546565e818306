"""pisco_beam_grid_adjoint_static, the allocation-free beam-grid adjoint, through the C ABI.

For callers that may not allocate device memory when they call: its scratch
is a static array inside the library.  Its output must match
pisco_beam_grid_adjoint's, on two calls in a row (the second call reuses
the array the first one left filled), within the tolerance of the atomic
summation order.  This file is collected last so a failure here comes after
every other test has run.
"""

import ctypes
import math

import numpy as np
import pytest
import torch

from paper_1908_05662_gb300 import pisco
from paper_1908_05662_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


@pytest.mark.parametrize("accumulate", [0, 1])
@pytest.mark.parametrize("precision,dtype,tol", [(pisco.PISCO_FP32, torch.float32, 1e-5),
                                                 (pisco.PISCO_FP64_PLAIN, torch.float64, 1e-12)])
def test_static_scratch_adjoint_matches_allocating_adjoint(precision, dtype, tol, accumulate):
    """Two calls in a row equal pisco_beam_grid_adjoint's result; with accumulate = 1 the
    result is added to what the output held (a seeded pre-fill)."""
    lib = pisco.load_library()
    nside, r, n = 32, math.radians(8.0), 61
    sky = _t(sy.gaussian_sky(nside, 5).numpy())
    grids = torch.as_tensor(sy.random_beam_maps(n, 12), device=DEV)[None]
    th, ph, ps = (_t(a) for a in sy.raster_scan(500, center=(1.2, 2.0), half_size=math.radians(4.0), rows=5))
    y = _t(np.random.default_rng(8).standard_normal(500), dtype)
    prefill = _t(np.random.default_rng(9).standard_normal((6, n, n)), dtype)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    with pisco.Plan(nside, r, sky, [(0.3, 0.05, 1.1)], grids, precision=precision) as plan:
        ref = torch.empty(6, n, n, dtype=dtype, device=DEV)
        st = lib.pisco_beam_grid_adjoint(plan.handle, 0, 500, th.data_ptr(), ph.data_ptr(), ps.data_ptr(),
                                         y.data_ptr(), ref.data_ptr(), 0, stream)
        assert st == pisco.PISCO_OK
        scale = ref.abs().max().item()
        if accumulate:
            ref = ref + prefill
        for _ in range(2):
            out = prefill.clone() if accumulate else torch.full((6, n, n), float("nan"), dtype=dtype, device=DEV)
            st = lib.pisco_beam_grid_adjoint_static(plan.handle, 0, 500, th.data_ptr(), ph.data_ptr(),
                                                    ps.data_ptr(), y.data_ptr(), out.data_ptr(), accumulate, stream)
            assert st == pisco.PISCO_OK, lib.pisco_last_error(plan.handle)
            torch.cuda.synchronize()
            torch.testing.assert_close(out, ref, rtol=0, atol=tol * scale)
        plan.sync_status()


@pytest.mark.parametrize("accumulate", [0, 1])
def test_static_scratch_empty_scan(accumulate):
    """n = 0 after a non-empty call: the array still holds that call's gradient, so the empty
    call must clear it and unfold zero: the output is zero (accumulate = 0) or unchanged."""
    lib = pisco.load_library()
    nside, r, n = 16, math.radians(10.0), 31
    sky = _t(sy.gaussian_sky(nside, 2).numpy())
    grids = torch.as_tensor(sy.random_beam_maps(n, 4), device=DEV)[None]
    th, ph, ps = (_t(a) for a in sy.raster_scan(64, center=(1.0, 1.0), half_size=0.1, rows=4))
    y = torch.ones(64, device=DEV)
    prefill = _t(np.random.default_rng(2).standard_normal((6, n, n)), torch.float32)
    with pisco.Plan(nside, r, sky, [(0.1, 0.0, 1.0)], grids) as plan:
        busy = torch.empty(6, n, n, device=DEV)
        assert lib.pisco_beam_grid_adjoint_static(plan.handle, 0, 64, th.data_ptr(), ph.data_ptr(), ps.data_ptr(),
                                                  y.data_ptr(), busy.data_ptr(), 0, None) == pisco.PISCO_OK
        torch.cuda.synchronize()
        assert busy.abs().max().item() > 0.0
        out = prefill.clone()
        st = lib.pisco_beam_grid_adjoint_static(plan.handle, 0, 0, None, None, None, None, out.data_ptr(),
                                                accumulate, None)
        assert st == pisco.PISCO_OK, lib.pisco_last_error(plan.handle)
        torch.cuda.synchronize()
        plan.sync_status()
    if accumulate:
        torch.testing.assert_close(out, prefill, rtol=0, atol=0)
    else:
        assert torch.count_nonzero(out).item() == 0


def test_static_scratch_rejects_grids_beyond_its_size():
    lib = pisco.load_library()
    nside, r, n = 8, math.radians(10.0), 513
    sky = _t(np.zeros((3, 12 * nside * nside)))
    grids = torch.zeros(1, 6, n, n, device=DEV)
    grids[0, 0] = 1.0
    th = _t(np.array([1.0]))
    y = torch.ones(1, device=DEV)
    out = torch.empty(6, n, n, device=DEV)
    with pisco.Plan(nside, r, sky, [(0.0, 0.0, 1.0)], grids) as plan:
        st = lib.pisco_beam_grid_adjoint_static(plan.handle, 0, 1, th.data_ptr(), th.data_ptr(), th.data_ptr(),
                                                y.data_ptr(), out.data_ptr(), 0, None)
        assert st == pisco.PISCO_EINVAL
        assert b"512" in lib.pisco_last_error(plan.handle)
