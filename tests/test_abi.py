"""The C-ABI library builds, loads and exports every entry point of include/pisco.h (CPU only)."""

import ctypes
import os
import re

import pytest

from paper_1908_05662_gb300 import pisco

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(pisco.LIB_PATH):
        from paper_1908_05662_gb300.build import build_library
        build_library()
    return pisco.load_library()


def _declared():
    with open(os.path.join(ROOT, "include", "pisco.h")) as f:
        text = f.read()
    return set(re.findall(r"^(?:pisco_status|void|const char\*)\s+(pisco_\w+)\s*\(", text, re.M))


def test_header_declares_the_binding_exports():
    assert _declared() == set(pisco.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_create_rejects_bad_arguments_before_touching_the_device(lib):
    handle = ctypes.c_void_p()
    det = (pisco.pisco_detector * 1)(pisco.pisco_detector(0.0, 0.0, 1.0))
    cases = [
        dict(nside=0, radius=0.1), dict(nside=9000, radius=0.1),
        dict(nside=8, radius=0.0), dict(nside=8, radius=2.0),
        dict(nside=8, radius=0.1, n_det=0), dict(nside=8, radius=0.1, grid_n=1),
        dict(nside=8, radius=0.1, dtype=7),
    ]
    for c in cases:
        st = lib.pisco_plan_create(ctypes.byref(handle), c["nside"], c["radius"], ctypes.c_void_p(16),
                                   c.get("dtype", 0), c.get("n_det", 1), det, c.get("grid_n", 11),
                                   ctypes.c_void_p(16), None, None, None)
        assert st == pisco.PISCO_EINVAL, c
        assert handle.value is None
        assert lib.pisco_last_error(None)


def test_multirealization_options_are_checked_before_touching_the_device(lib):
    """Realization count, stack dtype and the nside bound of the tensor-core path (its TMA row
    coordinates, 3 Npix rows, are 32-bit)."""
    handle = ctypes.c_void_p()
    det = (pisco.pisco_detector * 1)(pisco.pisco_detector(0.0, 0.0, 1.0))
    cases = [
        (8, pisco.PISCO_BF16_MR, pisco.PISCO_DTYPE_BF16, 48),    # not a multiple of 32
        (8, pisco.PISCO_BF16_MR, pisco.PISCO_DTYPE_BF16, 288),   # above 256
        (8, pisco.PISCO_BF16_MR, pisco.PISCO_DTYPE_F16, 64),     # FP16 stack on a BF16 plan
        (8, pisco.PISCO_FP16_MR, pisco.PISCO_DTYPE_F32, 64),     # FP32 sky on an FP16 plan
        (7724, pisco.PISCO_BF16_MR, pisco.PISCO_DTYPE_BF16, 32),  # 36 nside^2 >= 2^31
    ]
    for nside, precision, dtype, n_real in cases:
        opt = pisco.pisco_options(precision, 0, 0, 0, n_real)
        st = lib.pisco_plan_create(ctypes.byref(handle), nside, 0.1, ctypes.c_void_p(16), dtype, 1, det, 11,
                                   ctypes.c_void_p(16), None, ctypes.byref(opt), None)
        assert st == pisco.PISCO_EINVAL, (nside, precision, dtype, n_real)
        assert handle.value is None
        assert lib.pisco_last_error(None)


def test_calls_on_a_null_plan_are_rejected(lib):
    assert lib.pisco_convolve(None, 0, 0, None, None, None, None, None) == pisco.PISCO_EINVAL
    assert lib.pisco_adjoint(None, 0, 0, None, None, None, None, None, 0, None) == pisco.PISCO_EINVAL
    assert lib.pisco_disc_count(None, 0, None, None, None, None) == pisco.PISCO_EINVAL
    assert lib.pisco_sync_status(None, None) == pisco.PISCO_EINVAL
    assert lib.pisco_inject_mr_stall(None, 1000) == pisco.PISCO_EINVAL
    lib.pisco_plan_destroy(None)
    assert lib.pisco_plan_autotune(None, 0, 10, None, None, None, None, 1, None, None, None, None) == pisco.PISCO_EINVAL
    off2 = (ctypes.c_int64 * 2)(0, 4)
    assert lib.pisco_plan_autotune_batched(None, 1, off2, None, None, None, None, 1, None, None, None,
                                           None) == pisco.PISCO_EINVAL
    z = (ctypes.c_double * 2)(0.0, 1.0)
    assert lib.pisco_convolve_psb(None, 0, 0, None, None, None, 2, z, None, None) == pisco.PISCO_EINVAL
    off = (ctypes.c_int64 * 2)(0, 4)
    assert lib.pisco_convolve_batched(None, 1, off, None, None, None, None, None) == pisco.PISCO_EINVAL
    assert lib.pisco_beam_grid_adjoint(None, 0, 0, None, None, None, None, None, 0, None) == pisco.PISCO_EINVAL
    assert lib.pisco_beam_grid_adjoint_static(None, 0, 0, None, None, None, None, None, 0,
                                              None) == pisco.PISCO_EINVAL
    assert lib.pisco_adjoint_sky_beam(None, 0, 0, None, None, None, None, None, None, 0, None) == pisco.PISCO_EINVAL
    assert lib.pisco_omega_adjoint(None, 0, 0, None, None, None, None) == pisco.PISCO_EINVAL
    assert lib.pisco_update_beams(None, None, None, None) == pisco.PISCO_EINVAL
    assert lib.pisco_convolve_host(None, 0, 0, None, None, None, None) == pisco.PISCO_EINVAL
    om, sc = ctypes.c_double(), ctypes.c_double()
    assert lib.pisco_plan_omega(None, 0, ctypes.byref(om), ctypes.byref(sc)) == pisco.PISCO_EINVAL


def test_healpix_beam_resampling_rejects_bad_arguments_before_touching_the_device(lib):
    p = ctypes.c_void_p(16)
    for nside_b, n_maps, radius, grid_n in [(0, 6, 0.1, 11), (9000, 6, 0.1, 11), (4, 0, 0.1, 11),
                                           (4, 6, 0.0, 11), (4, 6, 1.6, 11), (4, 6, 0.1, 1), (4, 6, 0.1, 5000)]:
        st = lib.pisco_beam_grids_from_healpix(nside_b, n_maps, p, radius, grid_n, p, None)
        assert st == pisco.PISCO_EINVAL
        assert lib.pisco_last_error(None)


def test_map_making_rejects_bad_arguments_before_touching_the_device(lib):
    p = ctypes.c_void_p(16)
    ok_det = pisco.pisco_detector(0.0, 0.0, 1.0)
    nan_det = pisco.pisco_detector(float("nan"), 0.0, 1.0)
    for nside in (0, 8193):
        assert lib.pisco_ang2pix(nside, 1, p, p, p, None) == pisco.PISCO_EINVAL
        assert lib.pisco_map_solve(nside, p, 0.0, p, None) == pisco.PISCO_EINVAL
    assert lib.pisco_ang2pix(8, -1, p, p, p, None) == pisco.PISCO_EINVAL
    assert lib.pisco_ang2pix(8, 0, None, None, None, None) == pisco.PISCO_OK  # nothing to do
    cases = [dict(n=-1), dict(det=None), dict(det=nan_det), dict(dtype=pisco.PISCO_DTYPE_BF16), dict(nside=0)]
    for c in cases:
        det = c.get("det", ok_det)
        st = lib.pisco_map_accumulate(c.get("nside", 8), c.get("n", 4), p, p, p,
                                      None if det is None else ctypes.byref(det), p,
                                      c.get("dtype", pisco.PISCO_DTYPE_F32), p, 0, None)
        assert st == pisco.PISCO_EINVAL, c
        assert lib.pisco_last_error(None)
    for rcond in (-0.1, 1.5, float("nan")):
        assert lib.pisco_map_solve(8, p, rcond, p, None) == pisco.PISCO_EINVAL
