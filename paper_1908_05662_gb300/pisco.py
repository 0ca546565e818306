"""Thin Python binding of libpisco's C ABI (include/pisco.h).

Functions carry the C names and only marshal arguments: torch tensors become
device pointers, the current torch stream becomes the cudaStream_t, and a
non-zero status raises ``PiscoError``.  Every step of the convolution runs in
the CUDA library; there is no other implementation behind these calls, and
they raise if the library was not built.
"""

import ctypes
import os

import torch

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libpisco.so")

PISCO_OK, PISCO_EINVAL, PISCO_ENOMEM, PISCO_ECUDA, PISCO_ETIMEOUT, PISCO_EUNSUPPORTED, PISCO_EDEVICE = range(7)
PISCO_FP64_PLAIN, PISCO_FP32, PISCO_BF16_MR, PISCO_FP16_MR = 0, 1, 2, 3
PISCO_DTYPE_F32, PISCO_DTYPE_F64, PISCO_DTYPE_BF16, PISCO_DTYPE_F16 = 0, 1, 2, 3
PISCO_FETCH_TEXTURE, PISCO_FETCH_CELLS, PISCO_FETCH_PACKED, PISCO_FETCH_SHARED = 1, 2, 3, 4

STATUS_NAMES = {0: "PISCO_OK", 1: "PISCO_EINVAL", 2: "PISCO_ENOMEM", 3: "PISCO_ECUDA",
                4: "PISCO_ETIMEOUT", 5: "PISCO_EUNSUPPORTED", 6: "PISCO_EDEVICE"}

# Entry points declared in include/pisco.h, checked by the CPU test suite.
EXPORTS = ("pisco_plan_create", "pisco_plan_destroy", "pisco_last_error", "pisco_plan_omega",
           "pisco_convolve", "pisco_convolve_batched", "pisco_adjoint", "pisco_disc_count",
           "pisco_convolve_host", "pisco_sync_status", "pisco_beam_grid_adjoint", "pisco_omega_adjoint",
           "pisco_update_beams", "pisco_beam_grid_adjoint_static", "pisco_convolve_psb",
           "pisco_beam_grids_from_healpix", "pisco_ang2pix", "pisco_map_accumulate", "pisco_map_solve",
           "pisco_plan_autotune", "pisco_adjoint_sky_beam", "pisco_inject_mr_stall",
           "pisco_plan_autotune_batched")


class PiscoError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class pisco_detector(ctypes.Structure):
    _fields_ = [("zeta", ctypes.c_double), ("eps", ctypes.c_double), ("s_resp", ctypes.c_double)]


class pisco_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("tile_samples", ctypes.c_int),
                ("pixels_per_thread", ctypes.c_int), ("beam_fetch", ctypes.c_int), ("n_real", ctypes.c_int)]


_lib = None


def load_library(path=LIB_PATH):
    """Load libpisco.so once; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_1908_05662_gb300.build`")
    lib = ctypes.CDLL(path)
    vp, i64, c_int, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        "pisco_plan_create": (c_int, [ctypes.POINTER(vp), c_int, dbl, vp, c_int, c_int,
                                      ctypes.POINTER(pisco_detector), c_int, vp,
                                      ctypes.POINTER(dbl), ctypes.POINTER(pisco_options), vp]),
        "pisco_plan_destroy": (None, [vp]),
        "pisco_last_error": (ctypes.c_char_p, [vp]),
        "pisco_plan_omega": (c_int, [vp, c_int, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]),
        "pisco_convolve": (c_int, [vp, c_int, i64, vp, vp, vp, vp, vp]),
        "pisco_convolve_batched": (c_int, [vp, c_int, ctypes.POINTER(i64), vp, vp, vp, vp, vp]),
        "pisco_adjoint": (c_int, [vp, c_int, i64, vp, vp, vp, vp, vp, c_int, vp]),
        "pisco_disc_count": (c_int, [vp, i64, vp, vp, vp, vp]),
        "pisco_convolve_host": (c_int, [vp, c_int, i64, vp, vp, vp, vp]),
        "pisco_sync_status": (c_int, [vp, vp]),
        "pisco_inject_mr_stall": (c_int, [vp, i64]),
        "pisco_beam_grid_adjoint": (c_int, [vp, c_int, i64, vp, vp, vp, vp, vp, c_int, vp]),
        "pisco_omega_adjoint": (c_int, [vp, c_int, i64, vp, vp, vp, vp]),
        "pisco_update_beams": (c_int, [vp, vp, ctypes.POINTER(dbl), vp]),
        "pisco_beam_grid_adjoint_static": (c_int, [vp, c_int, i64, vp, vp, vp, vp, vp, c_int, vp]),
        "pisco_convolve_psb": (c_int, [vp, c_int, i64, vp, vp, vp, c_int, ctypes.POINTER(dbl), vp, vp]),
        "pisco_beam_grids_from_healpix": (c_int, [c_int, c_int, vp, dbl, c_int, vp, vp]),
        "pisco_ang2pix": (c_int, [c_int, i64, vp, vp, vp, vp]),
        "pisco_map_accumulate": (c_int, [c_int, i64, vp, vp, vp, ctypes.POINTER(pisco_detector), vp, c_int, vp,
                                         c_int, vp]),
        "pisco_map_solve": (c_int, [c_int, vp, dbl, vp, vp]),
        "pisco_adjoint_sky_beam": (c_int, [vp, c_int, i64, vp, vp, vp, vp, vp, vp, c_int, vp]),
        "pisco_plan_autotune": (c_int, [vp, c_int, i64, vp, vp, vp, vp, c_int, ctypes.POINTER(c_int),
                                        ctypes.POINTER(c_int), ctypes.POINTER(ctypes.c_float), vp]),
        "pisco_plan_autotune_batched": (c_int, [vp, c_int, ctypes.POINTER(i64), vp, vp, vp, vp, c_int,
                                                ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                                ctypes.POINTER(ctypes.c_float), vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(status, plan=None):
    if status != PISCO_OK:
        msg = load_library().pisco_last_error(plan)
        raise PiscoError(status, msg.decode() if msg else "")


def _f64(t):
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("pointing arrays must be contiguous float64 CUDA tensors")
    return t


def pisco_plan_create(nside, radius, sky, dets, beam_grids, omega_tilde=None,
                      precision=PISCO_FP32, tile_samples=0, pixels_per_thread=0, beam_fetch=0):
    """Create a plan; returns an opaque handle (int).  sky: (3, 12 nside^2) CUDA tensor
    (float32 or float64); dets: list of (zeta, eps, s_resp); beam_grids: (n_det, 6, N, N)
    float32 CUDA tensor."""
    lib = load_library()
    mr = precision in (PISCO_BF16_MR, PISCO_FP16_MR)
    if mr:
        want = torch.bfloat16 if precision == PISCO_BF16_MR else torch.float16
        if sky.dtype != want or not sky.is_cuda or sky.dim() != 3 or sky.shape[1] != 3:
            raise ValueError(f"a multi-realization plan takes a ({12 * nside * nside}, 3, n_real) {want} CUDA tensor")
    elif sky.dtype not in (torch.float32, torch.float64) or not sky.is_cuda:
        raise ValueError("sky must be a float32/float64 CUDA tensor")
    if beam_grids.dtype != torch.float32 or not beam_grids.is_cuda:
        raise ValueError("beam_grids must be a float32 CUDA tensor")
    sky, beam_grids = sky.contiguous(), beam_grids.contiguous()  # the plan copies both
    n_det = len(dets)
    if beam_grids.dim() != 4 or beam_grids.shape[0] != n_det or beam_grids.shape[1] != 6 \
            or beam_grids.shape[2] != beam_grids.shape[3]:
        raise ValueError("beam_grids must have shape (n_det, 6, N, N)")
    if not mr and tuple(sky.shape) != (3, 12 * nside * nside):
        raise ValueError("sky must have shape (3, 12 nside^2)")
    if mr and sky.shape[0] != 12 * nside * nside:
        raise ValueError("the realization stack must have shape (12 nside^2, 3, n_real)")
    arr = (pisco_detector * n_det)(*[pisco_detector(*map(float, d)) for d in dets])
    om = None if omega_tilde is None else (ctypes.c_double * n_det)(*map(float, omega_tilde))
    n_real = int(sky.shape[2]) if mr else 1
    opt = pisco_options(precision, tile_samples, pixels_per_thread, beam_fetch, n_real)
    handle = ctypes.c_void_p()
    dtype_code = {torch.float64: PISCO_DTYPE_F64, torch.float32: PISCO_DTYPE_F32,
                  torch.bfloat16: PISCO_DTYPE_BF16, torch.float16: PISCO_DTYPE_F16}[sky.dtype]
    st = lib.pisco_plan_create(ctypes.byref(handle), int(nside), float(radius), _ptr(sky), dtype_code,
                               n_det, arr, int(beam_grids.shape[-1]), _ptr(beam_grids), om,
                               ctypes.byref(opt), _stream())
    _check(st)
    return handle.value


def pisco_plan_destroy(plan):
    load_library().pisco_plan_destroy(plan)


def pisco_plan_omega(plan, det=0):
    om, sc = ctypes.c_double(), ctypes.c_double()
    _check(load_library().pisco_plan_omega(plan, det, ctypes.byref(om), ctypes.byref(sc)), plan)
    return om.value, sc.value


def pisco_convolve(plan, det, theta, phi, psi, tod):
    n = theta.numel()
    _check(load_library().pisco_convolve(plan, det, n, _ptr(_f64(theta)), _ptr(_f64(phi)),
                                         _ptr(_f64(psi)), _ptr(tod), _stream()), plan)
    return tod


def pisco_convolve_batched(plan, offsets, theta, phi, psi, tod):
    n_det = len(offsets) - 1
    off = (ctypes.c_int64 * len(offsets))(*map(int, offsets))
    _check(load_library().pisco_convolve_batched(plan, n_det, off, _ptr(_f64(theta)), _ptr(_f64(phi)),
                                                 _ptr(_f64(psi)), _ptr(tod), _stream()), plan)
    return tod


def pisco_beam_grids_from_healpix(maps, nside_b, radius, grid_n, grids=None):
    """Tangent-plane grids (..., grid_n, grid_n) float32 of HEALPix beam maps (..., 12 nside_b^2)."""
    if maps.dtype != torch.float32 or not maps.is_cuda:
        raise ValueError("maps must be a float32 CUDA tensor")
    maps = maps.contiguous()
    npix = 12 * nside_b * nside_b
    if maps.shape[-1] != npix:
        raise ValueError(f"maps must have last dimension 12 nside_b^2 = {npix}")
    lead = tuple(maps.shape[:-1])
    n_maps = maps.numel() // npix
    if grids is None:
        grids = torch.empty(lead + (grid_n, grid_n), dtype=torch.float32, device=maps.device)
    _check(load_library().pisco_beam_grids_from_healpix(int(nside_b), n_maps, _ptr(maps), float(radius),
                                                        int(grid_n), _ptr(grids), _stream()))
    return grids


def pisco_plan_autotune(plan, det, theta, phi, psi, reps=2):
    """Time the FP32 tile shapes on these pointings; the plan keeps the fastest.
    Returns (tile_samples, pixels_per_thread, ms per launch)."""
    scratch = torch.empty(theta.numel(), dtype=torch.float32, device=theta.device)
    t, p, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    _check(load_library().pisco_plan_autotune(plan, det, theta.numel(), _ptr(_f64(theta)), _ptr(_f64(phi)),
                                              _ptr(_f64(psi)), _ptr(scratch), int(reps), ctypes.byref(t),
                                              ctypes.byref(p), ctypes.byref(ms), _stream()), plan)
    return t.value, p.value, ms.value


def pisco_plan_autotune_batched(plan, offsets, theta, phi, psi, reps=2):
    """Time the FP32 tile shapes on a focal plane's slices (offsets as for convolve_batched); the
    plan keeps the fastest.  Returns (tile_samples, pixels_per_thread, ms per launch)."""
    n_det = len(offsets) - 1
    off = (ctypes.c_int64 * (n_det + 1))(*[int(x) for x in offsets])
    scratch = torch.empty(theta.numel(), dtype=torch.float32, device=theta.device)
    t, p, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    _check(load_library().pisco_plan_autotune_batched(plan, n_det, off, _ptr(_f64(theta)), _ptr(_f64(phi)),
                                                      _ptr(_f64(psi)), _ptr(scratch), int(reps), ctypes.byref(t),
                                                      ctypes.byref(p), ctypes.byref(ms), _stream()), plan)
    return t.value, p.value, ms.value


def pisco_ang2pix(nside, theta, phi, pix=None):
    """RING pixel (int64, -1 for invalid angles) of each direction."""
    if pix is None:
        pix = torch.empty(theta.numel(), dtype=torch.int64, device=theta.device)
    _check(load_library().pisco_ang2pix(int(nside), theta.numel(), _ptr(_f64(theta)), _ptr(_f64(phi)), _ptr(pix),
                                        _stream()))
    return pix


def pisco_map_accumulate(nside, theta, phi, psi, det, tod, acc=None, accumulate=False):
    """Per-pixel normal equations acc (10, 12 nside^2) float64 of one detector's TOD (float32/64)."""
    if acc is None:
        acc = torch.empty(10, 12 * nside * nside, dtype=torch.float64, device=theta.device)
    if tod.dtype not in (torch.float32, torch.float64) or not tod.is_cuda or not tod.is_contiguous():
        raise ValueError("tod must be a contiguous float32/float64 CUDA tensor")
    d = pisco_detector(*map(float, det))
    code = PISCO_DTYPE_F32 if tod.dtype == torch.float32 else PISCO_DTYPE_F64
    _check(load_library().pisco_map_accumulate(int(nside), theta.numel(), _ptr(_f64(theta)), _ptr(_f64(phi)),
                                               _ptr(_f64(psi)), ctypes.byref(d), _ptr(tod), code, _ptr(acc),
                                               int(bool(accumulate)), _stream()))
    return acc


def pisco_map_solve(nside, acc, rcond_min=1e-6, maps=None):
    """Binned I, Q, U maps (3, 12 nside^2) float64 from the normal equations (NaN where unsolved)."""
    if maps is None:
        maps = torch.empty(3, 12 * nside * nside, dtype=torch.float64, device=acc.device)
    _check(load_library().pisco_map_solve(int(nside), _ptr(acc), float(rcond_min), _ptr(maps), _stream()))
    return maps


def binned_map(nside, theta, phi, psi, det, tod, rcond_min=1e-6):
    """(maps (3, Npix) float64, hits (Npix,) int64) of one detector's TOD."""
    acc = pisco_map_accumulate(nside, theta, phi, psi, det, tod)
    return pisco_map_solve(nside, acc, rcond_min), acc[9].round().to(torch.int64)


def pisco_convolve_psb(plan, det, theta, phi, psi, zeta, tod):
    """TODs (len(zeta), n) of detector det's beam at polarisation angles zeta (radians)."""
    n = theta.numel()
    z = (ctypes.c_double * len(zeta))(*map(float, zeta))
    _check(load_library().pisco_convolve_psb(plan, det, n, _ptr(_f64(theta)), _ptr(_f64(phi)),
                                             _ptr(_f64(psi)), len(zeta), z, _ptr(tod), _stream()), plan)
    return tod


def pisco_adjoint(plan, det, theta, phi, psi, tod, maps, accumulate=False):
    n = theta.numel()
    _check(load_library().pisco_adjoint(plan, det, n, _ptr(_f64(theta)), _ptr(_f64(phi)),
                                        _ptr(_f64(psi)), _ptr(tod), _ptr(maps), int(bool(accumulate)),
                                        _stream()), plan)
    return maps


def pisco_adjoint_sky_beam(plan, det, theta, phi, psi, tod, maps, grad_grids, accumulate=False):
    n = theta.numel()
    _check(load_library().pisco_adjoint_sky_beam(plan, det, n, _ptr(_f64(theta)), _ptr(_f64(phi)),
                                                 _ptr(_f64(psi)), _ptr(tod), _ptr(maps), _ptr(grad_grids),
                                                 int(bool(accumulate)), _stream()), plan)
    return maps, grad_grids


def pisco_disc_count(plan, theta, phi, counts):
    n = theta.numel()
    _check(load_library().pisco_disc_count(plan, n, _ptr(_f64(theta)), _ptr(_f64(phi)), _ptr(counts),
                                           _stream()), plan)
    return counts


def pisco_convolve_host(plan, det, h_theta, h_phi, h_psi, h_tod):
    """Host-buffer variant: CPU tensors in, CPU tensor out (pinned memory overlaps copies)."""
    for t in (h_theta, h_phi, h_psi, h_tod):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError("pisco_convolve_host takes contiguous CPU tensors")
    n = h_theta.numel()
    _check(load_library().pisco_convolve_host(plan, det, n, _ptr(h_theta), _ptr(h_phi), _ptr(h_psi),
                                              _ptr(h_tod)), plan)
    return h_tod


def pisco_beam_grid_adjoint(plan, det, theta, phi, psi, tod, grad_grids, accumulate=False):
    n = theta.numel()
    _check(load_library().pisco_beam_grid_adjoint(plan, det, n, _ptr(_f64(theta)), _ptr(_f64(phi)),
                                                  _ptr(_f64(psi)), _ptr(tod), _ptr(grad_grids),
                                                  int(bool(accumulate)), _stream()), plan)
    return grad_grids


def pisco_beam_grid_adjoint_static(plan, det, theta, phi, psi, tod, grad_grids, accumulate=False):
    """pisco_beam_grid_adjoint without allocation (scratch in the library's static array, grid_n <= 512)."""
    n = theta.numel()
    _check(load_library().pisco_beam_grid_adjoint_static(plan, det, n, _ptr(_f64(theta)), _ptr(_f64(phi)),
                                                         _ptr(_f64(psi)), _ptr(tod), _ptr(grad_grids),
                                                         int(bool(accumulate)), _stream()), plan)
    return grad_grids


def pisco_omega_adjoint(plan, det, tod, tod_grad, grad_grids):
    _check(load_library().pisco_omega_adjoint(plan, det, tod.numel(), _ptr(tod), _ptr(tod_grad),
                                              _ptr(grad_grids), _stream()), plan)
    return grad_grids


def pisco_update_beams(plan, beam_grids, omega_tilde=None):
    if beam_grids.dtype != torch.float32 or not beam_grids.is_cuda:
        raise ValueError("beam_grids must be a float32 CUDA tensor")
    beam_grids = beam_grids.contiguous()
    om = None if omega_tilde is None else (ctypes.c_double * len(omega_tilde))(*map(float, omega_tilde))
    _check(load_library().pisco_update_beams(plan, _ptr(beam_grids), om, _stream()), plan)


def pisco_sync_status(plan):
    _check(load_library().pisco_sync_status(plan, _stream()), plan)


class Plan:
    """Owning wrapper: ``Plan(...)`` creates, ``close()`` / context exit destroys."""

    def __init__(self, nside, radius, sky, dets, beam_grids, omega_tilde=None, precision=PISCO_FP32,
                 tile_samples=0, pixels_per_thread=0, beam_fetch=0):
        self.nside, self.radius, self.precision = nside, radius, precision
        self.n_det = len(dets)
        self.grid_n = int(beam_grids.shape[-1])
        self.n_real = int(sky.shape[2]) if precision in (PISCO_BF16_MR, PISCO_FP16_MR) else 1
        self.handle = pisco_plan_create(nside, radius, sky, dets, beam_grids, omega_tilde, precision,
                                        tile_samples, pixels_per_thread, beam_fetch)

    @property
    def out_dtype(self):
        return torch.float64 if self.precision == PISCO_FP64_PLAIN else torch.float32

    def _out_shape(self, n):
        return (n, self.n_real) if self.n_real > 1 else (n,)

    def omega(self, det=0):
        return pisco_plan_omega(self.handle, det)

    def convolve(self, theta, phi, psi, det=0, out=None):
        if out is None:
            out = torch.empty(self._out_shape(theta.numel()), dtype=self.out_dtype, device=theta.device)
        return pisco_convolve(self.handle, det, theta, phi, psi, out)

    def autotune(self, theta, phi, psi, det=0, reps=2):
        """Pick the FP32 tile shape by timing it on these pointings: (tile_samples, pixels_per_thread, ms)."""
        return pisco_plan_autotune(self.handle, det, theta, phi, psi, reps)

    def autotune_batched(self, offsets, theta, phi, psi, reps=2):
        """Pick the FP32 tile shape by timing a focal-plane slice: (tile_samples, pixels_per_thread, ms)."""
        return pisco_plan_autotune_batched(self.handle, offsets, theta, phi, psi, reps)

    def convolve_batched(self, offsets, theta, phi, psi, out=None):
        if out is None:
            out = torch.empty(self._out_shape(theta.numel()), dtype=self.out_dtype, device=theta.device)
        return pisco_convolve_batched(self.handle, offsets, theta, phi, psi, out)

    def convolve_psb(self, theta, phi, psi, zeta, det=0, out=None):
        """One pass for detectors sharing det's beam, eps and s at angles zeta: (len(zeta), n) float32."""
        if out is None:
            out = torch.empty(len(zeta), theta.numel(), dtype=torch.float32, device=theta.device)
        return pisco_convolve_psb(self.handle, det, theta, phi, psi, zeta, out)

    def adjoint(self, theta, phi, psi, tod, det=0, maps=None, accumulate=False):
        if maps is None:
            maps = torch.empty(3, 12 * self.nside ** 2, dtype=self.out_dtype, device=theta.device)
        return pisco_adjoint(self.handle, det, theta, phi, psi, tod, maps, accumulate)

    def beam_grid_adjoint(self, theta, phi, psi, tod, det=0, grad=None, accumulate=False):
        if grad is None:
            grad = torch.empty(6, self.grid_n, self.grid_n, dtype=self.out_dtype, device=theta.device)
        return pisco_beam_grid_adjoint(self.handle, det, theta, phi, psi, tod, grad, accumulate)

    def adjoint_sky_beam(self, theta, phi, psi, tod, det=0, maps=None, grad=None, accumulate=False):
        """Both transposes in one pass (FP32 plans): (maps (3, Npix), grad (6, N, N))."""
        if maps is None:
            maps = torch.empty(3, 12 * self.nside ** 2, dtype=self.out_dtype, device=theta.device)
        if grad is None:
            grad = torch.empty(6, self.grid_n, self.grid_n, dtype=self.out_dtype, device=theta.device)
        return pisco_adjoint_sky_beam(self.handle, det, theta, phi, psi, tod, maps, grad, accumulate)

    def omega_adjoint(self, tod, tod_grad, grad, det=0):
        return pisco_omega_adjoint(self.handle, det, tod, tod_grad, grad)

    def update_beams(self, beam_grids, omega_tilde=None):
        pisco_update_beams(self.handle, beam_grids, omega_tilde)

    def disc_count(self, theta, phi):
        counts = torch.empty(theta.numel(), dtype=torch.int32, device=theta.device)
        return pisco_disc_count(self.handle, theta, phi, counts)

    def convolve_host(self, theta, phi, psi, det=0, out=None):
        out = torch.empty(theta.numel(), dtype=self.out_dtype) if out is None else out
        return pisco_convolve_host(self.handle, det, theta, phi, psi, out)

    def sync_status(self):
        pisco_sync_status(self.handle)

    def inject_mr_stall(self, cycles):
        """Test hook: the next multi-realization launch times out on a wait (PISCO_ETIMEOUT)."""
        _check(load_library().pisco_inject_mr_stall(self.handle, int(cycles)), self.handle)

    def close(self):
        if self.handle:
            pisco_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
