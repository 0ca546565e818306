// C ABI: argument validation, plan lifetime and launches.  The arithmetic
// lives in the kernels (pisco_plan.cu, pisco_fast.cuh, pisco_plain.cu, pisco_mr.cu).

#include "pisco_internal.cuh"

#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

using namespace pisco;

static thread_local char g_create_error[512] = "";

namespace pisco {
void set_error(pisco_plan* plan, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    char* dst = plan ? plan->msg : g_create_error;
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
}
}  // namespace pisco

#define PISCO_CUDA(plan, call)                                                        \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            set_error(plan, "%s failed: %s", #call, cudaGetErrorString(e_));          \
            return PISCO_ECUDA;                                                       \
        }                                                                             \
    } while (0)

// A pointer the kernels may dereference: device or managed memory of the current device.

bool pisco::is_device_ptr(const void* p) {
    if (p == nullptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static void free_plan(pisco_plan* p) {
    if (!p) return;
    cudaFree(p->d_rings);
    cudaFree(p->d_sky);
    cudaFree(p->d_beam);
    cudaFree(p->d_err);
    cudaFree(p->d_gscratch);
    if (p->h_tex)
        for (int k = 0; k < 3 * p->n_det; ++k)
            if (p->h_tex[k]) cudaDestroyTextureObject(p->h_tex[k]);
    if (p->h_arrays)
        for (int k = 0; k < 3 * p->n_det; ++k)
            if (p->h_arrays[k]) cudaFreeArray(p->h_arrays[k]);
    free(p->h_tex);
    free(p->h_arrays);
    for (int k = 0; k < 2; ++k) {
        if (p->hs[k]) cudaStreamDestroy(p->hs[k]);
        if (p->he[k]) cudaEventDestroy(p->he[k]);
        cudaFree(p->d_stage[k]);
    }
    free(p->h_omega);
    free(p->h_scale);
    free(p->h_dets);
    delete p;
}

// Packed-cell plans: the encoder flags a grid whose slopes fall outside the
// format's exponent range in word 2 of each detector's header (read after the
// plan kernels have finished).
static bool packed_range_ok(const pisco_plan* p, int* bad_det) {
    if (p->precision != PISCO_FP32 || p->beam_fetch != PISCO_FETCH_PACKED) return true;
    for (int d = 0; d < p->n_det; ++d) {
        unsigned flag = 0;
        if (cudaMemcpy(&flag, (const char*)p->d_beam + (size_t)d * p->beam_stride + 8, sizeof(unsigned),
                       cudaMemcpyDeviceToHost) != cudaSuccess || flag != 0) {
            cudaGetLastError();
            *bad_det = d;
            return false;
        }
    }
    return true;
}

// Folded node maps A, Bq', Cu' of every detector as 2-D float textures
// (created on first use, refilled by pisco_update_beams).
static cudaError_t build_textures(pisco_plan* p, const float* beam_grids, cudaStream_t s) {
    const int n = p->grid_n;
    const size_t nn = (size_t)n * n;
    cudaError_t e = cudaSuccess;
    if (!p->h_arrays) {
        p->h_arrays = (cudaArray_t*)calloc(3 * (size_t)p->n_det, sizeof(cudaArray_t));
        p->h_tex = (cudaTextureObject_t*)calloc(3 * (size_t)p->n_det, sizeof(cudaTextureObject_t));
        if (!p->h_arrays || !p->h_tex) return cudaErrorMemoryAllocation;
    }
    float* d_tmp = nullptr;
    e = cudaMalloc(&d_tmp, 3 * nn * sizeof(float));
    const cudaChannelFormatDesc desc = cudaCreateChannelDesc<float>();
    for (int d = 0; d < p->n_det && e == cudaSuccess; ++d) {
        e = launch_fold_nodes32(beam_grids + (size_t)d * 6 * nn, n, p->h_dets[d].eps, p->h_dets[d].zeta, d_tmp, s);
        for (int m = 0; m < 3 && e == cudaSuccess; ++m) {
            const int k = 3 * d + m;
            if (!p->h_arrays[k]) {
                e = cudaMallocArray(&p->h_arrays[k], &desc, n, n);
                if (e != cudaSuccess) break;
            }
            e = cudaMemcpy2DToArrayAsync(p->h_arrays[k], 0, 0, d_tmp + m * nn, n * sizeof(float), n * sizeof(float),
                                         n, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess || p->h_tex[k]) continue;
            cudaResourceDesc rd;
            memset(&rd, 0, sizeof(rd));
            rd.resType = cudaResourceTypeArray;
            rd.res.array.array = p->h_arrays[k];
            cudaTextureDesc td;
            memset(&td, 0, sizeof(td));
            td.addressMode[0] = cudaAddressModeClamp;
            td.addressMode[1] = cudaAddressModeClamp;
            td.filterMode = cudaFilterModePoint;
            td.readMode = cudaReadModeElementType;
            td.normalizedCoords = 0;
            e = cudaCreateTextureObject(&p->h_tex[k], &rd, &td, nullptr);
        }
        // the next detector reuses d_tmp: finish this one's copies first
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    cudaFree(d_tmp);
    return e;
}

extern "C" pisco_status pisco_plan_create(pisco_plan** out, int nside, double radius_rad, const void* sky,
                                          int sky_dtype, int n_det, const pisco_detector* dets, int grid_n,
                                          const float* beam_grids, const double* omega_tilde,
                                          const pisco_options* opt, void* stream) {
    if (!out) {
        set_error(nullptr, "out is NULL");
        return PISCO_EINVAL;
    }
    *out = nullptr;
    if (nside < 1 || nside > 8192) {
        set_error(nullptr, "nside %d outside [1, 8192]", nside);
        return PISCO_EINVAL;
    }
    if (!(radius_rad > 0.0 && radius_rad < 0.5 * kPi)) {
        set_error(nullptr, "radius %g outside (0, pi/2)", radius_rad);
        return PISCO_EINVAL;
    }
    const int precision0 = opt ? opt->precision : PISCO_FP32;
    const bool mr = precision0 == PISCO_BF16_MR || precision0 == PISCO_FP16_MR;
    if (!mr && sky_dtype != PISCO_DTYPE_F32 && sky_dtype != PISCO_DTYPE_F64) {
        set_error(nullptr, "sky_dtype %d is neither PISCO_DTYPE_F32 nor PISCO_DTYPE_F64", sky_dtype);
        return PISCO_EINVAL;
    }
    if (mr && sky_dtype != (precision0 == PISCO_BF16_MR ? PISCO_DTYPE_BF16 : PISCO_DTYPE_F16)) {
        set_error(nullptr, "a %s plan takes a %s realization stack", precision0 == PISCO_BF16_MR ? "BF16" : "FP16",
                  precision0 == PISCO_BF16_MR ? "PISCO_DTYPE_BF16" : "PISCO_DTYPE_F16");
        return PISCO_EINVAL;
    }
    const int n_real = mr ? opt->n_real : 1;
    if (mr && !(n_real >= 32 && n_real <= 256 && n_real % 32 == 0)) {
        set_error(nullptr, "n_real %d is not a multiple of 32 in [32, 256]", n_real);
        return PISCO_EINVAL;
    }
    if (mr && 36LL * nside * nside >= INT_MAX) {
        // the tensor-core kernel addresses the stack's 3 Npix rows with 32-bit TMA coordinates
        set_error(nullptr, "multi-realization plans take nside <= 7723 (got %d)", nside);
        return PISCO_EINVAL;
    }
    if (n_det < 1 || !dets) {
        set_error(nullptr, "need n_det >= 1 detectors (got %d, dets=%p)", n_det, (const void*)dets);
        return PISCO_EINVAL;
    }
    for (int d = 0; d < n_det; ++d) {
        if (!std::isfinite(dets[d].zeta) || !std::isfinite(dets[d].eps) || !std::isfinite(dets[d].s_resp)) {
            set_error(nullptr, "detector %d has a non-finite parameter", d);
            return PISCO_EINVAL;
        }
        if (omega_tilde && !(omega_tilde[d] > 0.0 && std::isfinite(omega_tilde[d]))) {
            set_error(nullptr, "omega_tilde[%d] = %g is not a positive finite number", d, omega_tilde[d]);
            return PISCO_EINVAL;
        }
    }
    if (grid_n < 2 || grid_n > 4096) {
        set_error(nullptr, "grid_n %d outside [2, 4096]", grid_n);
        return PISCO_EINVAL;
    }
    const int precision = precision0;
    if (precision != PISCO_FP32 && precision != PISCO_FP64_PLAIN && !mr) {
        set_error(nullptr, "precision %d is not a PISCO_* precision", precision);
        return PISCO_EINVAL;
    }
    int tile = opt && opt->tile_samples ? opt->tile_samples : 16;
    if (tile != 8 && tile != 16 && tile != 32) {
        set_error(nullptr, "tile_samples %d is not 8, 16 or 32", tile);
        return PISCO_EINVAL;
    }
    int np = opt && opt->pixels_per_thread ? opt->pixels_per_thread : 1;
    if (np != 1 && np != 2) {
        set_error(nullptr, "pixels_per_thread %d is not 1 or 2", np);
        return PISCO_EINVAL;
    }
    int fetch = opt && opt->beam_fetch ? opt->beam_fetch : PISCO_FETCH_CELLS;
    if (mr) fetch = PISCO_FETCH_CELLS;  // the multi-realization kernel reads coefficient cells
    if (fetch != PISCO_FETCH_TEXTURE && fetch != PISCO_FETCH_CELLS && fetch != PISCO_FETCH_PACKED &&
        fetch != PISCO_FETCH_SHARED) {
        set_error(nullptr, "beam_fetch %d is not PISCO_FETCH_TEXTURE, _CELLS, _PACKED or _SHARED", fetch);
        return PISCO_EINVAL;
    }
    if (fetch == PISCO_FETCH_SHARED && precision0 == PISCO_FP32 && grid_n > kSharedMaxGridN) {
        set_error(nullptr, "grid_n %d exceeds %d, the largest node grid PISCO_FETCH_SHARED stages in shared memory",
                  grid_n, kSharedMaxGridN);
        return PISCO_EINVAL;
    }
    if (!is_device_ptr(sky) || !is_device_ptr(beam_grids)) {
        set_error(nullptr, "sky and beam_grids must be device pointers");
        return PISCO_EINVAL;
    }

    pisco_plan* p = new (std::nothrow) pisco_plan();
    if (!p) {
        set_error(nullptr, "out of host memory");
        return PISCO_ENOMEM;
    }
    p->nside = nside;
    p->nrings = 4 * nside - 1;
    p->npix = 12LL * nside * nside;
    p->n_det = n_det;
    p->grid_n = grid_n;
    p->precision = precision;
    p->tile_samples = tile;
    p->pixels_per_thread = np;
    p->beam_fetch = fetch;
    p->n_real = n_real;
    p->radius = radius_rad;
    p->cos_r = cos(radius_rad);
    p->omega_pix = 4.0 * kPi / (double)p->npix;
    p->h_omega = (double*)calloc(n_det, sizeof(double));
    p->h_scale = (double*)calloc(n_det, sizeof(double));
    p->h_dets = (pisco_detector*)calloc(n_det, sizeof(pisco_detector));
    if (!p->h_omega || !p->h_scale || !p->h_dets) {
        free_plan(p);
        set_error(nullptr, "out of host memory");
        return PISCO_ENOMEM;
    }
    memcpy(p->h_dets, dets, n_det * sizeof(pisco_detector));

    const size_t nn = (size_t)grid_n * grid_n;
    const size_t nc = (size_t)(grid_n - 1) * (grid_n - 1);
    if (precision == PISCO_FP64_PLAIN) p->beam_stride = 3 * nn * sizeof(double);
    else if (mr) p->beam_stride = nc * 4 * sizeof(float4);
    else if (fetch == PISCO_FETCH_CELLS) p->beam_stride = nc * 4 * sizeof(float4);
    else if (fetch == PISCO_FETCH_PACKED) p->beam_stride = (nc + 1) * 32;  // 32-byte header + cells
    else if (fetch == PISCO_FETCH_SHARED) p->beam_stride = nn * sizeof(float4);  // folded nodes (A, Bq', Cu', 0)
    else p->beam_stride = 0;
    const size_t sky_bytes = mr ? (size_t)p->npix * 3 * n_real * 2
                             : precision == PISCO_FP32 ? p->npix * sizeof(float4) : 3 * p->npix * sizeof(double);
    double* d_omega = nullptr;
    cudaError_t e = cudaMalloc(&p->d_rings, p->nrings * sizeof(RingInfo));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_sky, sky_bytes);
    if (e == cudaSuccess && p->beam_stride) e = cudaMalloc(&p->d_beam, p->beam_stride * n_det);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&d_omega, n_det * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_omega);
        free_plan(p);
        set_error(nullptr, "device allocation failed: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? PISCO_ENOMEM : PISCO_ECUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemsetAsync(p->d_err, 0, sizeof(int), s);
    if (e == cudaSuccess && mr) {
        // realization stacks are stored as given ([Npix][3][n_real], 16-bit)
        e = cudaMemcpyAsync(p->d_sky, sky, sky_bytes, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = launch_plan_kernels(p, nullptr, -1, beam_grids, s, d_omega);
    } else if (e == cudaSuccess) {
        e = launch_plan_kernels(p, sky, sky_dtype, beam_grids, s, d_omega);
    }
    if (e == cudaSuccess && precision == PISCO_FP32 && fetch == PISCO_FETCH_TEXTURE) e = build_textures(p, beam_grids, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->h_omega, d_omega, n_det * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_omega);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_plan(p);
        set_error(nullptr, "plan set-up failed: %s", cudaGetErrorString(e));
        return PISCO_ECUDA;
    }
    int bad = -1;
    if (!packed_range_ok(p, &bad)) {
        set_error(nullptr, "detector %d: beam slopes outside the packed cells' range; use PISCO_FETCH_CELLS", bad);
        free_plan(p);
        return PISCO_EINVAL;
    }
    for (int d = 0; d < n_det; ++d) {
        if (omega_tilde) p->h_omega[d] = omega_tilde[d];
        if (!(p->h_omega[d] > 0.0) || !std::isfinite(p->h_omega[d])) {
            set_error(nullptr, "detector %d: Omega~ = %g from B_TT is not positive; pass omega_tilde", d,
                      p->h_omega[d]);
            free_plan(p);
            return PISCO_EINVAL;
        }
        p->h_scale[d] = 0.5 * dets[d].s_resp * p->omega_pix / p->h_omega[d];
    }
    *out = p;
    return PISCO_OK;
}

extern "C" void pisco_plan_destroy(pisco_plan* plan) {
    if (!plan) return;
    cudaDeviceSynchronize();
    free_plan(plan);
}

extern "C" const char* pisco_last_error(const pisco_plan* plan) { return plan ? plan->msg : g_create_error; }

extern "C" pisco_status pisco_plan_omega(const pisco_plan* plan, int det, double* omega_tilde, double* scale) {
    if (!plan || det < 0 || det >= plan->n_det) return PISCO_EINVAL;
    if (omega_tilde) *omega_tilde = plan->h_omega[det];
    if (scale) *scale = plan->h_scale[det];
    return PISCO_OK;
}

static LaunchParams base_params(const pisco_plan* p) {
    LaunchParams L;
    memset(&L, 0, sizeof(L));
    L.rings = p->d_rings;
    L.nrings = p->nrings;
    L.nside = p->nside;
    L.npix = p->npix;
    L.sky = p->d_sky;
    L.grid_n = p->grid_n;
    const double sin_r = sin(p->radius);
    L.sin_r = sin_r;
    L.h = 2.0 * sin_r / (double)(p->grid_n - 1);
    L.invh_f = (float)((double)(p->grid_n - 1) / (2.0 * sin_r));
    L.cg_f = (float)(0.5 * (double)(p->grid_n - 1));
    L.radius = p->radius;
    L.cos_r = p->cos_r;
    const double wr = 2.0 * sin(0.5 * p->radius) * sin(0.5 * p->radius);  // 1 - cos R
    L.wr_lo = (float)(wr * (1.0 - 2e-6));
    L.wr_hi = (float)(wr * (1.0 + 2e-6));
    L.group_cos = cos(0.25 * p->radius);
    L.group_dphi = (float)(0.5 * p->radius);
    L.err = p->d_err;
    return L;
}

pisco_status pisco::check_pointing(pisco_plan* plan, int64_t n, const double* a, const double* b,
                            const double* c) {
    if (n < 0) {
        set_error(plan, "n = %lld is negative", (long long)n);
        return PISCO_EINVAL;
    }
    if (n > 0 && (!is_device_ptr(a) || !is_device_ptr(b) || !is_device_ptr(c))) {
        set_error(plan, "theta, phi and psi must be device pointers");
        return PISCO_EINVAL;
    }
    return PISCO_OK;
}

pisco_status pisco::run(pisco_plan* plan, int mode, int d0, int nd, const int64_t* begin, const int64_t* count,
                 const double* theta, const double* phi, const double* psi, void* out, const void* tod_in,
                 int32_t* counts, cudaStream_t s, const PsbAngles* psb, void* out2, int grid_coef) {
    const long long per_tile = plan->precision == PISCO_FP64_PLAIN ? 1
                               : (plan->precision == PISCO_FP32 ? plan->tile_samples : 128);
    for (int c = 0; c < nd; c += kMaxDetPerLaunch) {
        LaunchParams L = base_params(plan);
        L.theta = theta;
        L.phi = phi;
        L.psi = psi;
        L.out = out;
        L.tod_in = tod_in;
        L.counts = counts;
        L.out2 = out2;
        L.grid_coef = grid_coef;
        const int m = nd - c < kMaxDetPerLaunch ? nd - c : kMaxDetPerLaunch;
        long long tiles = 0;
        int k = 0;
        for (int j = 0; j < m; ++j) {
            const int d = d0 + c + j;
            if (count[c + j] == 0) continue;
            DetEntry& e = L.det[k++];
            e.begin = begin[c + j];
            e.count = count[c + j];
            e.tile_begin = tiles;
            e.beam = plan->d_beam ? (const char*)plan->d_beam + (size_t)d * plan->beam_stride : nullptr;
            e.scale = plan->h_scale[d];
            for (int m = 0; m < 3; ++m) e.tex[m] = plan->h_tex ? plan->h_tex[3 * d + m] : 0;
            tiles += (e.count + per_tile - 1) / per_tile;
        }
        if (k == 0) continue;
        L.ndet = k;
        L.total_tiles = tiles;
        L.n_real = plan->n_real;
        if (psb) {
            L.n_zeta = psb->n;
            L.out_stride = psb->stride;
            for (int k = 0; k < psb->n; ++k) {
                L.psb_c2z[k] = psb->c2z[k];
                L.psb_s2z[k] = psb->s2z[k];
            }
        }
        cudaError_t e;
        if (plan->precision == PISCO_BF16_MR || plan->precision == PISCO_FP16_MR) {
            if (mode != kForward) {
                set_error(plan, "multi-realization plans support pisco_convolve and pisco_convolve_batched only");
                return PISCO_EUNSUPPORTED;
            }
            L.stall_cycles = plan->mr_stall;
            plan->mr_stall = 0;
            e = launch_mr(L, plan->precision == PISCO_FP16_MR, s);
        } else if (plan->precision == PISCO_FP64_PLAIN) e = launch_plain(L, mode, s);
        else if (plan->beam_fetch == PISCO_FETCH_CELLS)
            e = launch_fast_cells(L, mode, plan->tile_samples, plan->pixels_per_thread, s);
        else if (plan->beam_fetch == PISCO_FETCH_PACKED)
            e = launch_fast_packed(L, mode, plan->tile_samples, plan->pixels_per_thread, s);
        else if (plan->beam_fetch == PISCO_FETCH_SHARED)
            e = launch_fast_shared(L, mode, plan->tile_samples, plan->pixels_per_thread, s);
        else e = launch_fast_texture(L, mode, plan->tile_samples, plan->pixels_per_thread, s);
        if (e != cudaSuccess) {
            set_error(plan, "kernel launch failed: %s", cudaGetErrorString(e));
            return PISCO_ECUDA;
        }
    }
    return PISCO_OK;
}

extern "C" pisco_status pisco_convolve(pisco_plan* plan, int det, int64_t n, const double* theta,
                                       const double* phi, const double* psi, void* tod, void* stream) {
    if (!plan) return PISCO_EINVAL;
    if (det < 0 || det >= plan->n_det) {
        set_error(plan, "detector %d outside [0, %d)", det, plan->n_det);
        return PISCO_EINVAL;
    }
    pisco_status st = check_pointing(plan, n, theta, phi, psi);
    if (st != PISCO_OK) return st;
    if (n == 0) return PISCO_OK;
    if (!is_device_ptr(tod)) {
        set_error(plan, "tod must be a device pointer");
        return PISCO_EINVAL;
    }
    const int64_t begin = 0, count = n;
    return run(plan, kForward, det, 1, &begin, &count, theta, phi, psi, tod, nullptr, nullptr,
               (cudaStream_t)stream);
}

extern "C" pisco_status pisco_convolve_batched(pisco_plan* plan, int n_det, const int64_t* offsets,
                                               const double* theta, const double* phi, const double* psi,
                                               void* tod, void* stream) {
    if (!plan) return PISCO_EINVAL;
    if (n_det < 1 || n_det > plan->n_det || !offsets) {
        set_error(plan, "n_det %d outside [1, %d] or offsets NULL", n_det, plan->n_det);
        return PISCO_EINVAL;
    }
    if (offsets[0] != 0) {
        set_error(plan, "offsets[0] must be 0");
        return PISCO_EINVAL;
    }
    int64_t* count = (int64_t*)malloc(n_det * sizeof(int64_t));
    if (!count) return PISCO_ENOMEM;
    for (int d = 0; d < n_det; ++d) {
        count[d] = offsets[d + 1] - offsets[d];
        if (count[d] < 0) {
            free(count);
            set_error(plan, "offsets must be non-decreasing (detector %d)", d);
            return PISCO_EINVAL;
        }
    }
    const int64_t total = offsets[n_det];
    pisco_status st = check_pointing(plan, total, theta, phi, psi);
    if (st == PISCO_OK && total > 0 && !is_device_ptr(tod)) {
        set_error(plan, "tod must be a device pointer");
        st = PISCO_EINVAL;
    }
    if (st == PISCO_OK && total > 0)
        st = run(plan, kForward, 0, n_det, offsets, count, theta, phi, psi, tod, nullptr, nullptr,
                 (cudaStream_t)stream);
    free(count);
    return st;
}

extern "C" pisco_status pisco_convolve_psb(pisco_plan* plan, int det, int64_t n, const double* theta,
                                           const double* phi, const double* psi, int n_zeta, const double* zeta,
                                           void* tod, void* stream) {
    if (!plan) return PISCO_EINVAL;
    if (det < 0 || det >= plan->n_det) {
        set_error(plan, "detector %d outside [0, %d)", det, plan->n_det);
        return PISCO_EINVAL;
    }
    if (n_zeta < 1 || n_zeta > kMaxPsb || !zeta) {
        set_error(plan, "n_zeta %d outside [1, %d] or zeta NULL", n_zeta, kMaxPsb);
        return PISCO_EINVAL;
    }
    for (int k = 0; k < n_zeta; ++k)
        if (!std::isfinite(zeta[k])) {
            set_error(plan, "zeta[%d] is not finite", k);
            return PISCO_EINVAL;
        }
    if (plan->precision != PISCO_FP32 || plan->beam_fetch == PISCO_FETCH_TEXTURE) {
        set_error(plan, "pisco_convolve_psb needs an FP32 plan whose beam fetch is not PISCO_FETCH_TEXTURE");
        return PISCO_EUNSUPPORTED;
    }
    pisco_status st = check_pointing(plan, n, theta, phi, psi);
    if (st != PISCO_OK) return st;
    if (n == 0) return PISCO_OK;
    if (!is_device_ptr(tod)) {
        set_error(plan, "tod must be a device pointer");
        return PISCO_EINVAL;
    }
    PsbAngles a;
    a.n = n_zeta;
    a.stride = n;
    for (int k = 0; k < n_zeta; ++k) {
        const double d = 2.0 * (zeta[k] - plan->h_dets[det].zeta);
        a.c2z[k] = (float)cos(d);
        a.s2z[k] = (float)sin(d);
    }
    const int64_t begin = 0, count = n;
    return run(plan, kPsb, det, 1, &begin, &count, theta, phi, psi, tod, nullptr, nullptr, (cudaStream_t)stream,
               &a);
}

extern "C" pisco_status pisco_adjoint(pisco_plan* plan, int det, int64_t n, const double* theta,
                                      const double* phi, const double* psi, const void* tod, void* maps,
                                      int accumulate, void* stream) {
    if (!plan) return PISCO_EINVAL;
    if (det < 0 || det >= plan->n_det) {
        set_error(plan, "detector %d outside [0, %d)", det, plan->n_det);
        return PISCO_EINVAL;
    }
    pisco_status st = check_pointing(plan, n, theta, phi, psi);
    if (st != PISCO_OK) return st;
    if (!is_device_ptr(maps) || (n > 0 && !is_device_ptr(tod))) {
        set_error(plan, "tod and maps must be device pointers");
        return PISCO_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t elem = plan->precision == PISCO_FP32 ? sizeof(float) : sizeof(double);
    if (!accumulate) PISCO_CUDA(plan, cudaMemsetAsync(maps, 0, 3 * plan->npix * elem, s));
    if (n == 0) return PISCO_OK;
    const int64_t begin = 0, count = n;
    return run(plan, kAdjoint, det, 1, &begin, &count, theta, phi, psi, maps, tod, nullptr, s);
}

extern "C" pisco_status pisco_disc_count(pisco_plan* plan, int64_t n, const double* theta, const double* phi,
                                         int32_t* counts, void* stream) {
    if (!plan) return PISCO_EINVAL;
    pisco_status st = check_pointing(plan, n, theta, phi, theta);
    if (st != PISCO_OK) return st;
    if (n == 0) return PISCO_OK;
    if (!is_device_ptr(counts)) {
        set_error(plan, "counts must be a device pointer");
        return PISCO_EINVAL;
    }
    // psi does not change the disc: theta stands in for it.
    const int64_t begin = 0, count = n;
    return run(plan, kCount, 0, 1, &begin, &count, theta, phi, theta, nullptr, nullptr, counts,
               (cudaStream_t)stream);
}

extern "C" pisco_status pisco_convolve_host(pisco_plan* plan, int det, int64_t n, const double* h_theta,
                                            const double* h_phi, const double* h_psi, void* h_tod) {
    if (!plan) return PISCO_EINVAL;
    if (det < 0 || det >= plan->n_det) {
        set_error(plan, "detector %d outside [0, %d)", det, plan->n_det);
        return PISCO_EINVAL;
    }
    if (n < 0 || (n > 0 && (!h_theta || !h_phi || !h_psi || !h_tod))) {
        set_error(plan, "bad host buffers or n");
        return PISCO_EINVAL;
    }
    if (plan->n_real > 1) {
        set_error(plan, "pisco_convolve_host does not take multi-realization plans");
        return PISCO_EUNSUPPORTED;
    }
    if (n == 0) return PISCO_OK;
    const size_t out_elem = plan->precision == PISCO_FP32 ? sizeof(float) : sizeof(double);
    const int64_t chunk = 1 << 20;
    const size_t need = (size_t)chunk * (3 * sizeof(double) + out_elem);
    if (plan->stage_bytes < need) {
        for (int k = 0; k < 2; ++k) {
            cudaFree(plan->d_stage[k]);
            plan->d_stage[k] = nullptr;
            PISCO_CUDA(plan, cudaMalloc(&plan->d_stage[k], need));
            if (!plan->hs[k]) PISCO_CUDA(plan, cudaStreamCreateWithFlags(&plan->hs[k], cudaStreamNonBlocking));
            if (!plan->he[k]) PISCO_CUDA(plan, cudaEventCreateWithFlags(&plan->he[k], cudaEventDisableTiming));
        }
        plan->stage_bytes = need;
    }
    for (int64_t c0 = 0, idx = 0; c0 < n; c0 += chunk, ++idx) {
        const int k = (int)(idx & 1);
        const int64_t m = n - c0 < chunk ? n - c0 : chunk;
        cudaStream_t s = plan->hs[k];
        double* dth = (double*)plan->d_stage[k];
        double* dph = dth + chunk;
        double* dps = dph + chunk;
        void* dtod = dps + chunk;
        PISCO_CUDA(plan, cudaMemcpyAsync(dth, h_theta + c0, m * sizeof(double), cudaMemcpyHostToDevice, s));
        PISCO_CUDA(plan, cudaMemcpyAsync(dph, h_phi + c0, m * sizeof(double), cudaMemcpyHostToDevice, s));
        PISCO_CUDA(plan, cudaMemcpyAsync(dps, h_psi + c0, m * sizeof(double), cudaMemcpyHostToDevice, s));
        const int64_t begin = 0, count = m;
        pisco_status st = run(plan, kForward, det, 1, &begin, &count, dth, dph, dps, dtod, nullptr, nullptr, s);
        if (st != PISCO_OK) return st;
        PISCO_CUDA(plan, cudaMemcpyAsync((char*)h_tod + c0 * out_elem, dtod, m * out_elem, cudaMemcpyDeviceToHost, s));
    }
    PISCO_CUDA(plan, cudaStreamSynchronize(plan->hs[0]));
    PISCO_CUDA(plan, cudaStreamSynchronize(plan->hs[1]));
    return PISCO_OK;
}

extern "C" pisco_status pisco_inject_mr_stall(pisco_plan* plan, int64_t cycles) {
    if (!plan) return PISCO_EINVAL;
    if (plan->precision != PISCO_BF16_MR && plan->precision != PISCO_FP16_MR) {
        set_error(plan, "pisco_inject_mr_stall needs a multi-realization plan");
        return PISCO_EUNSUPPORTED;
    }
    if (cycles < 1 || cycles > 10000000000LL) {
        set_error(plan, "stall of %lld cycles outside [1, 1e10]", (long long)cycles);
        return PISCO_EINVAL;
    }
    plan->mr_stall = cycles;
    return PISCO_OK;
}

extern "C" pisco_status pisco_sync_status(pisco_plan* plan, void* stream) {
    if (!plan) return PISCO_EINVAL;
    int h = 0;
    PISCO_CUDA(plan, cudaStreamSynchronize((cudaStream_t)stream));
    PISCO_CUDA(plan, cudaMemcpy(&h, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h != 0) {
        PISCO_CUDA(plan, cudaMemset(plan->d_err, 0, sizeof(int)));
        set_error(plan, "a kernel recorded error flags 0x%x%s", h,
                  (h & 2) ? " (a bounded wait on an mbarrier gave up)" : "");
        return (h & 2) ? PISCO_ETIMEOUT : PISCO_EDEVICE;
    }
    return PISCO_OK;
}

extern "C" pisco_status pisco_update_beams(pisco_plan* plan, const float* beam_grids, const double* omega_tilde,
                                           void* stream) {
    if (!plan) return PISCO_EINVAL;
    if (!is_device_ptr(beam_grids)) {
        set_error(plan, "beam_grids must be a device pointer");
        return PISCO_EINVAL;
    }
    for (int d = 0; omega_tilde && d < plan->n_det; ++d)
        if (!(omega_tilde[d] > 0.0 && std::isfinite(omega_tilde[d]))) {
            set_error(plan, "omega_tilde[%d] = %g is not a positive finite number", d, omega_tilde[d]);
            return PISCO_EINVAL;
        }
    cudaStream_t s = (cudaStream_t)stream;
    double* d_omega = nullptr;
    PISCO_CUDA(plan, cudaMalloc(&d_omega, plan->n_det * sizeof(double)));
    double* h = (double*)malloc(plan->n_det * sizeof(double));
    cudaError_t e = h ? cudaSuccess : cudaErrorMemoryAllocation;
    if (e == cudaSuccess) e = launch_beam_kernels(plan, beam_grids, s, d_omega);
    if (e == cudaSuccess && plan->precision == PISCO_FP32 && plan->beam_fetch == PISCO_FETCH_TEXTURE)
        e = build_textures(plan, beam_grids, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d_omega, plan->n_det * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_omega);
    if (e != cudaSuccess) {
        free(h);
        set_error(plan, "beam update failed: %s", cudaGetErrorString(e));
        return PISCO_ECUDA;
    }
    int bad = -1;
    if (!packed_range_ok(plan, &bad)) {
        free(h);
        set_error(plan, "detector %d: beam slopes outside the packed cells' range; use PISCO_FETCH_CELLS", bad);
        return PISCO_EINVAL;
    }
    for (int d = 0; d < plan->n_det; ++d) {
        const double om = omega_tilde ? omega_tilde[d] : h[d];
        if (!(om > 0.0) || !std::isfinite(om)) {
            free(h);
            set_error(plan, "detector %d: Omega~ = %g from B_TT is not positive; pass omega_tilde", d, om);
            return PISCO_EINVAL;
        }
        plan->h_omega[d] = om;
        plan->h_scale[d] = 0.5 * plan->h_dets[d].s_resp * plan->omega_pix / om;
    }
    free(h);
    return PISCO_OK;
}

// Bytes of a plan's folded beam-grid gradient scratch: per cell coefficient for FP32
// plans, per node for the plain path.
static size_t plan_grad_scratch_bytes(const pisco_plan* plan) {
    if (plan->precision == PISCO_FP64_PLAIN) return folded_grad_bytes(plan->grid_n, 1);
    const size_t a = folded_coef_grad_bytes(plan->grid_n), b = folded_grad_bytes(plan->grid_n, 0);
    return a > b ? a : b;
}

extern "C" pisco_status pisco_beam_grid_adjoint(pisco_plan* plan, int det, int64_t n, const double* theta,
                                                const double* phi, const double* psi, const void* tod,
                                                void* grad_grids, int accumulate, void* stream) {
    if (!plan) return PISCO_EINVAL;
    if (det < 0 || det >= plan->n_det) {
        set_error(plan, "detector %d outside [0, %d)", det, plan->n_det);
        return PISCO_EINVAL;
    }
    pisco_status st = check_pointing(plan, n, theta, phi, psi);
    if (st != PISCO_OK) return st;
    if (!is_device_ptr(grad_grids) || (n > 0 && !is_device_ptr(tod))) {
        set_error(plan, "tod and grad_grids must be device pointers");
        return PISCO_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int f64 = plan->precision == PISCO_FP64_PLAIN;
    // FP32 plans accumulate per cell coefficient, the plain path per node
    const size_t bytes = plan_grad_scratch_bytes(plan);
    if (!plan->d_gscratch) PISCO_CUDA(plan, cudaMalloc(&plan->d_gscratch, bytes));
    PISCO_CUDA(plan, cudaMemsetAsync(plan->d_gscratch, 0, bytes, s));
    if (n > 0) {
        const int64_t begin = 0, count = n;
        st = run(plan, kGrid, det, 1, &begin, &count, theta, phi, psi, plan->d_gscratch, tod, nullptr, s, nullptr,
                 nullptr, f64 ? 0 : 1);
        if (st != PISCO_OK) return st;
    }
    if (f64)
        PISCO_CUDA(plan, launch_unfold_grid(plan->d_gscratch, plan->grid_n, plan->h_dets[det].eps,
                                            plan->h_dets[det].zeta, grad_grids, accumulate, 1, s));
    else
        PISCO_CUDA(plan, launch_unfold_coef_grid((const float*)plan->d_gscratch, plan->grid_n,
                                                 plan->h_dets[det].eps, plan->h_dets[det].zeta,
                                                 (float*)grad_grids, accumulate, s));
    return PISCO_OK;
}

extern "C" pisco_status pisco_adjoint_sky_beam(pisco_plan* plan, int det, int64_t n, const double* theta,
                                               const double* phi, const double* psi, const void* tod, void* maps,
                                               void* grad_grids, int accumulate, void* stream) {
    if (!plan) return PISCO_EINVAL;
    if (det < 0 || det >= plan->n_det) {
        set_error(plan, "detector %d outside [0, %d)", det, plan->n_det);
        return PISCO_EINVAL;
    }
    if (plan->precision != PISCO_FP32) {
        set_error(plan, "pisco_adjoint_sky_beam needs an FP32 plan; call pisco_adjoint and "
                        "pisco_beam_grid_adjoint on plain plans");
        return PISCO_EUNSUPPORTED;
    }
    pisco_status st = check_pointing(plan, n, theta, phi, psi);
    if (st != PISCO_OK) return st;
    if (!is_device_ptr(maps) || !is_device_ptr(grad_grids) || (n > 0 && !is_device_ptr(tod))) {
        set_error(plan, "tod, maps and grad_grids must be device pointers");
        return PISCO_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = plan_grad_scratch_bytes(plan);
    if (!plan->d_gscratch) PISCO_CUDA(plan, cudaMalloc(&plan->d_gscratch, bytes));
    PISCO_CUDA(plan, cudaMemsetAsync(plan->d_gscratch, 0, bytes, s));
    if (!accumulate) PISCO_CUDA(plan, cudaMemsetAsync(maps, 0, 3 * (size_t)plan->npix * sizeof(float), s));
    if (n > 0) {
        const int64_t begin = 0, count = n;
        st = run(plan, kBoth, det, 1, &begin, &count, theta, phi, psi, maps, tod, nullptr, s, nullptr,
                 plan->d_gscratch, 1);
        if (st != PISCO_OK) return st;
    }
    PISCO_CUDA(plan, launch_unfold_coef_grid((const float*)plan->d_gscratch, plan->grid_n, plan->h_dets[det].eps,
                                             plan->h_dets[det].zeta, (float*)grad_grids, accumulate, s));
    return PISCO_OK;
}

extern "C" pisco_status pisco_omega_adjoint(pisco_plan* plan, int det, int64_t n, const void* tod,
                                            const void* tod_grad, void* grad_grids, void* stream) {
    if (!plan) return PISCO_EINVAL;
    if (det < 0 || det >= plan->n_det || n < 0) {
        set_error(plan, "detector %d outside [0, %d) or n < 0", det, plan->n_det);
        return PISCO_EINVAL;
    }
    if (!is_device_ptr(grad_grids) || (n > 0 && (!is_device_ptr(tod) || !is_device_ptr(tod_grad)))) {
        set_error(plan, "tod, tod_grad and grad_grids must be device pointers");
        return PISCO_EINVAL;
    }
    const int f64 = plan->precision == PISCO_FP64_PLAIN;
    PISCO_CUDA(plan, launch_omega_adjoint(tod, tod_grad, n, f64, plan->h_omega[det], 1.0, plan->grid_n,
                                          sin(plan->radius), grad_grids, (cudaStream_t)stream));
    return PISCO_OK;
}
