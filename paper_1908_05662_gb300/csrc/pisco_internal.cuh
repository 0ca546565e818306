// Internal types shared by the translation units of libpisco.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pisco.h"

namespace pisco {

constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoPi = 6.28318530717958647692;

// One HEALPix RING ring (Sec. 5.1).  FP64 geometry plus the FP32 copies the
// fast path reads per pixel.
struct RingInfo {
    double z;         // cos(theta) of the ring
    double s;         // sin(theta), from (1 - z)(1 + z) so it keeps precision near the poles
    double theta;     // colatitude
    double phi0;      // phi of pixel j = 0
    double dphi;      // phi step
    long long first;  // pixel number of j = 0
    int count;        // pixels in the ring
    float s_f;        // (float) s
    float inv_s2_f;   // (float) 1 / s^2
    float dphi_f;     // (float) dphi
};
static_assert(sizeof(RingInfo) == 64, "RingInfo layout");

// One detector's slice of a launch.
struct DetEntry {
    long long begin;       // first sample, index into the pointing arrays
    long long count;       // number of samples
    long long tile_begin;  // first tile (block) index of this detector
    const void* beam;      // FP32: 64-byte cells [(N-1)^2][16 floats]; FP64: double nodes [3][N][N]
    double scale;          // (s/2) Omega_pix / Omega~
    cudaTextureObject_t tex[3];  // FP32 texture fetch: folded node maps A, Bq', Cu' as 2-D float textures
};

constexpr int kMaxDetPerLaunch = 64;

enum Mode { kForward = 0, kAdjoint = 1, kCount = 2, kGrid = 3, kPsb = 4, kBoth = 5 };

constexpr int kMaxPsb = 8;  // polarisation angles per shared-geometry pass

// Parameters of the FP32 tile kernel and of the FP64 plain kernel (by value).
struct LaunchParams {
    const RingInfo* rings;
    int nrings;
    int nside;
    long long npix;
    const void* sky;       // FP32: float4 [npix] (I, Q, U, 0); FP64: double [3][npix]
    int grid_n;
    float invh_f, cg_f;    // FP32 path: 1 / h and (N - 1) / 2
    double sin_r, h;       // FP64 path grid: sin(R) and node spacing
    double radius, cos_r;
    float wr_lo, wr_hi;    // (1 - cos R)(1 -/+ 2e-6): FP32 membership band
    double group_cos;      // samples within this cosine share one disc traversal
    float group_dphi;      // ... and within this longitude offset
    const double* theta;
    const double* phi;
    const double* psi;
    void* out;             // forward: tod; adjoint: maps [3][npix]
    const void* tod_in;    // adjoint input
    int32_t* counts;       // count mode output
    int* err;
    void* out2;            // sky and beam-grid transposes in one pass: the folded beam-grid gradient
    int grid_coef;         // FP32 folded gradient per cell coefficient ([(N-1)^2][3][4]) instead of per node
    int n_real;            // multi-realization plans: realizations per pixel
    int n_zeta;            // shared-geometry pass: number of polarisation angles
    long long out_stride;  // shared-geometry pass: elements between the TODs of two angles
    float psb_c2z[kMaxPsb], psb_s2z[kMaxPsb];  // cos, sin of 2 (zeta_k - zeta of the plan's detector)
    double mr_wr;            // multi-realization kernel: 1 - cos R, and its FP32 re-decision band edges
    float mr_wr_lo, mr_wr_hi;
    long long wait_limit;    // multi-realization kernel: SM clocks a wait on an mbarrier may take (0: ~2 s)
    long long stall_cycles;  // multi-realization kernel, test hook: > 0 makes it wait this long, before it
                             // issues any copy or MMA, on an mbarrier nothing arrives on (a timeout)
    int ndet;
    long long total_tiles;
    DetEntry det[kMaxDetPerLaunch];
};

}  // namespace pisco

struct pisco_plan {
    int nside;
    int nrings;
    long long npix;
    int n_det;
    int grid_n;
    int precision;
    int tile_samples;
    int pixels_per_thread;
    int beam_fetch;    // PISCO_FETCH_CELLS, _TEXTURE, _PACKED or _SHARED
    int n_real;        // realizations (multi-realization plans), else 1
    double radius;
    double cos_r;
    double omega_pix;
    pisco::RingInfo* d_rings;
    void* d_sky;       // float4 [npix] or double [3][npix]
    void* d_beam;      // per detector FP32 cells or FP64 nodes, contiguous
    size_t beam_stride;  // bytes per detector in d_beam
    cudaArray_t* h_arrays;           // [n_det][3] texture fetch: folded node maps
    cudaTextureObject_t* h_tex;      // [n_det][3]
    double* h_omega;
    double* h_scale;
    pisco_detector* h_dets;
    int* d_err;
    // staging for pisco_convolve_host
    cudaStream_t hs[2];
    cudaEvent_t he[2];
    void* d_stage[2];
    size_t stage_bytes;
    void* d_gscratch;  // beam-grid adjoint: folded gradient [3][N][N] (float or double)
    long long mr_stall;  // test hook: stall cycles for the next multi-realization launch (0: none)
    char msg[512];
};

namespace pisco {

// Polarisation angles of a shared-geometry pass, as rotations relative to the plan detector's zeta.
struct PsbAngles {
    int n;
    long long stride;  // elements between the TODs of two angles
    float c2z[kMaxPsb], s2z[kMaxPsb];
};

// Host helpers shared by the API translation units (defined in pisco_api.cu).
bool is_device_ptr(const void* p);
pisco_status check_pointing(pisco_plan* plan, int64_t n, const double* a, const double* b, const double* c);
// Launch one path over detectors [d0, d0 + nd) with per-detector sample ranges.
pisco_status run(pisco_plan* plan, int mode, int d0, int nd, const int64_t* begin, const int64_t* count,
                 const double* theta, const double* phi, const double* psi, void* out, const void* tod_in,
                 int32_t* counts, cudaStream_t s, const PsbAngles* psb = nullptr, void* out2 = nullptr,
                 int grid_coef = 0);

// Bytes of the folded beam-grid gradient scratch: FP32 plans interleave the three
// folded maps per node with a pad ([N][N][4] floats), the plain path keeps [3][N][N] doubles.
inline size_t folded_grad_bytes(int grid_n, int f64) {
    return (size_t)grid_n * grid_n * (f64 ? 3 * sizeof(double) : 4 * sizeof(float));
}
// The same gradient per cell coefficient (FP32 plans' own scratch): [(N-1)^2][3][4] floats.
inline size_t folded_coef_grad_bytes(int grid_n) { return (size_t)(grid_n - 1) * (grid_n - 1) * 12 * sizeof(float); }

// Launchers (defined in the kernel translation units).
cudaError_t launch_fast_texture(const LaunchParams& p, int mode, int tile_samples, int np, cudaStream_t s);
cudaError_t launch_fast_cells(const LaunchParams& p, int mode, int tile_samples, int np, cudaStream_t s);
cudaError_t launch_fast_packed(const LaunchParams& p, int mode, int tile_samples, int np, cudaStream_t s);
cudaError_t launch_fast_shared(const LaunchParams& p, int mode, int tile_samples, int np, cudaStream_t s);
// Largest node grid the shared-memory fetch stages (16 bytes per node; 182 KB at 108 nodes).
constexpr int kSharedMaxGridN = 108;
cudaError_t launch_plain(const LaunchParams& p, int mode, cudaStream_t s);
cudaError_t launch_mr(const LaunchParams& p, int f16, cudaStream_t s);
cudaError_t launch_plan_kernels(pisco_plan* plan, const void* sky, int sky_dtype,
                                const float* grids, cudaStream_t s, double* d_omega_out);
cudaError_t launch_fold_nodes32(const float* grids, int n, double eps, double zeta, float* out3, cudaStream_t s);
cudaError_t launch_beam_kernels(pisco_plan* plan, const float* grids, cudaStream_t s, double* d_omega_out);
cudaError_t launch_unfold_coef_grid(const float* cgrad, int n, double eps, double zeta, float* grad, int accumulate,
                                   cudaStream_t s);
cudaError_t launch_unfold_grid(const void* folded, int n, double eps, double zeta, void* grad, int accumulate,
                               int f64, cudaStream_t s);
cudaError_t launch_omega_adjoint(const void* tod, const void* y, long long n, int f64, double omega, double scale_tod,
                                 int grid_n, double sin_r, void* grad_tt, cudaStream_t s);

void set_error(pisco_plan* plan, const char* fmt, ...);

}  // namespace pisco

namespace pisco {

// Geometry of RING ring index r (0-based; ring number i = r + 1) of a map of the given nside.
static __device__ __forceinline__ RingInfo make_ring(int r, int nside) {
    const long long n = nside;
    const long long i = r + 1;
    RingInfo R;
    double omz;
    if (i < n) {
        omz = (double)(i * i) / (3.0 * (double)(n * n));
        R.z = 1.0 - omz;
        R.count = (int)(4 * i);
        R.dphi = kPi / (2.0 * (double)i);
        R.phi0 = 0.5 * R.dphi;
        R.first = 2 * i * (i - 1);
    } else if (i <= 3 * n) {
        R.z = 4.0 / 3.0 - 2.0 * (double)i / (3.0 * (double)n);
        omz = 1.0 - R.z;
        R.count = (int)(4 * n);
        R.dphi = kPi / (2.0 * (double)n);
        R.phi0 = 0.5 * (double)((i - n + 1) % 2) * R.dphi;
        R.first = 2 * n * (n - 1) + (i - n) * 4 * n;
    } else {
        const long long m = 4 * n - i;
        double opz = (double)(m * m) / (3.0 * (double)(n * n));
        R.z = -(1.0 - opz);
        omz = 1.0 - R.z;
        R.count = (int)(4 * m);
        R.dphi = kPi / (2.0 * (double)m);
        R.phi0 = 0.5 * R.dphi;
        R.first = 12 * n * n - 2 * m * (m + 1);
    }
    R.s = sqrt(omz * (1.0 + R.z));
    R.theta = atan2(R.s, R.z);
    R.s_f = (float)R.s;
    R.inv_s2_f = (float)(1.0 / (R.s * R.s));
    R.dphi_f = (float)R.dphi;
    return R;
}

// Continuous RING ring number (1-based) of colatitude cosine z (inverse of the
// ring heights of Sec. 5.1's scheme); used to bound the rings a disc can meet.
static __device__ __forceinline__ double ring_number(double z, int nside) {
    if (z > 2.0 / 3.0) return nside * sqrt(3.0 * (1.0 - z));
    if (z < -2.0 / 3.0) return 4.0 * nside - nside * sqrt(3.0 * (1.0 + z));
    return nside * (2.0 - 1.5 * z);
}

// 0-based ring index range [*ra, *rb] that contains every ring whose
// colatitude lies within `radius` of [tmin, tmax].
static __device__ __forceinline__ void ring_range(double tmin, double tmax, double radius, int nside,
                                           int* ra, int* rb) {
    const double za = cos(fmax(tmin - radius, 0.0));
    const double zb = cos(fmin(tmax + radius, kPi));
    int ia = (int)floor(ring_number(za, nside)) - 1;
    int ib = (int)ceil(ring_number(zb, nside)) + 1;
    if (ia < 1) ia = 1;
    if (ib > 4 * nside - 1) ib = 4 * nside - 1;
    *ra = ia - 1;
    *rb = ib - 1;
}

// The disc membership test k . p0 >= cos(radius) in FP64, evaluated in one
// fixed order without fused multiply-adds so every caller takes the same
// decision for the same pixel and pointing.
static __device__ __noinline__ bool exact_in_disc(const RingInfo* rings, int r, int jw, double px, double py,
                                           double pz, double cos_r) {
    const RingInfo& R = rings[r];
    double sp, cp;
    sincos(__dadd_rn(R.phi0, __dmul_rn((double)jw, R.dphi)), &sp, &cp);
    const double d = __dadd_rn(__dadd_rn(__dmul_rn(__dmul_rn(R.s, cp), px), __dmul_rn(__dmul_rn(R.s, sp), py)),
                               __dmul_rn(R.z, pz));
    return d >= cos_r;
}

}  // namespace pisco
