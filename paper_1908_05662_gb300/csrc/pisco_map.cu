// Binned map-making from TOD (the map-making step that follows TOD generation,
// Sec. 5.1 and Fig. 3; maps made from PISCO TOD in Sec. 6), and the RING pixel
// of a direction.
//
// Reading (the paper names no map-maker): per-pixel least squares with the
// pointing matrix of a delta beam at the boresight,
//     a_t = s/2 [(1 + eps), (1 - eps) cos 2 chi_t, (1 - eps) sin 2 chi_t],
// chi_t = psi_t + zeta (the co-polarisation angle at the beam centre,
// Appendix A at rho = 0), normal equations (sum a a^T) m = sum a d per pixel.
//
// pisco_map_accumulate: one thread per sample; the RING pixel by Gorski et
// al. (2005)'s boundary-line indexing in FP64 (products and sums rounded one
// at a time, no fused multiply-adds, so the integer decisions follow the
// written order), then 10 FP64 atomic adds into acc[10][Npix]:
//     0..5  sum a a^T  (II, IQ, IU, QQ, QU, UU)
//     6..8  sum a d    (I, Q, U)
//     9     hits
// pisco_map_solve: one thread per pixel; eigenvalues of the 3 x 3 matrix by
// the trigonometric closed form for symmetric 3 x 3 matrices (Smith, CACM
// 1961) give lambda_min / lambda_max; pixels with >= 3 hits and a reciprocal
// condition number >= rcond_min are solved by the adjugate, the rest are NaN.

#include "pisco_internal.cuh"

#include <cmath>

namespace pisco {
void set_error(pisco_plan* plan, const char* fmt, ...);
}  // namespace pisco

using namespace pisco;

namespace {

constexpr int kAcc = 10;

__device__ __forceinline__ long long ang2pix_ring(int nside, double theta, double phi) {
    const long long n = nside;
    const double z = cos(theta);
    const double za = fabs(z);
    double m = fmod(phi, kTwoPi);
    if (m < 0.0) m = __dadd_rn(m, kTwoPi);
    double tt = m / (0.5 * kPi);
    if (tt >= 4.0) tt = 0.0;
    if (za <= 2.0 / 3.0) {
        const double t1 = __dmul_rn((double)n, __dadd_rn(0.5, tt));
        const double t2 = __dmul_rn(__dmul_rn(0.75, (double)n), z);
        const long long jp = (long long)floor(__dsub_rn(t1, t2));
        const long long jm = (long long)floor(__dadd_rn(t1, t2));
        const long long ir = n + 1 + jp - jm;
        const long long kshift = 1 - (ir & 1);
        long long ip = (jp + jm - n + kshift + 1) / 2;
        ip %= 4 * n;
        if (ip < 0) ip += 4 * n;
        return 2 * n * (n - 1) + 4 * n * (ir - 1) + ip;
    }
    const double tp = __dsub_rn(tt, floor(tt));
    const double tmp = __dmul_rn((double)n, sqrt(__dmul_rn(3.0, __dsub_rn(1.0, za))));
    const long long jp = (long long)floor(__dmul_rn(tp, tmp));
    const long long jm = (long long)floor(__dmul_rn(__dsub_rn(1.0, tp), tmp));
    const long long ir = jp + jm + 1;
    long long ip = (long long)floor(__dmul_rn(tt, (double)ir));
    ip %= 4 * ir;
    if (ip < 0) ip += 4 * ir;
    return z > 0.0 ? 2 * ir * (ir - 1) + ip : 12 * n * n - 2 * ir * (ir + 1) + ip;
}

__device__ __forceinline__ bool valid_angles(double theta, double phi, double psi) {
    return isfinite(theta) && isfinite(phi) && isfinite(psi) && theta >= 0.0 && theta <= kPi;
}

__global__ void k_ang2pix(int nside, long long n, const double* __restrict__ theta, const double* __restrict__ phi,
                          long long* __restrict__ pix) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const double th = theta[t], ph = phi[t];
        pix[t] = valid_angles(th, ph, 0.0) ? ang2pix_ring(nside, th, ph) : -1;
    }
}

template <typename T>
__global__ void k_map_acc(int nside, long long n, const double* __restrict__ theta, const double* __restrict__ phi,
                          const double* __restrict__ psi, double zeta, double a_i, double a_p,
                          const T* __restrict__ tod, long long npix, double* __restrict__ acc) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const double th = theta[t], ph = phi[t], ps = psi[t];
        const double d = (double)tod[t];
        if (!valid_angles(th, ph, ps) || !isfinite(d)) continue;
        const long long p = ang2pix_ring(nside, th, ph);
        if (p < 0 || p >= npix) continue;  // cannot happen for theta in [0, pi]; keeps the adds in bounds
        double s2, c2;
        sincos(2.0 * (ps + zeta), &s2, &c2);
        const double a0 = a_i, a1 = a_p * c2, a2 = a_p * s2;
        double* q = acc + p;
        atomicAdd(q, a0 * a0);
        atomicAdd(q + npix, a0 * a1);
        atomicAdd(q + 2 * npix, a0 * a2);
        atomicAdd(q + 3 * npix, a1 * a1);
        atomicAdd(q + 4 * npix, a1 * a2);
        atomicAdd(q + 5 * npix, a2 * a2);
        atomicAdd(q + 6 * npix, a0 * d);
        atomicAdd(q + 7 * npix, a1 * d);
        atomicAdd(q + 8 * npix, a2 * d);
        atomicAdd(q + 9 * npix, 1.0);
    }
}

// Eigenvalues (ascending) of the symmetric matrix [[a, b, c], [b, d, e], [c, e, f]].
__device__ void sym3_eigenvalues(double a, double b, double c, double d, double e, double f, double* lo,
                                 double* hi) {
    const double p1 = b * b + c * c + e * e;
    const double q = (a + d + f) / 3.0;
    const double p2 = (a - q) * (a - q) + (d - q) * (d - q) + (f - q) * (f - q) + 2.0 * p1;
    if (p2 <= 0.0) {  // a multiple of the identity
        *lo = *hi = q;
        return;
    }
    const double p = sqrt(p2 / 6.0);
    const double ba = (a - q) / p, bd = (d - q) / p, bf = (f - q) / p, bb = b / p, bc = c / p, be = e / p;
    const double det = ba * (bd * bf - be * be) - bb * (bb * bf - be * bc) + bc * (bb * be - bd * bc);
    const double r = fmin(1.0, fmax(-1.0, 0.5 * det));
    const double ang = acos(r) / 3.0;
    *hi = q + 2.0 * p * cos(ang);
    *lo = q + 2.0 * p * cos(ang + 2.0 * kPi / 3.0);
}

__global__ void k_map_solve(long long npix, const double* __restrict__ acc, double rcond_min,
                            double* __restrict__ maps) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= npix) return;
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    const double hits = acc[9 * npix + p];
    double m0 = nan, m1 = nan, m2 = nan;
    if (hits >= 3.0) {
        const double a = acc[p], b = acc[npix + p], c = acc[2 * npix + p];
        const double d = acc[3 * npix + p], e = acc[4 * npix + p], f = acc[5 * npix + p];
        double lo, hi;
        sym3_eigenvalues(a, b, c, d, e, f, &lo, &hi);
        if (hi > 0.0 && lo / hi >= rcond_min) {
            // adjugate of the symmetric matrix
            const double A = d * f - e * e, B = c * e - b * f, C = b * e - c * d;
            const double D = a * f - c * c, E = b * c - a * e, F = a * d - b * b;
            const double det = a * A + b * B + c * C;
            const double y0 = acc[6 * npix + p], y1 = acc[7 * npix + p], y2 = acc[8 * npix + p];
            m0 = (A * y0 + B * y1 + C * y2) / det;
            m1 = (B * y0 + D * y1 + E * y2) / det;
            m2 = (C * y0 + E * y1 + F * y2) / det;
        }
    }
    maps[p] = m0;
    maps[npix + p] = m1;
    maps[2 * npix + p] = m2;
}

unsigned grid_for(long long n) {
    const long long b = (n + 255) / 256;
    return (unsigned)(b < 152LL * 64 ? (b > 0 ? b : 1) : 152LL * 64);
}

pisco_status check_nside(int nside) {
    if (nside < 1 || nside > 8192) {
        set_error(nullptr, "nside %d outside [1, 8192]", nside);
        return PISCO_EINVAL;
    }
    return PISCO_OK;
}

pisco_status launched() {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(nullptr, "kernel launch failed: %s", cudaGetErrorString(e));
        return PISCO_ECUDA;
    }
    return PISCO_OK;
}

}  // namespace

extern "C" pisco_status pisco_ang2pix(int nside, int64_t n, const double* theta, const double* phi, int64_t* pix,
                                      void* stream) {
    if (check_nside(nside) != PISCO_OK) return PISCO_EINVAL;
    if (n < 0) {
        set_error(nullptr, "n = %lld is negative", (long long)n);
        return PISCO_EINVAL;
    }
    if (n == 0) return PISCO_OK;
    if (!is_device_ptr(theta) || !is_device_ptr(phi) || !is_device_ptr(pix)) {
        set_error(nullptr, "theta, phi and pix must be device pointers");
        return PISCO_EINVAL;
    }
    k_ang2pix<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(nside, n, theta, phi, (long long*)pix);
    return launched();
}

extern "C" pisco_status pisco_map_accumulate(int nside, int64_t n, const double* theta, const double* phi,
                                             const double* psi, const pisco_detector* det, const void* tod,
                                             int tod_dtype, double* acc, int accumulate, void* stream) {
    if (check_nside(nside) != PISCO_OK) return PISCO_EINVAL;
    if (n < 0 || !det) {
        set_error(nullptr, "n = %lld is negative or det is NULL", (long long)n);
        return PISCO_EINVAL;
    }
    if (!std::isfinite(det->zeta) || !std::isfinite(det->eps) || !std::isfinite(det->s_resp)) {
        set_error(nullptr, "the detector has a non-finite parameter");
        return PISCO_EINVAL;
    }
    if (tod_dtype != PISCO_DTYPE_F32 && tod_dtype != PISCO_DTYPE_F64) {
        set_error(nullptr, "tod_dtype %d is neither PISCO_DTYPE_F32 nor PISCO_DTYPE_F64", tod_dtype);
        return PISCO_EINVAL;
    }
    if (!is_device_ptr(acc) ||
        (n > 0 && (!is_device_ptr(theta) || !is_device_ptr(phi) || !is_device_ptr(psi) || !is_device_ptr(tod)))) {
        set_error(nullptr, "theta, phi, psi, tod and acc must be device pointers");
        return PISCO_EINVAL;
    }
    const long long npix = 12LL * nside * nside;
    cudaStream_t s = (cudaStream_t)stream;
    if (!accumulate) {
        const cudaError_t e = cudaMemsetAsync(acc, 0, (size_t)kAcc * npix * sizeof(double), s);
        if (e != cudaSuccess) {
            set_error(nullptr, "cudaMemsetAsync failed: %s", cudaGetErrorString(e));
            return PISCO_ECUDA;
        }
    }
    if (n == 0) return PISCO_OK;
    const double a_i = 0.5 * det->s_resp * (1.0 + det->eps), a_p = 0.5 * det->s_resp * (1.0 - det->eps);
    if (tod_dtype == PISCO_DTYPE_F32)
        k_map_acc<float><<<grid_for(n), 256, 0, s>>>(nside, n, theta, phi, psi, det->zeta, a_i, a_p,
                                                      (const float*)tod, npix, acc);
    else
        k_map_acc<double><<<grid_for(n), 256, 0, s>>>(nside, n, theta, phi, psi, det->zeta, a_i, a_p,
                                                       (const double*)tod, npix, acc);
    return launched();
}

extern "C" pisco_status pisco_map_solve(int nside, const double* acc, double rcond_min, double* maps,
                                        void* stream) {
    if (check_nside(nside) != PISCO_OK) return PISCO_EINVAL;
    if (!(rcond_min >= 0.0 && rcond_min <= 1.0)) {
        set_error(nullptr, "rcond_min %g outside [0, 1]", rcond_min);
        return PISCO_EINVAL;
    }
    if (!is_device_ptr(acc) || !is_device_ptr(maps)) {
        set_error(nullptr, "acc and maps must be device pointers");
        return PISCO_EINVAL;
    }
    const long long npix = 12LL * nside * nside;
    k_map_solve<<<(unsigned)((npix + 255) / 256), 256, 0, (cudaStream_t)stream>>>(npix, acc, rcond_min, maps);
    return launched();
}
