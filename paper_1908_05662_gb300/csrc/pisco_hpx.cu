// HEALPix beam input: beamsor maps given as HEALPix RING maps (the paper's
// own representation, Sec. 5.1; beam NSIDE 4x the sky's in Sec. 5.3 and 6)
// resampled once onto the tangent-plane grid that the convolution kernels read.
//
// The beam centre is the map's north pole and the antenna coordinates are its
// spherical coordinates (rho = theta, sigma = phi), so grid node (u_i, v_j)
// samples rho = asin(sqrt(u^2 + v^2)), sigma = atan2(v, u).  The value there
// is the ring-wise bilinear interpolation of the map (the paper interpolates
// without naming a scheme, Sec. 4.2):
//   * along a ring, linear in phi between the two bracketing pixel centres;
//   * between the bracketing rings, linear in theta;
//   * above ring 1 (below the last ring), extrapolated from rings 1 and 2
//     (the last two) quadratic in theta, w = (theta^2 - theta_1^2) /
//     (theta_2^2 - theta_1^2), so a beam peak at the pole is not averaged down.
// Nodes with u^2 + v^2 > 1 lie off the hemisphere and are zero.  One thread
// per node, FP64 arithmetic, the ring geometry computed in registers.

#include "pisco_internal.cuh"

#include <cmath>

namespace pisco {
void set_error(pisco_plan* plan, const char* fmt, ...);
}  // namespace pisco

using namespace pisco;

namespace {

struct RingPair {
    long long p0, p1;  // bracketing pixels
    double f;          // weight of p1
};

__device__ __forceinline__ RingPair on_ring(const RingInfo& R, double phi) {
    const double x = (phi - R.phi0) / R.dphi;
    const double j = floor(x);
    long long j0 = (long long)j % R.count;
    if (j0 < 0) j0 += R.count;
    const long long j1 = j0 + 1 == R.count ? 0 : j0 + 1;
    return RingPair{R.first + j0, R.first + j1, x - j};
}

__global__ void k_hpx_grid(int nside, int n_maps, const float* __restrict__ maps, long long npix, double sin_r,
                           int n, float* __restrict__ grids) {
    const long long nn = (long long)n * n;
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= nn) return;
    const int i = (int)(idx % n), jn = (int)(idx / n);
    const double u = sin_r * (2.0 * i / (double)(n - 1) - 1.0);
    const double v = sin_r * (2.0 * jn / (double)(n - 1) - 1.0);
    const double r2 = u * u + v * v;
    if (r2 > 1.0) {
        for (int m = 0; m < n_maps; ++m) grids[m * nn + idx] = 0.0f;
        return;
    }
    const double rho = asin(sqrt(r2));
    const double sigma = atan2(v, u);
    const int nr = 4 * nside - 1;
    const RingInfo first = make_ring(0, nside), last = make_ring(nr - 1, nside);
    int r;
    double wt;
    if (rho < first.theta) {
        const RingInfo second = make_ring(1, nside);
        r = 0;
        wt = (rho * rho - first.theta * first.theta) / (second.theta * second.theta - first.theta * first.theta);
    } else if (rho >= last.theta) {
        const RingInfo prev = make_ring(nr - 2, nside);
        const double a = kPi - rho, b = kPi - last.theta, c = kPi - prev.theta;
        r = nr - 2;
        wt = 1.0 - (a * a - b * b) / (c * c - b * b);
    } else {
        // candidate from the continuous ring number, then step to theta_r <= rho < theta_{r+1}
        r = (int)floor(ring_number(cos(rho), nside)) - 1;
        r = r < 0 ? 0 : (r > nr - 2 ? nr - 2 : r);
        for (int k = 0; k < 4 && r < nr - 2 && make_ring(r + 1, nside).theta <= rho; ++k) ++r;
        for (int k = 0; k < 4 && r > 0 && make_ring(r, nside).theta > rho; ++k) --r;
        const double ta = make_ring(r, nside).theta, tb = make_ring(r + 1, nside).theta;
        wt = (rho - ta) / (tb - ta);
    }
    const RingPair a = on_ring(make_ring(r, nside), sigma);
    const RingPair b = on_ring(make_ring(r + 1, nside), sigma);
    const double wa0 = (1.0 - wt) * (1.0 - a.f), wa1 = (1.0 - wt) * a.f;
    const double wb0 = wt * (1.0 - b.f), wb1 = wt * b.f;
    for (int m = 0; m < n_maps; ++m) {
        const float* M = maps + (long long)m * npix;
        grids[m * nn + idx] = (float)(wa0 * (double)M[a.p0] + wa1 * (double)M[a.p1] + wb0 * (double)M[b.p0] +
                                      wb1 * (double)M[b.p1]);
    }
}

}  // namespace

extern "C" pisco_status pisco_beam_grids_from_healpix(int nside_b, int n_maps, const float* maps, double radius_rad,
                                                      int grid_n, float* grids, void* stream) {
    if (nside_b < 1 || nside_b > 8192) {
        set_error(nullptr, "nside_b %d outside [1, 8192]", nside_b);
        return PISCO_EINVAL;
    }
    if (n_maps < 1) {
        set_error(nullptr, "n_maps %d < 1", n_maps);
        return PISCO_EINVAL;
    }
    if (!(radius_rad > 0.0 && radius_rad < 0.5 * kPi)) {
        set_error(nullptr, "radius %g outside (0, pi/2)", radius_rad);
        return PISCO_EINVAL;
    }
    if (grid_n < 2 || grid_n > 4096) {
        set_error(nullptr, "grid_n %d outside [2, 4096]", grid_n);
        return PISCO_EINVAL;
    }
    if (!is_device_ptr(maps) || !is_device_ptr(grids)) {
        set_error(nullptr, "maps and grids must be device pointers");
        return PISCO_EINVAL;
    }
    const long long nn = (long long)grid_n * grid_n;
    const long long npix = 12LL * nside_b * nside_b;
    k_hpx_grid<<<(unsigned)((nn + 255) / 256), 256, 0, (cudaStream_t)stream>>>(nside_b, n_maps, maps, npix,
                                                                              sin(radius_rad), grid_n, grids);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(nullptr, "kernel launch failed: %s", cudaGetErrorString(e));
        return PISCO_ECUDA;
    }
    return PISCO_OK;
}
