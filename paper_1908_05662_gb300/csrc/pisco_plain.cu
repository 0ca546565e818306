// Plain FP64 path: one CTA per sample, everything in float64.
//
// The layout of Sec. 5.2 / Fig. 4 on the device: the block of a pointing
// loops over the rings its disc can meet (warps) and the disc pixels of each
// ring (lanes), evaluates each pair from global memory and reduces in shared
// memory.  The disc is queried on the device (ring range, then per ring the
// longitude range from the spherical law of cosines plus one pixel of margin,
// then the exact test k . p0 >= cos R).  Geometry by the vector route of
// Sec. 2: x = k . theta'0, y = k . phi'0; the beam is interpolated
// bilinearly from the three folded float64 node maps; chi enters as in the
// FP32 kernel through the z-components e1, e2 of the Ludwig-3 vectors.
// This is the straightforward FP64 path the optimised kernels are measured
// against.

#include "pisco_internal.cuh"

#include <climits>

namespace pisco {

constexpr int PT = 256;

template <int MODE>
__global__ void __launch_bounds__(PT) k_plain(const __grid_constant__ LaunchParams P) {
    __shared__ double sRed[PT / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double* __restrict__ sky = (const double*)P.sky;
    const long long npix = P.npix;
    const int n = P.grid_n;
    const long long nn = (long long)n * n;

    for (long long tile = blockIdx.x; tile < P.total_tiles; tile += gridDim.x) {
        int d = 0;
        while (d + 1 < P.ndet && P.det[d + 1].tile_begin <= tile) ++d;
        const DetEntry& det = P.det[d];
        const long long t = det.begin + (tile - det.tile_begin);
        const double th = P.theta[t], ph = P.phi[t], ps = P.psi[t];
        const bool ok = isfinite(th) && isfinite(ph) && isfinite(ps) && th >= 0.0 && th <= kPi;
        if (!ok) {
            if (tid == 0) {
                if (MODE == kForward) ((double*)P.out)[t] = __longlong_as_double(0x7ff8000000000000ll);
                if (MODE == kCount) P.counts[t] = -1;
            }
            continue;
        }
        double phw = ph - kTwoPi * floor(ph / kTwoPi);
        if (phw >= kTwoPi) phw -= kTwoPi;
        double st, ct, sp, cp, ss, cs;
        sincos(th, &st, &ct);
        sincos(phw, &sp, &cp);
        sincos(ps, &ss, &cs);
        const double px = st * cp, py = st * sp, pz = ct;
        // theta'0 = cos psi theta0 + sin psi phi0 ; phi'0 = -sin psi theta0 + cos psi phi0
        const double tax = cs * ct * cp - ss * sp, tay = cs * ct * sp + ss * cp, taz = -cs * st;
        const double fax = -ss * ct * cp - cs * sp, fay = -ss * ct * sp + cs * cp, faz = ss * st;
        const double yw = (MODE == kAdjoint || MODE == kGrid) ? ((const double*)P.tod_in)[t] * det.scale : 0.0;
        const double* __restrict__ nodes = (const double*)det.beam;

        int ra, rb;
        ring_range(th, th, P.radius, P.nside, &ra, &rb);
        double acc = 0.0;
        for (int r = ra + warp; r <= rb; r += PT / 32) {
            const RingInfo& R = P.rings[r];
            if (fabs(R.theta - th) > P.radius + 1e-9) continue;
            long long jlo = 0, cnt = R.count;
            const double denom = R.s * st;
            if (denom > 1e-9) {
                const double c = (P.cos_r - R.z * ct) / denom;
                if (c > 1.0 + 1e-9) continue;
                if (c > -1.0) {
                    const double half = acos(fmin(c, 1.0));
                    const long long a = (long long)floor((phw - half - R.phi0) / R.dphi) - 1;
                    const long long b = (long long)ceil((phw + half - R.phi0) / R.dphi) + 1;
                    if (b - a + 1 < R.count) {
                        jlo = a;
                        cnt = b - a + 1;
                    }
                }
            }
            for (long long jj = lane; jj < cnt; jj += 32) {
                long long jw = (jlo + jj) % R.count;
                if (jw < 0) jw += R.count;
                if (!exact_in_disc(P.rings, r, (int)jw, px, py, pz, P.cos_r)) continue;
                if (MODE == kCount) {
                    acc += 1.0;
                    continue;
                }
                const long long pix = R.first + jw;
                double sf, cf;
                sincos(R.phi0 + (double)jw * R.dphi, &sf, &cf);
                const double kx = R.s * cf, ky = R.s * sf, kz = R.z;
                const double dot = kx * px + ky * py + kz * pz;
                const double x = kx * tax + ky * tay + kz * taz;
                const double y = kx * fax + ky * fay + kz * faz;
                const double tu = (x + P.sin_r) / P.h, tv = (y + P.sin_r) / P.h;
                const int iu = (int)fmin(fmax(floor(tu), 0.0), (double)(n - 2));
                const int iv = (int)fmin(fmax(floor(tv), 0.0), (double)(n - 2));
                const double fx = tu - iu, fy = tv - iv;
                const long long base = (long long)iv * n + iu;
                const double w00 = (1.0 - fx) * (1.0 - fy), w10 = fx * (1.0 - fy);
                const double w01 = (1.0 - fx) * fy, w11 = fx * fy;
                double bm[3];
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    const double* g = nodes + m * nn + base;
                    bm[m] = w00 * g[0] + w10 * g[1] + w01 * g[n] + w11 * g[n + 1];
                }
                const double q = 1.0 / (1.0 + dot);
                const double mp = q * (x * taz + y * faz) + pz;
                const double e1 = taz - x * mp, e2 = faz - y * mp;
                const double re = e1 * e1 - e2 * e2, im2 = e1 * e2;
                const double inv = 1.0 / (R.s * R.s);
                if (MODE == kGrid) {
                    // d t / d(A, Bq', Cu') = (I, alpha, beta), spread over the cell's four nodes
                    const double I = sky[pix], Q = sky[npix + pix], U = sky[2 * npix + pix];
                    const double c[3] = {yw * I, yw * (re * Q - 2.0 * im2 * U) * inv, yw * (2.0 * im2 * Q + re * U) * inv};
                    double* g = (double*)P.out;
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        atomicAdd(g + m * nn + base, c[m] * w00);
                        atomicAdd(g + m * nn + base + 1, c[m] * w10);
                        atomicAdd(g + m * nn + base + n, c[m] * w01);
                        atomicAdd(g + m * nn + base + n + 1, c[m] * w11);
                    }
                    continue;
                }
                if (MODE == kForward) {
                    const double I = sky[pix], Q = sky[npix + pix], U = sky[2 * npix + pix];
                    acc += bm[0] * I + (bm[1] * (re * Q - 2.0 * im2 * U) + bm[2] * (2.0 * im2 * Q + re * U)) * inv;
                } else if (MODE == kAdjoint) {
                    double* maps = (double*)P.out;
                    atomicAdd(maps + pix, yw * bm[0]);
                    atomicAdd(maps + npix + pix, yw * (bm[1] * re + 2.0 * bm[2] * im2) * inv);
                    atomicAdd(maps + 2 * npix + pix, yw * (bm[2] * re - 2.0 * bm[1] * im2) * inv);
                }
            }
        }
        if (MODE == kForward || MODE == kCount) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) sRed[warp] = acc;
            __syncthreads();
            if (tid == 0) {
                double s = 0.0;
                for (int w = 0; w < PT / 32; ++w) s += sRed[w];
                if (MODE == kForward) ((double*)P.out)[t] = det.scale * s;
                else P.counts[t] = (int32_t)s;
            }
            __syncthreads();
        }
    }
}

cudaError_t launch_plain(const LaunchParams& p, int mode, cudaStream_t s) {
    if (p.total_tiles <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)min(p.total_tiles, (long long)INT_MAX);
    switch (mode) {
        case kForward: k_plain<kForward><<<grid, PT, 0, s>>>(p); break;
        case kAdjoint: k_plain<kAdjoint><<<grid, PT, 0, s>>>(p); break;
        case kGrid: k_plain<kGrid><<<grid, PT, 0, s>>>(p); break;
        default: k_plain<kCount><<<grid, PT, 0, s>>>(p); break;
    }
    return cudaGetLastError();
}

}  // namespace pisco
