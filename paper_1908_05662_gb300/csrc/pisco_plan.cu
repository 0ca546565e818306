// Plan-time kernels: HEALPix ring table, sky packing, beam folding, Omega~.
//
// Everything the hot path reads is built once here, on the device:
//  * the RING ring table (Sec. 5.1; z, phi offset, pixel count per ring);
//  * the sky as float4 (I, Q, U, 0) per pixel for the FP32 path, or three
//    float64 rows for the plain path;
//  * per detector, the six beamsor maps folded into the three that reach the
//    TOD.  D(chi) Lambda(chi) = (s/2)[(1+eps), (1-eps), 0, 0] (eqs. M_pol,
//    lambda_operator), so
//        A  = (1+eps) B_TT + (1-eps) B_TQ
//        Bq = (1+eps) B_QT + (1-eps) B_QQ
//        Cu = (1+eps) B_UT + (1-eps) B_UQ,
//    and the detector angle zeta enters chi = beta + zeta - sigma (Appendix A)
//    only through exp(2 i zeta), folded in as Bq' + i Cu' = (Bq + i Cu) e^{2 i zeta}.
//    Bilinear interpolation is linear, so folding before interpolating is exact.
//    FP32 plans store each grid cell as its bilinear coefficients
//    f(fx, fy) = c0 + c1 fx + c2 fy + c3 fx fy for the three maps, padded to
//    64 bytes so a cell spans two 32-byte sectors;
//    plain plans keep the folded node values in float64;
//    FP32 plans may instead keep the folded node values as three 2-D float
//    textures, fetched with 2 x 2 gathers;
//  * Omega~ = int B_TT dOmega (Sec. 3) by the trapezoid rule over the grid with
//    the orthographic area element du dv / sqrt(1 - u^2 - v^2).

#include "pisco_internal.cuh"

namespace pisco {

__global__ void k_rings(int nside, int nrings, RingInfo* out) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrings) return;
    out[r] = make_ring(r, nside);
}

template <typename T>
__global__ void k_sky32(const T* __restrict__ sky, long long npix, float4* __restrict__ out) {
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= npix) return;
    out[p] = make_float4((float)sky[p], (float)sky[npix + p], (float)sky[2 * npix + p], 0.0f);
}

template <typename T>
__global__ void k_sky64(const T* __restrict__ sky, long long npix, double* __restrict__ out) {
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= 3 * npix) return;
    out[p] = (double)sky[p];
}

struct Folded {
    double a, b, c;
};

__device__ __forceinline__ Folded fold_node(const float* __restrict__ g, long long nn, long long idx,
                                            double eps, double c2z, double s2z) {
    // map order TT, QT, UT, TQ, QQ, UQ
    double tt = g[idx], qt = g[nn + idx], ut = g[2 * nn + idx];
    double tq = g[3 * nn + idx], qq = g[4 * nn + idx], uq = g[5 * nn + idx];
    Folded f;
    f.a = (1.0 + eps) * tt + (1.0 - eps) * tq;
    double bq = (1.0 + eps) * qt + (1.0 - eps) * qq;
    double cu = (1.0 + eps) * ut + (1.0 - eps) * uq;
    f.b = bq * c2z - cu * s2z;
    f.c = bq * s2z + cu * c2z;
    return f;
}

__global__ void k_cells(const float* __restrict__ g, int n, double eps, double zeta,
                        float4* __restrict__ cells) {
    const int nc = n - 1;
    long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (cell >= (long long)nc * nc) return;
    const int i = (int)(cell % nc), j = (int)(cell / nc);
    const long long nn = (long long)n * n;
    double s2z, c2z;
    sincos(2.0 * zeta, &s2z, &c2z);
    Folded f00 = fold_node(g, nn, (long long)j * n + i, eps, c2z, s2z);
    Folded f10 = fold_node(g, nn, (long long)j * n + i + 1, eps, c2z, s2z);
    Folded f01 = fold_node(g, nn, (long long)(j + 1) * n + i, eps, c2z, s2z);
    Folded f11 = fold_node(g, nn, (long long)(j + 1) * n + i + 1, eps, c2z, s2z);
    cells[4 * cell + 0] = make_float4((float)f00.a, (float)(f10.a - f00.a), (float)(f01.a - f00.a),
                                      (float)(f11.a - f10.a - f01.a + f00.a));
    cells[4 * cell + 1] = make_float4((float)f00.b, (float)(f10.b - f00.b), (float)(f01.b - f00.b),
                                      (float)(f11.b - f10.b - f01.b + f00.b));
    cells[4 * cell + 2] = make_float4((float)f00.c, (float)(f10.c - f00.c), (float)(f01.c - f00.c),
                                      (float)(f11.c - f10.c - f01.c + f00.c));
    cells[4 * cell + 3] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Packed 32-byte cells (PISCO_FETCH_PACKED).  Per cell and folded map m the
// bilinear form f = c0 + d1 fx + d2 fy + d3 fx fy keeps c0 in FP32 and the three
// slopes as int16 on a block scale 2^(E - 31 + e_m), E one exponent per detector
// (from the largest slope of the grid) and e_m in [0, 31] per cell and map, so
// a slope is off by at most 2^-15 of the largest slope of its cell and map.
// Layout (eight 32-bit words): c0_A, c0_B, c0_C, (A1 | A2), (A3 | B1), (B2 | B3),
// (C1 | C2), (C3 | e_A | e_B << 5 | e_C << 10), slope k of map m in 16 bits
// (low half first).  A 32-byte header precedes the cells: word 0 = E - 31 + 127
// (the biased exponent of the unit scale), word 1 = the largest |slope| as
// float bits, word 2 = 1 when E falls outside the normal float range.
struct Slopes {
    double c0[3], d[3][3];
};

__device__ __forceinline__ Slopes cell_slopes(const float* __restrict__ g, int n, long long cell, double eps,
                                              double c2z, double s2z) {
    const int nc = n - 1;
    const int i = (int)(cell % nc), j = (int)(cell / nc);
    const long long nn = (long long)n * n;
    const Folded f00 = fold_node(g, nn, (long long)j * n + i, eps, c2z, s2z);
    const Folded f10 = fold_node(g, nn, (long long)j * n + i + 1, eps, c2z, s2z);
    const Folded f01 = fold_node(g, nn, (long long)(j + 1) * n + i, eps, c2z, s2z);
    const Folded f11 = fold_node(g, nn, (long long)(j + 1) * n + i + 1, eps, c2z, s2z);
    const double v00[3] = {f00.a, f00.b, f00.c}, v10[3] = {f10.a, f10.b, f10.c};
    const double v01[3] = {f01.a, f01.b, f01.c}, v11[3] = {f11.a, f11.b, f11.c};
    Slopes r;
    for (int m = 0; m < 3; ++m) {
        r.c0[m] = v00[m];
        r.d[m][0] = v10[m] - v00[m];
        r.d[m][1] = v01[m] - v00[m];
        r.d[m][2] = v11[m] - v10[m] - v01[m] + v00[m];
    }
    return r;
}

// Smallest k with |x| <= 2^k (x > 0).
__device__ __forceinline__ int ceil_log2(double x) {
    int k;
    const double f = frexp(x, &k);
    return f == 0.5 ? k - 1 : k;
}

__global__ void k_packed_max(const float* __restrict__ g, int n, double eps, double zeta, unsigned* header) {
    const long long nc = (long long)(n - 1) * (n - 1);
    const long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (cell >= nc) return;
    double s2z, c2z;
    sincos(2.0 * zeta, &s2z, &c2z);
    const Slopes r = cell_slopes(g, n, cell, eps, c2z, s2z);
    double mx = 0.0;
    for (int m = 0; m < 3; ++m)
        for (int k = 0; k < 3; ++k) mx = fmax(mx, fabs(r.d[m][k]));
    // non-negative floats order like their bit patterns
    atomicMax(header + 1, __float_as_uint((float)mx));
}

__global__ void k_packed_encode(const float* __restrict__ g, int n, double eps, double zeta,
                                unsigned* __restrict__ header, uint4* __restrict__ out) {
    const long long nc = (long long)(n - 1) * (n - 1);
    const long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const float gmax = __uint_as_float(header[1]);
    // unit scale 2^(E - 31); E such that the largest slope fits 32767 * 2^E
    const int E = gmax > 0.f ? ceil_log2(1.000001 * (double)gmax / 32767.0) : -90;
    const bool bad = E - 31 + 127 < 1 || E + 127 > 254;
    if (cell == 0) {
        header[0] = (unsigned)(E - 31 + 127);
        header[2] = bad ? 1u : 0u;
    }
    if (cell >= nc || bad) return;
    double s2z, c2z;
    sincos(2.0 * zeta, &s2z, &c2z);
    const Slopes r = cell_slopes(g, n, cell, eps, c2z, s2z);
    unsigned q[9], ex[3];
    for (int m = 0; m < 3; ++m) {
        double mx = 0.0;
        for (int k = 0; k < 3; ++k) mx = fmax(mx, fabs(r.d[m][k]));
        int e = mx > 0.0 ? ceil_log2(mx / 32767.0) - (E - 31) : 0;
        e = e < 0 ? 0 : (e > 31 ? 31 : e);
        ex[m] = (unsigned)e;
        const double inv = ldexp(1.0, -(E - 31 + e));
        for (int k = 0; k < 3; ++k) {
            double v = rint(r.d[m][k] * inv);
            v = fmin(32767.0, fmax(-32767.0, v));
            q[3 * m + k] = (unsigned)((int)v) & 0xffffu;
        }
    }
    uint4 lo, hi;
    lo.x = __float_as_uint((float)r.c0[0]);
    lo.y = __float_as_uint((float)r.c0[1]);
    lo.z = __float_as_uint((float)r.c0[2]);
    lo.w = q[0] | (q[1] << 16);
    hi.x = q[2] | (q[3] << 16);
    hi.y = q[4] | (q[5] << 16);
    hi.z = q[6] | (q[7] << 16);
    hi.w = q[8] | ((ex[0] | (ex[1] << 5) | (ex[2] << 10)) << 16);
    out[2 * (cell + 1)] = lo;  // cell 0 follows the 32-byte header
    out[2 * (cell + 1) + 1] = hi;
}

__global__ void k_nodes64(const float* __restrict__ g, int n, double eps, double zeta,
                          double* __restrict__ nodes) {
    const long long nn = (long long)n * n;
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= nn) return;
    double s2z, c2z;
    sincos(2.0 * zeta, &s2z, &c2z);
    Folded f = fold_node(g, nn, idx, eps, c2z, s2z);
    nodes[idx] = f.a;
    nodes[nn + idx] = f.b;
    nodes[2 * nn + idx] = f.c;
}

__global__ void k_nodes32(const float* __restrict__ g, int n, double eps, double zeta, float* __restrict__ out) {
    const long long nn = (long long)n * n;
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= nn) return;
    double s2z, c2z;
    sincos(2.0 * zeta, &s2z, &c2z);
    Folded f = fold_node(g, nn, idx, eps, c2z, s2z);
    out[idx] = (float)f.a;
    out[nn + idx] = (float)f.b;
    out[2 * nn + idx] = (float)f.c;
}

// Folded node values as one float4 (A, Bq', Cu', 0) per node, for the shared-memory fetch.
__global__ void k_nodes4(const float* __restrict__ g, int n, double eps, double zeta, float4* __restrict__ out) {
    const long long nn = (long long)n * n;
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= nn) return;
    double s2z, c2z;
    sincos(2.0 * zeta, &s2z, &c2z);
    Folded f = fold_node(g, nn, idx, eps, c2z, s2z);
    out[idx] = make_float4((float)f.a, (float)f.b, (float)f.c, 0.f);
}

// One block; fixed per-thread order and a fixed tree, so the result is deterministic.
__global__ void k_omega(const float* __restrict__ tt, int n, double sin_r, double* out) {
    __shared__ double red[256];
    const double h = 2.0 * sin_r / (double)(n - 1);
    double acc = 0.0;
    const long long nn = (long long)n * n;
    for (long long idx = threadIdx.x; idx < nn; idx += blockDim.x) {
        const int i = (int)(idx % n), j = (int)(idx / n);
        const double u = sin_r * (2.0 * i / (double)(n - 1) - 1.0);
        const double v = sin_r * (2.0 * j / (double)(n - 1) - 1.0);
        const double w = ((i == 0 || i == n - 1) ? 0.5 : 1.0) * ((j == 0 || j == n - 1) ? 0.5 : 1.0);
        acc += w * (double)tt[idx] / sqrt(1.0 - u * u - v * v);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] * h * h;
}

static inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_fold_nodes32(const float* grids, int n, double eps, double zeta, float* out3, cudaStream_t s) {
    k_nodes32<<<blocks_for((long long)n * n, 256), 256, 0, s>>>(grids, n, eps, zeta, out3);
    return cudaGetLastError();
}

// Folded-map gradient (A, Bq', Cu') -> gradient of the six input maps: the
// transpose of the folding above (A = (1+eps) TT + (1-eps) TQ, etc., and the
// rotation by 2 zeta).
template <typename T>
__global__ void k_unfold(const T* __restrict__ f, int n, double eps, double zeta, T* __restrict__ g, int accumulate) {
    const long long nn = (long long)n * n;
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= nn) return;
    double s2z, c2z;
    sincos(2.0 * zeta, &s2z, &c2z);
    // FP32 folded gradients are interleaved per node ([N][N][4]), FP64 ones are [3][N][N]
    const bool inter = sizeof(T) == sizeof(float);
    const double ga = inter ? f[4 * idx] : f[idx];
    const double gbp = inter ? f[4 * idx + 1] : f[nn + idx];
    const double gcp = inter ? f[4 * idx + 2] : f[2 * nn + idx];
    const double gbq = c2z * gbp + s2z * gcp;   // transpose of the 2 zeta rotation
    const double gcu = -s2z * gbp + c2z * gcp;
    const double v[6] = {(1.0 + eps) * ga, (1.0 + eps) * gbq, (1.0 + eps) * gcu,   // TT, QT, UT
                         (1.0 - eps) * ga, (1.0 - eps) * gbq, (1.0 - eps) * gcu};  // TQ, QQ, UQ
#pragma unroll
    for (int e = 0; e < 6; ++e) {
        const T add = (T)v[e];
        g[e * nn + idx] = accumulate ? g[e * nn + idx] + add : add;
    }
}

// Omega~ enters d through (s/2) Omega_pix / Omega~, so d L / d Omega~ = -sum_t y_t d_t / Omega~;
// Omega~ is the trapezoid sum of B_TT with weights J = h^2 w_i w_j / sqrt(1 - u_i^2 - v_j^2).
// One block: a fixed-order FP64 reduction, then the rank-one update of the TT gradient.
template <typename T>
__global__ void k_omega_adjoint(const T* __restrict__ tod, const T* __restrict__ y, long long n, double omega,
                                double scale_tod, int gn, double sin_r, T* __restrict__ g_tt) {
    __shared__ double red[1024];
    double acc = 0.0;
    for (long long t = threadIdx.x; t < n; t += blockDim.x) {
        const double d = (double)tod[t], w = (double)y[t];
        if (isfinite(d) && isfinite(w)) acc += d * w;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    const double dl_domega = -scale_tod * red[0] / omega;
    const double h = 2.0 * sin_r / (double)(gn - 1);
    const long long nn = (long long)gn * gn;
    for (long long idx = threadIdx.x; idx < nn; idx += blockDim.x) {
        const int i = (int)(idx % gn), j = (int)(idx / gn);
        const double u = sin_r * (2.0 * i / (double)(gn - 1) - 1.0);
        const double v = sin_r * (2.0 * j / (double)(gn - 1) - 1.0);
        const double w = ((i == 0 || i == gn - 1) ? 0.5 : 1.0) * ((j == 0 || j == gn - 1) ? 0.5 : 1.0);
        g_tt[idx] = (T)((double)g_tt[idx] + dl_domega * h * h * w / sqrt(1.0 - u * u - v * v));
    }
}

// Per-cell coefficient gradients G[cell][m] = dL/d(c0, c1, c2, c3) to the six input
// maps.  With c0 = f00, c1 = f10 - f00, c2 = f01 - f00, c3 = f11 - f10 - f01 + f00,
// node (i, j) collects g0 - g1 - g2 + g3 from cell (i, j) (its f00), g1 - g3 from
// cell (i-1, j) (f10), g2 - g3 from cell (i, j-1) (f01) and g3 from cell (i-1, j-1)
// (f11); then the transpose of the folding as in k_unfold.
__global__ void k_unfold_coef(const float* __restrict__ cg, int n, double eps, double zeta, float* __restrict__ g,
                              int accumulate) {
    const long long nn = (long long)n * n;
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= nn) return;
    const int nc = n - 1;
    const int i = (int)(idx % n), j = (int)(idx / n);
    double node[3] = {0.0, 0.0, 0.0};
    for (int m = 0; m < 3; ++m) {
        double v = 0.0;
        if (i < nc && j < nc) {
            const float* c = cg + 12 * ((long long)j * nc + i) + 4 * m;
            v += (double)c[0] - (double)c[1] - (double)c[2] + (double)c[3];
        }
        if (i > 0 && j < nc) {
            const float* c = cg + 12 * ((long long)j * nc + i - 1) + 4 * m;
            v += (double)c[1] - (double)c[3];
        }
        if (i < nc && j > 0) {
            const float* c = cg + 12 * ((long long)(j - 1) * nc + i) + 4 * m;
            v += (double)c[2] - (double)c[3];
        }
        if (i > 0 && j > 0) v += (double)cg[12 * ((long long)(j - 1) * nc + i - 1) + 4 * m + 3];
        node[m] = v;
    }
    double s2z, c2z;
    sincos(2.0 * zeta, &s2z, &c2z);
    const double gbq = c2z * node[1] + s2z * node[2];  // transpose of the 2 zeta rotation
    const double gcu = -s2z * node[1] + c2z * node[2];
    const double v[6] = {(1.0 + eps) * node[0], (1.0 + eps) * gbq, (1.0 + eps) * gcu,
                         (1.0 - eps) * node[0], (1.0 - eps) * gbq, (1.0 - eps) * gcu};
#pragma unroll
    for (int e = 0; e < 6; ++e) {
        const float add = (float)v[e];
        g[e * nn + idx] = accumulate ? g[e * nn + idx] + add : add;
    }
}

cudaError_t launch_unfold_coef_grid(const float* cgrad, int n, double eps, double zeta, float* grad, int accumulate,
                                   cudaStream_t s) {
    k_unfold_coef<<<blocks_for((long long)n * n, 256), 256, 0, s>>>(cgrad, n, eps, zeta, grad, accumulate);
    return cudaGetLastError();
}

cudaError_t launch_unfold_grid(const void* folded, int n, double eps, double zeta, void* grad, int accumulate,
                               int f64, cudaStream_t s) {
    const unsigned b = blocks_for((long long)n * n, 256);
    if (f64) k_unfold<double><<<b, 256, 0, s>>>((const double*)folded, n, eps, zeta, (double*)grad, accumulate);
    else k_unfold<float><<<b, 256, 0, s>>>((const float*)folded, n, eps, zeta, (float*)grad, accumulate);
    return cudaGetLastError();
}

cudaError_t launch_omega_adjoint(const void* tod, const void* y, long long n, int f64, double omega, double scale_tod,
                                 int grid_n, double sin_r, void* grad_tt, cudaStream_t s) {
    if (f64)
        k_omega_adjoint<double><<<1, 1024, 0, s>>>((const double*)tod, (const double*)y, n, omega, scale_tod, grid_n,
                                                   sin_r, (double*)grad_tt);
    else
        k_omega_adjoint<float><<<1, 1024, 0, s>>>((const float*)tod, (const float*)y, n, omega, scale_tod, grid_n,
                                                  sin_r, (float*)grad_tt);
    return cudaGetLastError();
}

cudaError_t launch_beam_kernels(pisco_plan* plan, const float* grids, cudaStream_t s, double* d_omega_out) {
    const int n = plan->grid_n;
    const long long nn = (long long)n * n;
    for (int d = 0; d < plan->n_det; ++d) {
        const float* g = grids + (long long)d * 6 * nn;
        char* dst = plan->d_beam ? (char*)plan->d_beam + (size_t)d * plan->beam_stride : nullptr;
        const pisco_detector& det = plan->h_dets[d];
        if (plan->precision != PISCO_FP64_PLAIN) {
            const long long nc = (long long)(n - 1) * (n - 1);
            if (plan->beam_fetch == PISCO_FETCH_CELLS) {
                k_cells<<<blocks_for(nc, 256), 256, 0, s>>>(g, n, det.eps, det.zeta, (float4*)dst);
            } else if (plan->beam_fetch == PISCO_FETCH_SHARED) {
                k_nodes4<<<blocks_for(nn, 256), 256, 0, s>>>(g, n, det.eps, det.zeta, (float4*)dst);
            } else if (plan->beam_fetch == PISCO_FETCH_PACKED) {
                cudaError_t e = cudaMemsetAsync(dst, 0, 32, s);
                if (e != cudaSuccess) return e;
                k_packed_max<<<blocks_for(nc, 256), 256, 0, s>>>(g, n, det.eps, det.zeta, (unsigned*)dst);
                k_packed_encode<<<blocks_for(nc, 256), 256, 0, s>>>(g, n, det.eps, det.zeta, (unsigned*)dst,
                                                                     (uint4*)dst);
            }
        } else {
            k_nodes64<<<blocks_for(nn, 256), 256, 0, s>>>(g, n, det.eps, det.zeta, (double*)dst);
        }
        k_omega<<<1, 256, 0, s>>>(g, n, sin(plan->radius), d_omega_out + d);
    }
    return cudaGetLastError();
}

cudaError_t launch_plan_kernels(pisco_plan* plan, const void* sky, int sky_dtype, const float* grids,
                                cudaStream_t s, double* d_omega_out) {
    k_rings<<<blocks_for(plan->nrings, 128), 128, 0, s>>>(plan->nside, plan->nrings, plan->d_rings);
    const long long npix = plan->npix;
    if (sky_dtype < 0) {
        // sky already in place (multi-realization plans)
    } else if (plan->precision == PISCO_FP32) {
        if (sky_dtype == PISCO_DTYPE_F32)
            k_sky32<float><<<blocks_for(npix, 256), 256, 0, s>>>((const float*)sky, npix, (float4*)plan->d_sky);
        else
            k_sky32<double><<<blocks_for(npix, 256), 256, 0, s>>>((const double*)sky, npix, (float4*)plan->d_sky);
    } else {
        if (sky_dtype == PISCO_DTYPE_F32)
            k_sky64<float><<<blocks_for(3 * npix, 256), 256, 0, s>>>((const float*)sky, npix, (double*)plan->d_sky);
        else
            k_sky64<double><<<blocks_for(3 * npix, 256), 256, 0, s>>>((const double*)sky, npix, (double*)plan->d_sky);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_beam_kernels(plan, grids, s, d_omega_out);
}

}  // namespace pisco
