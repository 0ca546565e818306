// FP32 tile kernel: TOD (forward), sky transpose (adjoint) and disc counts.
//
// One CTA owns a tile of S consecutive samples of one detector (Sec. 5.2 gives
// one block per pointing; consecutive samples of a scan share almost all of
// their disc, so here one disc traversal serves S pointings).  Per tile:
//
//  1. per sample, in FP64: the antenna basis (eq. antenna_base_vectors),
//     rounded to FP32 constants;
//  2. samples are grouped greedily into runs whose pointings lie within
//     R/4 of the run's first one and within R/2 in longitude; each run
//     shares one traversal of the union of its discs (the ring-ordered
//     disc query of Sec. 5.2, done on the device);
//  3. per (ring, sample), FP64 -> FP32: sin(theta_r - theta0) and
//     1 - cos(theta_r - theta0), so the in-frame offsets of every pixel are
//     formed from small, well-conditioned terms:
//        x0 = k . theta0_hat = sin(dtheta) - 2 cos(theta0) sin(theta_r) sin^2(dphi/2)
//        y0 = k . phi0_hat   = 2 sin(theta_r) sin(dphi/2) cos(dphi/2)
//        1 - k . p0          = (1 - cos dtheta) + 2 sin(theta0) sin(theta_r) sin^2(dphi/2)
//     with dphi/2 rotated from per-pixel and per-sample half-angles, and
//     (x, y) = (x0, y0) rotated by psi0 (Sec. 2): no O(1) terms cancel in FP32;
//  4. disc membership 1 - k . p0 <= 1 - cos R is decided in FP32; pairs
//     within 2e-6 (relative) of the boundary are settled by the FP64 test;
//  5. the three folded beam maps are interpolated bilinearly at the
//     orthographic grid coordinates (u, v) = (x, y) (Sec. 4.2), either from
//     64-byte coefficient cells read through L1/L2 (one 32-byte and one
//     16-byte load), from 32-byte packed cells (FP32 values, int16 slopes on
//     a per-cell power-of-two scale; one 32-byte load), from 2 x 2 texel
//     gathers of the node maps through the texture path (grids of 100s of KB
//     to MB, read at scattered cells), or from the four nodes of the cell in
//     shared memory (node grids up to 108^2, staged once per block);
//  6. the Ludwig-3 angle (Appendix A) enters through
//        e^{2 i chi} = e^{2 i zeta} (-e1 + i e2)^2 / sin^2(theta_k),
//        e1 = Z_theta - x (Z_p + m), e2 = Z_phi - y (Z_p + m),
//        m = (x Z_theta + y Z_phi) / (1 + k . p0),
//     where (Z_theta, Z_phi, Z_p) is the sky pole in the antenna basis; e1 and
//     e2 are z-components of the co- and cross-polar unit vectors
//     (e_co . theta_k = -(e_co . z)/sin theta_k, e_co . phi_k = (k x e_co) . z / sin theta_k).
//     e^{2 i zeta} is folded into the beam maps at plan time;
//  7. per-sample FP32 partial sums: warp shuffles, then FP64 across warps.
//
// The same traversal serves the transposes: the sky adjoint (atomic adds of
// each pixel's I, Q, U weights summed over the group's samples), the
// beam-grid adjoint (vector reductions into the folded node gradient,
// accumulated per cell in registers while consecutive samples stay in one
// cell), both in one pass (they share the geometry), and the disc count.
//
// A thread takes NP consecutive pixels of a ring: their sky values are loaded
// once per group and reused for all S samples, and each per-sample value read
// from shared memory serves NP pairs.

#pragma once

#include "pisco_internal.cuh"

#include <climits>

namespace pisco {

constexpr int NT = 256;
constexpr int NW = NT / 32;
constexpr int RC = 128;  // rings per chunk of the union disc

// 1 / x from the hardware reciprocal (about 1 ulp); it only scales the small
// correction m of the Ludwig-3 components, where 1e-7 relative is plenty.
static __device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Add the 12 accumulated gradients of one cell to the folded gradient and clear
// them.  Two layouts of the FP32 folded gradient:
//  * per node, [N][N][4] = (A, Bq', Cu', 0): gw holds the gradients of the four
//    nodes (i, j), (i+1, j), (i, j+1), (i+1, j+1) of each map, one 16-byte
//    vector reduction per node;
//  * per cell, [(N-1)^2][3][4]: gw holds, per map, the gradients of the cell's
//    bilinear coefficients (c0, c1, c2, c3) of f = c0 + c1 fx + c2 fy + c3 fx fy,
//    one 16-byte vector reduction per map (3 instead of 4); the unfolding
//    kernel turns them into node gradients.
static __device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

static __device__ __forceinline__ void flush_grid(float* g, int cell, int nc, int n, float* gw, int coef) {
    if (coef) {
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            if (gw[4 * m] != 0.f || gw[4 * m + 1] != 0.f || gw[4 * m + 2] != 0.f || gw[4 * m + 3] != 0.f)
                red_add_v4(g + 12 * (long long)cell + 4 * m, gw[4 * m], gw[4 * m + 1], gw[4 * m + 2], gw[4 * m + 3]);
            gw[4 * m] = gw[4 * m + 1] = gw[4 * m + 2] = gw[4 * m + 3] = 0.f;
        }
        return;
    }
    const int i = cell % nc, j = cell / nc;
    const long long base = (long long)j * n + i;
    const long long off[4] = {base, base + 1, base + n, base + n + 1};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (gw[k] != 0.f || gw[4 + k] != 0.f || gw[8 + k] != 0.f)
            red_add_v4(g + 4 * off[k], gw[k], gw[4 + k], gw[8 + k], 0.f);
        gw[k] = gw[4 + k] = gw[8 + k] = 0.f;
    }
}

// Bilinear value from a 2 x 2 texel gather, whose components are the nodes
// (i, j+1), (i+1, j+1), (i+1, j), (i, j) in that order.
static __device__ __forceinline__ float lerp_gather(const float4 g, float fx, float fy) {
    const float lo = fmaf(fx, g.z - g.w, g.w);  // row j
    const float hi = fmaf(fx, g.y - g.x, g.x);  // row j + 1
    return fmaf(fy, hi - lo, lo);
}

// Beam-cell loads: one 32-byte (256-bit vector, sm_100 and later) and one
// 16-byte read-only load per 64-byte cell, one sector each.  Cells are read at
// scattered places (the L1 hit rate is low), so they are not allocated in L1.
static __device__ __forceinline__ void ld_nc_v8(const float* p, float4& a, float4& b) {
    asm("ld.global.nc.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

static __device__ __forceinline__ float4 ld_nc_v4(const float* p) {
    float4 a;
    asm("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w)
        : "l"(p));
    return a;
}

// Signed 16-bit halves of a packed word, as floats.
static __device__ __forceinline__ float lo16(unsigned w) { return (float)(int)(short)(w & 0xffffu); }
static __device__ __forceinline__ float hi16(unsigned w) { return (float)((int)w >> 16); }

// Resident CTAs per SM the register allocation targets, per mode (measured on the
// single-detector workload, 16-sample tiles): 3 (80 registers, a few spilled to
// L1) runs the forward and sky-adjoint passes 10 % faster than 2 (128 registers);
// the shared-geometry pass keeps three accumulators per sample and is fastest at
// 2; the beam-grid transpose, bound by its atomic adds, at 4.
constexpr int fast_min_blocks(int mode) { return mode == kPsb ? 2 : (mode == kGrid ? 4 : 3); }
// Threads per block: NT, or for the shared-memory fetch (one block per SM, its shared memory
// holding the node grid) three times as many, the same 24 warps per SM.
constexpr int fast_threads(int fetch) { return fetch == PISCO_FETCH_SHARED ? 3 * NT : NT; }
constexpr int fast_blocks(int fetch, int mode) { return fetch == PISCO_FETCH_SHARED ? 1 : fast_min_blocks(mode); }

template <int S, int NP, int FETCH, int MODE>
__global__ void __launch_bounds__(fast_threads(FETCH), fast_blocks(FETCH, MODE))
    k_fast(const __grid_constant__ LaunchParams P) {
    constexpr int NTK = fast_threads(FETCH), NWK = NTK / 32;
    __shared__ double sTh[S], sPh[S], sPx[S], sPy[S], sPz[S];
    __shared__ float4 sA[S];  // cos(b/2), sin(b/2), cos psi0, sin psi0   (b = phi0 - phi_c)
    __shared__ float4 sB[S];  // cos theta0, sin theta0, Z_theta, Z_phi
    __shared__ float sBf[S];  // b
    __shared__ float sY[S];   // adjoint: tod * scale
    __shared__ int sValid[S];
    __shared__ int sGs[S], sGe[S];
    __shared__ int sNg;
    __shared__ double sPhiC;
    __shared__ int sRlo, sRhi;
    __shared__ float2 sPA[RC * S];  // per (ring, sample): sin(dtheta), 1 - cos(dtheta)
    __shared__ float sLo[RC], sHi[RC];
    __shared__ int sFlag[RC];
    __shared__ int sJlo[RC], sJref[RC], sFirst[RC], sRc[RC], sCnt[RC], sPref[RC + 1], sWarpTot[RC / 32];
    __shared__ float sAref[RC], sSr[RC], sInv[RC], sDph[RC];
    __shared__ float sRed[NWK][S];

    // shared-memory fetch: the folded node grid of the current detector, [N][N] (A, Bq', Cu', 0)
    extern __shared__ float4 sGridNodes[];
    int grid_det = -1;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float4* __restrict__ sky = (const float4*)P.sky;
    const int nc = P.grid_n - 1;
    const float gmax = (float)(P.grid_n - 2);
    // beam-grid transpose target: the output, or the second output when both transposes run
    float* const gout = (float*)(MODE == kBoth ? P.out2 : P.out);

    for (long long tile = blockIdx.x; tile < P.total_tiles; tile += gridDim.x) {
        int d = 0;
        while (d + 1 < P.ndet && P.det[d + 1].tile_begin <= tile) ++d;
        const DetEntry& det = P.det[d];
        const long long lt = tile - det.tile_begin;
        const long long t0 = det.begin + lt * S;
        const int ns = (int)min((long long)S, det.count - lt * S);
        const float* __restrict__ cells = (const float*)det.beam;
        // packed cells: biased exponent of the unit slope scale, from the 32-byte header
        const int qbase = FETCH == PISCO_FETCH_PACKED ? __ldg((const int*)det.beam) : 0;
        if (FETCH == PISCO_FETCH_SHARED && d != grid_det) {
            // stage this detector's node grid (once per block and detector of the persistent launch)
            __syncthreads();
            const float4* __restrict__ src = (const float4*)det.beam;
            for (int q = tid; q < P.grid_n * P.grid_n; q += NTK) sGridNodes[q] = __ldg(src + q);
            __syncthreads();
            grid_det = d;
        }

        // 1. per-sample constants
        if (tid < S) {
            const int i = tid;
            bool ok = i < ns;
            double th = 0.0, ph = 0.0, ps = 0.0;
            if (ok) {
                th = P.theta[t0 + i];
                ph = P.phi[t0 + i];
                ps = P.psi[t0 + i];
                ok = isfinite(th) && isfinite(ph) && isfinite(ps) && th >= 0.0 && th <= kPi;
            }
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = make_float4(0.f, 0.f, 0.f, 0.f);
            double px = 0.0, py = 0.0, pz = 0.0, phw = 0.0;
            if (ok) {
                phw = ph - kTwoPi * floor(ph / kTwoPi);
                if (phw >= kTwoPi) phw -= kTwoPi;
                double st, ct, sp, cp, ss, cs;
                sincos(th, &st, &ct);
                sincos(phw, &sp, &cp);
                sincos(ps, &ss, &cs);
                px = st * cp;
                py = st * sp;
                pz = ct;
                a.z = (float)cs;
                a.w = (float)ss;
                b = make_float4((float)ct, (float)st, (float)(-cs * st), (float)(ss * st));
                if (MODE == kAdjoint || MODE == kGrid || MODE == kBoth)
                    sY[i] = (float)((double)((const float*)P.tod_in)[t0 + i] * det.scale);
            }
            sTh[i] = th;
            sPh[i] = phw;
            sPx[i] = px;
            sPy[i] = py;
            sPz[i] = pz;
            sA[i] = a;
            sB[i] = b;
            sValid[i] = ok ? 1 : 0;
        }
        __syncthreads();

        // 2. greedy grouping of nearby samples
        if (tid == 0) {
            int ng = 0, i = 0;
            while (i < S) {
                if (!sValid[i]) {
                    ++i;
                    continue;
                }
                int j = i + 1;
                for (; j < S; ++j) {
                    if (!sValid[j]) continue;
                    const double c = sPx[i] * sPx[j] + sPy[i] * sPy[j] + sPz[i] * sPz[j];
                    double db = sPh[j] - sPh[i];
                    db -= kTwoPi * rint(db / kTwoPi);
                    if (c < P.group_cos || fabs(db) > (double)P.group_dphi) break;
                }
                sGs[ng] = i;
                sGe[ng] = j;
                ++ng;
                i = j;
            }
            sNg = ng;
        }
        __syncthreads();
        const int ngroups = sNg;

        for (int g = 0; g < ngroups; ++g) {
            const int gs = sGs[g], ge = sGe[g];
            if (tid < S && tid >= gs && tid < ge && sValid[tid]) {
                double db = sPh[tid] - sPh[gs];
                db -= kTwoPi * rint(db / kTwoPi);
                double sb, cb;
                sincos(0.5 * db, &sb, &cb);
                sA[tid].x = (float)cb;
                sA[tid].y = (float)sb;
                sBf[tid] = (float)db;
            }
            if (tid == 0) {
                sPhiC = sPh[gs];
                double tmin = 1e9, tmax = -1e9;
                for (int i = gs; i < ge; ++i)
                    if (sValid[i]) {
                        tmin = fmin(tmin, sTh[i]);
                        tmax = fmax(tmax, sTh[i]);
                    }
                int ra, rb;
                ring_range(tmin, tmax, P.radius, P.nside, &ra, &rb);
                sRlo = ra;
                sRhi = rb;
            }
            __syncthreads();

            // forward / count: acc.  Shared-geometry pass: acc = intensity part and accR + i accM =
            // polarised part for the cells' own zeta; another angle zeta_k multiplies the
            // polarised part by e^{2 i (zeta_k - zeta)}: zeta enters only through the folding's
            // e^{2 i zeta} (Sec. 3 eq. copol_bolo; a PSB pair is zeta and zeta - 90 deg)
            float acc[S], accR[MODE == kPsb ? S : 1], accM[MODE == kPsb ? S : 1];
#pragma unroll
            for (int i = 0; i < S; ++i) acc[i] = 0.f;
#pragma unroll
            for (int i = 0; i < (MODE == kPsb ? S : 1); ++i) accR[i] = accM[i] = 0.f;

            const int rlo = sRlo, rhi = sRhi;
            for (int c0 = rlo; c0 <= rhi; c0 += RC) {
                const int nr = min(RC, rhi - c0 + 1);

                // 3. per (ring, sample) offsets and the union of the discs' longitude ranges
                for (int item = tid; item < RC * S; item += NTK) {
                    const int ri = item / S, i = item % S;
                    float lo = __int_as_float(0x7f800000), hi = -__int_as_float(0x7f800000);
                    int full = 0;
                    float2 pa = make_float2(0.f, 1e30f);
                    if (ri < nr && i >= gs && i < ge && sValid[i]) {
                        const RingInfo& R = P.rings[c0 + ri];
                        const float h = (float)(0.5 * (R.theta - sTh[i]));
                        float sh, ch;
                        sincosf(h, &sh, &ch);
                        const float av = 2.f * sh * sh;
                        pa = make_float2(2.f * sh * ch, av);
                        if (av <= P.wr_hi) {
                            const float b2 = 2.f * sB[i].y * R.s_f;
                            const float tau = (P.wr_hi - av) / b2;
                            if (!(b2 > 0.f) || !(tau < 0.999f)) {
                                full = 1;
                            } else {
                                const float hw = 2.f * asinf(sqrtf(fmaxf(tau, 0.f)));
                                lo = sBf[i] - hw;
                                hi = sBf[i] + hw;
                            }
                        }
                    }
                    sPA[item] = pa;
#pragma unroll
                    for (int off = S / 2; off > 0; off >>= 1) {
                        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, off, S));
                        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, off, S));
                        full |= __shfl_xor_sync(0xffffffffu, full, off, S);
                    }
                    if (i == 0 && ri < nr) {
                        sLo[ri] = lo;
                        sHi[ri] = hi;
                        sFlag[ri] = full ? 2 : (lo <= hi ? 1 : 0);
                    }
                }
                __syncthreads();

                // per ring: pixel index range of the union; the prefix sum counts runs
                // of NP consecutive ring pixels (the last run of a ring is masked)
                int cnt = 0;
                if (tid < RC) {
                    int jlo = 0, jref = 0, first = 0, rc = 1;
                    float aref = 0.f, sr = 0.f, inv = 0.f, dph = 0.f;
                    if (tid < nr) {
                        const RingInfo& R = P.rings[c0 + tid];
                        const int flag = sFlag[tid];
                        first = (int)R.first;
                        rc = R.count;
                        sr = R.s_f;
                        inv = R.inv_s2_f;
                        dph = R.dphi_f;
                        const double phic = sPhiC;
                        jref = (int)rint((phic - R.phi0) / R.dphi);
                        aref = (float)(R.phi0 + (double)jref * R.dphi - phic);
                        if (flag == 2) {
                            cnt = R.count;
                            jlo = jref - R.count / 2;
                        } else if (flag == 1) {
                            const double ulo = (phic + (double)sLo[tid] - R.phi0) / R.dphi;
                            const double uhi = (phic + (double)sHi[tid] - R.phi0) / R.dphi;
                            const long long a = (long long)floor(ulo) - 1, b = (long long)ceil(uhi) + 1;
                            if (b - a + 1 >= R.count) {
                                cnt = R.count;
                                jlo = jref - R.count / 2;
                            } else {
                                cnt = (int)(b - a + 1);
                                jlo = (int)a;
                            }
                        }
                    }
                    sJlo[tid] = jlo;
                    sJref[tid] = jref;
                    sFirst[tid] = first;
                    sRc[tid] = rc;
                    sCnt[tid] = cnt;
                    sAref[tid] = aref;
                    sSr[tid] = sr;
                    sInv[tid] = inv;
                    sDph[tid] = dph;
                    int v = (cnt + NP - 1) / NP;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, v, o);
                        if (lane >= o) v += y;
                    }
                    if (lane == 31) sWarpTot[warp] = v;
                    cnt = v;  // inclusive prefix of runs within the warp
                }
                __syncthreads();
                if (tid < RC) {
                    int base = 0;
                    for (int w = 0; w < warp; ++w) base += sWarpTot[w];
                    sPref[tid + 1] = base + cnt;
                    if (tid == 0) sPref[0] = 0;
                }
                __syncthreads();

                // 4-7. runs of NP pixels x samples of the group: every per-sample value
                // read from shared memory serves NP pairs from registers
                const int totalq = sPref[nr];
                for (int qd = tid; qd < totalq; qd += NTK) {
                    int lo_ = 0, hi_ = nr - 1;
                    while (lo_ < hi_) {
                        const int mid = (lo_ + hi_ + 1) >> 1;
                        if (sPref[mid] <= qd) lo_ = mid;
                        else hi_ = mid - 1;
                    }
                    const int ri = lo_;
                    const int off0 = (qd - sPref[ri]) * NP;
                    const int cnt_r = sCnt[ri], rc = sRc[ri], jlo = sJlo[ri], jref = sJref[ri], first = sFirst[ri];
                    const float aref = sAref[ri], dph = sDph[ri], inv = sInv[ri];
                    const float sr2 = 2.f * sSr[ri];
                    float sa[NP], ca[NP], ip[NP], qp[NP], up[NP];
                    int jw[NP];
                    bool ok[NP];
#pragma unroll
                    for (int p4 = 0; p4 < NP; ++p4) {
                        const int j = jlo + off0 + p4;
                        int w = j % rc;
                        if (w < 0) w += rc;
                        jw[p4] = w;
                        ok[p4] = off0 + p4 < cnt_r;
                        const float aa = fmaf((float)(j - jref), dph, aref);
                        sincosf(0.5f * aa, &sa[p4], &ca[p4]);
                        float4 sk = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (ok[p4]) sk = __ldg(sky + first + w);
                        ip[p4] = sk.x;
                        qp[p4] = sk.y * inv;
                        up[p4] = sk.z * inv;
                    }
                    int lastcell[NP];
                    float4 cka[NP], ckb[NP], ckc[NP];
#pragma unroll
                    for (int p4 = 0; p4 < NP; ++p4) lastcell[p4] = -1;
                    float gI[NP], gQ[NP], gU[NP];
#pragma unroll
                    for (int p4 = 0; p4 < NP; ++p4) gI[p4] = gQ[p4] = gU[p4] = 0.f;
                    // beam-grid transpose: gradient of the four nodes of the current cell,
                    // kept in registers while consecutive samples stay in the cell
                    int gcell[NP];
                    float gw[NP][12];
#pragma unroll
                    for (int p4 = 0; p4 < NP; ++p4) {
                        gcell[p4] = -1;
#pragma unroll
                        for (int k = 0; k < 12; ++k) gw[p4][k] = 0.f;
                    }
#pragma unroll
                    for (int i = 0; i < S; ++i) {
                        if (i < gs || i >= ge) continue;
                        const float4 A4 = sA[i];
                        const float4 B4 = sB[i];
                        const float2 pa = sPA[ri * S + i];
                        const float k0 = B4.y * sr2;   // 2 sin(theta0) sin(theta_r)
                        const float k1 = -B4.x * sr2;  // -2 cos(theta0) sin(theta_r)
#pragma unroll
                        for (int p4 = 0; p4 < NP; ++p4) {
                            if (!ok[p4]) continue;
                            const float sh = fmaf(sa[p4], A4.x, -ca[p4] * A4.y);  // sin(dphi / 2)
                            const float ch = fmaf(ca[p4], A4.x, sa[p4] * A4.y);   // cos(dphi / 2)
                            const float sh2 = sh * sh;
                            const float w = fmaf(k0, sh2, pa.y);  // 1 - k . p0
                            if (w > P.wr_hi) continue;
                            if (w > P.wr_lo &&
                                !exact_in_disc(P.rings, c0 + ri, jw[p4], sPx[i], sPy[i], sPz[i], P.cos_r))
                                continue;
                            if (MODE == kCount) {
                                acc[i] += 1.f;
                                continue;
                            }
                            const float x0 = fmaf(k1, sh2, pa.x);
                            const float y0 = sr2 * sh * ch;
                            const float x = fmaf(A4.z, x0, A4.w * y0);   // k . theta'0
                            const float y = fmaf(A4.z, y0, -A4.w * x0);  // k . phi'0
                            const float fu = fmaf(x, P.invh_f, P.cg_f);
                            const float fv = fmaf(y, P.invh_f, P.cg_f);
                            const float flu = fminf(fmaxf(floorf(fu), 0.f), gmax);
                            const float flv = fminf(fmaxf(floorf(fv), 0.f), gmax);
                            const float fx = fmaf(x, P.invh_f, P.cg_f - flu);
                            const float fy = fmaf(y, P.invh_f, P.cg_f - flv);
                            if (MODE == kGrid || MODE == kBoth) {
                                const int cell = (int)flv * nc + (int)flu;
                                if (cell != gcell[p4]) {
                                    if (gcell[p4] >= 0) flush_grid(gout, gcell[p4], nc, P.grid_n, gw[p4], P.grid_coef);
                                    gcell[p4] = cell;
                                }
                                const float q = rcp_approx(2.f - w);
                                const float mp = fmaf(q, fmaf(x, B4.z, y * B4.w), B4.x);
                                const float e1 = fmaf(-x, mp, B4.z);
                                const float e2 = fmaf(-y, mp, B4.w);
                                const float re = fmaf(e1, e1, -e2 * e2);
                                const float im2 = e1 * e2;
                                const float yv = sY[i];
                                const float cA = yv * ip[p4];
                                const float cB = yv * fmaf(re, qp[p4], -2.f * im2 * up[p4]);
                                const float cC = yv * fmaf(2.f * im2, qp[p4], re * up[p4]);
                                // node weights, or the bilinear coefficients' weights (1, fx, fy, fx fy)
                                const float w11 = fx * fy;
                                const bool cf = P.grid_coef != 0;
                                const float w10 = cf ? fx : fx - w11, w01 = cf ? fy : fy - w11;
                                const float w00 = cf ? 1.f : (1.f - fx) - (fy - w11);
                                const float wt[4] = {w00, w10, w01, w11};
#pragma unroll
                                for (int k = 0; k < 4; ++k) {
                                    gw[p4][k] = fmaf(cA, wt[k], gw[p4][k]);
                                    gw[p4][4 + k] = fmaf(cB, wt[k], gw[p4][4 + k]);
                                    gw[p4][8 + k] = fmaf(cC, wt[k], gw[p4][8 + k]);
                                }
                                if (MODE == kGrid) continue;
                            }
                            float bA, bB, bC;
                            if (FETCH == PISCO_FETCH_CELLS) {
                                const int cell = (int)flv * nc + (int)flu;
                                // consecutive samples of a pixel often fall in the cell of
                                // the previous one: keep its coefficients in registers
                                if (cell != lastcell[p4]) {
                                    ld_nc_v8(cells + 16 * cell, cka[p4], ckb[p4]);
                                    ckc[p4] = ld_nc_v4(cells + 16 * cell + 8);
                                    lastcell[p4] = cell;
                                }
                                const float4 ka = cka[p4], kb = ckb[p4], kc = ckc[p4];
                                bA = fmaf(fy, fmaf(fx, ka.w, ka.z), fmaf(fx, ka.y, ka.x));
                                bB = fmaf(fy, fmaf(fx, kb.w, kb.z), fmaf(fx, kb.y, kb.x));
                                bC = fmaf(fy, fmaf(fx, kc.w, kc.z), fmaf(fx, kc.y, kc.x));
                            } else if (FETCH == PISCO_FETCH_PACKED) {
                                const int cell = (int)flv * nc + (int)flu;
                                if (cell != lastcell[p4]) {
                                    ld_nc_v8(cells + 8 * (cell + 1), cka[p4], ckb[p4]);  // after the header
                                    lastcell[p4] = cell;
                                }
                                const float4 lo = cka[p4], hi = ckb[p4];
                                const unsigned w3 = __float_as_uint(lo.w), w4 = __float_as_uint(hi.x);
                                const unsigned w5 = __float_as_uint(hi.y), w6 = __float_as_uint(hi.z);
                                const unsigned w7 = __float_as_uint(hi.w);
                                const unsigned ex = w7 >> 16;
                                const float sA = __int_as_float((qbase + (int)(ex & 31u)) << 23);
                                const float sB = __int_as_float((qbase + (int)((ex >> 5) & 31u)) << 23);
                                const float sC = __int_as_float((qbase + (int)((ex >> 10) & 31u)) << 23);
                                bA = fmaf(sA, fmaf(fy, fmaf(fx, lo16(w4), hi16(w3)), fx * lo16(w3)), lo.x);
                                bB = fmaf(sB, fmaf(fy, fmaf(fx, hi16(w5), lo16(w5)), fx * hi16(w4)), lo.y);
                                bC = fmaf(sC, fmaf(fy, fmaf(fx, lo16(w7), hi16(w6)), fx * lo16(w6)), lo.z);
                            } else if (FETCH == PISCO_FETCH_SHARED) {
                                // bilinear in FP32 from the cell's four nodes in shared memory
                                const int q00 = (int)flv * P.grid_n + (int)flu;
                                const float4 n00 = sGridNodes[q00], n10 = sGridNodes[q00 + 1];
                                const float4 n01 = sGridNodes[q00 + P.grid_n], n11 = sGridNodes[q00 + P.grid_n + 1];
                                const float ax = fmaf(fx, n10.x - n00.x, n00.x), bx = fmaf(fx, n11.x - n01.x, n01.x);
                                const float ay = fmaf(fx, n10.y - n00.y, n00.y), by = fmaf(fx, n11.y - n01.y, n01.y);
                                const float az = fmaf(fx, n10.z - n00.z, n00.z), bz = fmaf(fx, n11.z - n01.z, n01.z);
                                bA = fmaf(fy, bx - ax, ax);
                                bB = fmaf(fy, by - ay, ay);
                                bC = fmaf(fy, bz - az, az);
                            } else {
                                // texel centres sit at integer + 1/2: (flu + 1, flv + 1) selects
                                // nodes flu, flu + 1 and flv, flv + 1 exactly
                                const float xc = flu + 1.f, yc = flv + 1.f;
                                bA = lerp_gather(tex2Dgather<float4>(det.tex[0], xc, yc, 0), fx, fy);
                                bB = lerp_gather(tex2Dgather<float4>(det.tex[1], xc, yc, 0), fx, fy);
                                bC = lerp_gather(tex2Dgather<float4>(det.tex[2], xc, yc, 0), fx, fy);
                            }
                            const float q = rcp_approx(2.f - w);  // 1 / (1 + k . p0)
                            const float mp = fmaf(q, fmaf(x, B4.z, y * B4.w), B4.x);
                            const float e1 = fmaf(-x, mp, B4.z);
                            const float e2 = fmaf(-y, mp, B4.w);
                            const float re = fmaf(e1, e1, -e2 * e2);
                            const float im2 = e1 * e2;
                            if (MODE == kForward) {
                                const float al = fmaf(re, qp[p4], -2.f * im2 * up[p4]);
                                const float be = fmaf(2.f * im2, qp[p4], re * up[p4]);
                                acc[i] = fmaf(bA, ip[p4], fmaf(bB, al, fmaf(bC, be, acc[i])));
                            } else if (MODE == kPsb) {
                                const float al = fmaf(re, qp[p4], -2.f * im2 * up[p4]);
                                const float be = fmaf(2.f * im2, qp[p4], re * up[p4]);
                                acc[i] = fmaf(bA, ip[p4], acc[i]);
                                accR[i] = fmaf(bB, al, fmaf(bC, be, accR[i]));
                                accM[i] = fmaf(bC, al, fmaf(-bB, be, accM[i]));
                            } else {
                                const float yv = sY[i];
                                gI[p4] = fmaf(yv, bA, gI[p4]);
                                gQ[p4] = fmaf(yv, fmaf(bB, re, 2.f * bC * im2), gQ[p4]);
                                gU[p4] = fmaf(yv, fmaf(bC, re, -2.f * bB * im2), gU[p4]);
                            }
                        }
                    }
                    if (MODE == kGrid || MODE == kBoth) {
#pragma unroll
                        for (int p4 = 0; p4 < NP; ++p4)
                            if (gcell[p4] >= 0) flush_grid(gout, gcell[p4], nc, P.grid_n, gw[p4], P.grid_coef);
                    }
                    if (MODE == kAdjoint || MODE == kBoth) {
                        float* maps = (float*)P.out;
#pragma unroll
                        for (int p4 = 0; p4 < NP; ++p4) {
                            if (ok[p4] && (gI[p4] != 0.f || gQ[p4] != 0.f || gU[p4] != 0.f)) {
                                const long long pix = (long long)first + jw[p4];
                                atomicAdd(maps + pix, gI[p4]);
                                atomicAdd(maps + P.npix + pix, gQ[p4] * inv);
                                atomicAdd(maps + 2 * P.npix + pix, gU[p4] * inv);
                            }
                        }
                    }
                }
                __syncthreads();
            }

            if (MODE == kForward || MODE == kCount) {
#pragma unroll
                for (int i = 0; i < S; ++i) {
                    if (i < gs || i >= ge) continue;
                    float v = acc[i];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == 0) sRed[warp][i] = v;
                }
                __syncthreads();
                if (tid >= gs && tid < ge && sValid[tid]) {
                    double s = 0.0;
#pragma unroll
                    for (int w = 0; w < NWK; ++w) s += (double)sRed[w][tid];
                    if (MODE == kForward) ((float*)P.out)[t0 + tid] = (float)(det.scale * s);
                    else P.counts[t0 + tid] = (int32_t)s;
                }
                __syncthreads();
            }
            if (MODE == kPsb) {
                double part[3] = {0.0, 0.0, 0.0};
#pragma unroll
                for (int c = 0; c < 3; ++c) {
#pragma unroll
                    for (int i = 0; i < S; ++i) {
                        if (i < gs || i >= ge) continue;
                        float v = c == 0 ? acc[i] : (c == 1 ? accR[i] : accM[i]);
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                        if (lane == 0) sRed[warp][i] = v;
                    }
                    __syncthreads();
                    if (tid >= gs && tid < ge && sValid[tid])
                        for (int w = 0; w < NWK; ++w) part[c] += (double)sRed[w][tid];
                    __syncthreads();
                }
                if (tid >= gs && tid < ge && sValid[tid]) {
                    float* out = (float*)P.out;
                    for (int k = 0; k < P.n_zeta; ++k)
                        out[k * P.out_stride + t0 + tid] =
                            (float)(det.scale * (part[0] + (double)P.psb_c2z[k] * part[1] - (double)P.psb_s2z[k] * part[2]));
                }
            }
        }

        if (tid < ns && !sValid[tid]) {
            if (MODE == kForward) ((float*)P.out)[t0 + tid] = __int_as_float(0x7fc00000);
            if (MODE == kPsb)
                for (int k = 0; k < P.n_zeta; ++k) ((float*)P.out)[k * P.out_stride + t0 + tid] = __int_as_float(0x7fc00000);
            if (MODE == kCount) P.counts[t0 + tid] = -1;
        }
        __syncthreads();
    }
}

// One launch of mode MODE: a grid of one block per tile, or, for the shared-memory fetch, a
// persistent grid of the resident blocks (each stages the node grid once).
template <int S, int NP, int FETCH, int MODE>
static cudaError_t launch_mode(const LaunchParams& p, cudaStream_t s) {
    unsigned grid = (unsigned)min(p.total_tiles, (long long)INT_MAX);
    size_t dyn = 0;
    if constexpr (FETCH == PISCO_FETCH_SHARED) {
        dyn = (size_t)p.grid_n * p.grid_n * sizeof(float4);
        cudaError_t e = cudaFuncSetAttribute(k_fast<S, NP, FETCH, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)dyn);
        if (e != cudaSuccess) return e;
        int dev = 0, n_sm = 0, per_sm = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fast<S, NP, FETCH, MODE>, fast_threads(FETCH), dyn);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        grid = (unsigned)min((long long)grid, (long long)n_sm * per_sm);
    }
    k_fast<S, NP, FETCH, MODE><<<grid, fast_threads(FETCH), dyn, s>>>(p);
    return cudaGetLastError();
}

template <int S, int NP, int FETCH>
static cudaError_t launch_s(const LaunchParams& p, int mode, cudaStream_t s) {
    if (p.total_tiles <= 0) return cudaSuccess;
    if (mode == kPsb) {
        // three accumulators per sample: instantiated for beam cells only
        if constexpr (FETCH != PISCO_FETCH_TEXTURE) return launch_mode<S, NP, FETCH, kPsb>(p, s);
        return cudaErrorInvalidValue;
    }
    switch (mode) {
        case kForward: return launch_mode<S, NP, FETCH, kForward>(p, s);
        case kAdjoint: return launch_mode<S, NP, FETCH, kAdjoint>(p, s);
        case kGrid: return launch_mode<S, NP, FETCH, kGrid>(p, s);
        case kBoth: return launch_mode<S, NP, FETCH, kBoth>(p, s);
        default: return launch_mode<S, NP, FETCH, kCount>(p, s);
    }
}

// Dispatch over the tile size and pixels per thread for one fetch mode.
template <int FETCH>
static cudaError_t launch_fetch(const LaunchParams& p, int mode, int tile_samples, int np, cudaStream_t s) {
    const bool one = np == 1;
    switch (tile_samples) {
        case 8: return one ? launch_s<8, 1, FETCH>(p, mode, s) : launch_s<8, 2, FETCH>(p, mode, s);
        case 32: return one ? launch_s<32, 1, FETCH>(p, mode, s) : launch_s<32, 2, FETCH>(p, mode, s);
        default: return one ? launch_s<16, 1, FETCH>(p, mode, s) : launch_s<16, 2, FETCH>(p, mode, s);
    }
}

}  // namespace pisco
