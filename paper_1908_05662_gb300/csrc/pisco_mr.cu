// Multi-realization convolution on the tensor cores.
//
// With R sky realizations S_r sharing one scan and one beam, the TOD is a
// dense contraction (eq. discrete_beam_conv_tensor with the per-pair weights
// factored out):
//     d_r(t) = scale * sum_k sum_{m = I,Q,U} W[t][k][m] S_r[k][m],
//     W[t][k] = (A, (Bq' re + 2 Cu' im2) / sin^2 theta_k, (Cu' re - 2 Bq' im2) / sin^2 theta_k),
// the pair weights of the FP32 kernel.  One CTA owns 16 consecutive samples
// (the tile and union disc of the FP32 kernel).  For each batch of 32 union
// pixels it
//   1. stages the realizations of the batch, [pixel][I,Q,U][R] in 16-bit, in
//      shared memory (rows k = 3 pixel + m, realizations contiguous);
//   2. computes the 32 x 16 pair weights in FP32 (zero outside a sample's
//      disc) and splits each into two 16-bit parts, W = W_hi + W_lo with
//      W_lo the rounded remainder, [sample][k] (the weights keep ~16
//      significant bits; only the stored realizations are 16-bit);
//   3. accumulates D[r][t] += sum_k S[k][r] (W_hi[t][k] + W_lo[t][k]) with
//      m16n8k16 MMAs (realizations = M, samples = N), FP32 accumulators in
//      registers; warp w owns realizations 32 w .. 32 w + 31.
// Realization stacks are [Npix][3][R] 16-bit (BF16 or FP16), R a multiple of
// 32 up to 256; the output is FP32 [n][R].

#include "pisco_internal.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <climits>

namespace pisco {

namespace {

constexpr int MT = 256;         // threads
constexpr int MS = 16;          // samples per tile
constexpr int MRC = 128;        // rings per chunk
constexpr int KPIX = 32;        // union pixels per batch
constexpr int KB = 3 * KPIX;    // contraction length per batch
constexpr int SKY_LD = 264;     // 16-bit elements per staged realization row (256 + 8: ldmatrix rows on distinct banks)
constexpr int W_LD = KB + 8;    // 16-bit elements per weight row (conflict-free B-fragment loads)
constexpr int MR_DYN_SMEM = (KB * SKY_LD + 2 * MS * W_LD) * 2;

// x split into a rounded 16-bit part and the rounded remainder.
__device__ __forceinline__ void split16(float x, int f16, unsigned short& hi, unsigned short& lo) {
    if (f16) {
        const __half h = __float2half_rn(x);
        const __half l = __float2half_rn(x - __half2float(h));
        hi = *reinterpret_cast<const unsigned short*>(&h);
        lo = *reinterpret_cast<const unsigned short*>(&l);
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
        hi = *reinterpret_cast<const unsigned short*>(&h);
        lo = *reinterpret_cast<const unsigned short*>(&l);
    }
}

__device__ __forceinline__ void mma16816(float* d, const unsigned* a, unsigned b0, unsigned b1, int f16) {
    if (f16) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    } else {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
}

__device__ __forceinline__ void ldsm_x4_trans(unsigned* a, const void* p) {
    const unsigned addr = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3])
                 : "r"(addr));
}

__device__ __forceinline__ void ldg_cell(const float* p, float4& a, float4& b, float4& c) {
    asm("ld.global.nc.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
    asm("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
        : "=f"(c.x), "=f"(c.y), "=f"(c.z), "=f"(c.w)
        : "l"(p + 8));
}

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

}  // namespace

template <int F16>
__global__ void __launch_bounds__(MT, 2) k_mr(const __grid_constant__ LaunchParams P) {
    __shared__ double sTh[MS], sPh[MS], sPx[MS], sPy[MS], sPz[MS];
    __shared__ float4 sA[MS], sB[MS];
    __shared__ float sBf[MS];
    __shared__ int sValid[MS], sGs[MS], sGe[MS];
    __shared__ int sNg, sRlo, sRhi;
    __shared__ double sPhiC;
    __shared__ float2 sPA[MRC * MS];
    __shared__ float sLo[MRC], sHi[MRC];
    __shared__ int sFlag[MRC], sJlo[MRC], sJref[MRC], sFirst[MRC], sRc[MRC], sCnt[MRC], sPref[MRC + 1], sWarpTot[MRC / 32];
    __shared__ float sAref[MRC], sSr[MRC], sInv[MRC], sDph[MRC];
    // per batch pixel data
    __shared__ int bRi[KPIX], bJw[KPIX], bOk[KPIX];
    __shared__ float bSa[KPIX], bCa[KPIX];
    extern __shared__ __align__(16) unsigned short mr_dyn[];
    unsigned short* sSky = mr_dyn;               // [KB][SKY_LD]
    unsigned short* sW = mr_dyn + KB * SKY_LD;   // [MS][W_LD] high parts
    unsigned short* sWl = sW + MS * W_LD;        // [MS][W_LD] low parts

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned short* __restrict__ sky16 = (const unsigned short*)P.sky;
    const int nreal = P.n_real;
    const int nc = P.grid_n - 1;
    const float gmax = (float)(P.grid_n - 2);
    const bool mma_warp = warp * 32 < nreal;

    for (long long tile = blockIdx.x; tile < P.total_tiles; tile += gridDim.x) {
        int d = 0;
        while (d + 1 < P.ndet && P.det[d + 1].tile_begin <= tile) ++d;
        const DetEntry& det = P.det[d];
        const long long lt = tile - det.tile_begin;
        const long long t0 = det.begin + lt * MS;
        const int ns = (int)min((long long)MS, det.count - lt * MS);
        const float* __restrict__ cells = (const float*)det.beam;

        if (tid < MS) {
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
        if (tid == 0) {
            int ng = 0, i = 0;
            while (i < MS) {
                if (!sValid[i]) {
                    ++i;
                    continue;
                }
                int j = i + 1;
                for (; j < MS; ++j) {
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

        // accumulators: [m-tile][n-tile][4], realizations warp*32 + mt*16 + ..., samples nt*8 + ...
        float acc[2][2][4];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;

        for (int g = 0; g < ngroups; ++g) {
            const int gs = sGs[g], ge = sGe[g];
            if (tid < MS && tid >= gs && tid < ge && sValid[tid]) {
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
            const int rlo = sRlo, rhi = sRhi;
            for (int c0 = rlo; c0 <= rhi; c0 += MRC) {
                const int nr = min(MRC, rhi - c0 + 1);
                for (int item = tid; item < MRC * MS; item += MT) {
                    const int ri = item / MS, i = item % MS;
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
                    for (int off = MS / 2; off > 0; off >>= 1) {
                        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, off, MS));
                        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, off, MS));
                        full |= __shfl_xor_sync(0xffffffffu, full, off, MS);
                    }
                    if (i == 0 && ri < nr) {
                        sLo[ri] = lo;
                        sHi[ri] = hi;
                        sFlag[ri] = full ? 2 : (lo <= hi ? 1 : 0);
                    }
                }
                __syncthreads();
                int cnt = 0;
                if (tid < MRC) {
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
                    int v = cnt;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, v, o);
                        if (lane >= o) v += y;
                    }
                    if (lane == 31) sWarpTot[warp] = v;
                    cnt = v;
                }
                __syncthreads();
                if (tid < MRC) {
                    int base = 0;
                    for (int w = 0; w < warp; ++w) base += sWarpTot[w];
                    sPref[tid + 1] = base + cnt;
                    if (tid == 0) sPref[0] = 0;
                }
                __syncthreads();

                const int total = sPref[nr];
                for (int b0 = 0; b0 < total; b0 += KPIX) {
                    // 1a. pixel data of the batch
                    if (tid < KPIX) {
                        const int f = b0 + tid;
                        int ok = f < total;
                        int ri = 0, jw = 0;
                        float sa = 0.f, ca = 1.f;
                        if (ok) {
                            int lo_ = 0, hi_ = nr - 1;
                            while (lo_ < hi_) {
                                const int mid = (lo_ + hi_ + 1) >> 1;
                                if (sPref[mid] <= f) lo_ = mid;
                                else hi_ = mid - 1;
                            }
                            ri = lo_;
                            const int j = sJlo[ri] + (f - sPref[ri]);
                            const int rc = sRc[ri];
                            jw = j % rc;
                            if (jw < 0) jw += rc;
                            const float aa = fmaf((float)(j - sJref[ri]), sDph[ri], sAref[ri]);
                            sincosf(0.5f * aa, &sa, &ca);
                        }
                        bRi[tid] = ri;
                        bJw[tid] = jw;
                        bOk[tid] = ok;
                        bSa[tid] = sa;
                        bCa[tid] = ca;
                    }
                    __syncthreads();
                    // 1b. stage the realizations of the batch: 32 pixels x 3 rows x R values
                    {
                        const int chunks = nreal / 8;  // 16-byte chunks per row
                        for (int q = tid; q < KB * chunks; q += MT) {
                            const int row = q / chunks, cch = q % chunks;
                            const int p = row / 3, m = row % 3;
                            uint4 v = make_uint4(0u, 0u, 0u, 0u);
                            if (bOk[p]) {
                                const long long pix = (long long)sFirst[bRi[p]] + bJw[p];
                                v = __ldg((const uint4*)(sky16 + (pix * 3 + m) * nreal) + cch);
                            }
                            *(uint4*)(sSky + row * SKY_LD + 8 * cch) = v;
                        }
                    }
                    // 2. pair weights: pixel p = tid % 32, samples tid / 32 and tid / 32 + 8
#pragma unroll
                    for (int h2 = 0; h2 < 2; ++h2) {
                        const int p = tid & 31, i = (tid >> 5) + 8 * h2;
                        float wI = 0.f, wQ = 0.f, wU = 0.f;
                        if (i >= gs && i < ge && bOk[p]) {
                            const int ri = bRi[p];
                            const float sr2 = 2.f * sSr[ri], inv = sInv[ri];
                            const float4 A4 = sA[i];
                            const float4 B4 = sB[i];
                            const float2 pa = sPA[ri * MS + i];
                            const float sa = bSa[p], ca = bCa[p];
                            const float sh = fmaf(sa, A4.x, -ca * A4.y);
                            const float ch = fmaf(ca, A4.x, sa * A4.y);
                            const float sh2 = sh * sh;
                            const float w = fmaf(B4.y * sr2, sh2, pa.y);
                            bool in = w <= P.wr_hi;
                            if (in && w > P.wr_lo)
                                in = exact_in_disc(P.rings, c0 + ri, bJw[p], sPx[i], sPy[i], sPz[i], P.cos_r);
                            if (in) {
                                const float x0 = fmaf(-B4.x * sr2, sh2, pa.x);
                                const float y0 = sr2 * sh * ch;
                                const float x = fmaf(A4.z, x0, A4.w * y0);
                                const float y = fmaf(A4.z, y0, -A4.w * x0);
                                const float fu = fmaf(x, P.invh_f, P.cg_f);
                                const float fv = fmaf(y, P.invh_f, P.cg_f);
                                const float flu = fminf(fmaxf(floorf(fu), 0.f), gmax);
                                const float flv = fminf(fmaxf(floorf(fv), 0.f), gmax);
                                const float fx = fmaf(x, P.invh_f, P.cg_f - flu);
                                const float fy = fmaf(y, P.invh_f, P.cg_f - flv);
                                const int cell = (int)flv * nc + (int)flu;
                                float4 ka, kb, kc;
                                ldg_cell(cells + 16 * cell, ka, kb, kc);
                                const float bA = fmaf(fy, fmaf(fx, ka.w, ka.z), fmaf(fx, ka.y, ka.x));
                                const float bB = fmaf(fy, fmaf(fx, kb.w, kb.z), fmaf(fx, kb.y, kb.x));
                                const float bC = fmaf(fy, fmaf(fx, kc.w, kc.z), fmaf(fx, kc.y, kc.x));
                                const float q = rcp_approx(2.f - w);
                                const float mp = fmaf(q, fmaf(x, B4.z, y * B4.w), B4.x);
                                const float e1 = fmaf(-x, mp, B4.z);
                                const float e2 = fmaf(-y, mp, B4.w);
                                const float re = fmaf(e1, e1, -e2 * e2);
                                const float im2 = e1 * e2;
                                wI = bA;
                                wQ = fmaf(bB, re, 2.f * bC * im2) * inv;
                                wU = fmaf(bC, re, -2.f * bB * im2) * inv;
                            }
                        }
                        unsigned short* wh = sW + i * W_LD + 3 * p;
                        unsigned short* wl = sWl + i * W_LD + 3 * p;
                        split16(wI, F16, wh[0], wl[0]);
                        split16(wQ, F16, wh[1], wl[1]);
                        split16(wU, F16, wh[2], wl[2]);
                    }
                    __syncthreads();
                    // 3. tensor cores: D[r][t] += sum_k S[k][r] W[t][k]
                    if (mma_warp) {
                        const int gq = lane >> 2, cq = lane & 3;
                        const int mj = lane >> 3, mi = lane & 7;
#pragma unroll
                        for (int k0 = 0; k0 < KB; k0 += 16) {
                            unsigned afr[2][4];
#pragma unroll
                            for (int mt = 0; mt < 2; ++mt) {
                                const int k = k0 + mi + ((mj >> 1) << 3);
                                const int r = warp * 32 + mt * 16 + ((mj & 1) << 3);
                                ldsm_x4_trans(afr[mt], sSky + k * SKY_LD + r);
                            }
#pragma unroll
                            for (int nt = 0; nt < 2; ++nt) {
                                const int off = (nt * 8 + gq) * W_LD + k0 + 2 * cq;
                                const unsigned h0 = *(const unsigned*)(sW + off);
                                const unsigned h1 = *(const unsigned*)(sW + off + 8);
                                const unsigned l0 = *(const unsigned*)(sWl + off);
                                const unsigned l1 = *(const unsigned*)(sWl + off + 8);
#pragma unroll
                                for (int mt = 0; mt < 2; ++mt) {
                                    mma16816(acc[mt][nt], afr[mt], h0, h1, F16);
                                    mma16816(acc[mt][nt], afr[mt], l0, l1, F16);
                                }
                            }
                        }
                    }
                    __syncthreads();
                }
            }
        }

        // output: D[t0 + t][r] = scale * acc, NaN rows for invalid samples
        if (mma_warp) {
            const int gq = lane >> 2, cq = lane & 3;
            float* out = (float*)P.out;
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int r = warp * 32 + mt * 16 + gq + ((c >> 1) << 3);
                        const int t = nt * 8 + 2 * cq + (c & 1);
                        if (t < ns) {
                            const float v = sValid[t] ? (float)(det.scale * (double)acc[mt][nt][c])
                                                      : __int_as_float(0x7fc00000);
                            out[(t0 + t) * nreal + r] = v;
                        }
                    }
        }
        __syncthreads();
    }
}

cudaError_t launch_mr(const LaunchParams& p, int f16, cudaStream_t s) {
    if (p.total_tiles <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)min(p.total_tiles, (long long)INT_MAX);
    cudaError_t e;
    if (f16) {
        e = cudaFuncSetAttribute(k_mr<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, MR_DYN_SMEM);
        if (e != cudaSuccess) return e;
        k_mr<1><<<grid, MT, MR_DYN_SMEM, s>>>(p);
    } else {
        e = cudaFuncSetAttribute(k_mr<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, MR_DYN_SMEM);
        if (e != cudaSuccess) return e;
        k_mr<0><<<grid, MT, MR_DYN_SMEM, s>>>(p);
    }
    return cudaGetLastError();
}

}  // namespace pisco
