// Multi-realization convolution on the tensor cores.
//
// With R sky realizations S_r sharing one scan and one beam, the TOD is a
// dense contraction (eq. discrete_beam_conv_tensor with the per-pair weights
// factored out):
//     d_r(t) = scale * sum_k sum_{m = I,Q,U} W[t][k][m] S_r[k][m],
//     W[t][k] = (A, (Bq' re + 2 Cu' im2) / sin^2 theta_k, (Cu' re - 2 Bq' im2) / sin^2 theta_k),
// the pair weights of the FP32 kernel.  One CTA owns 16 consecutive samples
// (the tile and union disc of the FP32 kernel).  For each super-batch of 64
// union pixels it
//   1. streams the realizations, [pixel][I,Q,U][R] in 16-bit, as four slabs of
//      16 pixels through two shared-memory buffers (rows k = 3 pixel + m,
//      realizations contiguous) with bulk copies (TMA) completing on one
//      mbarrier per buffer, each slab issued as soon as its buffer is free;
//   2. computes the 64 x 16 pair weights in FP32 (zero outside a sample's
//      disc; four samples per thread, while the first slabs stream) and
//      splits each into two 16-bit parts, W = W_hi + W_lo with
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
constexpr int KPIX = 16;        // union pixels per batch
constexpr int KB = 3 * KPIX;    // contraction length per slab
constexpr int SB_SLABS = 4;     // slabs per super-batch
constexpr int SBPIX = SB_SLABS * KPIX;  // union pixels per super-batch (weights computed together)
constexpr int SKY_LD = 264;     // 16-bit elements per staged realization row (256 + 8: ldmatrix rows on distinct banks)
constexpr int W_LD = KB + 8;    // 16-bit elements per weight row (conflict-free B-fragment loads)
constexpr int MR_DYN_SMEM = (2 * KB * SKY_LD + 2 * SB_SLABS * MS * W_LD) * 2;

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

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

// Wait for the mbarrier phase with the given parity; gives up after about two
// seconds of SM clock and returns false (the caller records the error).
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    const unsigned addr = smem_u32(bar);
    const long long t0 = clock64();
    while (true) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > 4000000000ll) return false;
    }
}

// Pixel data of union pixel f of the current chunk (thread tid of a batch).
__device__ __forceinline__ void batch_pixel(int b0, int tid, int nr, int total, const int* sPref, const int* sJlo,
                                            const int* sRc, const int* sJref, const float* sDph, const float* sAref,
                                            const int* sFirst, int* bRi, int* bJw, int* bOk, float* bSa, float* bCa,
                                            long long* bPix) {
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
    bPix[tid] = ok ? (long long)sFirst[ri] + jw : 0;
}

// Warp 0 copies the realization rows [pixel][I,Q,U][R] of a batch into slab
// buffer `buf` with bulk copies (TMA) that complete on the buffer's mbarrier:
// lane 0 arms it with the byte count, lane p < KPIX copies pixel p's 3 rows.
__device__ __forceinline__ void issue_slab(int lane, const int* ok, const long long* pix,
                                           const unsigned short* sky16, int nreal, unsigned short* sSky,
                                           unsigned long long* mbar, int buf) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const unsigned row_bytes = (unsigned)nreal * 2u;
    int nvalid = 0;
#pragma unroll
    for (int p = 0; p < KPIX; ++p) nvalid += ok[p];
    const unsigned bar = smem_u32(mbar + buf);
    if (lane == 0) {
        unsigned long long state;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
                     : "=l"(state)
                     : "r"(bar), "r"((unsigned)(3 * nvalid) * row_bytes)
                     : "memory");
    }
    __syncwarp();
    if (lane < KPIX && ok[lane]) {
        for (int m = 0; m < 3; ++m) {
            const unsigned short* src = sky16 + (pix[lane] * 3 + m) * nreal;
            unsigned short* dst = sSky + ((size_t)buf * KB + 3 * lane + m) * SKY_LD;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                ::"r"(smem_u32(dst)), "l"(src), "r"(row_bytes), "r"(bar)
                : "memory");
        }
    }
}

// In-frame geometry of one (pixel, sample) pair, as in the FP32 kernel: returns
// false when the pair is certainly outside the disc (1 - k.p0 above the band).
struct PairGeom {
    float w, x, y, fx, fy, flu, flv;
};

__device__ __forceinline__ bool pair_geometry(const LaunchParams& P, const float4 A4, const float4 B4, const float2 pa,
                                              float sa, float ca, float sr2, float gmax, PairGeom& g) {
    const float sh = fmaf(sa, A4.x, -ca * A4.y);
    const float ch = fmaf(ca, A4.x, sa * A4.y);
    const float sh2 = sh * sh;
    g.w = fmaf(B4.y * sr2, sh2, pa.y);
    if (g.w > P.wr_hi) return false;
    const float x0 = fmaf(-B4.x * sr2, sh2, pa.x);
    const float y0 = sr2 * sh * ch;
    g.x = fmaf(A4.z, x0, A4.w * y0);
    g.y = fmaf(A4.z, y0, -A4.w * x0);
    const float fu = fmaf(g.x, P.invh_f, P.cg_f);
    const float fv = fmaf(g.y, P.invh_f, P.cg_f);
    g.flu = fminf(fmaxf(floorf(fu), 0.f), gmax);
    g.flv = fminf(fmaxf(floorf(fv), 0.f), gmax);
    g.fx = fmaf(g.x, P.invh_f, P.cg_f - g.flu);
    g.fy = fmaf(g.y, P.invh_f, P.cg_f - g.flv);
    return true;
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
    // pixel data of the current super-batch
    __shared__ int bRi[SBPIX], bJw[SBPIX], bOk[SBPIX];
    __shared__ long long bPix[SBPIX];
    __shared__ float bSa[SBPIX], bCa[SBPIX];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ int failed;
    extern __shared__ __align__(16) unsigned short mr_dyn[];
    unsigned short* sSky = mr_dyn;                  // [2][KB][SKY_LD] realization slabs
    unsigned short* sW = mr_dyn + 2 * KB * SKY_LD;  // [SB_SLABS][MS][W_LD] high parts
    unsigned short* sWl = sW + SB_SLABS * MS * W_LD;  // [SB_SLABS][MS][W_LD] low parts

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned short* __restrict__ sky16 = (const unsigned short*)P.sky;
    const int nreal = P.n_real;
    const int nc = P.grid_n - 1;
    const float gmax = (float)(P.grid_n - 2);
    const bool mma_warp = warp * 32 < nreal;

    // Both slab buffers start zeroed (a row a batch leaves unwritten then holds
    // finite stale values, multiplied by zero weights); then the mbarriers.
    for (int q = tid; q < 2 * KB * SKY_LD / 8; q += MT) ((uint4*)sSky)[q] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        mbar_init(mbar + 0);
        mbar_init(mbar + 1);
        failed = 0;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    unsigned phase[2] = {0u, 0u};

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
                for (int s0 = 0; s0 < total; s0 += SBPIX) {
                    const int nslab = min(SB_SLABS, (total - s0 + KPIX - 1) / KPIX);
                    // pixel data of the super-batch (one pixel per thread)
                    if (tid < SBPIX)
                        batch_pixel(s0, tid, nr, total, sPref, sJlo, sRc, sJref, sDph, sAref, sFirst, bRi, bJw, bOk,
                                    bSa, bCa, bPix);
                    __syncthreads();
                    // the first two slabs start streaming while the weights are computed
                    if (warp == 0) {
                        issue_slab(lane, bOk, bPix, sky16, nreal, sSky, mbar, 0);
                        if (nslab > 1) issue_slab(lane, bOk + KPIX, bPix + KPIX, sky16, nreal, sSky, mbar, 1);
                    }
                    // 2. pair weights: pixel p = tid % 64 for samples tid / 64 + 4 j, j = 0..3.
                    //    Pass 1 finds the four beam cells and prefetches them into L1 so their
                    //    latencies overlap; pass 2 recomputes the (cheap) geometry and reads them.
                    {
                        const int p = tid & (SBPIX - 1), i0 = tid / SBPIX;
                        const int q = p / KPIX, pl = p % KPIX;
                        const bool pok = bOk[p];
                        const int ri = bRi[p];
                        const float sr2 = 2.f * sSr[ri], inv = sInv[ri];
                        const float sa = bSa[p], ca = bCa[p];
                        int cellv[MS / 4];
#pragma unroll
                        for (int j = 0; j < MS / 4; ++j) {
                            const int i = i0 + 4 * j;
                            cellv[j] = -1;
                            if (pok && i >= gs && i < ge) {
                                PairGeom g;
                                if (pair_geometry(P, sA[i], sB[i], sPA[ri * MS + i], sa, ca, sr2, gmax, g) &&
                                    (g.w <= P.wr_lo ||
                                     exact_in_disc(P.rings, c0 + ri, bJw[p], sPx[i], sPy[i], sPz[i], P.cos_r))) {
                                    cellv[j] = (int)g.flv * nc + (int)g.flu;
                                    asm volatile("prefetch.global.L1 [%0];" ::"l"(cells + 16 * cellv[j]));
                                }
                            }
                        }
#pragma unroll
                        for (int j = 0; j < MS / 4; ++j) {
                            const int i = i0 + 4 * j;
                            float wI = 0.f, wQ = 0.f, wU = 0.f;
                            if (cellv[j] >= 0) {
                                const float4 B4 = sB[i];
                                PairGeom g;
                                pair_geometry(P, sA[i], B4, sPA[ri * MS + i], sa, ca, sr2, gmax, g);
                                const float* cp = cells + 16 * cellv[j];
                                const float4 ka = __ldg((const float4*)cp), kb = __ldg((const float4*)(cp + 4));
                                const float4 kc = __ldg((const float4*)(cp + 8));
                                const float bA = fmaf(g.fy, fmaf(g.fx, ka.w, ka.z), fmaf(g.fx, ka.y, ka.x));
                                const float bB = fmaf(g.fy, fmaf(g.fx, kb.w, kb.z), fmaf(g.fx, kb.y, kb.x));
                                const float bC = fmaf(g.fy, fmaf(g.fx, kc.w, kc.z), fmaf(g.fx, kc.y, kc.x));
                                const float qr = rcp_approx(2.f - g.w);
                                const float mp = fmaf(qr, fmaf(g.x, B4.z, g.y * B4.w), B4.x);
                                const float e1 = fmaf(-g.x, mp, B4.z);
                                const float e2 = fmaf(-g.y, mp, B4.w);
                                const float re = fmaf(e1, e1, -e2 * e2);
                                const float im2 = e1 * e2;
                                wI = bA;
                                wQ = fmaf(bB, re, 2.f * bC * im2) * inv;
                                wU = fmaf(bC, re, -2.f * bB * im2) * inv;
                            }
                            const int off = (q * MS + i) * W_LD + 3 * pl;
                            split16(wI, F16, sW[off], sWl[off]);
                            split16(wQ, F16, sW[off + 1], sWl[off + 1]);
                            split16(wU, F16, sW[off + 2], sWl[off + 2]);
                        }
                    }
                    __syncthreads();
                    // 3. stream the slabs through the two buffers:
                    //    D[r][t] += sum_k S[k][r] (W_hi[t][k] + W_lo[t][k])
                    for (int q = 0; q < nslab; ++q) {
                        const int buf = q & 1;
                        if (!mbar_wait(mbar + buf, phase[buf])) {
                            atomicOr(P.err, 2);
                            failed = 1;
                        }
                        phase[buf] ^= 1u;
                        if (mma_warp && !failed) {
                            const unsigned short* slab = sSky + buf * KB * SKY_LD;
                            const unsigned short* wh = sW + q * MS * W_LD;
                            const unsigned short* wl = sWl + q * MS * W_LD;
                            const int gq = lane >> 2, cq = lane & 3;
                            const int mj = lane >> 3, mi = lane & 7;
#pragma unroll
                            for (int k0 = 0; k0 < KB; k0 += 16) {
                                unsigned afr[2][4];
#pragma unroll
                                for (int mt = 0; mt < 2; ++mt) {
                                    const int k = k0 + mi + ((mj >> 1) << 3);
                                    const int r = warp * 32 + mt * 16 + ((mj & 1) << 3);
                                    ldsm_x4_trans(afr[mt], slab + k * SKY_LD + r);
                                }
#pragma unroll
                                for (int nt = 0; nt < 2; ++nt) {
                                    const int off = (nt * 8 + gq) * W_LD + k0 + 2 * cq;
                                    const unsigned h0 = *(const unsigned*)(wh + off);
                                    const unsigned h1 = *(const unsigned*)(wh + off + 8);
                                    const unsigned l0 = *(const unsigned*)(wl + off);
                                    const unsigned l1 = *(const unsigned*)(wl + off + 8);
#pragma unroll
                                    for (int mt = 0; mt < 2; ++mt) {
                                        mma16816(acc[mt][nt], afr[mt], h0, h1, F16);
                                        mma16816(acc[mt][nt], afr[mt], l0, l1, F16);
                                    }
                                }
                            }
                        }
                        __syncthreads();
                        if (failed) {
                            // a copy never arrived: wait (bounded) for the other buffer's copy, then stop
                            if (q + 1 < nslab) mbar_wait(mbar + (buf ^ 1), phase[buf ^ 1]);
                            return;
                        }
                        // the buffer just read is free: stream slab q + 2 into it
                        if (q + 2 < nslab && warp == 0)
                            issue_slab(lane, bOk + (q + 2) * KPIX, bPix + (q + 2) * KPIX, sky16, nreal, sSky, mbar, buf);
                    }
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
