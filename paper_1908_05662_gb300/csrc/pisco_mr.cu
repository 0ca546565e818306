// Multi-realization convolution on the fifth-generation tensor cores (tcgen05).
//
// With R sky realizations S_r sharing one scan and one beam, the TOD is a
// dense contraction (eq. discrete_beam_conv_tensor with the per-pair weights
// factored out):
//     d_r(t) = scale * sum_k sum_{m = I,Q,U} W[t][k][m] S_r[k][m],
//     W[t][k] = (A, (Bq' re + 2 Cu' im2) / sin^2 theta_k, (Cu' re - 2 Bq' im2) / sin^2 theta_k),
// the pair weights of the FP32 kernel.  One CTA owns 128 consecutive samples
// of one detector, the M dimension of the MMA; the realizations are N (up to
// 256), so the whole 128 x R accumulator lives in tensor memory (TMEM) for
// the tile.  The CTA traverses the union of the 128 discs ring by ring (the
// ring-ordered disc query of the FP32 kernel) and, per batch of 16 union
// pixels (K = 48: pixel x I, Q, U):
//   1. copies the realization rows [pixel][I,Q,U][R] (16-bit) straight into
//      the B operand's MN-major core-matrix layout (8 k-rows x 16 bytes per
//      core matrix, no swizzle): a core matrix whose 8 rows are consecutive
//      in the stack (pixels of one ring run) comes by TMA: one 3-D tile load
//      per 8-row block fills its core matrices for all realizations (8 rows x
//      R realizations, completing on the buffer's load mbarrier); blocks with
//      a run boundary inside, or in the batch's tail, are 16-byte asynchronous
//      copies and zeros;
//   2. computes the 128 x 16 pair weights in FP32 (zero outside a sample's
//      disc) and splits each into two 16-bit parts, W = W_hi + W_lo
//      (W_lo the rounded remainder), written in the A operand's K-major
//      core-matrix layout;
//   3. one thread issues tcgen05.mma (kind::f16, FP32 accumulate in TMEM) for
//      W_hi and W_lo over the three K-steps of 16, then tcgen05.commit to the
//      batch buffer's mbarrier.
// Operand buffers are double-buffered: the MMAs of one batch run while the
// TMA loads and the threads' weights fill the next; a buffer is rewritten only
// after the mbarrier of the MMAs that read it has completed, and its MMAs are
// issued only after its load mbarrier has.  At the end of the tile
// the sixteen warps read the accumulator rows back with tcgen05.ld (warp w
// sees TMEM lanes 32 (w % 4) ..; warps w, w + 4, w + 8, w + 12 take a quarter
// of the realizations each) and store d[t][r] = scale * D[t][r].  Every wait on an mbarrier is
// bounded; on a timeout the kernel records error bit 2, drains what it
// issued and releases its TMEM.
// Realization stacks are [Npix][3][R] 16-bit (BF16 or FP16), R a multiple of
// 32 up to 256; the output is FP32 [n][R].

#include "pisco_internal.cuh"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <climits>

namespace pisco {

namespace {

constexpr int MT = 512;              // threads
constexpr int MS = 128;              // samples per tile = MMA M
constexpr int MRC = 32;              // rings per chunk of the union disc
constexpr int KPIX = 16;             // union pixels per batch
constexpr int KB = 3 * KPIX;         // contraction length per batch (3 K-steps of 16)
constexpr int MAXR = 256;            // realizations (MMA N) at most
// A operand (weights, K-major): core matrix (t / 8, k / 8), 8 rows of 16 bytes
constexpr int A_LBO = 128;                 // bytes between core matrices adjacent in K
constexpr int A_SBO = (KB / 8) * 128;      // bytes between core matrices adjacent in M (768)
constexpr int A_BYTES = MS * KB * 2;       // one 16-bit weight part of a batch (12 KB)
// B operand (realizations, MN-major): core matrix (k / 8, r / 8), 8 k-rows of 16 bytes
constexpr int B_SBO = 128;                 // bytes between core matrices adjacent in N
constexpr int B_BYTES = KB * MAXR * 2;     // a batch's realization rows (24 KB at R = 256)
// dynamic shared memory: [2 buffers] x (B, A_hi, A_lo)
constexpr int BUF_BYTES = B_BYTES + 2 * A_BYTES;
constexpr int MR_DYN_SMEM = 2 * BUF_BYTES + 1024;  // + alignment slack

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

// Shared-memory matrix descriptor of the fifth-generation MMA: start address,
// leading (K-direction) and stride (M/N-direction) byte offsets between core
// matrices, descriptor version 1, no swizzle.
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (unsigned long long)((addr >> 4) & 0x3FFFu) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulate, A and B both BF16 (or
// both FP16), A K-major, B MN-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ unsigned instr_desc(int f16, int n, int m) {
    const unsigned fmt = f16 ? 0u : 1u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | (0u << 15) | (1u << 16) | ((unsigned)(n >> 3) << 17) |
           ((unsigned)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(unsigned dtmem, unsigned long long ad, unsigned long long bd, unsigned idesc,
                                        unsigned accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(unsigned long long* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// The calling thread arrives on the mbarrier and raises its expected transaction count by `bytes`.
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// TMA tile load of a 3-D tensor's box at coordinates (0, y, 0) into dst, which must
// be 128-byte aligned; completes `bar`'s transaction count by the box's bytes.
__device__ __forceinline__ void tma_tile3(void* dst, const CUtensorMap* map, int y, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)map), "r"(0), "r"(y), "r"(0), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// Pixel data of union pixel f of the current chunk.
__device__ __forceinline__ void batch_pixel(int b0, int tid, int nr, int total, const int* sPref, const int* sJlo,
                                            const int* sRc, const int* sJref, const float* sDph, const float* sAref,
                                            const int* sFirst, int* bRi, int* bJw, int* bOk, float* bSa, float* bCa,
                                            long long* bPix, unsigned* bFlag) {
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
    const long long pix = ok ? (long long)sFirst[ri] + jw : 0;
    bRi[tid] = ri;
    bJw[tid] = jw;
    bOk[tid] = ok;
    bSa[tid] = sa;
    bCa[tid] = ca;
    bPix[tid] = pix;
    // core matrix kb holds rows k = 8 kb .. 8 kb + 7 (k = 3 p + m): one TMA tile when its
    // pixels are valid and consecutive in the stack (rows 3 pix + m then run on)
    const long long nxt = __shfl_down_sync(0xffffu, pix, 1, KPIX);
    const unsigned okm = __ballot_sync(0xffffu, ok);
    const unsigned conm = __ballot_sync(0xffffu, ok && tid < KPIX - 1 && nxt == pix + 1);
    if (tid == 0) {
        unsigned fl = 0;
        for (int kb = 0; kb < KB / 8; ++kb) {
            const int pa = (8 * kb) / 3, pz = (8 * kb + 7) / 3;
            const unsigned mo = ((2u << pz) - 1u) & ~((1u << pa) - 1u);  // pixels pa .. pz
            const unsigned mc = ((1u << pz) - 1u) & ~((1u << pa) - 1u);  // steps pa -> pa + 1 .. pz - 1 -> pz
            if ((okm & mo) == mo && (conm & mc) == mc) fl |= 1u << kb;
        }
        *bFlag = fl;
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

// `rows` is the realization stack seen as a 3-D tensor of 16-bit values: element
// (c, y, q) = realization 8 q + c of row y = 3 p + m (map m of pixel p), with a box of
// 8 x 8 x R/8 whose shared-memory image [q][8 rows][8] is the B operand's core matrices
// (k-block, q) at 128-byte strides.
template <int F16>
__global__ void __launch_bounds__(MT, 1) k_mr(const __grid_constant__ LaunchParams P,
                                              const __grid_constant__ CUtensorMap rows) {
    __shared__ double sTh[MS], sPh[MS], sPx[MS], sPy[MS], sPz[MS];
    __shared__ float4 sA[MS], sB[MS];
    __shared__ float sBf[MS];
    __shared__ int sValid[MS];
    __shared__ int sAny, sRlo, sRhi;
    __shared__ double sPhiC;
    __shared__ float2 sPA[MRC * MS];
    __shared__ float sLo[MRC], sHi[MRC];
    __shared__ int sFlag[MRC], sJlo[MRC], sJref[MRC], sFirst[MRC], sRc[MRC], sPref[MRC + 1];
    __shared__ float sAref[MRC], sSr[MRC], sInv[MRC], sDph[MRC];
    // pixel data of the current and the next batch
    __shared__ int bRi[2][KPIX], bJw[2][KPIX], bOk[2][KPIX];
    __shared__ long long bPix[2][KPIX];
    __shared__ unsigned bFlag[2];  // core matrices of the batch loaded by TMA (bit kb)
    __shared__ float bSa[2][KPIX], bCa[2][KPIX];
    __shared__ __align__(8) unsigned long long mbar[2];  // MMAs of buffer b done
    __shared__ __align__(8) unsigned long long lbar[2];  // TMA loads into buffer b done
    __shared__ unsigned tmem_base;
    __shared__ int failed;
    extern __shared__ unsigned char mr_dyn_raw[];
    // operand buffers, 1024-byte aligned: buffer b = [B | A_hi | A_lo]
    unsigned char* dyn = mr_dyn_raw + ((1024u - (smem_u32(mr_dyn_raw) & 1023u)) & 1023u);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned short* __restrict__ sky16 = (const unsigned short*)P.sky;
    const int nreal = P.n_real;
    const int nc = P.grid_n - 1;
    const float gmax = (float)(P.grid_n - 2);
    const int b_lbo = (nreal / 8) * 128;  // B: bytes between core matrices adjacent in K
    const unsigned ncols = nreal <= 32 ? 32u : (nreal <= 64 ? 64u : (nreal <= 128 ? 128u : 256u));
    const unsigned idesc = instr_desc(F16, nreal, MS);

    // zeroed operand buffers, the two mbarriers, the accumulator columns
    for (int q = tid; q < 2 * BUF_BYTES / 16; q += MT) ((uint4*)dyn)[q] = make_uint4(0u, 0u, 0u, 0u);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(mbar + 0);
        mbar_init(mbar + 1);
        mbar_init(lbar + 0);
        mbar_init(lbar + 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_base;
    unsigned phase[2] = {0u, 0u};
    unsigned lphase[2] = {0u, 0u};  // load mbarrier parities (thread 0 waits on them)
    bool lfail = false;             // thread 0: a wait for loads timed out (shared flag set before a barrier)
    bool pend[2] = {false, false};

    // wait for the MMAs that read buffer b (all threads); false after a timeout
    auto drain = [&](int b) -> bool {
        if (!pend[b]) return true;
        pend[b] = false;
        const bool ok = mbar_wait(mbar + b, phase[b]);
        phase[b] ^= 1u;
        return ok;
    };

    for (long long tile = blockIdx.x; tile < P.total_tiles && !failed; tile += gridDim.x) {
        int d = 0;
        while (d + 1 < P.ndet && P.det[d + 1].tile_begin <= tile) ++d;
        const DetEntry& det = P.det[d];
        const long long lt = tile - det.tile_begin;
        const long long t0 = det.begin + lt * MS;
        const int ns = (int)min((long long)MS, det.count - lt * MS);
        const float* __restrict__ cells = (const float*)det.beam;

        // 1. per-sample constants (FP64), relative to the first valid sample's longitude
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
            int first = -1;
            double tmin = 1e9, tmax = -1e9;
            for (int i = 0; i < MS; ++i)
                if (sValid[i]) {
                    if (first < 0) first = i;
                    tmin = fmin(tmin, sTh[i]);
                    tmax = fmax(tmax, sTh[i]);
                }
            sAny = first >= 0;
            sPhiC = first >= 0 ? sPh[first] : 0.0;
            int ra = 0, rb = -1;
            if (first >= 0) ring_range(tmin, tmax, P.radius, P.nside, &ra, &rb);
            sRlo = ra;
            sRhi = rb;
        }
        __syncthreads();
        if (tid < MS && sValid[tid]) {
            double db = sPh[tid] - sPhiC;
            db -= kTwoPi * rint(db / kTwoPi);
            double sb, cb;
            sincos(0.5 * db, &sb, &cb);
            sA[tid].x = (float)cb;
            sA[tid].y = (float)sb;
            sBf[tid] = (float)db;
        }
        __syncthreads();

        int batch = 0;  // batches issued in this tile (the first one overwrites the accumulator)
        const int rlo = sRlo, rhi = sRhi;
        for (int c0 = rlo; c0 <= rhi && !failed; c0 += MRC) {
            const int nr = min(MRC, rhi - c0 + 1);
            // 2. per (ring, sample): sin(dtheta), 1 - cos(dtheta); union of the discs' longitude ranges.
            //    Thread (ring tid / 16, samples tid % 16 + 16 j).
            {
                const int ri = tid >> 4, sub = tid & 15;
                float lo = __int_as_float(0x7f800000), hi = -__int_as_float(0x7f800000);
                int full = 0;
                const bool ring_ok = ri < nr;
                const RingInfo* R = ring_ok ? &P.rings[c0 + ri] : nullptr;
#pragma unroll 4
                for (int j = 0; j < MS / 16; ++j) {
                    const int i = sub + 16 * j;
                    float2 pa = make_float2(0.f, 1e30f);
                    if (ring_ok && sValid[i]) {
                        const float h = (float)(0.5 * (R->theta - sTh[i]));
                        float sh, ch;
                        sincosf(h, &sh, &ch);
                        const float av = 2.f * sh * sh;
                        pa = make_float2(2.f * sh * ch, av);
                        if (av <= P.wr_hi) {
                            const float b2 = 2.f * sB[i].y * R->s_f;
                            const float tau = (P.wr_hi - av) / b2;
                            if (!(b2 > 0.f) || !(tau < 0.999f)) {
                                full = 1;
                            } else {
                                const float hw = 2.f * asinf(sqrtf(fmaxf(tau, 0.f)));
                                lo = fminf(lo, sBf[i] - hw);
                                hi = fmaxf(hi, sBf[i] + hw);
                            }
                        }
                    }
                    sPA[ri * MS + i] = pa;
                }
#pragma unroll
                for (int off = 8; off > 0; off >>= 1) {
                    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, off, 16));
                    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, off, 16));
                    full |= __shfl_xor_sync(0xffffffffu, full, off, 16);
                }
                if (sub == 0) {
                    sLo[ri] = lo;
                    sHi[ri] = hi;
                    sFlag[ri] = ring_ok ? (full ? 2 : (lo <= hi ? 1 : 0)) : 0;
                }
            }
            __syncthreads();
            // 3. per ring: index range of the union, and its prefix over the chunk (one warp)
            if (warp == 0) {
                int cnt = 0, jlo = 0, jref = 0, first = 0, rc = 1;
                float aref = 0.f, sr = 0.f, inv = 0.f, dph = 0.f;
                if (lane < nr) {
                    const RingInfo& R = P.rings[c0 + lane];
                    const int flag = sFlag[lane];
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
                        const double ulo = (phic + (double)sLo[lane] - R.phi0) / R.dphi;
                        const double uhi = (phic + (double)sHi[lane] - R.phi0) / R.dphi;
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
                sJlo[lane] = jlo;
                sJref[lane] = jref;
                sFirst[lane] = first;
                sRc[lane] = rc;
                sAref[lane] = aref;
                sSr[lane] = sr;
                sInv[lane] = inv;
                sDph[lane] = dph;
                int v = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, v, o);
                    if (lane >= o) v += y;
                }
                sPref[lane + 1] = v;
                if (lane == 0) sPref[0] = 0;
            }
            __syncthreads();

            const int total = sPref[nr];
            // the first batch's pixel data; each batch then prepares the next one's
            if (tid < KPIX && total > 0)
                batch_pixel(0, tid, nr, total, sPref, sJlo, sRc, sJref, sDph, sAref, sFirst, bRi[0], bJw[0], bOk[0],
                            bSa[0], bCa[0], bPix[0], bFlag + 0);
            __syncthreads();
            int fb = 0;  // batch within the chunk
            for (int f0 = 0; f0 < total && !failed; f0 += KPIX, ++batch, ++fb) {
                const int buf = batch & 1, pb = fb & 1;
                unsigned char* bB = dyn + buf * BUF_BYTES;
                unsigned char* bAh = bB + B_BYTES;
                unsigned char* bAl = bAh + A_BYTES;
                // the MMAs of two batches ago read this buffer
                if (!drain(buf) || lfail) atomicOr(&failed, 1);
                // 4. realization rows into the B operand, core matrix (kb, q) = rows k = 8 kb .. 8 kb + 7
                //    (k = 3 p + m) x realizations 8 q .. 8 q + 7: by TMA (warp 0) when its rows are
                //    consecutive in the stack, else as 16-byte chunks (all threads) or zeros
                {
                    const int qn = nreal / 8;
                    const unsigned fl = bFlag[pb];
                    if (warp == 0) {
                        if (lane == 0) mbar_expect_tx(lbar + buf, (unsigned)(__popc(fl) * qn * 128));
                        __syncwarp();
                        const int kb = lane, k0 = 8 * lane;
                        if (kb < KB / 8 && ((fl >> kb) & 1u))
                            tma_tile3(bB + kb * b_lbo, &rows, (int)(bPix[pb][k0 / 3] * 3 + k0 % 3), lbar + buf);
                    }
                    if (fl != (1u << (KB / 8)) - 1u) {
                        for (int c = tid; c < KB * qn; c += MT) {
                            const int k = c / qn, q = c % qn;
                            if ((fl >> (k >> 3)) & 1u) continue;
                            const int p = k / 3, m = k % 3;
                            unsigned char* dst = bB + (k >> 3) * b_lbo + q * B_SBO + (k & 7) * 16;
                            if (bOk[pb][p]) cp_async16(dst, sky16 + (bPix[pb][p] * 3 + m) * (long long)nreal + 8 * q);
                            else *(uint4*)dst = make_uint4(0u, 0u, 0u, 0u);
                        }
                    }
                    asm volatile("cp.async.commit_group;" ::: "memory");
                }
                // 5. pair weights, thread (pixel tid % 16, samples tid / 16 + 32 j), into the A operand
                {
                    const int p = tid & (KPIX - 1), tb = tid >> 4;
                    const bool pok = bOk[pb][p];
                    const int ri = bRi[pb][p];
                    const float sr2 = 2.f * sSr[ri], inv = sInv[ri];
                    const float sa = bSa[pb][p], ca = bCa[pb][p];
#pragma unroll
                    for (int j = 0; j < MS / 32; ++j) {
                        const int t = tb + 32 * j;
                        float wI = 0.f, wQ = 0.f, wU = 0.f;
                        PairGeom g;
                        if (pok && sValid[t] &&
                            pair_geometry(P, sA[t], sB[t], sPA[ri * MS + t], sa, ca, sr2, gmax, g) &&
                            (g.w <= P.wr_lo ||
                             exact_in_disc(P.rings, c0 + ri, bJw[pb][p], sPx[t], sPy[t], sPz[t], P.cos_r))) {
                            const float4 B4 = sB[t];
                            const float* cp = cells + 16 * ((int)g.flv * nc + (int)g.flu);
                            const float4 ka = __ldg((const float4*)cp), kb = __ldg((const float4*)(cp + 4));
                            const float4 kc = __ldg((const float4*)(cp + 8));
                            const float bA = fmaf(g.fy, fmaf(g.fx, ka.w, ka.z), fmaf(g.fx, ka.y, ka.x));
                            const float bBq = fmaf(g.fy, fmaf(g.fx, kb.w, kb.z), fmaf(g.fx, kb.y, kb.x));
                            const float bC = fmaf(g.fy, fmaf(g.fx, kc.w, kc.z), fmaf(g.fx, kc.y, kc.x));
                            const float qr = rcp_approx(2.f - g.w);
                            const float mp = fmaf(qr, fmaf(g.x, B4.z, g.y * B4.w), B4.x);
                            const float e1 = fmaf(-g.x, mp, B4.z);
                            const float e2 = fmaf(-g.y, mp, B4.w);
                            const float re = fmaf(e1, e1, -e2 * e2);
                            const float im2 = e1 * e2;
                            wI = bA;
                            wQ = fmaf(bBq, re, 2.f * bC * im2) * inv;
                            wU = fmaf(bC, re, -2.f * bBq * im2) * inv;
                        }
                        const float wv[3] = {wI, wQ, wU};
#pragma unroll
                        for (int m = 0; m < 3; ++m) {
                            const int k = 3 * p + m;
                            const int off = (t >> 3) * A_SBO + (k >> 3) * A_LBO + (t & 7) * 16 + (k & 7) * 2;
                            unsigned short h, l;
                            split16(wv[m], F16, h, l);
                            *(unsigned short*)(bAh + off) = h;
                            *(unsigned short*)(bAl + off) = l;
                        }
                    }
                }
                if (tid < KPIX && f0 + KPIX < total)
                    batch_pixel(f0 + KPIX, tid, nr, total, sPref, sJlo, sRc, sJref, sDph, sAref, sFirst, bRi[pb ^ 1],
                                bJw[pb ^ 1], bOk[pb ^ 1], bSa[pb ^ 1], bCa[pb ^ 1], bPix[pb ^ 1], bFlag + (pb ^ 1));
                asm volatile("cp.async.wait_group 0;" ::: "memory");
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncthreads();
                if (failed) {
                    // leave no TMA load in flight: thread 0 waits (bounded) for this batch's loads
                    if (tid == 0) mbar_wait(lbar + buf, lphase[buf]);
                    break;
                }
                // 6. one thread waits for the batch's loads and issues its MMAs:
                //    D[t][r] += sum_k (W_hi + W_lo)[t][k] S[k][r]; the commit is made even when the
                //    loads timed out (no MMAs then), so the MMA mbarrier phases stay in step
                if (tid == 0) {
                    const bool loaded = mbar_wait(lbar + buf, lphase[buf]);
                    lphase[buf] ^= 1u;
                    if (!loaded) {
                        atomicOr(P.err, 2);
                        lfail = true;
                    } else {
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                        for (int ks = 0; ks < KB / 16; ++ks) {
                            const unsigned long long bd = smem_desc(smem_u32(bB + ks * 2 * b_lbo), b_lbo, B_SBO);
                            const unsigned long long ah = smem_desc(smem_u32(bAh + ks * 2 * A_LBO), A_LBO, A_SBO);
                            const unsigned long long al = smem_desc(smem_u32(bAl + ks * 2 * A_LBO), A_LBO, A_SBO);
                            mma_f16(tmem, ah, bd, idesc, (batch > 0 || ks > 0) ? 1u : 0u);
                            mma_f16(tmem, al, bd, idesc, 1u);
                        }
                    }
                    mma_commit(mbar + buf);
                }
                pend[buf] = true;
            }
        }

        // 7. epilogue: wait for every MMA of the tile, read D back, d = scale * D (NaN for invalid samples)
        const bool ok0 = drain(0), ok1 = drain(1);
        if (!ok0 || !ok1 || lfail) {
            atomicOr(P.err, 2);
            failed = 1;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        __syncthreads();
        if (failed) break;
        {
            // warp w reads TMEM lanes 32 (w % 4) .. (its samples) and a quarter of the realizations
            const int t = (warp & 3) * 32 + lane;
            const int half = nreal / 4;
            const int cbeg = (warp >> 2) * half;
            float* out = (float*)P.out;
            const bool valid_row = t < ns;
            const bool computed = batch > 0;
            for (int c = cbeg; c < cbeg + half; c += 8) {
                unsigned r[8];
                const unsigned addr = tmem + ((unsigned)((warp & 3) * 32) << 16) + (unsigned)c;
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                               "=r"(r[7])
                             : "r"(addr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (valid_row) {
                    float v[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        v[j] = !sValid[t] ? __int_as_float(0x7fc00000)
                                          : (computed ? (float)(det.scale * (double)__uint_as_float(r[j])) : 0.f);
                    float4* o = (float4*)(out + (t0 + t) * nreal + c);
                    o[0] = make_float4(v[0], v[1], v[2], v[3]);
                    o[1] = make_float4(v[4], v[5], v[6], v[7]);
                }
            }
        }
        // the next tile's first MMA overwrites the accumulator: all reads done first
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }

    // release the accumulator columns (nothing is left in flight: every commit was waited for,
    // or the wait timed out and the error flag is set)
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

namespace {

// cuTensorMapEncodeTiled, looked up once through the runtime (no link to the driver library).
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_tiled() {
    static EncodeTiled fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return (EncodeTiled)f;
    }();
    return fn;
}

}  // namespace

cudaError_t launch_mr(const LaunchParams& p, int f16, cudaStream_t s) {
    if (p.total_tiles <= 0) return cudaSuccess;
    // the stack [3 Npix][R] of 16-bit values as (8 realizations, rows, R / 8 groups): innermost
    // box extent 16 bytes, every box starts at column 0 of its group (16-byte aligned)
    const EncodeTiled encode = encode_tiled();
    if (!encode || 3 * p.npix >= INT_MAX || p.n_real % 8 != 0 || p.n_real > 256) return cudaErrorInvalidValue;
    CUtensorMap rows;
    const cuuint64_t dims[3] = {8, (cuuint64_t)(3 * p.npix), (cuuint64_t)(p.n_real / 8)};
    const cuuint64_t strides[2] = {(cuuint64_t)p.n_real * 2, 16};
    const cuuint32_t box[3] = {8, 8, (cuuint32_t)(p.n_real / 8)}, estr[3] = {1, 1, 1};
    if (encode(&rows, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<void*>(p.sky), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const unsigned grid = (unsigned)min(p.total_tiles, (long long)INT_MAX);
    cudaError_t e;
    if (f16) {
        e = cudaFuncSetAttribute(k_mr<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, MR_DYN_SMEM);
        if (e != cudaSuccess) return e;
        k_mr<1><<<grid, MT, MR_DYN_SMEM, s>>>(p, rows);
    } else {
        e = cudaFuncSetAttribute(k_mr<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, MR_DYN_SMEM);
        if (e != cudaSuccess) return e;
        k_mr<0><<<grid, MT, MR_DYN_SMEM, s>>>(p, rows);
    }
    return cudaGetLastError();
}

}  // namespace pisco
