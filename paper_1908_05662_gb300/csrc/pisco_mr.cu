// Multi-realization convolution on the fifth-generation tensor cores (tcgen05).
//
// With R sky realizations S_r sharing one scan and one beam, the TOD is a
// dense contraction (eq. discrete_beam_conv_tensor with the per-pair weights
// factored out):
//     d_r(t) = scale * sum_k sum_{m = I,Q,U} W[t][k][m] S_r[k][m],
//     W[t][k] = (A, (Bq' re + 2 Cu' im2) / sin^2 theta_k, (Cu' re - 2 Bq' im2) / sin^2 theta_k),
// the pair weights of the FP32 kernel.  One CTA (persistent, one per SM) takes
// tiles of 128 consecutive samples of one detector: the M dimension of the
// MMA; the realizations are N (up to 256), so the 128 x R FP32 accumulator
// lives in tensor memory (TMEM) for the whole tile.  The CTA walks the union
// of the tile's 128 discs ring by ring (the ring-ordered disc query of the
// FP32 kernel, Sec. 5.2), in batches of 16 union pixels.  Each ring's run of
// union pixels is cut into blocks of 8 pixels that are consecutive in the
// RING numbering (a run that wraps past longitude 0 is split there), and a
// batch is two such blocks.  The contraction index of a batch is map-major,
// k = 16 m + p (m = I, Q, U; p = pixel of the batch), so that
//   * the realization rows of one block, [8 pixels][I, Q, U][R] in the stack,
//     land by one 4-D TMA tile load as the B operand in the MN-major layout
//     with 64-byte swizzling: atoms of 8 pixels x 32 realizations (rows of
//     64 bytes), ordered [R/32][3 maps][8 pixels][32 realizations], so the
//     copy engine moves 64-byte rows (192 per block at R = 256);
//   * a thread's four weights of one map are one 8-byte row segment of the A
//     operand's K-major core matrices (no swizzling).
//
// Warp roles (640 threads):
//   warp 0      one thread issues the MMAs: per batch, for the three maps,
//               W_hi x S and W_lo x S (kind::f16) into two FP32 accumulators in
//               TMEM (2 x R columns; the epilogue adds them),
//               then tcgen05.commit to the stage's "empty" barrier, and at the
//               tile's end to the accumulator's "full" barrier;
//   warp 1      the scheduler: per batch, the stage's control word and the two
//               TMA loads of the realization rows;
//   warps 2-3   the planner, one tile and up to two windows ahead of the
//               others: per tile the samples' constants (FP64 basis, FP32
//               copies), per chunk of 32 rings the union of the tile's discs
//               (a longitude range per ring, cut into blocks of 8 pixels), per
//               window of 32 batches the pixel table (ring, in-ring index,
//               half-angle of the longitude offset);
//   warps 4-19  the weight producers: thread (sample t, pixel quad q) computes
//               the FP32 weights of 4 pairs (geometry, 64-byte beam cell, the
//               Ludwig-3 rotation), splits each into two 16-bit parts
//               W = W_hi + W_lo (W_lo the rounded remainder) and stores them;
//               at a tile's end they read the accumulator back (tcgen05.ld)
//               and write d[t][r] = scale * D[t][r].
// mbarriers link them: a ring of NST operand stages ("loads": TMA bytes +
// scheduler -> MMA; "full": 16 producer warps -> MMA; "empty": MMA commit ->
// scheduler and producers), two window buffers ("window full": planner ->
// scheduler and producers; "window empty": back), two tile buffers of
// per-sample data ("tile free": producers after their epilogue -> planner)
// and the accumulator ("full": MMA -> producers; "empty": back).  No role
// waits on a CTA-wide barrier between the prologue and the end.
//
// Precision of the disc decision.  The FP32 offsets of a pair come from the
// half-angles of the pixel's and the sample's longitudes relative to the
// tile's reference; their absolute error grows with those angles.  Per chunk
// the planner bounds the resulting relative error of 1 - k . p0 from the
// largest half-angles of the chunk's pixels and the tile's samples; where the
// bound exceeds the kernel's FP64 re-decision band (2e-5 relative; tiles whose
// samples lie far apart, which scans do not produce) the chunk takes the half-angles in FP64
// (stored as FP32 value + remainder) and forms sin(dphi / 2) as a double-FP32
// product difference, so every path reaches the FP64 decision of the oracle.
//
// Every wait on an mbarrier is bounded (about two seconds of SM clock, or a
// test-set limit); on a timeout the kernel records error bit 2, every role
// stops issuing, waits (bounded) for the copies and MMAs it issued, and the
// block releases its TMEM and returns.
// Realization stacks are [Npix][3][R] 16-bit (BF16 or FP16), R a multiple of
// 32 up to 256; the output is FP32 [n][R].

#include "pisco_internal.cuh"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <climits>

namespace pisco {

namespace {

constexpr int MS = 128;                   // samples per tile = MMA M
constexpr int NPW = 16;                   // weight-producer warps
constexpr int NRW = 4;                    // role warps: MMA issuer, scheduler, two planner warps
constexpr int MT = 32 * (NRW + NPW);      // threads
constexpr int MRC = 32;                   // rings per chunk of the union
constexpr int KPIX = 16;                  // union pixels per batch (two blocks of 8)
constexpr int KB = 3 * KPIX;              // contraction length per batch (3 K-steps of 16)
constexpr int NST = 3;                    // pipeline stages (3 leave L1 room for the beam cells)
constexpr int WINB = 32;                  // batches per window of the pixel table
constexpr int WPIX = 16 * WINB;           // pixels per window
constexpr int WBLK = 2 * WINB;            // blocks of 8 pixels per window
constexpr int MAXR = 256;                 // realizations (MMA N) at most
// A operand (weights, K-major): core matrix (t / 8, k / 8), 8 rows of 16 bytes
constexpr int A_LBO = 128;                // bytes between core matrices adjacent in K
constexpr int A_SBO = (KB / 8) * 128;     // bytes between core matrices adjacent in M (768)
constexpr int A_BYTES = MS * KB * 2;      // one 16-bit weight part of a batch (12 KB)
// B operand (realizations, MN-major, 64-byte swizzle): per block [R/32][3 maps][8 pixels][32 realizations]
constexpr int B_ATOM = 8 * 64;            // one swizzle atom: 8 pixels (K) x 32 realizations (N)
constexpr int B_LBO = 3 * B_ATOM;         // bytes between atoms adjacent in N
constexpr unsigned kSwizzle64 = 4u;       // descriptor layout type: 64-byte swizzling
__host__ __device__ constexpr int block_bytes(int nreal) { return 48 * nreal; }  // one block: 8 pixels x 3 maps x R
__host__ __device__ constexpr int stage_bytes(int nreal) { return 2 * A_BYTES + 2 * block_bytes(nreal); }
enum { CT_FIRST = 1, CT_LAST = 2, CT_END = 4 };            // stage control word
enum { W_TFIRST = 1, W_TLAST = 2, W_END = 4 };             // window flags: a tile's first / last window
struct WinMeta {
    int nb;       // batches in the window
    int precise;  // the chunk takes the double-FP32 longitude offsets
    int flags;
    int tb;       // the tile buffer of its per-sample data
};
struct TileMeta {
    long long t0;  // first sample of the tile
    int ns;        // samples in the tile
    int d;         // detector
};
constexpr float kEps32 = 5.9604645e-8f;   // FP32 unit roundoff
constexpr double kBand = 2e-5;            // relative half-width of the FP64 re-decision band (the
                                          // launcher sets the band edges from it)

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(unsigned addr, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    return done != 0;
}

// The same test, letting the thread sleep until the phase completes or about a microsecond
// passes, so that waiting warps leave the issue slots to the others.
__device__ __forceinline__ bool mbar_try_sleep(unsigned addr, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(addr), "r"(parity), "r"(1000u)
        : "memory");
    return done != 0;
}

// Wait for the phase of the given parity.  Gives up when the block's failure
// flag is raised, or after `limit` SM clocks, when it raises the flag and
// records error bit 2.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, volatile int* failed,
                                          long long limit, int* err) {
    const unsigned a = smem_u32(bar);
    if (mbar_try(a, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try_sleep(a, parity)) return true;
        if (*failed) return false;
        if (clock64() - t0 > limit) {
            *failed = 1;
            atomicOr(err, 2);
            return false;
        }
    }
}

// Bounded wait that ignores the failure flag (draining after a failure).
__device__ __forceinline__ bool mbar_drain(unsigned long long* bar, unsigned parity, long long limit) {
    const unsigned a = smem_u32(bar);
    const long long t0 = clock64();
    while (!mbar_try_sleep(a, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// The calling thread arrives on the mbarrier and raises its expected transaction count by `bytes`.
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// The block's failure flag as lane 0 of the warp sees it (a warp-uniform value).
__device__ __forceinline__ bool warp_failed(volatile int* failed) {
    return __shfl_sync(0xffffffffu, *failed, 0) != 0;
}

// The planner's two warps meet at named barrier 1.
__device__ __forceinline__ void plan_sync() { asm volatile("bar.sync 1, 64;" ::: "memory"); }

// mbar_wait by lane 0 of a warp, the outcome broadcast to the warp (whose later reads are
// ordered after lane 0's).
__device__ __forceinline__ bool warp_wait(unsigned long long* bar, unsigned parity, volatile int* failed,
                                          long long limit, int* err) {
    bool ok = true;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, failed, limit, err);
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    __syncwarp();
    return ok;
}

// Shared-memory matrix descriptor of the fifth-generation MMA: start address,
// leading and stride byte offsets, descriptor version 1, layout type (bits
// 61-63).  Without swizzling the leading offset steps between core matrices
// along K and the stride offset along M/N; in a swizzled MN-major layout the
// leading offset steps between atoms along N and the stride offset between
// groups of 8 rows along K.
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr, unsigned lbo, unsigned sbo,
                                                        unsigned layout = 0u) {
    return (unsigned long long)((addr >> 4) & 0x3FFFu) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) |
           ((unsigned long long)layout << 61);
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

// TMA tile load of the 4-D realization tensor's box at (0, pix, 0, 0) into dst
// (512-byte aligned, the period of the 64-byte swizzle, which the copy engine
// and the MMA both take from the shared-memory address); completes `bar`'s
// transaction count by the box's bytes.
__device__ __forceinline__ void tma_tile4(void* dst, const CUtensorMap* map, int pix, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)map), "r"(0), "r"(pix), "r"(0), "r"(0), "r"(smem_u32(bar))
        : "memory");
}

// 64-byte beam cell: one 32-byte and one 16-byte read-only load, cached in L1 (a
// lane's next pixel of the ring often falls in the cell a later sample of its
// warp has just read).
__device__ __forceinline__ void ld_cell(const float* p, float4& a, float4& b, float4& c) {
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
    asm("ld.global.nc.v4.f32 {%0,%1,%2,%3}, [%4];"
        : "=f"(c.x), "=f"(c.y), "=f"(c.z), "=f"(c.w)
        : "l"(p + 8));
}

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Four values as two 16-bit parts each, packed in pairs: hi = rounded value,
// lo = rounded remainder (element i of a pair in the low half).
template <int F16>
__device__ __forceinline__ void split4(const float v[4], uint2& hi, uint2& lo) {
    unsigned h[2], l[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        if (F16) {
            const __half2 a = __floats2half2_rn(v[2 * j], v[2 * j + 1]);
            const float2 af = __half22float2(a);
            const __half2 b = __floats2half2_rn(v[2 * j] - af.x, v[2 * j + 1] - af.y);
            h[j] = *reinterpret_cast<const unsigned*>(&a);
            l[j] = *reinterpret_cast<const unsigned*>(&b);
        } else {
            const __nv_bfloat162 a = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
            const float2 af = __bfloat1622float2(a);
            const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * j] - af.x, v[2 * j + 1] - af.y);
            h[j] = *reinterpret_cast<const unsigned*>(&a);
            l[j] = *reinterpret_cast<const unsigned*>(&b);
        }
    }
    hi = make_uint2(h[0], h[1]);
    lo = make_uint2(l[0], l[1]);
}

}  // namespace

// `rows` is the realization stack seen as a 4-D tensor of 16-bit values: element
// (c, p, m, q) = realization 32 q + c of map m of pixel p, with a box of 32 x 8 x 3 x R/32
// whose shared-memory image [q][m][8 pixels][32], 64-byte swizzled, is one block's atoms.
template <int F16>
__global__ void __launch_bounds__(MT, 1) k_mr(const __grid_constant__ LaunchParams P,
                                              const __grid_constant__ CUtensorMap rows) {
    // per-sample data of two tiles: the planner fills one while the producers use the other
    __shared__ float4 tA[2][MS];  // cos(b/2), sin(b/2), cos psi0, sin psi0   (b = phi0 - phi_c)
    __shared__ float4 tB[2][MS];  // cos theta0, sin theta0, Z_theta, Z_phi
    __shared__ float4 tC[2][MS];  // theta0 as FP32 value + remainder; FP32 remainders of cos(b/2), sin(b/2)
    __shared__ double tP[2][3][MS];  // unit vector p0 (the FP64 decision in the band)
    __shared__ int tValid[2][MS];
    __shared__ TileMeta tMeta[2];
    // the planner's own per-tile and per-chunk data
    __shared__ double pPh[MS];  // longitude of the sample in [0, 2 pi)
    __shared__ float2 pBs[MS];  // b, 1 / (2 sin theta0)
    __shared__ float sRedF[2][4];
    __shared__ int sRedI[2], sPlanOk, sNb, sNblocks, sPrecise;
    __shared__ float sULo[MRC], sUHi[MRC];
    __shared__ int sUFull[MRC];
    __shared__ int sJref[MRC], sFirst[MRC];
    __shared__ float sArefF[MRC], sDphF[MRC], sSr2[MRC], sInv[MRC];
    __shared__ double sArefD[MRC], sDphD[MRC], sThR[MRC];
    __shared__ int sEntJw[2 * MRC], sEntJ[2 * MRC], sEntLen[2 * MRC], sEntPref[2 * MRC + 1];
    // two windows of WINB batches: per pixel and per block of 8 pixels
    __shared__ __align__(16) float wSa[2][WPIX];
    __shared__ __align__(16) float wCa[2][WPIX];
    __shared__ __align__(16) float wSal[2][WPIX];
    __shared__ __align__(16) float wCal[2][WPIX];
    __shared__ int wJw[2][WPIX];
    __shared__ int wNv[2][WBLK], wPix0[2][WBLK], wRing[2][WBLK];
    __shared__ float wThh[2][WBLK], wThl[2][WBLK], wSr2[2][WBLK], wInv[2][WBLK];
    __shared__ WinMeta wMeta[2];
    // stages
    __shared__ int sCtrl[NST];
    __shared__ __align__(8) unsigned long long bLoad[NST], bFull[NST], bEmpty[NST];
    __shared__ __align__(8) unsigned long long bWinFull[2], bWinEmpty[2], bTileFree[2];
    __shared__ __align__(8) unsigned long long bAccFull, bAccEmpty, bFin, bStall;
    __shared__ unsigned tmem_base;
    __shared__ volatile int failed;
    extern __shared__ unsigned char mr_dyn_raw[];
    // operand stages, 1024-byte aligned: stage s = [A_hi | A_lo | B block 0 | B block 1]
    unsigned char* dyn = mr_dyn_raw + ((1024u - (smem_u32(mr_dyn_raw) & 1023u)) & 1023u);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nreal = P.n_real;
    const int sbytes = stage_bytes(nreal);
    const int bbytes = block_bytes(nreal);
    // two accumulators of ncols columns: W_hi x S and W_lo x S (the small second one keeps its
    // rounding errors small; the epilogue adds them)
    const unsigned ncols = nreal <= 32 ? 32u : (nreal <= 64 ? 64u : (nreal <= 128 ? 128u : 256u));
    const long long limit = P.wait_limit > 0 ? P.wait_limit : 4000000000ll;

    // zeroed operand stages (a batch whose block has no pixels reads whatever its B buffer
    // holds, always finite, times zero weights), barriers, accumulator columns
    for (int q = tid; q < NST * sbytes / 16; q += MT) ((uint4*)dyn)[q] = make_uint4(0u, 0u, 0u, 0u);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(2 * ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(bLoad + s, 1);
            mbar_init(bFull + s, NPW);
            mbar_init(bEmpty + s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(bWinFull + b, 1);
            mbar_init(bWinEmpty + b, NPW + 1);
            mbar_init(bTileFree + b, NPW);
        }
        mbar_init(&bAccFull, 1);
        mbar_init(&bAccEmpty, NPW);
        mbar_init(&bFin, 1);
        mbar_init(&bStall, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
        // test hook: wait on a barrier nothing arrives on, before any copy or MMA is issued
        if (P.stall_cycles > 0) mbar_wait(&bStall, 0, &failed, P.stall_cycles, P.err);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_base;

    if (warp == 0) {
        // ------------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const unsigned idesc = instr_desc(F16, nreal, MS);
            unsigned it = 0;
            int tiles = 0;
            bool pending = false;  // MMAs issued whose completion no one has waited for
            while (true) {
                const int s = (int)(it % NST);
                const unsigned ph = (it / NST) & 1u;
                if (!mbar_wait(bLoad + s, ph, &failed, limit, P.err)) break;
                const int ctrl = sCtrl[s];
                if (ctrl & CT_END) break;
                if (!mbar_wait(bFull + s, ph, &failed, limit, P.err)) break;
                const bool first = (ctrl & CT_FIRST) != 0;
                if (first && tiles > 0 && !mbar_wait(&bAccEmpty, (unsigned)((tiles - 1) & 1), &failed, limit, P.err))
                    break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                unsigned char* st = dyn + s * sbytes;
                const unsigned ah = smem_u32(st), al = smem_u32(st + A_BYTES), bb = smem_u32(st + 2 * A_BYTES);
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    const unsigned long long bd = smem_desc(bb + m * B_ATOM, B_LBO, (unsigned)bbytes, kSwizzle64);
                    const unsigned acc = (first && m == 0) ? 0u : 1u;
                    mma_f16(tmem, smem_desc(ah + m * 2 * A_LBO, A_LBO, A_SBO), bd, idesc, acc);
                    mma_f16(tmem + ncols, smem_desc(al + m * 2 * A_LBO, A_LBO, A_SBO), bd, idesc, acc);
                }
                mma_commit(bEmpty + s);
                pending = true;
                if (ctrl & CT_LAST) {
                    mma_commit(&bAccFull);
                    ++tiles;
                    pending = false;  // the producers wait for it before their epilogue
                }
                ++it;
            }
            if (failed && pending) {
                // leave no MMA in flight
                mma_commit(&bFin);
                mbar_drain(&bFin, 0, limit);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------------------------ scheduler
        // per batch of the published windows: the stage's control word and the TMA loads of
        // its two blocks of realization rows
        unsigned w = 0, it = 0;
        bool ok = true;
        while (ok) {
            const int wb = (int)(w & 1u);
            ok = warp_wait(bWinFull + wb, (w >> 1) & 1u, &failed, limit, P.err);
            if (!ok) break;
            const WinMeta m = wMeta[wb];
            if (m.flags & W_END) break;
            for (int fb = 0; fb < m.nb; ++fb) {
                const int s = (int)(it % NST);
                const unsigned u = it / NST;
                if (u > 0 && !warp_wait(bEmpty + s, (u - 1) & 1u, &failed, limit, P.err)) {
                    ok = false;
                    break;
                }
                const int nv0 = wNv[wb][2 * fb], nv1 = wNv[wb][2 * fb + 1];
                if (lane == 0) {
                    sCtrl[s] = ((m.flags & W_TFIRST) && fb == 0 ? CT_FIRST : 0) |
                               ((m.flags & W_TLAST) && fb == m.nb - 1 ? CT_LAST : 0);
                    mbar_expect_tx(bLoad + s, (unsigned)(((nv0 > 0) + (nv1 > 0)) * bbytes));
                }
                __syncwarp();
                if (lane < 2 && (lane == 0 ? nv0 : nv1) > 0)
                    tma_tile4(dyn + s * sbytes + 2 * A_BYTES + lane * bbytes, &rows, wPix0[wb][2 * fb + lane],
                              bLoad + s);
                ++it;
            }
            if (!ok) break;
            __syncwarp();
            if (lane == 0) mbar_arrive(bWinEmpty + wb);
            ++w;
        }
        if (!warp_failed(&failed)) {
            // the end marker
            const int s = (int)(it % NST);
            const unsigned u = it / NST;
            if (u == 0 || warp_wait(bEmpty + s, (u - 1) & 1u, &failed, limit, P.err)) {
                if (lane == 0) {
                    sCtrl[s] = CT_END;
                    mbar_expect_tx(bLoad + s, 0u);
                }
            }
        }
        if (failed && lane == 0) {
            // leave no TMA load in flight: wait (bounded) for the last load of every stage
            for (int s = 0; s < NST; ++s)
                if (it > (unsigned)s) mbar_drain(bLoad + s, ((it - 1 - s) / NST) & 1u, limit);
        }
        __syncwarp();
    } else if (warp < NRW) {
        // ------------------------------------------------------------------ planner (warps 2 and 3)
        // per tile the samples' constants, per chunk of MRC rings the union of the discs and its
        // blocks, per window the pixel table; it runs up to two windows (and one tile) ahead.
        // Its two warps split the samples and the pixels and meet at a named barrier; warp 2
        // takes every wait and every decision and shares it through shared memory.
        const int pl = tid - 64, pq = warp - 2;  // planner thread 0 .. 63, planner warp
        const double wr = P.mr_wr;  // 1 - cos R
        const float wr_hi = P.mr_wr_hi;
        unsigned w = 0;             // windows published
        int tk = 0;                 // tiles planned
        bool ok = true;
        for (long long tile = blockIdx.x; tile < P.total_tiles; tile += gridDim.x, ++tk) {
            const int tb = tk & 1;
            // the producers have finished the tile two back (its epilogue reads tValid and tMeta)
            if (pq == 0) {
                bool okt = !warp_failed(&failed);
                if (okt && tk >= 2) okt = warp_wait(bTileFree + tb, (unsigned)(((tk - 2) >> 1) & 1), &failed, limit, P.err);
                if (lane == 0) sPlanOk = okt ? 1 : 0;
            }
            plan_sync();
            if (!sPlanOk) {
                ok = false;
                break;
            }
            int d = 0;
            while (d + 1 < P.ndet && P.det[d + 1].tile_begin <= tile) ++d;
            const DetEntry& det = P.det[d];
            const long long lt = tile - det.tile_begin;
            const long long t0 = det.begin + lt * MS;
            const int ns = (int)min((long long)MS, det.count - lt * MS);

            // 1. per-sample constants (FP64 basis, FP32 copies); the colatitude range (rounded
            //    outwards to FP32), the largest sin theta0 and the first valid sample
            float tmin = __int_as_float(0x7f800000), tmax = 0.f, s0 = 0.f;
            int first = MS;
#pragma unroll 1
            for (int i = pl; i < MS; i += 64) {
                bool v = i < ns;
                double th = 0.0, ph = 0.0, ps = 0.0;
                if (v) {
                    th = P.theta[t0 + i];
                    ph = P.phi[t0 + i];
                    ps = P.psi[t0 + i];
                    v = isfinite(th) && isfinite(ph) && isfinite(ps) && th >= 0.0 && th <= kPi;
                }
                float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a, c = a;
                double px = 0.0, py = 0.0, pz = 0.0, phw = 0.0;
                float inv2s = 0.f;
                if (v) {
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
                    c.x = (float)th;
                    c.y = (float)(th - (double)c.x);
                    inv2s = 0.5f / b.y;  // +inf at the poles: the whole ring is then taken
                    tmin = fminf(tmin, __double2float_rd(th));
                    tmax = fmaxf(tmax, __double2float_ru(th));
                    s0 = fmaxf(s0, b.y);
                    first = min(first, i);
                }
                tA[tb][i] = a;
                tB[tb][i] = b;
                tC[tb][i] = c;
                tP[tb][0][i] = px;
                tP[tb][1][i] = py;
                tP[tb][2][i] = pz;
                tValid[tb][i] = v ? 1 : 0;
                pPh[i] = phw;
                pBs[i] = make_float2(0.f, inv2s);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                tmin = fminf(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
                tmax = fmaxf(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
                s0 = fmaxf(s0, __shfl_xor_sync(0xffffffffu, s0, o));
                first = min(first, __shfl_xor_sync(0xffffffffu, first, o));
            }
            if (lane == 0) {
                sRedF[pq][0] = tmin;
                sRedF[pq][1] = tmax;
                sRedF[pq][2] = s0;
                sRedI[pq] = first;
            }
            plan_sync();
            tmin = fminf(sRedF[0][0], sRedF[1][0]);
            tmax = fmaxf(sRedF[0][1], sRedF[1][1]);
            s0 = fmaxf(sRedF[0][2], sRedF[1][2]);
            first = min(sRedI[0], sRedI[1]);
            const double phic = first < MS ? pPh[first] : 0.0;
            int rlo = 0, rhi = -1;
            if (first < MS) ring_range((double)tmin, (double)tmax, P.radius, P.nside, &rlo, &rhi);
            //    the longitude offsets b from the tile's reference, as half-angle sines and cosines
            float bmax = 0.f;
#pragma unroll 1
            for (int i = pl; i < MS; i += 64) {
                if (tValid[tb][i]) {
                    double db = pPh[i] - phic;
                    db -= kTwoPi * rint(db / kTwoPi);
                    double sb, cb;
                    sincos(0.5 * db, &sb, &cb);
                    const float cbf = (float)cb, sbf = (float)sb;
                    tA[tb][i].x = cbf;
                    tA[tb][i].y = sbf;
                    tC[tb][i].z = (float)(cb - (double)cbf);
                    tC[tb][i].w = (float)(sb - (double)sbf);
                    pBs[i].x = (float)db;
                    bmax = fmaxf(bmax, fabsf(sbf));
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) bmax = fmaxf(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
            if (lane == 0) sRedF[pq][3] = bmax;
            if (pl == 0) {
                TileMeta tm;
                tm.t0 = t0;
                tm.ns = ns;
                tm.d = d;
                tMeta[tb] = tm;
            }
            plan_sync();
            bmax = fmaxf(sRedF[0][3], sRedF[1][3]);

            bool any_window = false;
            const int nch = rhi >= rlo ? (rhi - rlo) / MRC + 1 : 1;
            for (int ch = 0; ok && ch < nch; ++ch) {
                const int c0 = rlo + ch * MRC;
                const int nr = rhi >= rlo ? min(MRC, rhi - c0 + 1) : 0;
                const bool last_chunk = ch == nch - 1;
                // 2. ring c0 + lane: the union of the discs' longitude ranges (relative to phi_c)
                //    over this warp's half of the samples
                float lo = __int_as_float(0x7f800000), hi = -__int_as_float(0x7f800000);
                int full = 0;
                const RingInfo* R = lane < nr ? &P.rings[c0 + lane] : nullptr;
                if (R) {
                    const double thr = R->theta;
                    const float thh = (float)thr, thl = (float)(thr - (double)thh);
                    const float inv_sr = 1.f / R->s_f;
#pragma unroll 2
                    for (int i = 64 * pq; i < 64 * pq + 64; ++i) {
                        if (!tValid[tb][i]) continue;
                        const float4 c = tC[tb][i];
                        // half the colatitude difference: the FP32 values of nearby colatitudes
                        // subtract exactly, the remainders restore the rest
                        const float h = 0.5f * ((thh - c.x) + (thl - c.y));
                        const float sh = sinf(h);
                        const float av = 2.f * sh * sh;
                        if (av <= wr_hi) {
                            // sin^2 of half the longitude half-width: (wr - av) / (2 sin theta0 sin theta_r)
                            const float2 bs = pBs[i];
                            const float tau = (wr_hi - av) * bs.y * inv_sr;
                            if (!(tau < 0.999f)) {
                                full = 1;
                            } else {
                                const float hw = 2.f * asinf(sqrtf(fmaxf(tau, 0.f)));
                                lo = fminf(lo, bs.x - hw);
                                hi = fmaxf(hi, bs.x + hw);
                            }
                        }
                    }
                }
                if (pq == 1) {
                    sULo[lane] = lo;
                    sUHi[lane] = hi;
                    sUFull[lane] = full;
                }
                plan_sync();
                if (pq == 0) {
                    lo = fminf(lo, sULo[lane]);
                    hi = fmaxf(hi, sUHi[lane]);
                    full |= sUFull[lane];
                    // flag 2 = the whole ring, 1 = the range [lo, hi], 0 = no pixel
                    const int flag = R ? (full ? 2 : (lo <= hi ? 1 : 0)) : 0;
                    // 3. per ring the index range of the union, split where it wraps past
                    //    longitude 0, in blocks of 8; the precision bound of the chunk
                    int cnt = 0, jlo = 0, jref = 0, firstpix = 0, rc = 1;
                    double arefd = 0.0, dphd = 0.0, thr = 0.0;
                    float sr2 = 0.f, inv = 0.f, amax = 0.f, srmax = 0.f;
                    if (R) {
                        firstpix = (int)R->first;
                        rc = R->count;
                        sr2 = 2.f * R->s_f;
                        inv = R->inv_s2_f;
                        dphd = R->dphi;
                        thr = R->theta;
                        jref = (int)rint((phic - R->phi0) / R->dphi);
                        arefd = R->phi0 + (double)jref * R->dphi - phic;
                        if (flag == 2) {
                            cnt = R->count;
                            jlo = jref - R->count / 2;
                            amax = 1.f;
                        } else if (flag == 1) {
                            const double ulo = (phic + (double)lo - R->phi0) / R->dphi;
                            const double uhi = (phic + (double)hi - R->phi0) / R->dphi;
                            const long long a = (long long)floor(ulo) - 1, b = (long long)ceil(uhi) + 1;
                            if (b - a + 1 >= R->count) {
                                cnt = R->count;
                                jlo = jref - R->count / 2;
                                amax = 1.f;
                            } else {
                                cnt = (int)(b - a + 1);
                                jlo = (int)a;
                                // largest half-angle of the run's pixels (one pixel of margin each side)
                                const float ea = fabsf((float)(((double)a - jref) * R->dphi + arefd));
                                const float eb = fabsf((float)(((double)b - jref) * R->dphi + arefd));
                                amax = fminf(1.f, fabsf(sinf(0.5f * fminf(fmaxf(ea, eb), 3.1415927f))) + 1e-3f);
                            }
                        }
                        if (flag != 0) srmax = R->s_f;
                    }
                    int w0 = 0, l1 = 0, l2 = 0;
                    if (cnt > 0) {
                        w0 = jlo % rc;
                        if (w0 < 0) w0 += rc;
                        l1 = min(cnt, rc - w0);
                        l2 = cnt - l1;
                    }
                    const int b0 = (l1 + 7) >> 3, b1 = (l2 + 7) >> 3;
                    sJref[lane] = jref;
                    sFirst[lane] = firstpix;
                    sArefF[lane] = (float)arefd;
                    sArefD[lane] = arefd;
                    sDphF[lane] = (float)dphd;
                    sDphD[lane] = dphd;
                    sThR[lane] = thr;
                    sSr2[lane] = sr2;
                    sInv[lane] = inv;
                    sEntJw[2 * lane] = w0;
                    sEntJ[2 * lane] = jlo;
                    sEntLen[2 * lane] = l1;
                    sEntJw[2 * lane + 1] = 0;
                    sEntJ[2 * lane + 1] = jlo + l1;
                    sEntLen[2 * lane + 1] = l2;
                    int v = b0 + b1;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, v, o);
                        if (lane >= o) v += y;
                    }
                    const int excl = v - b0 - b1;
                    sEntPref[2 * lane] = excl;
                    sEntPref[2 * lane + 1] = excl + b0;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
                        srmax = fmaxf(srmax, __shfl_xor_sync(0xffffffffu, srmax, o));
                    }
                    if (lane == 31) {
                        sEntPref[2 * MRC] = v;
                        sNblocks = v;
                        int nb = (v + 1) >> 1;
                        if (last_chunk && nb == 0) nb = 1;  // every tile ends on a batch flagged last
                        sNb = nb;
                        // bound of the relative error of 1 - k . p0 from the FP32 half-angles
                        // (A = max |sin a/2| of the chunk's pixels, B = max |sin b/2| of the tile's
                        // samples, k0 = 2 sin theta0 sin theta_r):
                        //   beta <= 14 u + 2 u sqrt(k0 / wr) (6.2 A + 4 B + 3.2 A B)
                        // with u the FP32 unit roundoff; the fast path needs beta <= the band
                        const double am = amax, bm = bmax;
                        const double beta = 14.0 * kEps32 + 2.0 * kEps32 * sqrt(2.0 * (double)s0 * (double)srmax / wr) *
                                                                (6.2 * am + 4.0 * bm + 3.2 * am * bm);
                        sPrecise = beta > kBand ? 1 : 0;
                    }
                }
                plan_sync();
                const int nb = sNb, nblocks = sNblocks, precise = sPrecise;

                // the chunk's batches, in windows of WINB batches (2 WINB blocks)
                for (int wb0 = 0; wb0 < nb; wb0 += WINB) {
                    const int wnb = min(WINB, nb - wb0);
                    const int wb = (int)(w & 1u);
                    if (pq == 0) {
                        const bool okw = w < 2 || warp_wait(bWinEmpty + wb, ((w >> 1) - 1) & 1u, &failed, limit, P.err);
                        if (lane == 0) sPlanOk = okw ? 1 : 0;
                    }
                    plan_sync();
                    if (!sPlanOk) {
                        ok = false;
                        break;
                    }
                    // 4. pixel q of the window: block g = 2 wb0 + q / 8, pixel q % 8 of the block
#pragma unroll 1
                    for (int q = pl; q < WPIX; q += 64) {
                        const int g = 2 * wb0 + (q >> 3), pp = q & 7;
                        float sa = 0.f, ca = 1.f, sal = 0.f, cal = 0.f;
                        int jw = 0;
                        if (g < nblocks) {
                            int lo_ = 0, hi_ = 2 * MRC - 1;
                            while (lo_ < hi_) {
                                const int mid = (lo_ + hi_ + 1) >> 1;
                                if (sEntPref[mid] <= g) lo_ = mid;
                                else hi_ = mid - 1;
                            }
                            const int e = lo_, ri = e >> 1;
                            const int bk = g - sEntPref[e];
                            const int off = 8 * bk + pp;
                            jw = sEntJw[e] + off;
                            const int j = sEntJ[e] + off;
                            if (precise) {
                                const double aa = (double)(j - sJref[ri]) * sDphD[ri] + sArefD[ri];
                                double sd, cd;
                                sincos(0.5 * aa, &sd, &cd);
                                sa = (float)sd;
                                ca = (float)cd;
                                sal = (float)(sd - (double)sa);
                                cal = (float)(cd - (double)ca);
                            } else {
                                const float aa = fmaf((float)(j - sJref[ri]), sDphF[ri], sArefF[ri]);
                                sincosf(0.5f * aa, &sa, &ca);
                            }
                            if (pp == 0) {
                                const int wbk = q >> 3;
                                wNv[wb][wbk] = min(8, sEntLen[e] - 8 * bk);
                                wPix0[wb][wbk] = sFirst[ri] + sEntJw[e] + 8 * bk;
                                wRing[wb][wbk] = c0 + ri;
                                const float th_h = (float)sThR[ri];
                                wThh[wb][wbk] = th_h;
                                wThl[wb][wbk] = (float)(sThR[ri] - (double)th_h);
                                wSr2[wb][wbk] = sSr2[ri];
                                wInv[wb][wbk] = sInv[ri];
                            }
                        } else if (pp == 0) {
                            wNv[wb][q >> 3] = 0;
                        }
                        wSa[wb][q] = sa;
                        wCa[wb][q] = ca;
                        wSal[wb][q] = sal;
                        wCal[wb][q] = cal;
                        wJw[wb][q] = jw;
                    }
                    plan_sync();  // the window's entries are written
                    if (pl == 0) {
                        WinMeta m;
                        m.nb = wnb;
                        m.precise = precise;
                        m.flags = (any_window ? 0 : W_TFIRST) | (last_chunk && wb0 + wnb == nb ? W_TLAST : 0);
                        m.tb = tb;
                        wMeta[wb] = m;
                        mbar_arrive(bWinFull + wb);
                    }
                    any_window = true;
                    ++w;
                }
            }
            if (!ok) break;
        }
        if (ok && pq == 0 && !warp_failed(&failed)) {
            // the end marker
            const int wb = (int)(w & 1u);
            if (w < 2 || warp_wait(bWinEmpty + wb, ((w >> 1) - 1) & 1u, &failed, limit, P.err)) {
                if (lane == 0) {
                    wMeta[wb].flags = W_END;
                    mbar_arrive(bWinFull + wb);
                }
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------------ weight producers
        const int pt = tid - 32 * NRW;             // producer thread index
        const int pw = pt >> 5;                    // producer warp 0 .. 15
        // its sample and pixel quad (block my_q >> 1); a warp takes 32 consecutive samples of one
        // quad, whose pairs mostly fall inside (or outside) the disc together.  The quad turns
        // with the batch, so the quads that end a block (more often empty) fall to every warp
        const int my_t = 32 * (pw & 3) + lane;
        const int q0 = pw >> 2;
        const int nc = P.grid_n - 1;
        const float gmax = (float)(P.grid_n - 2);
        const float wlo = P.mr_wr_lo, whi = P.mr_wr_hi;
        unsigned w = 0, it = 0;
        int tile_k = 0;                            // tiles finished (accumulator barrier parity)
        // the sample's constants for the current tile
        float4 A4 = make_float4(0.f, 0.f, 0.f, 0.f), B4 = A4;
        float2 Bl = make_float2(0.f, 0.f);
        float th0h = 0.f, th0l = 0.f;              // the sample's colatitude as FP32 value + remainder
        bool tvalid = false;
        int pa_ring = -1;
        float2 pa = make_float2(0.f, 1e30f);
        const float* __restrict__ cells = nullptr;
        bool ok = true;
        while (ok) {
            const int wb = (int)(w & 1u);
            ok = warp_wait(bWinFull + wb, (w >> 1) & 1u, &failed, limit, P.err);
            if (!ok) break;
            const WinMeta m = wMeta[wb];
            if (m.flags & W_END) break;
            const int tb = m.tb;
            if (m.flags & W_TFIRST) {
                tvalid = tValid[tb][my_t] != 0;
                A4 = tA[tb][my_t];
                B4 = tB[tb][my_t];
                const float4 c = tC[tb][my_t];
                th0h = c.x;
                th0l = c.y;
                Bl = make_float2(c.z, c.w);
                pa_ring = -1;
                cells = (const float*)P.det[tMeta[tb].d].beam;
            }
            const bool prec = m.precise != 0;
            for (int fb = 0; fb < m.nb; ++fb) {
                const int s = (int)(it % NST);
                const unsigned u = it / NST;
                bool okw = true;
                if (u > 0) okw = mbar_wait(bEmpty + s, (u - 1) & 1u, &failed, limit, P.err);
                if (!__all_sync(0xffffffffu, okw)) {
                    ok = false;
                    break;
                }
                const int my_q = (q0 + (int)it) & 3;
                const int b = my_q >> 1, half = 4 * (my_q & 1);
                const int wbk = 2 * fb + b;  // the thread's block in the window
                const int px0 = 8 * wbk + half;  // its first pixel in the window
                const int nv = wNv[wb][wbk];
                float wt[3][4];
#pragma unroll
                for (int mm = 0; mm < 3; ++mm)
#pragma unroll
                    for (int i = 0; i < 4; ++i) wt[mm][i] = 0.f;
                if (nv > half) {  // warp-uniform: the quad has pixels
                    const int rg = wRing[wb][wbk];
                    if (rg != pa_ring) {
                        // half the colatitude difference: the FP32 values of nearby rings
                        // subtract exactly, the remainders restore the rest
                        const float h = 0.5f * ((wThh[wb][wbk] - th0h) + (wThl[wb][wbk] - th0l));
                        float shh, chh;
                        sincosf(h, &shh, &chh);
                        pa = make_float2(2.f * shh * chh, 2.f * shh * shh);
                        pa_ring = rg;
                    }
                    const float sr2 = wSr2[wb][wbk], inv = wInv[wb][wbk];
                    const float4 sa4 = *(const float4*)&wSa[wb][px0];
                    const float4 ca4 = *(const float4*)&wCa[wb][px0];
                    const float sav[4] = {sa4.x, sa4.y, sa4.z, sa4.w};
                    const float cav[4] = {ca4.x, ca4.y, ca4.z, ca4.w};
                    float4 salv4 = make_float4(0.f, 0.f, 0.f, 0.f), calv4 = salv4;
                    if (prec) {
                        salv4 = *(const float4*)&wSal[wb][px0];
                        calv4 = *(const float4*)&wCal[wb][px0];
                    }
                    const float salv[4] = {salv4.x, salv4.y, salv4.z, salv4.w};
                    const float calv[4] = {calv4.x, calv4.y, calv4.z, calv4.w};
                    const float k0 = B4.y * sr2, k1 = -B4.x * sr2;
                    unsigned band = 0u;  // pairs within the FP32 band of the disc boundary
                    // two pairs at a time: both pairs' geometry, then both beam cells in flight
                    // together, then both pairs' weights (a pair no lane has inside skips its load
                    // and weights; lanes outside a pair's disc compute it and keep zero)
#pragma unroll
                    for (int hp = 0; hp < 4; hp += 2) {
                        float wv[2], x[2], y[2], fx[2], fy[2];
                        const float* cp[2];
                        bool in[2];
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            const int i = hp + j;
                            float sh;
                            if (prec) {
                                // sin((a - b)/2) with the products' rounding errors kept
                                const float p1 = sav[i] * A4.x, p2 = cav[i] * A4.y;
                                const float e1 = fmaf(sav[i], A4.x, -p1), e2 = fmaf(cav[i], A4.y, -p2);
                                const float tl = fmaf(salv[i], A4.x, sav[i] * Bl.x) - fmaf(calv[i], A4.y, cav[i] * Bl.y);
                                sh = (p1 - p2) + (tl + (e1 - e2));
                            } else {
                                sh = fmaf(sav[i], A4.x, -cav[i] * A4.y);
                            }
                            const float chv = fmaf(cav[i], A4.x, sav[i] * A4.y);
                            const float sh2 = sh * sh;
                            wv[j] = fmaf(k0, sh2, pa.y);  // 1 - k . p0
                            in[j] = tvalid && half + i < nv && wv[j] <= whi;
                            if (in[j] && wv[j] > wlo) band |= 1u << i;  // settled in FP64 below
                            const float x0 = fmaf(k1, sh2, pa.x);
                            const float y0 = sr2 * sh * chv;
                            x[j] = fmaf(A4.z, x0, A4.w * y0);   // k . theta'0
                            y[j] = fmaf(A4.z, y0, -A4.w * x0);  // k . phi'0
                            // clamped to the grid, so every lane's cell address is valid
                            const float flu = fminf(fmaxf(floorf(fmaf(x[j], P.invh_f, P.cg_f)), 0.f), gmax);
                            const float flv = fminf(fmaxf(floorf(fmaf(y[j], P.invh_f, P.cg_f)), 0.f), gmax);
                            fx[j] = fmaf(x[j], P.invh_f, P.cg_f - flu);
                            fy[j] = fmaf(y[j], P.invh_f, P.cg_f - flv);
                            cp[j] = cells + 16 * ((int)flv * nc + (int)flu);
                        }
                        const bool any0 = __any_sync(0xffffffffu, in[0]), any1 = __any_sync(0xffffffffu, in[1]);
                        float4 ka[2], kb[2], kc[2];
                        if (any0) ld_cell(cp[0], ka[0], kb[0], kc[0]);
                        if (any1) ld_cell(cp[1], ka[1], kb[1], kc[1]);
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            if (!(j == 0 ? any0 : any1)) continue;
                            const int i = hp + j;
                            const float bA = fmaf(fy[j], fmaf(fx[j], ka[j].w, ka[j].z), fmaf(fx[j], ka[j].y, ka[j].x));
                            const float bBq = fmaf(fy[j], fmaf(fx[j], kb[j].w, kb[j].z), fmaf(fx[j], kb[j].y, kb[j].x));
                            const float bC = fmaf(fy[j], fmaf(fx[j], kc[j].w, kc[j].z), fmaf(fx[j], kc[j].y, kc[j].x));
                            const float qr = rcp_approx(2.f - wv[j]);  // 1 / (1 + k . p0)
                            const float mp = fmaf(qr, fmaf(x[j], B4.z, y[j] * B4.w), B4.x);
                            const float e1 = fmaf(-x[j], mp, B4.z);
                            const float e2 = fmaf(-y[j], mp, B4.w);
                            const float re = fmaf(e1, e1, -e2 * e2);
                            const float im2 = e1 * e2;
                            wt[0][i] = in[j] ? bA : 0.f;
                            wt[1][i] = in[j] ? fmaf(bBq, re, 2.f * bC * im2) * inv : 0.f;
                            wt[2][i] = in[j] ? fmaf(bC, re, -2.f * bBq * im2) * inv : 0.f;
                        }
                    }
                    // pairs in the band take the FP64 decision shared with the other paths
                    if (band) {
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            if (((band >> i) & 1u) &&
                                !exact_in_disc(P.rings, rg, wJw[wb][px0 + i], tP[tb][0][my_t], tP[tb][1][my_t],
                                               tP[tb][2][my_t], P.cos_r))
                                wt[0][i] = wt[1][i] = wt[2][i] = 0.f;
                    }
                }
                // the A operand rows: map m, part hi / lo, 8 bytes at core matrix
                // (my_t / 8, 2 m + b), row my_t % 8, bytes 8 (my_q % 2) ..
                unsigned char* st = dyn + s * sbytes;
                const int off = (my_t >> 3) * A_SBO + b * A_LBO + (my_t & 7) * 16 + (my_q & 1) * 8;
#pragma unroll
                for (int mm = 0; mm < 3; ++mm) {
                    uint2 hi, lo;
                    split4<F16>(wt[mm], hi, lo);
                    *(uint2*)(st + off + mm * 2 * A_LBO) = hi;
                    *(uint2*)(st + A_BYTES + off + mm * 2 * A_LBO) = lo;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(bFull + s);
                ++it;
            }
            if (!ok) break;
            __syncwarp();
            if (lane == 0) mbar_arrive(bWinEmpty + wb);
            if (m.flags & W_TLAST) {
                // the epilogue, D read back from TMEM (warp w reads lanes 32 (w % 4) ..)
                ok = warp_wait(&bAccFull, (unsigned)(tile_k & 1), &failed, limit, P.err);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const TileMeta tm = tMeta[tb];
                const int quad = warp & 3, t = 32 * quad + lane;
                const int part = nreal / 4;
                const int cbeg = ((warp - NRW) >> 2) * part;
                float* out = (float*)P.out;
                const float scale_f = (float)P.det[tm.d].scale;
                const bool row = t < tm.ns;
                const bool vrow = row && tValid[tb][t];
                for (int c = cbeg; c < cbeg + part; c += 8) {
                    unsigned r[8], rl[8];
                    const unsigned addr = tmem + ((unsigned)(32 * quad) << 16) + (unsigned)c;
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                                   "=r"(r[6]), "=r"(r[7])
                                 : "r"(addr));
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                 : "=r"(rl[0]), "=r"(rl[1]), "=r"(rl[2]), "=r"(rl[3]), "=r"(rl[4]), "=r"(rl[5]),
                                   "=r"(rl[6]), "=r"(rl[7])
                                 : "r"(addr + ncols));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (row) {
                        float v[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            v[j] = vrow ? scale_f * (__uint_as_float(r[j]) + __uint_as_float(rl[j]))
                                        : __int_as_float(0x7fc00000);
                        float4* o = (float4*)(out + (tm.t0 + t) * nreal + c);
                        o[0] = make_float4(v[0], v[1], v[2], v[3]);
                        o[1] = make_float4(v[4], v[5], v[6], v[7]);
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&bAccEmpty);
                    mbar_arrive(bTileFree + tb);
                }
                ++tile_k;
            }
            ++w;
        }
    }

    // release the accumulator columns
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * ncols) : "memory");
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

cudaError_t launch_mr(const LaunchParams& p0, int f16, cudaStream_t s) {
    if (p0.total_tiles <= 0) return cudaSuccess;
    LaunchParams p = p0;
    const double wr = 2.0 * sin(0.5 * p.radius) * sin(0.5 * p.radius);  // 1 - cos R
    p.mr_wr = wr;
    p.mr_wr_lo = (float)(wr * (1.0 - kBand));
    p.mr_wr_hi = (float)(wr * (1.0 + kBand));
    const EncodeTiled encode = encode_tiled();
    if (!encode || p.npix >= INT_MAX || p.n_real % 32 != 0 || p.n_real < 32 || p.n_real > MAXR)
        return cudaErrorInvalidValue;
    // the stack [Npix][3][R] of 16-bit values as (32 realizations, pixel, map, R / 32 groups): innermost
    // box extent 64 bytes (the 64-byte swizzle span), every box starts at realization 0 of its pixel
    // (16-byte aligned); the shared-memory destinations are 1024-byte aligned
    CUtensorMap rows;
    const cuuint64_t dims[4] = {32, (cuuint64_t)p.npix, 3, (cuuint64_t)(p.n_real / 32)};
    const cuuint64_t strides[3] = {(cuuint64_t)p.n_real * 6, (cuuint64_t)p.n_real * 2, 64};
    const cuuint32_t box[4] = {32, 8, 3, (cuuint32_t)(p.n_real / 32)}, estr[4] = {1, 1, 1, 1};
    if (encode(&rows, CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, const_cast<void*>(p.sky), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    static int n_sm = 0;
    if (n_sm == 0) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess || n_sm <= 0) n_sm = 1;
    }
    // persistent: one CTA per SM (the operand stages take most of its shared memory)
    const unsigned grid = (unsigned)min(p.total_tiles, (long long)n_sm);
    const int smem = NST * stage_bytes(p.n_real) + 1024;
    cudaError_t e;
    if (f16) {
        e = cudaFuncSetAttribute(k_mr<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        k_mr<1><<<grid, MT, smem, s>>>(p, rows);
    } else {
        e = cudaFuncSetAttribute(k_mr<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        k_mr<0><<<grid, MT, smem, s>>>(p, rows);
    }
    return cudaGetLastError();
}

}  // namespace pisco
