/*
 * pisco.h -- C ABI of the GB300 pixel-space convolver (PISCO, arXiv:1908.05662).
 *
 * One TOD sample is the pixelised convolution of Sec. 4.2
 * (eq. discrete_beam_conv_tensor):
 *
 *   d(theta0, phi0, psi0) = (s/2) (Omega_pix / Omega~) sum_k [ (1+eps) row_T(k) + (1-eps) row_Q(k) ]
 *   row_T = B_TT I' + B_QT Q' + B_UT U',   row_Q = B_TQ I' + B_QQ Q' + B_UQ U',
 *   (I', Q', U') = Lambda(-chi_k) (I_k, Q_k, U_k)       (eq. lambda_operator)
 *
 * over the HEALPix RING pixels k whose centre lies within `radius` of the
 * pointing (k . p0 >= cos radius), with the beamsor elements re-pixelised
 * bilinearly at the pixel's antenna coordinates (Sec. 2, Appendix A) and
 * chi_k the Ludwig-3 co-polarisation angle (Appendix A).  D Lambda(chi) =
 * (s/2)[(1+eps), (1-eps), 0, 0] (eq. M_pol), so only six beamsor elements
 * enter; the library folds them into three maps per detector at plan time.
 *
 * Conventions shared by every call:
 *  - Pointers are plain device pointers unless a parameter says "host".
 *    The caller owns every pointer it passes; the plan copies sky and beams
 *    at creation, so the caller may free them afterwards.  Outputs are
 *    caller-allocated.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Device work
 *    is stream-ordered and asynchronous; calls return after enqueueing.
 *    Calls that share one plan must be ordered on one stream (they share the
 *    plan's read-only tables only, but pisco_convolve_host also uses
 *    plan-owned staging buffers).
 *  - Argument errors are detected before any launch and return
 *    PISCO_EINVAL with a message in pisco_last_error().  CUDA errors return
 *    PISCO_ECUDA.
 *  - Pointing angles are float64 radians: theta (colatitude) in [0, pi],
 *    phi any finite value, psi any finite value.  A sample whose angles are
 *    non-finite or whose theta lies outside [0, pi] produces NaN (and -1 in
 *    pisco_disc_count) without touching memory for it.
 *  - Sky maps: [3][12 nside^2], rows I, Q, U in RING order, contiguous.
 *  - Beam grids: [n_det][6][grid_n][grid_n] float32, maps ordered
 *    TT, QT, UT, TQ, QQ, UQ (element B_XY: X = input Stokes column,
 *    Y = output row of eq. beamsor).  Element [j][i] is the beamsor at
 *    tangent-plane coordinates u_i = sin(R)(2i/(grid_n-1) - 1) along theta'0
 *    and v_j (same formula) along phi'0 (orthographic coordinates
 *    u = k . theta'0, v = k . phi'0; eq. antenna_base_vectors).
 */
#ifndef PISCO_H
#define PISCO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pisco_status {
    PISCO_OK = 0,
    PISCO_EINVAL = 1,        /* bad argument; nothing was enqueued */
    PISCO_ENOMEM = 2,        /* device or host allocation failed */
    PISCO_ECUDA = 3,         /* a CUDA runtime call failed */
    PISCO_ETIMEOUT = 4,      /* a bounded device wait gave up (reported by pisco_sync_status) */
    PISCO_EUNSUPPORTED = 5,  /* valid request this build does not implement */
    PISCO_EDEVICE = 6        /* a kernel recorded an invariant violation (reserved) */
} pisco_status;

/* Arithmetic of a plan (pisco_options.precision).  tile_samples and
 * pixels_per_thread change only the work split of the FP32 kernel (results
 * differ at FP32 rounding level), never the arithmetic. */
enum {
    PISCO_FP64_PLAIN = 0, /* FP64 throughout, one CTA per sample: the plain reference path */
    PISCO_FP32 = 1,       /* FP32 arithmetic, FP64 only where offsets would cancel */
    PISCO_BF16_MR = 2,    /* n_real sky realizations in BF16; FP32 weights split into two BF16 parts (hi + lo);
                             fifth-generation tensor cores (tcgen05), FP32 accumulate in tensor memory;
                             realization rows gathered into shared memory by TMA; 128-sample tiles.
                             Realization values must be finite: every pixel of a tile's disc union
                             enters the contraction, with weight zero outside a sample's disc */
    PISCO_FP16_MR = 3     /* the same with FP16 realizations and weight parts */
};

/* Element type of caller arrays (sky_dtype). */
enum { PISCO_DTYPE_F32 = 0, PISCO_DTYPE_F64 = 1, PISCO_DTYPE_BF16 = 2, PISCO_DTYPE_F16 = 3 };

/* One detector (Sec. 3 eq. copol_bolo, Sec. 4.1 eq. M_pol): polarisation
 * angle zeta (radians) from theta'0, polarisation efficiency 1 - eps,
 * responsivity s. */
typedef struct pisco_detector {
    double zeta;
    double eps;
    double s_resp;
} pisco_detector;

typedef struct pisco_options {
    int precision;     /* PISCO_FP64_PLAIN or PISCO_FP32 */
    int tile_samples;       /* FP32 path: consecutive samples sharing one disc traversal: 8, 16 or 32 (0 = 16) */
    int pixels_per_thread;  /* FP32 path: consecutive ring pixels per thread: 1 or 2 (0 = 1) */
    int beam_fetch;         /* FP32 path: PISCO_FETCH_CELLS, _TEXTURE, _PACKED or _SHARED (0 = cells) */
    int n_real;             /* PISCO_*_MR plans: realizations, a multiple of 32 in [32, 256] */
} pisco_options;

/* How the FP32 kernel reads the beam (pisco_options.beam_fetch):
 *  PISCO_FETCH_CELLS    64-byte cells of FP32 bilinear coefficients through L1/L2;
 *  PISCO_FETCH_TEXTURE  2 x 2 texel gathers of the folded node maps (same arithmetic);
 *  PISCO_FETCH_PACKED   32-byte cells: per map the FP32 value at the cell's first
 *                       node and the three bilinear slopes as int16 on a per-cell
 *                       power-of-two scale (each slope within 2^-15 of the largest
 *                       slope of its cell and map).  Half the bytes per pair of
 *                       the FP32 cells; the plan fails with PISCO_EINVAL when the
 *                       grid's slopes lie outside about 2^-80 .. 2^140;
 *  PISCO_FETCH_SHARED   the folded node grid (FP32 A, Bq', Cu' per node, 16 bytes)
 *                       staged in shared memory once per block of a persistent
 *                       launch (Sec. 5.2 keeps the beam in fast on-chip memory);
 *                       grid_n <= 108, else PISCO_EINVAL; same arithmetic as the
 *                       cells (bilinear in FP32 from the four nodes). */
enum { PISCO_FETCH_TEXTURE = 1, PISCO_FETCH_CELLS = 2, PISCO_FETCH_PACKED = 3, PISCO_FETCH_SHARED = 4 };

typedef struct pisco_plan pisco_plan;  /* opaque, owned by the library */

/*
 * pisco_plan_create -- build the device tables for one sky and n_det beams.
 *
 * Sec. 5.1: PISCO receives the sky maps, the beamsor and the focal plane
 * (zeta per detector); Sec. 5.2's beam interpolation grid is assembled here.
 *   nside        HEALPix resolution, 1 <= nside <= 8192 (<= 7723 for PISCO_*_MR plans).
 *   radius_rad   disc cut-off rho_max (Sec. 5.3, Table 1) = beam grid radius,
 *                0 < radius < pi/2.
 *   sky          device, [3][12 nside^2] of sky_dtype (I, Q, U; V is zero, Sec. 6.2);
 *                for PISCO_BF16_MR / PISCO_FP16_MR plans a realization stack
 *                [12 nside^2][3][n_real] of PISCO_DTYPE_BF16 / PISCO_DTYPE_F16
 *                (realizations contiguous per pixel and Stokes parameter).
 *   n_det, dets  host array of n_det >= 1 detectors.
 *   grid_n       nodes per grid side, 2 <= grid_n <= 4096.
 *   beam_grids   device float32 [n_det][6][grid_n][grid_n].
 *   omega_tilde  host [n_det] normalisations Omega~ = int B_TT dOmega (Sec. 3), or
 *                NULL to compute each from B_TT by the trapezoid rule over the
 *                grid with area element du dv / sqrt(1 - u^2 - v^2).
 *   opt          NULL for defaults (PISCO_FP32, 16 samples per tile).
 *   stream       stream for the set-up kernels; the call synchronises it once.
 * On success *out holds a new plan.  On failure *out is NULL and
 * pisco_last_error(NULL) describes the error.
 */
pisco_status pisco_plan_create(pisco_plan** out, int nside, double radius_rad,
                               const void* sky, int sky_dtype,
                               int n_det, const pisco_detector* dets,
                               int grid_n, const float* beam_grids,
                               const double* omega_tilde,
                               const pisco_options* opt, void* stream);

/*
 * pisco_beam_grids_from_healpix -- beamsor maps given as HEALPix RING maps (the
 * paper's representation: Sec. 5.1, beam NSIDE 4x the sky's in Sec. 5.3 and
 * Sec. 6) resampled onto the tangent-plane grid that pisco_plan_create takes.
 * The beam centre is the maps' north pole and (rho, sigma) are their (theta,
 * phi); node (u_i, v_j), u_i = sin(R)(2i/(grid_n-1) - 1), takes the value at
 * rho = asin(sqrt(u^2 + v^2)), sigma = atan2(v, u) by ring-wise bilinear
 * interpolation (the paper interpolates without naming a scheme, Sec. 4.2):
 * linear in phi along a ring, linear in theta between rings, quadratic in
 * theta from rings 1 and 2 above ring 1.  Nodes with u^2 + v^2 > 1 are zero.
 *   nside_b     HEALPix resolution of the beam maps, 1 <= nside_b <= 8192.
 *   n_maps      number of maps (6 per detector, ordered as beam_grids).
 *   maps        device float32 [n_maps][12 nside_b^2], RING order.
 *   radius_rad  grid radius R, 0 < R < pi/2 (the plan's radius).
 *   grid_n      nodes per grid side, 2 <= grid_n <= 4096.
 *   grids       device float32 [n_maps][grid_n][grid_n]; overwritten.
 * FP64 arithmetic, one thread per node, no allocation; errors as for
 * pisco_plan_create (pisco_last_error(NULL)).
 */
pisco_status pisco_beam_grids_from_healpix(int nside_b, int n_maps, const float* maps, double radius_rad,
                                           int grid_n, float* grids, void* stream);

/*
 * Map-making (Sec. 5.1: TOD go on to "a map-making code"; Sec. 6 makes maps
 * from PISCO TOD of pixels observed at their centres at three angles).  The
 * paper names no map-maker; these calls are the binned (naive) one:
 * per-pixel least squares with the pointing matrix of a delta beam at the
 * boresight, a_t = s/2 [(1 + eps), (1 - eps) cos 2 chi_t, (1 - eps) sin 2 chi_t]
 * (eq. M_pol), chi_t = psi_t + zeta (Appendix A at rho = 0), pixel = the RING
 * pixel containing (theta_t, phi_t) (Gorski et al. 2005).
 *
 * pisco_ang2pix -- RING pixel of each direction.
 *   theta, phi  device float64 [n]; pix device int64 [n], -1 for non-finite
 *               angles or theta outside [0, pi].
 *
 * pisco_map_accumulate -- adds one detector's samples to the per-pixel normal
 * equations acc, device float64 [10][12 nside^2] laid out as
 *   acc[0..5]  sum a a^T   (II, IQ, IU, QQ, QU, UU)
 *   acc[6..8]  sum a d     (I, Q, U)
 *   acc[9]     hits.
 *   det         host pointer to the detector (zeta, eps, s_resp).
 *   tod         device [n] of tod_dtype (PISCO_DTYPE_F32 or PISCO_DTYPE_F64).
 *   accumulate  0: acc is zeroed first; otherwise the samples are added (call
 *               once per detector to bin a focal plane).
 * Samples with non-finite angles or data, or theta outside [0, pi], are
 * skipped.  FP64 atomic adds: the summation order, hence the last bits, vary
 * from run to run.
 *
 * pisco_map_solve -- maps, device float64 [3][12 nside^2] (I, Q, U): per
 * pixel, m = (sum a a^T)^-1 sum a d where hits >= 3 and the reciprocal
 * condition number lambda_min / lambda_max >= rcond_min (in [0, 1]); NaN
 * elsewhere.  Hits are acc[9].
 *
 * All three take 1 <= nside <= 8192 and report argument errors through
 * pisco_last_error(NULL).
 */
pisco_status pisco_ang2pix(int nside, int64_t n, const double* theta, const double* phi, int64_t* pix,
                           void* stream);
pisco_status pisco_map_accumulate(int nside, int64_t n, const double* theta, const double* phi,
                                  const double* psi, const pisco_detector* det, const void* tod,
                                  int tod_dtype, double* acc, int accumulate, void* stream);
pisco_status pisco_map_solve(int nside, const double* acc, double rcond_min, double* maps, void* stream);

/* Free a plan and its device memory (synchronises the device first).  NULL is a no-op. */
void pisco_plan_destroy(pisco_plan* plan);

/* Message of the last error on `plan`, or of the last failed create when plan is NULL. */
const char* pisco_last_error(const pisco_plan* plan);

/* Host copy of Omega~ and of the TOD scale (s/2) Omega_pix / Omega~ of detector det. */
pisco_status pisco_plan_omega(const pisco_plan* plan, int det, double* omega_tilde, double* scale);

/*
 * pisco_convolve -- TOD of detector `det` for n pointings (Sec. 4.2, eq.
 * discrete_beam_conv_tensor; Sec. 5.2's per-pointing loop L1 over the disc loop L2).
 *   theta, phi, psi  device float64 [n].
 *   tod              device [n]: float32 for a PISCO_FP32 plan, float64 for
 *                    PISCO_FP64_PLAIN; float32 [n][n_real] for PISCO_*_MR plans
 *                    (one TOD per realization, the dense contraction
 *                    d_r(t) = sum_k W_t(k) . S_r(k) run on the tensor cores);
 *                    overwritten.  Multi-realization plans support
 *                    pisco_convolve and pisco_convolve_batched only
 *                    (PISCO_EUNSUPPORTED otherwise).
 * n = 0 is a valid no-op.  Long scans may be split into consecutive calls on
 * sub-ranges (pointer offsets); results do not depend on the split.
 */
pisco_status pisco_convolve(pisco_plan* plan, int det, int64_t n,
                            const double* theta, const double* phi, const double* psi,
                            void* tod, void* stream);

/*
 * pisco_convolve_batched -- a focal plane in one launch (Sec. 5.1: several
 * detectors in one pointing stream).  Detector d (0 <= d < n_det <= plan's
 * n_det) owns samples offsets[d] .. offsets[d+1]-1 of the concatenated
 * arrays; offsets is a host array of n_det + 1 non-decreasing values with
 * offsets[0] = 0.  tod is concatenated the same way.  Plain plans run one
 * launch per detector.
 */
pisco_status pisco_convolve_batched(pisco_plan* plan, int n_det, const int64_t* offsets,
                                    const double* theta, const double* phi, const double* psi,
                                    void* tod, void* stream);

/*
 * pisco_convolve_psb -- TODs of detectors that share detector `det`'s beam,
 * pointing, eps and s and differ only in their polarisation angle, from one
 * traversal of the discs (Sec. 3 eq. copol_bolo: a PSB is a pair at zeta and
 * zeta - 90 deg; Sec. 5.3's benchmark convolves two such detectors with the
 * same beams).  zeta enters d_t only as e^{2 i zeta} on the polarised part of
 * the folded beam, so the kernel accumulates the intensity part and the
 * complex polarised part once and writes, for every k,
 *   tod[k][t] = pisco_convolve's d_t for a detector with zeta = zeta[k].
 *   zeta    host [n_zeta] polarisation angles in radians (1 <= n_zeta <= 8);
 *           they replace detector det's own zeta.
 *   tod     device float32 [n_zeta][n] (row k = angle k); overwritten, NaN for
 *           invalid pointings as in pisco_convolve.
 * FP32 plans, any beam fetch but PISCO_FETCH_TEXTURE (PISCO_EUNSUPPORTED otherwise); the
 * pass runs the FP32 kernel with three accumulators per sample, so its
 * results agree with n_zeta pisco_convolve calls to FP32 rounding, not
 * bit for bit.  The paper computes each detector separately; this pass is an
 * evaluation of the same sums that shares their geometry.
 */
pisco_status pisco_convolve_psb(pisco_plan* plan, int det, int64_t n,
                                const double* theta, const double* phi, const double* psi,
                                int n_zeta, const double* zeta, void* tod, void* stream);

/*
 * pisco_adjoint -- transpose of pisco_convolve with respect to the sky:
 * maps[m][k] (+)= sum_t tod[t] * d d_t / d S^m_k for m = I, Q, U.
 *   tod    device [n], float32 (FP32 plan) or float64 (plain plan).
 *   maps   device [3][12 nside^2] of the same type; zeroed first unless
 *          accumulate != 0.  Uses atomic adds: the summation order, hence
 *          the last bits, vary from run to run.
 */
pisco_status pisco_adjoint(pisco_plan* plan, int det, int64_t n,
                           const double* theta, const double* phi, const double* psi,
                           const void* tod, void* maps, int accumulate, void* stream);

/*
 * pisco_beam_grid_adjoint -- transpose of pisco_convolve with respect to the
 * six beam grids, Omega~ held fixed:
 *   grad_grids[e][j][i] (+)= sum_t tod[t] * d d_t / d beam_grids[det][e][j][i].
 * Every beam element enters d_t linearly through the bilinear weights of the
 * cell a pixel falls in (Sec. 4.2) and through the folding of the six maps
 * (eqs. M_pol, lambda_operator); this is that linear map transposed.
 *   tod         device [n], float32 (FP32 plan) or float64 (plain plan).
 *   grad_grids  device [6][grid_n][grid_n] of the same type, maps ordered as
 *               beam_grids; overwritten unless accumulate != 0.
 * Uses a plan-owned scratch buffer (allocated on the first call) of
 * 12 (grid_n - 1)^2 floats (FP32 plans: per cell, the gradients of the three
 * folded maps' bilinear coefficients) or 3 grid_n^2 doubles (plain plans),
 * and atomic adds (the last bits vary from run to run).  The
 * dependence of Omega~ on B_TT is added by pisco_omega_adjoint.
 */
pisco_status pisco_beam_grid_adjoint(pisco_plan* plan, int det, int64_t n,
                                     const double* theta, const double* phi, const double* psi,
                                     const void* tod, void* grad_grids, int accumulate, void* stream);

/*
 * pisco_adjoint_sky_beam -- pisco_adjoint and pisco_beam_grid_adjoint in one
 * traversal of the discs (the two transposes of the same linear map share
 * every pair's geometry and beam value): maps (+)= A_S^T tod and
 * grad_grids (+)= A_G^T tod, with the layouts, the accumulate flag and the
 * scratch of those two calls.  FP32 plans only (PISCO_EUNSUPPORTED
 * otherwise); tod, maps and grad_grids float32.
 */
pisco_status pisco_adjoint_sky_beam(pisco_plan* plan, int det, int64_t n,
                                    const double* theta, const double* phi, const double* psi,
                                    const void* tod, void* maps, void* grad_grids, int accumulate,
                                    void* stream);

/*
 * pisco_beam_grid_adjoint_static -- pisco_beam_grid_adjoint that allocates
 * nothing.  The paper has no counterpart: this entry point exists for
 * callers that may not allocate device memory when they call (a real-time
 * loop with a fixed memory budget, an allocator that forbids cudaMalloc after
 * start-up).  Same arguments, layout and result as pisco_beam_grid_adjoint;
 * the folded-gradient scratch is a static device array of 6 MiB inside the
 * library instead of a plan buffer, so the plan's grid_n must be <= 512
 * (PISCO_EINVAL otherwise).  The first call on a device looks the array's
 * address up (once per device; make it before any stream capture).  Every
 * call uses the same array and clears it first: calls whose kernels overlap
 * on the GPU race.  No cudaMalloc, cudaFree or allocating library call.
 */
pisco_status pisco_beam_grid_adjoint_static(pisco_plan* plan, int det, int64_t n,
                                            const double* theta, const double* phi, const double* psi,
                                            const void* tod, void* grad_grids, int accumulate, void* stream);

/*
 * pisco_omega_adjoint -- the Omega~ term of the beam gradient.  Omega~ =
 * int B_TT dOmega (Sec. 3) scales every sample by 1/Omega~, so with the
 * forward TOD d (from pisco_convolve) and its gradient y:
 *   grad_grids[TT][j][i] += -(sum_t y_t d_t / Omega~) * dOmega~/dB_TT[j][i],
 * dOmega~/dB_TT being the trapezoid weights of the grid rule.  Skip it when
 * the plan was given omega_tilde explicitly.  tod, tod_grad: device [n];
 * grad_grids: device [6][grid_n][grid_n]; float32 or float64 as the plan.
 */
pisco_status pisco_omega_adjoint(pisco_plan* plan, int det, int64_t n, const void* tod,
                                 const void* tod_grad, void* grad_grids, void* stream);

/*
 * pisco_update_beams -- replace the beams of an existing plan (same n_det and
 * grid_n; detector parameters unchanged): refolds the grids and recomputes
 * Omega~ (or takes omega_tilde, host [n_det], when not NULL).  Synchronises
 * `stream` once.
 */
pisco_status pisco_update_beams(pisco_plan* plan, const float* beam_grids, const double* omega_tilde,
                                void* stream);

/*
 * pisco_disc_count -- number of sky pixels in the disc of each pointing
 * (the pixel list of Sec. 5.2, cut at rho_max as in Table 1), decided by
 * the plan's own path (the FP32 path filters in FP32 and settles pixels
 * within 2e-6 of the boundary in FP64).  counts: device int32 [n]; -1 for
 * an invalid sample.
 */
pisco_status pisco_disc_count(pisco_plan* plan, int64_t n, const double* theta,
                              const double* phi, int32_t* counts, void* stream);

/*
 * pisco_convolve_host -- pisco_convolve with HOST buffers: copies the
 * pointing to the device in chunks, convolves and copies the TOD back,
 * overlapping the copies of one chunk with the kernel of the previous one
 * on two internal streams.  Synchronous: returns when h_tod is written.
 * Pinned host memory gives asynchronous copies; pageable memory works.
 */
pisco_status pisco_convolve_host(pisco_plan* plan, int det, int64_t n,
                                 const double* h_theta, const double* h_phi,
                                 const double* h_psi, void* h_tod);

/*
 * pisco_plan_autotune -- chooses the FP32 kernel's tile shape for this plan.
 * Sec. 5.2 fixes one block per pointing; here the shape (tile_samples in
 * {8, 16, 32} consecutive samples per disc traversal x pixels_per_thread in
 * {1, 2}) is a tuning choice whose best value depends on the scan and the
 * disc size.  Every shape runs pisco_convolve on the n pointings given (a
 * representative slice of the scan, e.g. 1e5 - 1e6 samples) once untimed and
 * `reps` times timed with CUDA events on `stream`; the fastest is kept by the
 * plan for its later calls.
 *   tod_scratch        device float32 [n], overwritten (the TOD of the last shape tried).
 *   reps               timed launches per shape, 1 .. 100.
 *   tile_samples, pixels_per_thread, best_ms
 *                      host outputs (each may be NULL): the chosen shape and its
 *                      mean time per launch in milliseconds.
 * Synchronises `stream`.  FP32 plans only (PISCO_EUNSUPPORTED otherwise); on
 * error the plan keeps its previous shape.
 */
pisco_status pisco_plan_autotune(pisco_plan* plan, int det, int64_t n,
                                 const double* theta, const double* phi, const double* psi,
                                 void* tod_scratch, int reps, int* tile_samples,
                                 int* pixels_per_thread, float* best_ms, void* stream);

/*
 * pisco_inject_mr_stall -- test hook for the failure detection of the
 * multi-realization kernel (no counterpart in the paper).  The next launch of
 * pisco_convolve or pisco_convolve_batched on this (PISCO_BF16_MR or
 * PISCO_FP16_MR) plan first waits `cycles` SM clocks on an mbarrier that
 * nothing arrives on, before it issues any copy or MMA: the wait gives up,
 * the kernel records error bit 2, writes no TOD, releases its tensor memory
 * and returns, and pisco_sync_status reports PISCO_ETIMEOUT.  Later launches
 * run normally.  cycles in [1, 1e10]; PISCO_EUNSUPPORTED for other plans.
 */
pisco_status pisco_inject_mr_stall(pisco_plan* plan, int64_t cycles);

/*
 * pisco_plan_autotune_batched -- pisco_plan_autotune for a focal plane (Sec.
 * 5.1): every shape runs pisco_convolve_batched on the given slices of the
 * detectors' scans (offsets: host [n_det + 1], as in pisco_convolve_batched;
 * e.g. the first 1e4 - 1e5 samples of every detector), and the plan keeps the
 * fastest shape for all its detectors.  tod_scratch: device float32
 * [offsets[n_det]], overwritten.  Other arguments, outputs and errors as for
 * pisco_plan_autotune.
 */
pisco_status pisco_plan_autotune_batched(pisco_plan* plan, int n_det, const int64_t* offsets,
                                         const double* theta, const double* phi, const double* psi,
                                         void* tod_scratch, int reps, int* tile_samples,
                                         int* pixels_per_thread, float* best_ms, void* stream);

/* Synchronise the plan's work on `stream` and report any error a kernel
 * recorded since the last call, clearing it: PISCO_ETIMEOUT when a bounded
 * device wait gave up (flag 2: every mbarrier wait of the multi-realization
 * kernel, on its MMAs, its TMA loads and its warps' hand-offs, gives up after
 * about two seconds, and the kernel then stops issuing, frees its tensor
 * memory and returns), PISCO_EDEVICE for any other flag (no kernel records
 * one at present: the value is kept for invariant checks). */
pisco_status pisco_sync_status(pisco_plan* plan, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PISCO_H */
