// Tile-shape autotuner for the FP32 tile kernel.
//
// The FP32 path's tile shape (consecutive samples sharing one disc traversal,
// ring pixels per thread) trades the reuse of each pixel's sky value and
// half-angle against registers and the length of the per-sample loop; the
// best shape depends on the scan's speed against the sky pixel size and on
// the disc size.  pisco_plan_autotune times every shape the kernel is built
// for on a representative slice of the caller's pointing, with CUDA events on
// the caller's stream, and keeps the fastest for the plan's later calls.

#include "pisco_internal.cuh"

#include <cstdlib>

namespace pisco {
void set_error(pisco_plan* plan, const char* fmt, ...);
}  // namespace pisco

using namespace pisco;

namespace {

// Times every tile shape on detectors [d0, d0 + nd) with per-detector sample ranges (one untimed
// launch per shape, then `reps` timed ones) and keeps the fastest.  Arguments already checked.
pisco_status tune(pisco_plan* plan, int d0, int nd, const int64_t* begin, const int64_t* count,
                  const double* theta, const double* phi, const double* psi, void* tod_scratch, int reps,
                  int* tile_samples, int* pixels_per_thread, float* best_ms, cudaStream_t s) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        set_error(plan, "cudaEventCreate failed");
        return PISCO_ECUDA;
    }
    const int tiles[3] = {8, 16, 32}, nps[2] = {1, 2};
    const int old_tile = plan->tile_samples, old_np = plan->pixels_per_thread;
    int best_tile = old_tile, best_np = old_np;
    float best = -1.f;
    pisco_status st = PISCO_OK;
    for (int a = 0; a < 3 && st == PISCO_OK; ++a)
        for (int b = 0; b < 2 && st == PISCO_OK; ++b) {
            plan->tile_samples = tiles[a];
            plan->pixels_per_thread = nps[b];
            st = run(plan, kForward, d0, nd, begin, count, theta, phi, psi, tod_scratch, nullptr, nullptr, s);
            cudaError_t e = cudaEventRecord(e0, s);
            for (int r = 0; r < reps && st == PISCO_OK && e == cudaSuccess; ++r)
                st = run(plan, kForward, d0, nd, begin, count, theta, phi, psi, tod_scratch, nullptr, nullptr, s);
            if (st != PISCO_OK) break;
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                set_error(plan, "timing failed: %s", cudaGetErrorString(e));
                st = PISCO_ECUDA;
                break;
            }
            ms /= (float)reps;
            if (best < 0.f || ms < best) {
                best = ms;
                best_tile = tiles[a];
                best_np = nps[b];
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != PISCO_OK) {
        plan->tile_samples = old_tile;
        plan->pixels_per_thread = old_np;
        return st;
    }
    plan->tile_samples = best_tile;
    plan->pixels_per_thread = best_np;
    if (tile_samples) *tile_samples = best_tile;
    if (pixels_per_thread) *pixels_per_thread = best_np;
    if (best_ms) *best_ms = best;
    return PISCO_OK;
}

}  // namespace

extern "C" pisco_status pisco_plan_autotune(pisco_plan* plan, int det, int64_t n, const double* theta,
                                            const double* phi, const double* psi, void* tod_scratch, int reps,
                                            int* tile_samples, int* pixels_per_thread, float* best_ms,
                                            void* stream) {
    if (!plan) return PISCO_EINVAL;
    if (plan->precision != PISCO_FP32) {
        set_error(plan, "pisco_plan_autotune tunes FP32 plans only");
        return PISCO_EUNSUPPORTED;
    }
    if (det < 0 || det >= plan->n_det) {
        set_error(plan, "detector %d outside [0, %d)", det, plan->n_det);
        return PISCO_EINVAL;
    }
    if (n < 1 || reps < 1 || reps > 100) {
        set_error(plan, "n = %lld must be >= 1 and reps = %d in [1, 100]", (long long)n, reps);
        return PISCO_EINVAL;
    }
    pisco_status st = check_pointing(plan, n, theta, phi, psi);
    if (st != PISCO_OK) return st;
    if (!is_device_ptr(tod_scratch)) {
        set_error(plan, "tod_scratch must be a device pointer");
        return PISCO_EINVAL;
    }
    const int64_t begin = 0, count = n;
    return tune(plan, det, 1, &begin, &count, theta, phi, psi, tod_scratch, reps, tile_samples, pixels_per_thread,
                best_ms, (cudaStream_t)stream);
}

extern "C" pisco_status pisco_plan_autotune_batched(pisco_plan* plan, int n_det, const int64_t* offsets,
                                                    const double* theta, const double* phi, const double* psi,
                                                    void* tod_scratch, int reps, int* tile_samples,
                                                    int* pixels_per_thread, float* best_ms, void* stream) {
    if (!plan) return PISCO_EINVAL;
    if (plan->precision != PISCO_FP32) {
        set_error(plan, "pisco_plan_autotune_batched tunes FP32 plans only");
        return PISCO_EUNSUPPORTED;
    }
    if (n_det < 1 || n_det > plan->n_det || !offsets || offsets[0] != 0) {
        set_error(plan, "n_det %d outside [1, %d], or offsets NULL or not starting at 0", n_det, plan->n_det);
        return PISCO_EINVAL;
    }
    if (reps < 1 || reps > 100) {
        set_error(plan, "reps = %d outside [1, 100]", reps);
        return PISCO_EINVAL;
    }
    int64_t* count = (int64_t*)malloc(n_det * sizeof(int64_t));
    if (!count) return PISCO_ENOMEM;
    pisco_status st = PISCO_OK;
    for (int d = 0; d < n_det && st == PISCO_OK; ++d) {
        count[d] = offsets[d + 1] - offsets[d];
        if (count[d] < 0) {
            set_error(plan, "offsets must be non-decreasing (detector %d)", d);
            st = PISCO_EINVAL;
        }
    }
    const int64_t total = st == PISCO_OK ? offsets[n_det] : 0;
    if (st == PISCO_OK && total < 1) {
        set_error(plan, "the slices hold no samples");
        st = PISCO_EINVAL;
    }
    if (st == PISCO_OK) st = check_pointing(plan, total, theta, phi, psi);
    if (st == PISCO_OK && !is_device_ptr(tod_scratch)) {
        set_error(plan, "tod_scratch must be a device pointer");
        st = PISCO_EINVAL;
    }
    if (st == PISCO_OK)
        st = tune(plan, 0, n_det, offsets, count, theta, phi, psi, tod_scratch, reps, tile_samples,
                  pixels_per_thread, best_ms, (cudaStream_t)stream);
    free(count);
    return st;
}
