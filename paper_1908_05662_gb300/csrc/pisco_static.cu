// pisco_beam_grid_adjoint_static: the beam-grid adjoint without any allocation.
//
// pisco_beam_grid_adjoint needs a scratch buffer for the folded node gradient
// (3 grid_n^2 elements) and allocates it in the plan on its first call.  Code
// that may not allocate device memory at the point of the call (a real-time
// loop with a frozen memory budget, an allocator that forbids cudaMalloc
// after start-up) uses this entry point instead: the scratch is the file-scope
// array below, present on every GPU that loads the library until the process
// exits.  Its device address is looked up once per device, with that device
// current, on the first call made there; make that first call before any
// stream capture.  All calls share the one array and leave their result in it,
// so calls whose kernels overlap on the GPU race; each call clears the part it
// uses before the kernels run.

#include "pisco_internal.cuh"

#include <cmath>
#include <mutex>

using namespace pisco;

namespace {

// Largest grid this entry point accepts: 3 x 512^2 float64 = 6 MiB of scratch.
constexpr int kStaticMaxGridN = 512;
constexpr size_t kStaticScratchBytes = 3ull * kStaticMaxGridN * kStaticMaxGridN * sizeof(double);

__device__ __align__(256) unsigned char g_grid_scratch[kStaticScratchBytes];
static_assert(kStaticScratchBytes >= 4ull * kStaticMaxGridN * kStaticMaxGridN * sizeof(float),
              "the static scratch holds the interleaved FP32 folded gradient too");

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mutex;

// Device address of g_grid_scratch on the current device (looked up once per device).
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_grid_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" pisco_status pisco_beam_grid_adjoint_static(pisco_plan* plan, int det, int64_t n, const double* theta,
                                                       const double* phi, const double* psi, const void* tod,
                                                       void* grad_grids, int accumulate, void* stream) {
    if (!plan) return PISCO_EINVAL;
    if (det < 0 || det >= plan->n_det) {
        set_error(plan, "detector %d outside [0, %d)", det, plan->n_det);
        return PISCO_EINVAL;
    }
    if (plan->grid_n > kStaticMaxGridN) {
        set_error(plan, "grid_n %d exceeds %d, the largest grid the static scratch of "
                        "pisco_beam_grid_adjoint_static holds; use pisco_beam_grid_adjoint",
                  plan->grid_n, kStaticMaxGridN);
        return PISCO_EINVAL;
    }
    pisco_status st = check_pointing(plan, n, theta, phi, psi);
    if (st != PISCO_OK) return st;
    if (!is_device_ptr(grad_grids) || (n > 0 && !is_device_ptr(tod))) {
        set_error(plan, "tod and grad_grids must be device pointers");
        return PISCO_EINVAL;
    }
    void* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) {
        set_error(plan, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
        return PISCO_ECUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int f64 = plan->precision == PISCO_FP64_PLAIN;
    const size_t bytes = folded_grad_bytes(plan->grid_n, f64);
    e = cudaMemsetAsync(scratch, 0, bytes, s);
    if (e != cudaSuccess) {
        set_error(plan, "clearing the static scratch failed: %s", cudaGetErrorString(e));
        return PISCO_ECUDA;
    }
    if (n > 0) {
        const int64_t begin = 0, count = n;
        st = run(plan, kGrid, det, 1, &begin, &count, theta, phi, psi, scratch, tod, nullptr, s);
        if (st != PISCO_OK) return st;
    }
    e = launch_unfold_grid(scratch, plan->grid_n, plan->h_dets[det].eps, plan->h_dets[det].zeta, grad_grids,
                           accumulate, f64, s);
    if (e != cudaSuccess) {
        set_error(plan, "kernel launch failed: %s", cudaGetErrorString(e));
        return PISCO_ECUDA;
    }
    return PISCO_OK;
}
