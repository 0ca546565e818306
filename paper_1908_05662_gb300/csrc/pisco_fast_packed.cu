// Instantiations of the FP32 tile kernel that read 32-byte packed beam cells.
#include "pisco_fast.cuh"

namespace pisco {
cudaError_t launch_fast_packed(const LaunchParams& p, int mode, int tile_samples, int np, cudaStream_t s) {
    return launch_fetch<PISCO_FETCH_PACKED>(p, mode, tile_samples, np, s);
}
}  // namespace pisco
