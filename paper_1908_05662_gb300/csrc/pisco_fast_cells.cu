// Instantiations of the FP32 tile kernel that read 64-byte beam cells through L1/L2.
#include "pisco_fast.cuh"

namespace pisco {
cudaError_t launch_fast_cells(const LaunchParams& p, int mode, int tile_samples, int np, cudaStream_t s) {
    return launch_fetch<PISCO_FETCH_CELLS>(p, mode, tile_samples, np, s);
}
}  // namespace pisco
