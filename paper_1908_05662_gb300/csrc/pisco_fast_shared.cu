// Instantiations of the FP32 tile kernel that read the folded node grid from shared memory.
#include "pisco_fast.cuh"

namespace pisco {
cudaError_t launch_fast_shared(const LaunchParams& p, int mode, int tile_samples, int np, cudaStream_t s) {
    return launch_fetch<PISCO_FETCH_SHARED>(p, mode, tile_samples, np, s);
}
}  // namespace pisco
