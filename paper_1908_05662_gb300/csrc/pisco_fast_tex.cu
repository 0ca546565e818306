// Instantiations of the FP32 tile kernel that read the beam through the texture path.
#include "pisco_fast.cuh"

namespace pisco {
cudaError_t launch_fast_texture(const LaunchParams& p, int mode, int tile_samples, int np, cudaStream_t s) {
    return launch_fetch<PISCO_FETCH_TEXTURE>(p, mode, tile_samples, np, s);
}
}  // namespace pisco
