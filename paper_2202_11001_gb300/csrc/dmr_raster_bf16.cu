// Rasterise-and-sample kernels for bf16 image storage (see dmr_device.cuh).
#include "dmr_device.cuh"

namespace dmr {

void launch_raster_bf16(const DevProblem* probs, const Batch& b, int warps, int vpw, int n_sm, cudaStream_t st,
                       cudaStream_t side, cudaEvent_t fork) {
  raster_launch<ST_BF16>(probs, b, warps, vpw, n_sm, st, side, fork);
}

}  // namespace dmr
