// vegas_batch_fill4.cu -- the batched fill with 4 resident CTAs per SM
// (at most 64 registers a thread), and the variant dispatch.
#include "vegas_batch_fill.cuh"

namespace vg {

int launch_batch_fill_v2(const BatchLaunch& L, int grid, int smem, cudaStream_t s);
int batch_fill_occupancy_v2(int smem);

int launch_batch_fill(int variant, const BatchLaunch& L, int grid, int smem, cudaStream_t s) {
  if (variant == 0) return launch_batch_fill_variant<4>(L, grid, smem, s);
  if (variant == 1) return launch_batch_fill_v2(L, grid, smem, s);
  return VEGAS_EINVAL;
}

int batch_fill_occupancy(int variant, int smem) {
  if (variant == 0) return batch_fill_occupancy_variant<4>(smem);
  if (variant == 1) return batch_fill_occupancy_v2(smem);
  return 0;
}

}  // namespace vg
