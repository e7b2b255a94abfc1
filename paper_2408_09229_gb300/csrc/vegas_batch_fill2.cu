// vegas_batch_fill2.cu -- the batched fill with 2 resident CTAs per SM
// (at most 128 registers a thread: the 16-axis paths do not spill).
#include "vegas_batch_fill.cuh"

namespace vg {

int launch_batch_fill_v2(const BatchLaunch& L, int grid, int smem, cudaStream_t s) {
  return launch_batch_fill_variant<2>(L, grid, smem, s);
}

int batch_fill_occupancy_v2(int smem) { return batch_fill_occupancy_variant<2>(smem); }

}  // namespace vg
