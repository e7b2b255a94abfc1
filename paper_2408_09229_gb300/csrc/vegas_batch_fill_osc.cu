// vegas_batch_fill_osc.cu -- the batched fill's kernels for the oscillatory integrals
// (widths 4, 8 and 16; both register budgets).  One file per family, so that
// the instances compile in parallel.
#include "vegas_batch_fill.cuh"

namespace vg {

int launch_batch_fill_osc(int variant, int dmax, int group, const BatchLaunch& L, int grid, int smem, cudaStream_t s) {
  return launch_batch_fill_family<VEGAS_OSCILLATORY>(variant, dmax, group, L, grid, smem, s);
}

int batch_fill_occupancy_osc(int variant, int dmax, int smem) {
  return batch_fill_family_occupancy<VEGAS_OSCILLATORY>(variant, dmax, smem);
}

}  // namespace vg
