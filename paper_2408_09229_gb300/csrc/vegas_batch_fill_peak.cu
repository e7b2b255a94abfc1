// vegas_batch_fill_peak.cu -- the batched fill's kernels for the product-peak integrals
// (widths 4, 8 and 16; both register budgets).  One file per family, so that
// the instances compile in parallel.
#include "vegas_batch_fill.cuh"

namespace vg {

int launch_batch_fill_peak(int variant, int dmax, int group, const BatchLaunch& L, int grid, int smem, cudaStream_t s) {
  return launch_batch_fill_family<VEGAS_PRODUCT_PEAK>(variant, dmax, group, L, grid, smem, s);
}

int batch_fill_occupancy_peak(int variant, int dmax, int smem) {
  return batch_fill_family_occupancy<VEGAS_PRODUCT_PEAK>(variant, dmax, smem);
}

}  // namespace vg
