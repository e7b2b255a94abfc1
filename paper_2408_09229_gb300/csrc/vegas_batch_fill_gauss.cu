// vegas_batch_fill_gauss.cu -- the batched fill's kernels for the diagonal-ridge (Gaussian sum) integrals
// (widths 4, 8 and 16; both register budgets).  One file per family, so that
// the instances compile in parallel.
#include "vegas_batch_fill.cuh"

namespace vg {

int launch_batch_fill_gauss(int variant, int dmax, int group, const BatchLaunch& L, int grid, int smem, cudaStream_t s) {
  return launch_batch_fill_family<VEGAS_GAUSS_SUM>(variant, dmax, group, L, grid, smem, s);
}

int batch_fill_occupancy_gauss(int variant, int dmax, int smem) {
  return batch_fill_family_occupancy<VEGAS_GAUSS_SUM>(variant, dmax, smem);
}

}  // namespace vg
