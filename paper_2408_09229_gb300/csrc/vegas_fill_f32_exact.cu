// vegas_fill_f32_exact.cu -- FP32 instantiations of the fill kernel for d = DMAX
// (4 or 8) with the map table in shared memory, for both tile sizes, and their launcher.
#include "vegas_fill_dispatch.cuh"

namespace vg {
namespace {
using Unit = FillUnit<float, true, false, AllFamilies, IntList<4, 8>, true>;
}  // namespace

int launch_fill_f32_exact(int integrand, int dmax, FillArgs& a, int grid, cudaStream_t s) {
  return Unit::launch(integrand, dmax, a, grid, s);
}

int fill_occupancy_f32_exact(int integrand, int dmax, int tile_log2, int smem) {
  return Unit::occupancy(integrand, dmax, tile_log2, smem);
}

}  // namespace vg
