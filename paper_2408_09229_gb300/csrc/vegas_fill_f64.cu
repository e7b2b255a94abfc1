// vegas_fill_f64.cu -- FP64 instantiations of the fill kernel (map table in
// global memory; widths 4 to 32) and their launcher.
#include "vegas_fill_dispatch.cuh"

namespace vg {
namespace {
using Unit = FillUnit<double, false, false, AllFamilies, IntList<4, 8, 16, 32>>;
}  // namespace

int launch_fill_f64(int integrand, int dmax, FillArgs& a, int grid, cudaStream_t s) {
  return Unit::launch(integrand, dmax, a, grid, s);
}

int fill_occupancy_f64(int integrand, int dmax, int tile_log2, int smem) {
  return Unit::occupancy(integrand, dmax, tile_log2, smem);
}

}  // namespace vg
