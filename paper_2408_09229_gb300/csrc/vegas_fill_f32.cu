// vegas_fill_f32.cu -- FP32 instantiations of the fill kernel (map table in
// global memory; every family, the learned proposal's tabulated and point
// passes; widths 4 to 32) and their launcher.
#include "vegas_fill_dispatch.cuh"

namespace vg {
namespace {
using Ids = IntList<VEGAS_GAUSS_SUM, VEGAS_PRODUCT_PEAK, VEGAS_OSCILLATORY, VEGAS_SIN_EXP, VEGAS_LINEAR, VEGAS_COSINE,
                    VEGAS_EXPONENTIAL, VEGAS_ROOS_ARNOLD, VEGAS_MOROKOFF_CAFLISCH, VEGAS_MAP_DENSITY,
                    kIntegrandTabulated, kIntegrandPoints>;
using Unit = FillUnit<float, false, false, Ids, IntList<4, 8, 16, 32>>;
}  // namespace

int launch_fill_f32(int integrand, int dmax, FillArgs& a, int grid, cudaStream_t s) {
  return Unit::launch(integrand, dmax, a, grid, s);
}

int fill_occupancy_f32(int integrand, int dmax, int tile_log2, int smem) {
  return Unit::occupancy(integrand, dmax, tile_log2, smem);
}

}  // namespace vg
