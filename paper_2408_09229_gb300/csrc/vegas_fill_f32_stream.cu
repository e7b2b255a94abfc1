// vegas_fill_f32_stream.cu -- FP32 fill instantiations with the streamed point
// path (DMAX 16 and 32; see stream_point_eval in vegas_fill.cuh) and their
// launcher.
#include "vegas_fill_dispatch.cuh"

namespace vg {
namespace {
using Ids = IntList<VEGAS_GAUSS_SUM, VEGAS_PRODUCT_PEAK, VEGAS_OSCILLATORY, VEGAS_LINEAR, VEGAS_COSINE,
                    VEGAS_EXPONENTIAL, VEGAS_ROOS_ARNOLD, VEGAS_MOROKOFF_CAFLISCH, kIntegrandTabulated,
                    kIntegrandPoints>;
using Unit = FillUnit<float, false, true, Ids, IntList<16, 32>>;
}  // namespace

int launch_fill_f32_stream(int integrand, int dmax, FillArgs& a, int grid, cudaStream_t s) {
  return Unit::launch(integrand, dmax, a, grid, s);
}

int fill_occupancy_f32_stream(int integrand, int dmax, int tile_log2, int smem) {
  return Unit::occupancy(integrand, dmax, tile_log2, smem);
}

}  // namespace vg
