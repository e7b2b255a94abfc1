// vegas_fill_f32_stream.cu -- FP32 fill instantiations with the streamed point
// path (DMAX 16 and 32; see stream_point_eval in vegas_fill.cuh) and their
// launcher.
#include "vegas_fill.cuh"

namespace vg {
namespace {

template <int ID, int DMAX>
int launch_one(FillArgs& a, int grid, cudaStream_t s) {
  auto k = fill_kernel<ID, float, DMAX, false, true>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, a.sm_total);
  if (e != cudaSuccess) return VEGAS_ECUDA;
  k<<<grid, kFillThreads, a.sm_total, s>>>(a);
  return cuda_status(cudaGetLastError());
}

template <int ID, int DMAX>
int occupancy_one(int smem) {
  auto k = fill_kernel<ID, float, DMAX, false, true>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kFillThreads, smem) != cudaSuccess) return 0;
  return n;
}

template <int DMAX, typename F>
int dispatch_id(int integrand, F&& f) {
  switch (integrand) {
    case VEGAS_GAUSS_SUM: return f(std::integral_constant<int, VEGAS_GAUSS_SUM>{});
    case VEGAS_PRODUCT_PEAK: return f(std::integral_constant<int, VEGAS_PRODUCT_PEAK>{});
    case VEGAS_OSCILLATORY: return f(std::integral_constant<int, VEGAS_OSCILLATORY>{});
    case VEGAS_LINEAR: return f(std::integral_constant<int, VEGAS_LINEAR>{});
    case VEGAS_COSINE: return f(std::integral_constant<int, VEGAS_COSINE>{});
    case VEGAS_EXPONENTIAL: return f(std::integral_constant<int, VEGAS_EXPONENTIAL>{});
    case VEGAS_ROOS_ARNOLD: return f(std::integral_constant<int, VEGAS_ROOS_ARNOLD>{});
    case VEGAS_MOROKOFF_CAFLISCH: return f(std::integral_constant<int, VEGAS_MOROKOFF_CAFLISCH>{});
    case kIntegrandTabulated: return f(std::integral_constant<int, kIntegrandTabulated>{});
    case kIntegrandPoints: return f(std::integral_constant<int, kIntegrandPoints>{});
    default: return -1;
  }
}

template <typename F>
int dispatch(int integrand, int dmax, F&& f) {
  switch (dmax) {
    case 16: return dispatch_id<16>(integrand, [&](auto id) { return f(id, std::integral_constant<int, 16>{}); });
    case 32: return dispatch_id<32>(integrand, [&](auto id) { return f(id, std::integral_constant<int, 32>{}); });
    default: return -1;
  }
}

}  // namespace

int launch_fill_f32_stream(int integrand, int dmax, FillArgs& a, int grid, cudaStream_t s) {
  const int r = dispatch(integrand, dmax, [&](auto id, auto dm) { return launch_one<decltype(id)::value, decltype(dm)::value>(a, grid, s); });
  return r == -1 ? VEGAS_EINVAL : r;
}

int fill_occupancy_f32_stream(int integrand, int dmax, int smem) {
  const int r = dispatch(integrand, dmax, [&](auto id, auto dm) { return occupancy_one<decltype(id)::value, decltype(dm)::value>(smem); });
  return r < 0 ? 0 : r;
}

}  // namespace vg
