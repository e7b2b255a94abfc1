// vegas_fill_dispatch.cuh -- the launcher shared by the fill instantiation
// units.  Each unit (one precision and point path per translation unit, so that
// the instances compile in parallel) names the integrand families and widths it
// instantiates as two lists; FillUnit maps the run-time (integrand, dmax) pair
// onto fill_kernel<ID, T, DMAX, EXACT, STREAM>, launches it or asks for its
// occupancy.  A pair outside the lists gives VEGAS_EINVAL from launch and 0
// from occupancy.
#pragma once
#include <type_traits>

#include "vegas_fill.cuh"

namespace vg {

template <int... Is>
struct IntList {};

// f(std::integral_constant<int, I>{}) for the I of the list equal to v; -1 when none is
template <typename F, int... Is>
int pick_int(int v, IntList<Is...>, F&& f) {
  int r = -1;
  (void)((v == Is ? (r = f(std::integral_constant<int, Is>{}), true) : false) || ...);
  return r;
}

// TILED: the kernels are built for each tile size (tile_log2 10 and 11 at compile time); otherwise one kernel
// reads the tile from its arguments.
template <typename T, bool EXACT, bool STREAM, typename Ids, typename Dims, bool TILED = false>
struct FillUnit {
  template <int ID, int DMAX, int TLC>
  static int launch_one(FillArgs& a, int grid, cudaStream_t s) {
    auto k = fill_kernel<ID, T, DMAX, EXACT, STREAM, TLC>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, a.sm_total) != cudaSuccess)
      return VEGAS_ECUDA;
    k<<<grid, kFillThreads, a.sm_total, s>>>(a);
    return cuda_status(cudaGetLastError());
  }

  template <int ID, int DMAX, int TLC>
  static int occupancy_one(int smem) {
    auto k = fill_kernel<ID, T, DMAX, EXACT, STREAM, TLC>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kFillThreads, smem) != cudaSuccess) return 0;
    return n;
  }

  // f(id, dm, tl) with all three as integral constants (tl 0 unless TILED); -1 when not instantiated
  template <typename F>
  static int dispatch(int integrand, int dmax, int tile_log2, F&& f) {
    return pick_int(dmax, Dims{}, [&](auto dm) {
      return pick_int(integrand, Ids{}, [&](auto id) {
        if constexpr (TILED)
          return pick_int(tile_log2, IntList<kTileLog2Min, kTileLog2Max>{}, [&](auto tl) { return f(id, dm, tl); });
        else
          return f(id, dm, std::integral_constant<int, 0>{});
      });
    });
  }

  static int launch(int integrand, int dmax, FillArgs& a, int grid, cudaStream_t s) {
    const int r = dispatch(integrand, dmax, a.tile_log2, [&](auto id, auto dm, auto tl) {
      return launch_one<decltype(id)::value, decltype(dm)::value, decltype(tl)::value>(a, grid, s);
    });
    return r == -1 ? VEGAS_EINVAL : r;
  }

  static int occupancy(int integrand, int dmax, int tile_log2, int smem) {
    const int r = dispatch(integrand, dmax, tile_log2, [&](auto id, auto dm, auto tl) {
      return occupancy_one<decltype(id)::value, decltype(dm)::value, decltype(tl)::value>(smem);
    });
    return r < 0 ? 0 : r;
  }
};

// the closed-form integrand families of Table 3 and the Gaussian sums
using AllFamilies = IntList<VEGAS_GAUSS_SUM, VEGAS_PRODUCT_PEAK, VEGAS_OSCILLATORY, VEGAS_SIN_EXP, VEGAS_LINEAR,
                            VEGAS_COSINE, VEGAS_EXPONENTIAL, VEGAS_ROOS_ARNOLD, VEGAS_MOROKOFF_CAFLISCH,
                            VEGAS_MAP_DENSITY>;

}  // namespace vg
