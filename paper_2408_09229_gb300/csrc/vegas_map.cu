// vegas_map.cu -- adjustWeights + updateMap and combineIterationsResults of
// Algorithm 1 in cuVegas (Sec. 2.1.1 map refinement with damping alpha;
// Sec. 2.1.3, Eqs. (8)-(9)).  Both are small: one CTA per axis for the map
// and one CTA for the combination.
#include <cmath>

#include "vegas_device.cuh"
#include "vegas_internal.h"
#include "vegas_map.cuh"

namespace vg {

__global__ void __launch_bounds__(256) refine_kernel(int G, double alpha, const double* __restrict__ bins,
                                                     const double* __restrict__ e_in, double* __restrict__ e_out) {
  extern __shared__ double sh[];
  const int k = blockIdx.x;
  refine_axis_body(G, alpha, bins + (size_t)k * G, e_in + (size_t)k * (G + 1), e_out + (size_t)k * (G + 1), sh);
}

__global__ void __launch_bounds__(kCombineThreads) combine_kernel(const double* est, const double* sig, int n,
                                                                   int skip, double* out, bool lagged) {
  combine_block(est, sig, n, skip, out, lagged);
}

// handle path: store (I_t, sigma_t) of iteration t from the fill's (I, var), then combine
__global__ void __launch_bounds__(kCombineThreads) record_combine_kernel(const double* result, int t, double* est,
                                                                         double* sig, int skip, double* out,
                                                                         bool lagged) {
  if (threadIdx.x == 0) {
    est[t] = result[0];
    sig[t] = sqrt(result[1]);
  }
  __syncthreads();
  combine_block(est, sig, t + 1, skip, out, lagged);
}

int launch_record_combine(const double* d_result, int t, double* d_est, double* d_sig, int skip, double* d_out,
                          bool lagged, cudaStream_t s) {
  record_combine_kernel<<<1, kCombineThreads, 0, s>>>(d_result, t, d_est, d_sig, skip, d_out, lagged);
  return cuda_status(cudaGetLastError());
}

}  // namespace vg

using namespace vg;

extern "C" int vegas_refine(int32_t dim, int32_t nbins, double alpha, const double* d_bins, const double* d_edges_in,
                            double* d_edges_out, void* stream) {
  if (dim < 1 || dim > kMaxDim || nbins < 2 || nbins > kMaxBins || !(alpha >= 0.0) || !d_bins || !d_edges_in ||
      !d_edges_out || d_edges_in == d_edges_out)
    return VEGAS_EINVAL;
  const size_t smem = sizeof(double) * 2 * (size_t)nbins;
  if (smem > 48 * 1024)
    VG_CHECK(cudaFuncSetAttribute(refine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  refine_kernel<<<dim, 256, smem, (cudaStream_t)stream>>>(nbins, alpha, d_bins, d_edges_in, d_edges_out);
  return cuda_status(cudaGetLastError());
}

extern "C" int vegas_combine(const double* d_it_est, const double* d_it_sigma, int32_t n, int32_t skip, double* d_out,
                             void* stream) {
  if (n < 1 || skip < 0 || !d_it_est || !d_it_sigma || !d_out) return VEGAS_EINVAL;
  combine_kernel<<<1, kCombineThreads, 0, (cudaStream_t)stream>>>(d_it_est, d_it_sigma, n, skip, d_out, false);
  return cuda_status(cudaGetLastError());
}

extern "C" int vegas_combine_weighted(const double* d_it_est, const double* d_it_sigma, int32_t n, int32_t skip,
                                      int32_t weighting, double* d_out, void* stream) {
  if (n < 1 || skip < 0 || !d_it_est || !d_it_sigma || !d_out ||
      (weighting != VEGAS_WEIGHT_INVERSE_VARIANCE && weighting != VEGAS_WEIGHT_LAGGED))
    return VEGAS_EINVAL;
  combine_kernel<<<1, kCombineThreads, 0, (cudaStream_t)stream>>>(d_it_est, d_it_sigma, n, skip, d_out,
                                                                   weighting == VEGAS_WEIGHT_LAGGED);
  return cuda_status(cudaGetLastError());
}
