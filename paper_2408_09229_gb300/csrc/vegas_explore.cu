// vegas_explore.cu -- exploration for the learned proposal (not in cuVegas,
// arXiv 2408.09229).  A VEGAS+ map (Sec. 2.1.1) adapted from a uniform start
// follows whichever peak its first samples happen to favour; maps adapted
// with different seeds favour different peaks.  Their samples are pooled into
// one weighted training set for the flow by the balance heuristic (Veach and
// Guibas, SIGGRAPH 1995): sample r comes from map k = r mod S, and its weight
// is |f(x)| / q(x) with q = (1/S) sum_k q_k, q_k(x) = prod_a 1 / (N_g dx_a)
// the density of map k on the interval that holds x_a.  Each sample's
// uniform numbers are one Philox4x32-10 call per four axes, counter
// (r, axis group, "EXPR"), key = the 64-bit seed.
#include <algorithm>

#include "vegas_device.cuh"
#include "vegas_internal.h"

namespace vg {
namespace {

constexpr uint32_t kExploreTag = 0x45585052u;  // "EXPR"

__global__ void __launch_bounds__(256) explore_points_kernel(int d, int G, int S, const double* __restrict__ maps,
                                                             int64_t m, uint32_t k0, uint32_t k1,
                                                             float* __restrict__ X, double* __restrict__ q) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= m) return;
  const size_t stride = (size_t)d * (G + 1);
  const double* E = maps + (size_t)(r % S) * stride;
  double xa[kMaxDim];
  for (int g0 = 0; g0 < d; g0 += 4) {
    const uint4 b = philox4x32_10(make_uint4((uint32_t)r, (uint32_t)(r >> 32), (uint32_t)g0, kExploreTag), k0, k1);
    const uint32_t u[4] = {b.x, b.y, b.z, b.w};
    for (int t = 0; t < 4 && g0 + t < d; ++t) {
      const int a = g0 + t;
      // y = (u + 1/2) 2^-32 in (0, 1); z = y N_g is exact (33 + 16 significant bits)
      const double z = ((double)u[t] + 0.5) * 0x1p-32 * (double)G;
      const int i = min((int)z, G - 1);
      const double* e = E + (size_t)a * (G + 1);
      const double x = fma(z - (double)i, e[i + 1] - e[i], e[i]);
      xa[a] = x;
      X[r * d + a] = (float)x;
    }
  }
  // the mixture density: for every map, the interval j of each coordinate (e_j <= x < e_{j+1}, j in [0, G-1])
  double qs = 0.0;
  for (int k = 0; k < S; ++k) {
    const double* F = maps + (size_t)k * stride;
    double p = 1.0;
    for (int a = 0; a < d; ++a) {
      const double* e = F + (size_t)a * (G + 1);
      int lo = 0, hi = G;  // e_lo <= x unless lo = 0; x < e_hi unless hi = G
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (e[mid] <= xa[a]) lo = mid;
        else hi = mid;
      }
      p *= (double)G * (e[lo + 1] - e[lo]);
    }
    qs += 1.0 / p;
  }
  q[r] = qs / (double)S;
}

__global__ void explore_weights_kernel(const float* __restrict__ f, const double* __restrict__ q, int64_t m,
                                       float* __restrict__ w) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= m) return;
  const double v = fabs((double)f[r]) / q[r];
  w[r] = isfinite(v) ? (float)v : 0.0f;  // a non-finite weight counts as 0
}

}  // namespace

int explore_points(int d, int G, int S, const double* maps, int64_t m, uint64_t seed, float* X, double* q,
                   cudaStream_t s) {
  if (m == 0) return VEGAS_OK;
  const unsigned grid = (unsigned)((m + 255) / 256);
  explore_points_kernel<<<grid, 256, 0, s>>>(d, G, S, maps, m, (uint32_t)seed, (uint32_t)(seed >> 32), X, q);
  return cuda_status(cudaGetLastError());
}

int explore_weights(const float* f, const double* q, int64_t m, float* w, cudaStream_t s) {
  if (m == 0) return VEGAS_OK;
  explore_weights_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(f, q, m, w);
  return cuda_status(cudaGetLastError());
}

}  // namespace vg

extern "C" int vegas_explore_points(int32_t dim, int32_t nbins, int32_t nmaps, const double* d_maps,
                                    int64_t samples_per_map, uint64_t seed, float* d_x, double* d_q, void* stream) {
  if (dim < 1 || dim > vg::kMaxDim || nbins < 2 || nbins > vg::kMaxBins || nmaps < 1 || nmaps > vg::kMaxExploreMaps ||
      samples_per_map < 0 || samples_per_map > vg::kMaxEval / nmaps)
    return VEGAS_EINVAL;
  const int64_t m = samples_per_map * nmaps;
  if (m > 0 && (!d_maps || !d_x || !d_q)) return VEGAS_EINVAL;
  return vg::explore_points(dim, nbins, nmaps, d_maps, m, seed, d_x, d_q, (cudaStream_t)stream);
}
