// vegas_probe.cu -- issue-rate probes of the arithmetic pipes the fill kernel
// uses (FP32 FMA, FP64 FMA, MUFU ex2, 32-bit multiply-high, the FP64
// exponential of the FP64 form's Gaussian integrand, exp2_64ths) and of the shared
// memory integer atomics its map-weight histogram accumulates with.  Each thread runs
// eight independent dependent chains; every block times itself with the SM
// cycle counter.  The rate is operations per SM per clock, taken from the
// median block with four blocks resident per SM.  These rates, times the SM
// count and clock, are the denominators of the fill kernel's roofline.
#include <algorithm>
#include <vector>

#include "vegas_device.cuh"
#include "vegas_internal.h"

namespace vg {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeIters = 4096;
constexpr int kChains = 8;

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) probe_kernel(float seedf, double* sink, long long* cycles) {
  float f[kChains];
  double g[kChains];
  uint32_t u[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    f[c] = seedf * (float)(threadIdx.x + c + 1) * 1e-6f;
    g[c] = (double)f[c];
    u[c] = threadIdx.x * 2654435761u + c;
  }
  __syncthreads();
  const long long t0 = clock64();
#pragma unroll 4
  for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      if constexpr (KIND == 0) f[c] = fmaf(f[c], 0.999999f, 1e-7f);
      else if constexpr (KIND == 1) g[c] = fma(g[c], 0.999999, 1e-7);
      else if constexpr (KIND == 2) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(f[c]));
      else if constexpr (KIND == 5) g[c] = exp2_64ths(-g[c]);  // converges to 0.989..., stays in range
      else u[c] = __umulhi(u[c], 0x9E3779B9u) + c;
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  double acc = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc += (double)f[c] + g[c] + (double)u[c];
  if (acc == 12345.678) sink[0] = acc;  // keeps the chains alive
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// 32-bit integer atomic adds to shared memory, every lane of a warp on its own
// bank (the fill's fixed-point histogram when its intervals do not collide);
// the return value is unused, as in the fill
__global__ void __launch_bounds__(kProbeThreads) probe_atomics_kernel(double* sink, long long* cycles) {
  __shared__ uint32_t hs[kChains * kProbeThreads];
#pragma unroll
  for (int c = 0; c < kChains; ++c) hs[c * kProbeThreads + threadIdx.x] = 0u;
  __syncthreads();
  const long long t0 = clock64();
#pragma unroll 4
  for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) atomicAdd(&hs[c * kProbeThreads + threadIdx.x], (uint32_t)it | 1u);
  }
  __syncthreads();
  const long long t1 = clock64();
  uint32_t acc = 0u;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc += hs[c * kProbeThreads + threadIdx.x];
  if (acc == 12345u) sink[0] = (double)acc;  // keeps the adds alive
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

template <int KIND>
int run_probe(int sms, double* d_sink, long long* d_cyc, double& rate) {
  const int blocks = 4 * sms;
  for (int rep = 0; rep < 2; ++rep) {  // warm-up, then the timed launch
    if constexpr (KIND == 4) probe_atomics_kernel<<<blocks, kProbeThreads>>>(d_sink, d_cyc);
    else probe_kernel<KIND><<<blocks, kProbeThreads>>>(1.0f, d_sink, d_cyc);
  }
  VG_CHECK(cudaGetLastError());
  VG_CHECK(cudaDeviceSynchronize());
  std::vector<long long> cyc(blocks);
  VG_CHECK(cudaMemcpy(cyc.data(), d_cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost));
  std::sort(cyc.begin(), cyc.end());
  const double med = (double)cyc[blocks / 2];
  const double ops_per_sm = 4.0 * kProbeThreads * (double)kProbeIters * kChains;
  rate = ops_per_sm / med;
  return VEGAS_OK;
}

}  // namespace
}  // namespace vg

namespace {
// one probe of kind KIND on the current device, with its own small buffers
template <int KIND>
int probe_one(double& rate) {
  int dev = 0, sms = 0;
  VG_CHECK(cudaGetDevice(&dev));
  VG_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  double* d_sink = nullptr;
  long long* d_cyc = nullptr;
  if (cudaMalloc(&d_sink, sizeof(double)) != cudaSuccess) return VEGAS_ENOMEM;
  if (cudaMalloc(&d_cyc, sizeof(long long) * 4 * sms) != cudaSuccess) {
    cudaFree(d_sink);
    return VEGAS_ENOMEM;
  }
  const int rc = vg::run_probe<KIND>(sms, d_sink, d_cyc, rate);
  cudaFree(d_sink);
  cudaFree(d_cyc);
  return rc;
}
}  // namespace

namespace {
__global__ void exp64_eval_kernel(const double* __restrict__ x, double* __restrict__ y, int64_t n, int which) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = which == 0 ? vg::exp_table64(x[i]) : which == 2 ? vg::exp2_64ths(x[i]) : exp(x[i]);
}
}  // namespace

extern "C" int vegas_exp64_eval(const double* d_x, double* d_y, int64_t n, int32_t which, void* stream) {
  if (n < 0 || (n > 0 && (!d_x || !d_y)) || which < 0 || which > 2) return VEGAS_EINVAL;
  if (n == 0) return VEGAS_OK;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
  exp64_eval_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(d_x, d_y, n, which);
  return vg::cuda_status(cudaGetLastError());
}

extern "C" int vegas_probe_exp64(double* rate) {
  if (!rate) return VEGAS_EINVAL;
  return probe_one<5>(*rate);
}

extern "C" int vegas_probe_shared_atomics(double* rate) {
  if (!rate) return VEGAS_EINVAL;
  return probe_one<4>(*rate);
}

extern "C" int vegas_probe_pipes(double rates[4]) {
  if (!rates) return VEGAS_EINVAL;
  int dev = 0, sms = 0;
  VG_CHECK(cudaGetDevice(&dev));
  VG_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  double* d_sink = nullptr;
  long long* d_cyc = nullptr;
  if (cudaMalloc(&d_sink, sizeof(double)) != cudaSuccess) return VEGAS_ENOMEM;
  if (cudaMalloc(&d_cyc, sizeof(long long) * 4 * sms) != cudaSuccess) {
    cudaFree(d_sink);
    return VEGAS_ENOMEM;
  }
  int rc = vg::run_probe<0>(sms, d_sink, d_cyc, rates[0]);
  if (rc == VEGAS_OK) rc = vg::run_probe<1>(sms, d_sink, d_cyc, rates[1]);
  if (rc == VEGAS_OK) rc = vg::run_probe<2>(sms, d_sink, d_cyc, rates[2]);
  if (rc == VEGAS_OK) rc = vg::run_probe<3>(sms, d_sink, d_cyc, rates[3]);
  cudaFree(d_sink);
  cudaFree(d_cyc);
  return rc;
}
