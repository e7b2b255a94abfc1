// vegas_alloc.cu -- updateEvalsPerCube + mapEvalsToCubes of Algorithm 1
// (Sec. 2.1.2 of cuVegas: n_h proportional to sigma_h damped by beta, with
// sum n_h = N_eval, Eq. (7)).
//
// n_h = 2 + a share of R = neval - 2 N_h proportional to the quantised weight
// q_h = rint(2^24 2^(ell_h - max ell)), with ell_h = (beta/2) log2 var_h from
// the fill.  Cumulative rounding gives the shares:
//   off_h = 2h + floor(R Q_h / Q),  Q_h = sum_{h'<h} q_h',  Q = Q_{N_h},
// so sum n_h = neval exactly and n_h >= 2.  Integer arithmetic makes every
// decision, so the counts are a function of the ell_h bits alone.  The
// offsets of the scan are the thread-to-cube mapping; the fill reads them
// and never materialises a per-evaluation array.
//
// Passes: (0) max ell, (1) per-block sums of q, (2) scan of the block sums in
// one CTA, (3) per-block scan and offsets.  The uniform allocation (first
// iteration, beta = 0, every variance zero) needs pass 3 only.
#include <algorithm>
#include <mutex>

#include "vegas_alloc.cuh"
#include "vegas_device.cuh"
#include "vegas_internal.h"

namespace vg {
namespace {

__global__ void key_init_kernel(int* key) { *key = float_key(-__int_as_float(0x7f800000)); }

__global__ void max_kernel(const float* __restrict__ ell, int64_t n, int* key) {
  float m = -__int_as_float(0x7f800000);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, ell[i]);
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(key, float_key(m));
}

__global__ void __launch_bounds__(kAllocThreads) block_sum_kernel(const float* __restrict__ ell, int64_t n,
                                                                  const int* key, int uniform, uint64_t* bsum) {
  block_sum_body(ell, n, key, uniform, bsum, blockIdx.x);
}

__global__ void __launch_bounds__(1024) block_scan_kernel(uint64_t* bsum, int64_t nb) { block_scan_body(bsum, nb); }

__global__ void __launch_bounds__(kAllocThreads) offsets_kernel(const float* __restrict__ ell, int64_t n,
                                                                int64_t neval, const int* key, int uniform,
                                                                const uint64_t* __restrict__ bpre,
                                                                int64_t* __restrict__ offsets) {
  offsets_body(ell, n, neval, key, uniform, bpre, offsets, blockIdx.x);
}

}  // namespace
}  // namespace vg

using namespace vg;

extern "C" size_t vegas_allocate_scratch_bytes(int64_t ncubes) {
  if (ncubes < 1) return 0;
  return alloc_layout(ncubes).total;
}

namespace vg {
// d_key: the order-preserving key of max ell when the caller already has it
// (the fill computes it), or NULL to compute it here
int allocate_impl(const float* d_ell, int64_t ncubes, int64_t neval, int uniform, int64_t* d_offsets,
                  void* d_scratch, size_t scratch_bytes, cudaStream_t s, const int* d_key) {
  if (ncubes < 1 || ncubes >= (int64_t(1) << 31) || neval < 2 * ncubes || neval > kMaxEval) return VEGAS_EINVAL;
  if (!d_offsets || !d_scratch || (!uniform && !d_ell)) return VEGAS_EINVAL;
  const AllocScratch L = alloc_layout(ncubes);
  if (scratch_bytes < L.total) return VEGAS_ENOSPACE;
  unsigned char* sc = (unsigned char*)d_scratch;
  int* own_key = (int*)(sc + L.key);
  uint64_t* bsum = (uint64_t*)(sc + L.bsum);
  const int* key = own_key;
  if (d_key && !uniform) {
    key = d_key;
  } else {
    key_init_kernel<<<1, 1, 0, s>>>(own_key);
    VG_CHECK(cudaGetLastError());
    if (!uniform) {
      const int grid = (int)std::min<int64_t>((ncubes + 255) / 256, 4096);
      max_kernel<<<grid, 256, 0, s>>>(d_ell, ncubes, own_key);
      VG_CHECK(cudaGetLastError());
    }
  }
  if (!uniform) {
    block_sum_kernel<<<(unsigned)L.nblocks, kAllocThreads, 0, s>>>(d_ell, ncubes, key, 0, bsum);
    VG_CHECK(cudaGetLastError());
    block_scan_kernel<<<1, 1024, 0, s>>>(bsum, L.nblocks);
    VG_CHECK(cudaGetLastError());
  }
  offsets_kernel<<<(unsigned)L.nblocks, kAllocThreads, 0, s>>>(d_ell, ncubes, neval, key, uniform, bsum, d_offsets);
  VG_CHECK(cudaGetLastError());
  return VEGAS_OK;
}
}  // namespace vg

extern "C" int vegas_allocate(const float* d_ell, int64_t ncubes, int64_t neval, int uniform, int64_t* d_offsets,
                              void* d_scratch, size_t scratch_bytes, void* stream) {
  return vg::allocate_impl(d_ell, ncubes, neval, uniform, d_offsets, d_scratch, scratch_bytes, (cudaStream_t)stream,
                           nullptr);
}

// ---------------------------------------------------------------------------
// vegas_allocate_static: the same allocation with no caller scratch and no
// allocation at all.  Its scratch (the per-block sums and the max key) is a
// fixed array in device global memory, sized for VEGAS_ALLOCATE_STATIC_MAX_CUBES
// cubes, that every GPU which loads this library holds until the process exits.
// ---------------------------------------------------------------------------
namespace vg {
namespace {

constexpr size_t kStaticScratchBytes =
    256 + sizeof(uint64_t) * (size_t)((VEGAS_ALLOCATE_STATIC_MAX_CUBES + kBlockCubes - 1) / kBlockCubes + 1) + 256;

__device__ __align__(256) unsigned char g_allocate_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
void* g_static_scratch[kMaxDevices] = {};

// Device address of g_allocate_scratch on the current device.  In host code
// the array's name is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress with that device current.  The lookup runs on every call
// made outside stream capture, so that a call after cudaDeviceReset sees the
// array of the new context; a call on a capturing stream uses the address that
// the last call outside capture found on the device.
int static_scratch(cudaStream_t s, void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return VEGAS_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return VEGAS_EINVAL;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const cudaError_t qe = cudaStreamIsCapturing(s, &cs);
  if (qe != cudaSuccess) (void)cudaGetLastError();  // e.g. the legacy stream while another stream captures
  const bool capturing = qe != cudaSuccess || cs != cudaStreamCaptureStatusNone;
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!capturing || !g_static_scratch[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_allocate_scratch) != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return VEGAS_ECUDA;
    }
    g_static_scratch[dev] = p;
  }
  *out = g_static_scratch[dev];
  return VEGAS_OK;
}

}  // namespace
}  // namespace vg

extern "C" int vegas_allocate_static(const float* d_ell, int64_t ncubes, int64_t neval, int uniform,
                                     int64_t* d_offsets, void* stream) {
  if (ncubes < 1 || neval < 2 * ncubes || neval > kMaxEval) return VEGAS_EINVAL;
  if (ncubes > VEGAS_ALLOCATE_STATIC_MAX_CUBES) return VEGAS_ENOSPACE;
  if (!d_offsets || (!uniform && !d_ell)) return VEGAS_EINVAL;
  void* base = nullptr;
  const int rc = static_scratch((cudaStream_t)stream, &base);
  if (rc != VEGAS_OK) return rc;
  const AllocScratch L = alloc_layout(ncubes);
  if (L.total > kStaticScratchBytes) return VEGAS_ENOSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* sc = (unsigned char*)base;
  int* key = (int*)(sc + L.key);
  uint64_t* bsum = (uint64_t*)(sc + L.bsum);
  // the key is re-initialised and every block sum rewritten on each call, so
  // nothing left by an earlier call is read
  key_init_kernel<<<1, 1, 0, s>>>(key);
  VG_CHECK(cudaGetLastError());
  if (!uniform) {
    const int grid = (int)std::min<int64_t>((ncubes + 255) / 256, 4096);
    max_kernel<<<grid, 256, 0, s>>>(d_ell, ncubes, key);
    VG_CHECK(cudaGetLastError());
    block_sum_kernel<<<(unsigned)L.nblocks, kAllocThreads, 0, s>>>(d_ell, ncubes, key, 0, bsum);
    VG_CHECK(cudaGetLastError());
    block_scan_kernel<<<1, 1024, 0, s>>>(bsum, L.nblocks);
    VG_CHECK(cudaGetLastError());
  }
  offsets_kernel<<<(unsigned)L.nblocks, kAllocThreads, 0, s>>>(d_ell, ncubes, neval, key, uniform, bsum, d_offsets);
  VG_CHECK(cudaGetLastError());
  return VEGAS_OK;
}
