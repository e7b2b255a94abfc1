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

#include "vegas_device.cuh"
#include "vegas_internal.h"

namespace vg {
namespace {

constexpr int kBlockCubes = kAllocThreads * kAllocItems;

struct AllocScratch {
  size_t key, bsum, total;
  int64_t nblocks;
};

AllocScratch alloc_layout(int64_t ncubes) {
  AllocScratch L{};
  L.nblocks = (ncubes + kBlockCubes - 1) / kBlockCubes;
  L.key = 0;
  L.bsum = 256;
  L.total = L.bsum + sizeof(uint64_t) * (size_t)(L.nblocks + 1) + 256;
  return L;
}

__global__ void key_init_kernel(int* key) { *key = float_key(-__int_as_float(0x7f800000)); }

__global__ void max_kernel(const float* __restrict__ ell, int64_t n, int* key) {
  float m = -__int_as_float(0x7f800000);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, ell[i]);
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(key, float_key(m));
}

__device__ __forceinline__ bool is_uniform(const int* key, int uniform) {
  return uniform || *key == float_key(-__int_as_float(0x7f800000));
}

__device__ __forceinline__ uint64_t weight_of(const float* __restrict__ ell, int64_t h, bool uni, float emax) {
  return uni ? 1ull : (uint64_t)quant_weight(ell[h], emax);
}

// the quantised weights of cubes [base, base + kAllocItems): four 16-byte
// loads issued together when the run is whole and aligned, scalar loads else
__device__ __forceinline__ void load_weights(const float* __restrict__ ell, int64_t base, int64_t n, bool uni,
                                             float emax, uint32_t (&q)[kAllocItems]) {
  if (uni) {
#pragma unroll
    for (int i = 0; i < kAllocItems; ++i) q[i] = base + i < n ? 1u : 0u;
    return;
  }
  if (base + kAllocItems <= n && ((reinterpret_cast<uintptr_t>(ell + base) & 15) == 0)) {
    const float4* p = reinterpret_cast<const float4*>(ell + base);
    float4 v[kAllocItems / 4];
#pragma unroll
    for (int i = 0; i < kAllocItems / 4; ++i) v[i] = __ldg(p + i);
#pragma unroll
    for (int i = 0; i < kAllocItems / 4; ++i) {
      q[4 * i] = quant_weight(v[i].x, emax);
      q[4 * i + 1] = quant_weight(v[i].y, emax);
      q[4 * i + 2] = quant_weight(v[i].z, emax);
      q[4 * i + 3] = quant_weight(v[i].w, emax);
    }
  } else {
#pragma unroll
    for (int i = 0; i < kAllocItems; ++i) q[i] = base + i < n ? quant_weight(ell[base + i], emax) : 0u;
  }
}

// pass 1: sum of q over each block of kBlockCubes cubes
__global__ void __launch_bounds__(kAllocThreads) block_sum_kernel(const float* __restrict__ ell, int64_t n,
                                                                  const int* key, int uniform, uint64_t* bsum) {
  __shared__ uint64_t red[kAllocThreads / 32];
  const bool uni = is_uniform(key, uniform);
  const float emax = key_float(*key);
  uint32_t q[kAllocItems];
  load_weights(ell, (int64_t)blockIdx.x * kBlockCubes + (int64_t)threadIdx.x * kAllocItems, n, uni, emax, q);
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < kAllocItems; ++i) s += q[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t t = 0;
    for (int w = 0; w < kAllocThreads / 32; ++w) t += red[w];
    bsum[blockIdx.x] = t;
  }
}

// pass 2: exclusive scan of the block sums, in place; bsum[nb] = Q
__global__ void __launch_bounds__(1024) block_scan_kernel(uint64_t* bsum, int64_t nb) {
  __shared__ uint64_t warp_tot[32];
  __shared__ uint64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const uint64_t v = i < nb ? bsum[i] : 0ull;
    uint64_t x = v;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
      uint64_t t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0ull;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      warp_tot[lane] = t;  // inclusive scan of warp totals
    }
    __syncthreads();
    const uint64_t before = carry + (w > 0 ? warp_tot[w - 1] : 0ull) + (x - v);
    if (i < nb) bsum[i] = before;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = before + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[nb] = carry;
}

// floor(R * Qh / Q) exactly: a double estimate, corrected with 128-bit products
__device__ __forceinline__ uint64_t share_floor(uint64_t R, uint64_t Qh, uint64_t Q, double r_over_q) {
  uint64_t c = (uint64_t)((double)Qh * r_over_q);
  const unsigned __int128 P = (unsigned __int128)R * Qh;
  unsigned __int128 CQ = (unsigned __int128)c * Q;
  for (int it = 0; it < 8 && CQ > P; ++it) {
    --c;
    CQ -= Q;
  }
  for (int it = 0; it < 8 && CQ + Q <= P; ++it) {
    ++c;
    CQ += Q;
  }
  return c;
}

// pass 3: block scan of q and the offsets off_h = 2h + floor(R Q_h / Q).
// Every thread works on a run of kAllocItems consecutive cubes; the offsets
// go out through shared memory so that the global stores are coalesced.
// Padding keeps the runs free of bank conflicts.
__device__ __forceinline__ int pad16(int x) { return x + (x >> 4); }  // 8-byte words

__global__ void __launch_bounds__(kAllocThreads) offsets_kernel(const float* __restrict__ ell, int64_t n,
                                                                int64_t neval, const int* key, int uniform,
                                                                const uint64_t* __restrict__ bpre,
                                                                int64_t* __restrict__ offsets) {
  __shared__ uint64_t warp_tot[kAllocThreads / 32];
  __shared__ int64_t stage[kBlockCubes + kBlockCubes / 16];
  __shared__ double r_over_q_s;
  const bool uni = is_uniform(key, uniform);
  const float emax = uni ? 0.0f : key_float(*key);
  const int64_t nb = (n + kBlockCubes - 1) / kBlockCubes;
  const uint64_t R = (uint64_t)(neval - 2 * n);
  const uint64_t Q = uni ? (uint64_t)n : bpre[nb];
  // FP64 is scarce on this GPU: one division per block, none per cube
  if (threadIdx.x == 0) r_over_q_s = (double)R / (double)Q;
  const int64_t block0 = (int64_t)blockIdx.x * kBlockCubes;
  const int64_t base = block0 + (int64_t)threadIdx.x * kAllocItems;
  uint32_t q[kAllocItems];
  load_weights(ell, base, n, uni, emax, q);
  uint64_t tsum = 0;
#pragma unroll
  for (int i = 0; i < kAllocItems; ++i) tsum += q[i];
  // exclusive scan of the thread sums across the block
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t x = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  uint64_t wbefore = 0;
  for (int k = 0; k < w; ++k) wbefore += warp_tot[k];
  uint64_t Qh = (uni ? (uint64_t)blockIdx.x * kBlockCubes : bpre[blockIdx.x]) + wbefore + (x - tsum);
  // the thread's first share exactly, then share_{h+1} = share_h + floor((rem_h + R q_h) / Q)
  // with rem_h = R Q_h - share_h Q carried exactly; FP32 estimates every step and
  // integer compares correct it, so no step needs FP64
  uint64_t share = share_floor(R, Qh, Q, r_over_q_s);
  uint64_t rem = (uint64_t)((unsigned __int128)R * Qh - (unsigned __int128)share * Q);
  const float inv_q = 1.0f / ((float)(uint32_t)(Q >> 32) * 4294967296.0f + (float)(uint32_t)Q);
#pragma unroll
  for (int i = 0; i < kAllocItems; ++i) {
    const int64_t h = base + i;
    stage[pad16(threadIdx.x * kAllocItems + i)] = 2 * h + (int64_t)share;
    const uint64_t X = rem + R * (uint64_t)q[i];  // < 2^57
    // X to float from its 32-bit halves (32-bit conversions, no FP64 pipe)
    const float xf = fmaf((float)(uint32_t)(X >> 32), 4294967296.0f, (float)(uint32_t)X);
    uint64_t inc = (uint64_t)(uint32_t)fminf(xf * inv_q, 4294967040.0f);
    if (inc > (1ull << 20)) {  // a heavy cube: the FP32 estimate is too coarse
      inc = share_floor(X, 1, Q, (double)X / (double)Q);
    } else {
      // inc is within one of floor(X/Q) <= 2^20, so inc Q <= X + Q < 2^58: 64 bits suffice
      uint64_t t = inc * Q;
      for (int it = 0; it < 8 && t > X; ++it) {
        --inc;
        t -= Q;
      }
      for (int it = 0; it < 8 && t + Q <= X; ++it) {
        ++inc;
        t += Q;
      }
    }
    share += inc;
    rem = X - inc * Q;
  }
  __syncthreads();
#pragma unroll 4
  for (int i = threadIdx.x; i < kBlockCubes; i += kAllocThreads)
    if (block0 + i < n) offsets[block0 + i] = stage[pad16(i)];
  if (base <= n - 1 && n - 1 < base + kAllocItems) offsets[n] = neval;  // the thread of the last cube
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
// cudaGetSymbolAddress, once per device, with that device current.
int static_scratch(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return VEGAS_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return VEGAS_EINVAL;
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_scratch[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_allocate_scratch) != cudaSuccess || !p) return VEGAS_ECUDA;
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
  const int rc = static_scratch(&base);
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
