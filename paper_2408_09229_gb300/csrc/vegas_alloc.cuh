// vegas_alloc.cuh -- device code of the allocation passes (updateEvalsPerCube
// + mapEvalsToCubes of Algorithm 1, Sec. 2.1.2 and Eq. (7) of cuVegas), shared
// by the single-integral entry points and the batched driver.
//
// n_h = 2 + a share of R = neval - 2 N_h proportional to the quantised weight
// q_h = rint(2^24 2^(ell_h - max ell)), with ell_h = (beta/2) log2 var_h from
// the fill.  Cumulative rounding gives the shares:
//   off_h = 2h + floor(R Q_h / Q),  Q_h = sum_{h'<h} q_h',  Q = Q_{N_h},
// so sum n_h = neval exactly and n_h >= 2.  Integer arithmetic makes every
// decision, so the counts are a function of the ell_h bits alone.
#pragma once
#include <algorithm>
#include <cstdint>

#include "vegas_device.cuh"
#include "vegas_internal.h"

namespace vg {

constexpr int kBlockCubes = kAllocThreads * kAllocItems;

struct AllocScratch {
  size_t key, bsum, total;
  int64_t nblocks;
};

inline AllocScratch alloc_layout(int64_t ncubes) {
  AllocScratch L{};
  L.nblocks = (ncubes + kBlockCubes - 1) / kBlockCubes;
  L.key = 0;
  L.bsum = 256;
  L.total = L.bsum + sizeof(uint64_t) * (size_t)(L.nblocks + 1) + 256;
  return L;
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
__device__ __forceinline__ void block_sum_body(const float* __restrict__ ell, int64_t n, const int* key, int uniform,
                                               uint64_t* bsum, int64_t blk) {
  __shared__ uint64_t red[kAllocThreads / 32];
  const bool uni = is_uniform(key, uniform);
  const float emax = key_float(*key);
  uint32_t q[kAllocItems];
  load_weights(ell, blk * kBlockCubes + (int64_t)threadIdx.x * kAllocItems, n, uni, emax, q);
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
    bsum[blk] = t;
  }
}

// pass 2: exclusive scan of the block sums, in place; bsum[nb] = Q
__device__ __forceinline__ void block_scan_body(uint64_t* bsum, int64_t nb) {
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

__device__ __forceinline__ void offsets_body(const float* __restrict__ ell, int64_t n, int64_t neval, const int* key,
                                             int uniform, const uint64_t* __restrict__ bpre,
                                             int64_t* __restrict__ offsets, int64_t blk) {
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
  const int64_t block0 = blk * kBlockCubes;
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
  uint64_t Qh = (uni ? (uint64_t)blk * kBlockCubes : bpre[blk]) + wbefore + (x - tsum);
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


}  // namespace vg
