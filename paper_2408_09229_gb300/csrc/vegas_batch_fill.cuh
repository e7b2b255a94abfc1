// vegas_batch_fill.cuh -- the batched fill: one persistent launch evaluates
// the tiles of every running integral of a batch (Algorithm 2 of cuVegas per
// integral; the batch shares the launch).
//
// The integrals fall into groups of one family and width; each group has its
// own persistent kernel (one instance of the tile code: the registers of that
// instance alone).  The CTAs take chunks of chunk_tiles consecutive tiles of
// the group's work list from the group's counter, so integrals of different
// cost balance out.
// A CTA keeps one integral's state in shared memory: its FillArgs, its map
// table, its derived parameters and its map-weight histogram.  When the next
// tile belongs to another integral the CTA flushes that state (the
// histogram and the iteration sums go to the integral's global accumulators
// with FP64 atomic adds, the largest ell with an integer atomic max) and
// loads the next one.  Consecutive tiles of a chunk mostly share their
// integral, so the flushes are rare.  Cubes that cross a tile edge leave
// Carry records exactly as in the single-integral fill.
//
// The sums over CTAs arrive in a run-dependent order, so the batched results
// are reproducible to FP64 rounding, not bit for bit.
#pragma once
#include "vegas_batch.cuh"
#include "vegas_fill.cuh"

namespace vg {

template <int ID, int DMAX>
__device__ __forceinline__ void batch_tile_one(const FillArgs& sa, const BatchLaunch& L, unsigned char* smem,
                                               FillState<float>& st, int tile) {
  // the shared-memory views are rebuilt per tile (a few adds) instead of being held across the loop
  const FillShared<float> S = fill_shared<float>(smem, sa, true);
  const float ps0 = S.prm[0], ps1 = S.prm[1];
  const int pK = (ID == VEGAS_GAUSS_SUM) ? (int)S.prm[2] : 0;
  // 16-axis integrals take the streamed point path (64 registers, no spills)
  fill_tile<ID, float, DMAX, false, (DMAX >= 16)>(sa, L.rk0, L.rk1, S, st, tile, ps0, ps1, pK, nullptr);
}

// the CTA's share of integral p: iteration sums, largest ell, flags and the
// map-weight histogram go to p's global accumulators
__device__ __forceinline__ void batch_flush(const BatchLaunch& L, int p, const FillArgs& sa, unsigned char* smem,
                                            const FillState<float>& st) {
  const int tid = threadIdx.x;
  const FillShared<float> S = fill_shared<float>(smem, sa, true);
  const double si = block_sum(st.acc_i.value(), S.red);
  const double sv = block_sum(st.acc_v.value(), S.red);
  if (tid == 0) {
    atomicAdd(L.acc + 2 * p, si);
    atomicAdd(L.acc + 2 * p + 1, sv);
  }
  float lmax = st.lmax;
  for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  if ((tid & 31) == 0) atomicMax(L.key + p, float_key(lmax));
  if (__syncthreads_or(st.bad) && tid == 0) atomicOr(L.flags + p, 1);
  double* bins = L.prob[p].bins;
  const int dG = sa.d * sa.G;
  for (int b = tid; b < dG; b += kFillThreads) {
    const float pend = st.inv_scale > 0.0f ? __fmul_rn((float)S.hist_u[b], st.inv_scale) : 0.0f;
    double v;
    if (sa.acc32) {
      v = (double)S.hist_accf[b] + (double)pend;
    } else {
      ff acc = S.hist_acc[b];
      if (st.inv_scale > 0.0f) acc = ff_add(acc, pend);
      v = ff_to_double(acc);
    }
    if (v != 0.0) atomicAdd(bins + b, ldexp(v, 2 * st.vexp));
  }
  __syncthreads();
}

// The fill of one group (one family ID at width DMAX): persistent CTAs over the group's tiles.
template <int MINB, int ID, int DMAX>
__global__ void __launch_bounds__(kFillThreads, MINB) batch_fill_kernel(const __grid_constant__ BatchLaunch L,
                                                                        int group) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(16) FillArgs sa;
  __shared__ int s_chunk;
  const int tid = threadIdx.x;
  const int32_t* pre = L.grp_tile + (size_t)group * (L.P + 1);
  const int total = pre[L.P];
  int cur = -1;
  FillState<float> st;
  for (;;) {
    if (tid == 0) s_chunk = (int)atomicAdd(L.counter + 2 + group, 1u);
    __syncthreads();
    const int64_t t0 = (int64_t)s_chunk * L.chunk_tiles;
    __syncthreads();  // s_chunk is rewritten only after every thread has read it
    if (t0 >= total) break;
    const int t1 = (int)min((int64_t)total, t0 + L.chunk_tiles);
    for (int gt = (int)t0; gt < t1; ++gt) {
      const int p = batch_find(pre, L.P, gt);
      if (p != cur) {
        if (cur >= 0) batch_flush(L, cur, sa, smem, st);
        // load integral p: arguments, map table, derived parameters, zeroed histogram
        const uint32_t* src = reinterpret_cast<const uint32_t*>(&L.prob[p].a);
        uint32_t* dst = reinterpret_cast<uint32_t*>(&sa);
        for (int i = tid; i < (int)(sizeof(FillArgs) / 4); i += kFillThreads) dst[i] = src[i];
        __syncthreads();
        {
          const FillShared<float> S = fill_shared<float>(smem, sa, true);
          fill_prologue<float>(sa, S, sa.d, true, 1.0);
          prep_params<ID, float, DMAX>(sa.params_raw, sa.np_raw, sa.d, S.prm);
        }
        st = FillState<float>{};
        st.vexp = sa.vexp ? *sa.vexp : 0;
        st.J0 = ldexpf(1.0f, -st.vexp);
        cur = p;
        __syncthreads();
      }
      batch_tile_one<ID, DMAX>(sa, L, smem, st, gt - pre[p]);
    }
  }
  if (cur >= 0) batch_flush(L, cur, sa, smem, st);
}

template <int MINB, int ID, int DMAX>
int launch_batch_fill_kernel(const BatchLaunch& L, int group, int grid, int smem, cudaStream_t s) {
  auto k = batch_fill_kernel<MINB, ID, DMAX>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return VEGAS_ECUDA;
  k<<<grid, kFillThreads, smem, s>>>(L, group);
  return cuda_status(cudaGetLastError());
}

template <int MINB, int ID, int DMAX>
int batch_fill_kernel_occupancy(int smem) {
  auto k = batch_fill_kernel<MINB, ID, DMAX>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kFillThreads, smem) != cudaSuccess) return 0;
  return n;
}

// the launcher and occupancy query of family ID, for the variant's register budget and the width
template <int ID>
int launch_batch_fill_family(int variant, int dmax, int group, const BatchLaunch& L, int grid, int smem,
                             cudaStream_t s) {
  // variant 0: the fewest registers without local-memory spills in the persistent kernel: 64 at 4 axes (4 CTAs
  // an SM), 80 at 8 (3 CTAs), 128 for the 16-axis streamed path (2 CTAs).  Variant 1: 128 at every width.
  if (variant == 0) {
    if (dmax == 4) return launch_batch_fill_kernel<4, ID, 4>(L, group, grid, smem, s);
    if (dmax == 8) return launch_batch_fill_kernel<3, ID, 8>(L, group, grid, smem, s);
  }
  if (dmax == 4) return launch_batch_fill_kernel<2, ID, 4>(L, group, grid, smem, s);
  if (dmax == 8) return launch_batch_fill_kernel<2, ID, 8>(L, group, grid, smem, s);
  return launch_batch_fill_kernel<2, ID, 16>(L, group, grid, smem, s);
}

template <int ID>
int batch_fill_family_occupancy(int variant, int dmax, int smem) {
  if (variant == 0) {
    if (dmax == 4) return batch_fill_kernel_occupancy<4, ID, 4>(smem);
    if (dmax == 8) return batch_fill_kernel_occupancy<3, ID, 8>(smem);
  }
  if (dmax == 4) return batch_fill_kernel_occupancy<2, ID, 4>(smem);
  if (dmax == 8) return batch_fill_kernel_occupancy<2, ID, 8>(smem);
  return batch_fill_kernel_occupancy<2, ID, 16>(smem);
}

}  // namespace vg
