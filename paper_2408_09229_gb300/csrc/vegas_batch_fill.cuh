// vegas_batch_fill.cuh -- the batched fill: one persistent launch evaluates
// the tiles of every running integral of a batch (Algorithm 2 of cuVegas per
// integral; the batch shares the launch).
//
// The CTAs take chunks of chunk_tiles consecutive tiles of the batch's work
// list from a global counter, so integrals of different cost balance out.
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

// derived parameters of the integral in sa, for its family and width
__device__ __forceinline__ void batch_prep(const FillArgs& sa, int dmax, float* prm) {
  const int d = sa.d;
#define VG_PREP(ID, DM) prep_params<ID, float, DM>(sa.params_raw, sa.np_raw, d, prm)
  switch (sa.iid * 4 + (dmax == 4 ? 0 : dmax == 8 ? 1 : 2)) {
    case VEGAS_GAUSS_SUM * 4 + 0: VG_PREP(VEGAS_GAUSS_SUM, 4); break;
    case VEGAS_GAUSS_SUM * 4 + 1: VG_PREP(VEGAS_GAUSS_SUM, 8); break;
    case VEGAS_GAUSS_SUM * 4 + 2: VG_PREP(VEGAS_GAUSS_SUM, 16); break;
    case VEGAS_PRODUCT_PEAK * 4 + 0: VG_PREP(VEGAS_PRODUCT_PEAK, 4); break;
    case VEGAS_PRODUCT_PEAK * 4 + 1: VG_PREP(VEGAS_PRODUCT_PEAK, 8); break;
    case VEGAS_PRODUCT_PEAK * 4 + 2: VG_PREP(VEGAS_PRODUCT_PEAK, 16); break;
    case VEGAS_OSCILLATORY * 4 + 0: VG_PREP(VEGAS_OSCILLATORY, 4); break;
    case VEGAS_OSCILLATORY * 4 + 1: VG_PREP(VEGAS_OSCILLATORY, 8); break;
    default: VG_PREP(VEGAS_OSCILLATORY, 16); break;
  }
#undef VG_PREP
}

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

__device__ __forceinline__ void batch_tile(const FillArgs& sa, int dmax, const BatchLaunch& L, unsigned char* smem,
                                           FillState<float>& st, int tile) {
  switch (sa.iid * 4 + (dmax == 4 ? 0 : dmax == 8 ? 1 : 2)) {
    case VEGAS_GAUSS_SUM * 4 + 0: batch_tile_one<VEGAS_GAUSS_SUM, 4>(sa, L, smem, st, tile); break;
    case VEGAS_GAUSS_SUM * 4 + 1: batch_tile_one<VEGAS_GAUSS_SUM, 8>(sa, L, smem, st, tile); break;
    case VEGAS_GAUSS_SUM * 4 + 2: batch_tile_one<VEGAS_GAUSS_SUM, 16>(sa, L, smem, st, tile); break;
    case VEGAS_PRODUCT_PEAK * 4 + 0: batch_tile_one<VEGAS_PRODUCT_PEAK, 4>(sa, L, smem, st, tile); break;
    case VEGAS_PRODUCT_PEAK * 4 + 1: batch_tile_one<VEGAS_PRODUCT_PEAK, 8>(sa, L, smem, st, tile); break;
    case VEGAS_PRODUCT_PEAK * 4 + 2: batch_tile_one<VEGAS_PRODUCT_PEAK, 16>(sa, L, smem, st, tile); break;
    case VEGAS_OSCILLATORY * 4 + 0: batch_tile_one<VEGAS_OSCILLATORY, 4>(sa, L, smem, st, tile); break;
    case VEGAS_OSCILLATORY * 4 + 1: batch_tile_one<VEGAS_OSCILLATORY, 8>(sa, L, smem, st, tile); break;
    default: batch_tile_one<VEGAS_OSCILLATORY, 16>(sa, L, smem, st, tile); break;
  }
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

template <int MINB>
__global__ void __launch_bounds__(kFillThreads, MINB) batch_fill_kernel(const __grid_constant__ BatchLaunch L) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(16) FillArgs sa;
  __shared__ int s_chunk;
  const int tid = threadIdx.x;
  const int total = L.act_tile[L.P];
  int cur = -1, dmax = 4;
  FillState<float> st;
  for (;;) {
    if (tid == 0) s_chunk = (int)atomicAdd(L.counter, 1u);
    __syncthreads();
    const int64_t t0 = (int64_t)s_chunk * L.chunk_tiles;
    __syncthreads();  // s_chunk is rewritten only after every thread has read it
    if (t0 >= total) break;
    const int t1 = (int)min((int64_t)total, t0 + L.chunk_tiles);
    for (int gt = (int)t0; gt < t1; ++gt) {
      const int p = batch_find(L.act_tile, L.P, gt);
      if (p != cur) {
        if (cur >= 0) batch_flush(L, cur, sa, smem, st);
        // load integral p: arguments, map table, derived parameters, zeroed histogram
        const uint32_t* src = reinterpret_cast<const uint32_t*>(&L.prob[p].a);
        uint32_t* dst = reinterpret_cast<uint32_t*>(&sa);
        for (int i = tid; i < (int)(sizeof(FillArgs) / 4); i += kFillThreads) dst[i] = src[i];
        __syncthreads();
        dmax = L.prob[p].dmax;
        {
          const FillShared<float> S = fill_shared<float>(smem, sa, true);
          fill_prologue<float>(sa, S, sa.d, true);
          batch_prep(sa, dmax, S.prm);
        }
        st = FillState<float>{};
        st.vexp = sa.vexp ? *sa.vexp : 0;
        st.J0 = ldexpf(1.0f, -st.vexp);
        cur = p;
        __syncthreads();
      }
      batch_tile(sa, dmax, L, smem, st, gt - L.act_tile[p]);
    }
  }
  if (cur >= 0) batch_flush(L, cur, sa, smem, st);
}

template <int MINB>
int launch_batch_fill_variant(const BatchLaunch& L, int grid, int smem, cudaStream_t s) {
  auto k = batch_fill_kernel<MINB>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return VEGAS_ECUDA;
  k<<<grid, kFillThreads, smem, s>>>(L);
  return cuda_status(cudaGetLastError());
}

template <int MINB>
int batch_fill_occupancy_variant(int smem) {
  auto k = batch_fill_kernel<MINB>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kFillThreads, smem) != cudaSuccess) return 0;
  return n;
}

}  // namespace vg
