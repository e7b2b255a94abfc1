// vegas_fill.cuh -- the fill kernel (Algorithm 2, vegasFill, of cuVegas), as a
// template over integrand, precision and maximum dimension.
//
// Work decomposition (Sec. 3.1: every thread does the same number of
// evaluations).  Evaluations j in [0, neval) are cut into tiles of kTile
// consecutive indices; a persistent grid walks the tiles round-robin.  A tile
// meets at most kMaxCubesPerTile hypercubes because n_h >= 2.  It stages their
// offsets in shared memory, and each thread takes kSamplesPerThread consecutive
// evaluations.  A thread binary-searches the cube of its first evaluation and
// steps forward from there; no evaluation-to-cube array is ever built.
//
// Accumulation without global atomics (the paper's atomicAdd of Sec. 3.3.3):
//  * cube weights: every J f goes to a shared array.  The cubes that lie inside
//    the tile get their two-pass (count, mean, centred second moment) from
//    one thread, or from one warp for long runs.  A cube that crosses a tile
//    edge leaves a Carry record, and a fix-up kernel merges the records
//    (Chan's pairwise formula) in tile order.
//  * map weights: a per-CTA histogram in shared memory (shared atomics),
//    written once per CTA to a partial array that a second kernel sums in a
//    fixed order.
//  * iteration estimate / variance: per-thread sums, reduced per CTA, then
//    summed over CTAs in a fixed order.
#pragma once
#include <type_traits>

#include "vegas_device.cuh"
#include "vegas_internal.h"

namespace vg {

template <typename T>
struct alignas(4 * sizeof(T)) TabEntry {
  T e, dx, jk, pad;  // left edge, width, N_g * width of one map interval
};

template <typename T>
struct Acc;  // per-thread accumulator of the iteration sums
template <>
struct Acc<double> {
  double v = 0.0;
  __device__ void add(double x) { v += x; }
  __device__ double value() const { return v; }
};
template <>
struct Acc<float> {
  ff v{0.0f, 0.0f};
  __device__ void add(ff x) { v = ff_add(v, x); }
  __device__ void add(float x) { v = ff_add(v, x); }
  __device__ double value() const { return ff_to_double(v); }
};

__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(ff v) { return ff_to_double(v); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ ff warp_sum(ff v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ff w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = ff_add(v, w);
  }
  return v;
}

// sum over the block in a fixed order; the result is valid in thread 0
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += red[i];
  return r;
}

// Turn the caller's parameters into the derived form used by vg::integrand.
template <int ID, typename T>
__device__ void prep_params(const double* __restrict__ raw, int np, int d, T* out) {
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    double v = raw[i];
    if constexpr (ID == VEGAS_GAUSS_SUM) {
      if (i == 1) {
        const double s2 = 2.0 * v * v;
        v = sizeof(T) == 8 ? -1.0 / s2 : -1.4426950408889634 / s2;  // exp or exp2 exponent
      } else if (i == 2) {
        v = (double)((np - 3) / d);
      }
    } else if constexpr (ID == VEGAS_PRODUCT_PEAK) {
      if (i < d) v = 1.0 / (v * v);
    } else if constexpr (ID == VEGAS_OSCILLATORY) {
      if (i == 0) v = 6.283185307179586 * v;
    }
    out[i] = (T)v;
  }
  if constexpr (ID == VEGAS_MOROKOFF_CAFLISCH) {
    if (threadIdx.x == 0) {
      out[0] = (T)pow(1.0 + 1.0 / d, (double)d);
      out[1] = (T)(1.0 / d);
    }
  }
}

// Point of evaluation j in cube h: Philox coordinates, z = (c + u) N_g / s,
// interval i = min(floor z, N_g - 1), x = e_i + (z - i) dx_i, J = prod N_g dx_i.
template <typename T, int DMAX>
__device__ __forceinline__ void make_point(const FillArgs& a, uint32_t h, int64_t j, const T* __restrict__ gz,
                                           const TabEntry<T>* __restrict__ tab, T (&x)[DMAX], int (&bin)[DMAX],
                                           T& J) {
  const int G = a.G;
  uint32_t rest = h;
  J = T(1);
  uint4 r = make_uint4(0u, 0u, 0u, 0u);
  const uint32_t jlo = (uint32_t)j, jhi = (uint32_t)((uint64_t)j >> 32);
#pragma unroll
  for (int k = 0; k < DMAX; ++k) {
    if (k < a.d) {
      const uint32_t q = (uint32_t)(((uint64_t)rest * a.magic[k]) >> a.shift[k]);  // rest / s_k
      const uint32_t ck = rest - q * a.nstrat[k];
      rest = q;
      T z;
      if constexpr (sizeof(T) == 8) {
        if ((k & 1) == 0)
          r = philox4x32_10(make_uint4(jlo, jhi, a.iter, (a.pid << 16) | (uint32_t)(k >> 1)), a.key0, a.key1);
        const uint32_t whi = (k & 1) ? r.z : r.x, wlo = (k & 1) ? r.w : r.y;
        const uint64_t bits = (((uint64_t)whi << 32) | wlo) >> 11;
        const double u = __dmul_rn(__ull2double_rn(bits), 0x1p-53);
        z = __dmul_rn(__dadd_rn((double)ck, u), gz[k]);
      } else {
        if ((k & 3) == 0)
          r = philox4x32_10(make_uint4(jlo, jhi, a.iter, (a.pid << 16) | (uint32_t)(k >> 2)), a.key0, a.key1);
        const uint32_t w = (k & 3) == 0 ? r.x : (k & 3) == 1 ? r.y : (k & 3) == 2 ? r.z : r.w;
        const float u = __fmul_rn(__uint2float_rn(w >> 8), 0x1p-24f);
        z = __fmul_rn(__fadd_rn((float)ck, u), gz[k]);
      }
      int i = (int)z;  // z >= 0: truncation is floor
      i = i < G - 1 ? i : G - 1;
      const T dz = z - (T)i;  // exact
      const TabEntry<T> te = tab[k * G + i];
      x[k] = fma(dz, te.dx, te.e);
      J = J * te.jk;
      bin[k] = k * G + i;
    }
  }
}

template <int ID, typename T, int DMAX>
__global__ void __launch_bounds__(kFillThreads) fill_kernel(const __grid_constant__ FillArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x;
  const int d = a.d, G = a.G, dG = a.d * a.G;
  TabEntry<T>* tab = a.table_smem ? (TabEntry<T>*)(smem + a.sm_table) : (TabEntry<T>*)a.gtable;
  T* hist_s = (T*)(smem + a.sm_hist);
  double* hist_g = a.hist_part + (size_t)blockIdx.x * dG;
  T* prm = (T*)(smem + a.sm_params);
  int64_t* off_s = (int64_t*)(smem + a.sm_off);
  T* invn = (T*)(smem + a.sm_invn);
  T* vals = (T*)(smem + a.sm_vals);
  int* longlist = (int*)(smem + a.sm_long);
  T* gz = (T*)(smem + a.sm_misc);
  int* misc = (int*)(smem + a.sm_misc + kMaxDim * sizeof(T));  // [0] long count, [1] cubes in tile
  double* red = (double*)(smem + a.sm_misc + kMaxDim * sizeof(T) + 16);

  // ---- prologue: map table, histogram, parameters, z scales ----
  if (a.table_smem) {
    for (int b = tid; b < dG; b += kFillThreads) {
      const int k = b / G, i = b - k * G;
      const double e0 = a.edges[k * (G + 1) + i], e1 = a.edges[k * (G + 1) + i + 1];
      const double dx = __dsub_rn(e1, e0), jk = __dmul_rn((double)G, dx);
      tab[b] = TabEntry<T>{(T)e0, (T)dx, (T)jk, T(0)};
    }
  }
  if (a.hist_smem)
    for (int b = tid; b < dG; b += kFillThreads) hist_s[b] = T(0);
  prep_params<ID, T>(a.params_raw, a.np_raw, d, prm);
  if (tid < d) {
    if constexpr (sizeof(T) == 8) gz[tid] = __ddiv_rn((double)G, (double)a.nstrat[tid]);
    else gz[tid] = __fdiv_rn((float)G, (float)a.nstrat[tid]);
  }
  __syncthreads();

  Acc<T> acc_i, acc_v;
  float lmax = -__int_as_float(0x7f800000);
  bool bad = false;

  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const int64_t j0 = (int64_t)tile * kTile;
    const int len = (int)min((int64_t)kTile, a.neval - j0);
    const int h0 = a.tile_first[tile];
    const int64_t jend = j0 + len;

    // ---- offsets and 1/n_h of the cubes the tile can meet ----
    for (int c = tid; c <= kMaxCubesPerTile; c += kFillThreads) {
      const int64_t h = (int64_t)h0 + c;
      const int64_t o0 = h <= a.NH ? a.offsets[h] : INT64_MAX;
      off_s[c] = o0;
      if (c < kMaxCubesPerTile) {
        T inv = T(0);
        if (o0 < jend) {
          const int64_t o1 = a.offsets[h + 1];
          inv = T(1) / (T)(o1 - o0);
        }
        invn[c] = inv;
      }
    }
    if (tid == 0) {
      misc[0] = 0;
      a.carries[2 * tile] = Carry{-1, 0, 0.0, 0.0};
      a.carries[2 * tile + 1] = Carry{-1, 0, 0.0, 0.0};
    }
    __syncthreads();

    // ---- evaluations: point, map, integrand, J f, map weights ----
    const int jl0 = tid * kSamplesPerThread;
    if (jl0 < len) {
      const int64_t jfirst = j0 + jl0;
      int lo = 0, hi = kMaxCubesPerTile - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off_s[mid] <= jfirst) lo = mid;
        else hi = mid - 1;
      }
      int c = lo;
#pragma unroll 1
      for (int s = 0; s < kSamplesPerThread; ++s) {
        const int jl = jl0 + s;
        if (jl >= len) break;
        const int64_t j = j0 + jl;
        while (off_s[c + 1] <= j) ++c;
        T x[DMAX];
        int bin[DMAX];
        T J;
        make_point<T, DMAX>(a, (uint32_t)(h0 + c), j, gz, tab, x, bin, J);
        const T f = integrand<ID, T, DMAX>(x, d, prm, a.np_derived);
        if (!isfinite(f)) bad = true;
        const T v = J * f;
        vals[jl] = v;
        const T wv = v * v * invn[c];
#pragma unroll
        for (int k = 0; k < DMAX; ++k) {
          if (k < d) {
            if (a.hist_smem) atomicAdd(hist_s + bin[k], wv);
            else atomicAdd(hist_g + bin[k], (double)wv);
          }
        }
        if (jl == len - 1) misc[1] = c + 1;
      }
    }
    __syncthreads();

    // ---- cube statistics ----
    const int ncub = misc[1];
    // one cube segment done: a cube inside the tile is final, one crossing an
    // edge becomes a Carry for the fix-up kernel
    auto finish = [&](int c, int L, auto mean, T m2) {
      const int64_t o0 = off_s[c], o1 = off_s[c + 1];
      const bool before = o0 < j0, after = o1 > jend;
      const int h = h0 + c;
      if (before || after) {
        a.carries[2 * tile + (before ? 0 : 1)] = Carry{h, L, to_double(mean), (double)m2};
        return;
      }
      const int64_t n = o1 - o0;
      float ell;
      acc_i.add(mean);
      if constexpr (sizeof(T) == 8) {
        acc_v.add(m2 / ((double)n * (double)(n - 1)));
        ell = __fmul_rn(a.half_beta, log2r(m2 / (double)(n - 1)));
      } else {
        acc_v.add(m2 / ((float)n * (float)(n - 1)));
        ell = __fmul_rn(a.half_beta, log2r(__fdiv_rn(m2, (float)(n - 1))));
      }
      a.ell[h] = ell;
      lmax = fmaxf(lmax, ell);
      if (a.cube_mean) {
        a.cube_mean[h] = to_double(mean);
        a.cube_m2[h] = (double)m2;
      }
    };

    for (int c = tid; c < ncub; c += kFillThreads) {
      const int64_t o0 = off_s[c], o1 = off_s[c + 1];
      const int r0 = (int)max(o0 - j0, (int64_t)0), r1 = (int)min(o1 - j0, (int64_t)len);
      const int L = r1 - r0;
      if (L > kLongSegment) {
        longlist[atomicAdd(&misc[0], 1)] = c;
        continue;
      }
      if constexpr (sizeof(T) == 8) {
        double s = 0.0;
        for (int r = r0; r < r1; ++r) s += vals[r];
        const double mean = s / (double)L;
        double q = 0.0;
        for (int r = r0; r < r1; ++r) {
          const double dv = vals[r] - mean;
          q = fma(dv, dv, q);
        }
        finish(c, L, mean, q);
      } else {
        ff s{0.0f, 0.0f};
        for (int r = r0; r < r1; ++r) s = ff_add(s, vals[r]);
        const float Lf = (float)L;
        const float mh = __fdiv_rn(s.hi, Lf);
        const float ml = __fdiv_rn(__fadd_rn(fmaf(-mh, Lf, s.hi), s.lo), Lf);
        float q = 0.0f;
        for (int r = r0; r < r1; ++r) {
          const float dv = vals[r] - mh;
          q = fmaf(dv, dv, q);
        }
        finish(c, L, ff{mh, ml}, q);
      }
    }
    __syncthreads();
    const int nlong = misc[0];
    const int warp = tid >> 5, lane = tid & 31;
    for (int e = warp; e < nlong; e += kFillThreads / 32) {
      const int c = longlist[e];
      const int64_t o0 = off_s[c], o1 = off_s[c + 1];
      const int r0 = (int)max(o0 - j0, (int64_t)0), r1 = (int)min(o1 - j0, (int64_t)len);
      const int L = r1 - r0;
      if constexpr (sizeof(T) == 8) {
        double s = 0.0;
        for (int r = r0 + lane; r < r1; r += 32) s += vals[r];
        s = warp_sum(s);
        const double mean = s / (double)L;
        double q = 0.0;
        for (int r = r0 + lane; r < r1; r += 32) {
          const double dv = vals[r] - mean;
          q = fma(dv, dv, q);
        }
        q = warp_sum(q);
        if (lane == 0) finish(c, L, mean, q);
      } else {
        ff s{0.0f, 0.0f};
        for (int r = r0 + lane; r < r1; r += 32) s = ff_add(s, vals[r]);
        s = warp_sum(s);
        const float Lf = (float)L;
        const float mh = __fdiv_rn(s.hi, Lf);
        const float ml = __fdiv_rn(__fadd_rn(fmaf(-mh, Lf, s.hi), s.lo), Lf);
        float q = 0.0f;
        for (int r = r0 + lane; r < r1; r += 32) {
          const float dv = vals[r] - mh;
          q = fmaf(dv, dv, q);
        }
        const ff qq = warp_sum(ff{q, 0.0f});
        if (lane == 0) finish(c, L, ff{mh, ml}, __fadd_rn(qq.hi, qq.lo));
      }
    }
    __syncthreads();
  }

  // ---- epilogue: CTA partial sums, max weight, flags, histogram ----
  const double si = block_sum(acc_i.value(), red);
  const double sv = block_sum(acc_v.value(), red);
  if (tid == 0) {
    a.cta_part[2 * blockIdx.x] = si;
    a.cta_part[2 * blockIdx.x + 1] = sv;
  }
  for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  if ((tid & 31) == 0) atomicMax(a.ellmax_key, float_key(lmax));
  if (__syncthreads_or(bad) && tid == 0) atomicOr(a.flags, 1);
  if (a.hist_smem)
    for (int b = tid; b < dG; b += kFillThreads) hist_g[b] = (double)hist_s[b];
}

}  // namespace vg
