// vegas_fill.cuh -- the fill kernel (Algorithm 2, vegasFill, of cuVegas), as a
// template over integrand, precision and maximum dimension.
//
// Work decomposition (Sec. 3.1: every thread does the same number of
// evaluations).  Evaluations j in [0, neval) are cut into tiles of 2^tile_log2
// (1024 or 2048) consecutive indices; a persistent grid walks the tiles
// round-robin.  A tile of n evaluations meets at most n / 2 + 3 hypercubes
// because n_h >= 2.  It stages their offsets, relative to the tile start, in
// shared memory.  Each thread takes n / 256 consecutive evaluations.  Every cube writes its index
// into a start-cube table for the threads whose first evaluation it holds; a
// thread starts there and steps forward.  No evaluation-to-cube array is ever
// built.
//
// Accumulation without global atomics (the paper's atomicAdd of Sec. 3.3.3):
//  * cube weights: every J f goes to a shared array.  The cubes that lie inside
//    the tile get their two-pass (count, mean, centred second moment) from
//    one thread, or from one warp for long runs.  A cube that crosses a tile
//    edge leaves a Carry record, and a fix-up kernel merges the records
//    (Chan's pairwise formula) in tile order.
//  * map weights: a per-CTA histogram.  The FP64 form adds with shared FP64
//    atomics.  The 32 lanes of a warp share a stratum on the high axes, so
//    their adds collide on a handful of bins; the FP64 histogram is therefore
//    kept in up to 16 copies, lane l adding into copy l mod copies.  Shared
//    floating-point atomics measured slower than integer ones, so the FP32
//    form adds in two phases per tile:
//    the tile's largest weight fixes a power-of-two scale, the weights go in
//    as 32-bit fixed-point integers through native shared integer atomics,
//    and every tile's totals are folded into float-float accumulators.
//    The per-CTA histograms are summed in a fixed order by a second kernel.
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

// Number of shared-memory elements of the derived parameters.  The Gaussian
// centres are padded to rows of DMAX so that a row loads as vectors.
__host__ __device__ inline int gauss_kp(int K) { return (K + 3) & ~3; }  // peaks padded to 4
__host__ __device__ inline int derived_smem_count(int integrand, int d, int dmax, int np) {
  if (integrand == VEGAS_GAUSS_SUM) {
    const int K = (np - 3) / d;
    return 4 + K * dmax + (dmax >= 16 ? dmax * gauss_kp(K) : 0);
  }
  if (integrand == VEGAS_PRODUCT_PEAK) return 2 * dmax;
  if (integrand == VEGAS_OSCILLATORY) return 4 + dmax;
  if (integrand == VEGAS_MOROKOFF_CAFLISCH) return 4;
  if (integrand == VEGAS_MAP_DENSITY) return np;
  return 0;
}

// Turn the caller's parameters into the derived form read by vg::integrand:
//   GAUSS_SUM         [A, c, K, sigma, mu rows of DMAX]  c = -log2(e)/(2 s^2) (FP32, exp2);
//                     FP64: sigma = sqrt(32/ln2)/s in slot 3 and the centres times sigma
//                     (the point comes scaled from the map table);
//                     FP32 with DMAX = 4: slot 3 holds sigma = sqrt(log2(e)/(2 s^2)), the
//                     centres are scaled by sigma and stored in pairs of peaks, [K/2][axis][2],
//                     so that one 16-byte load holds two axes of both peaks, an odd last peak
//                     as a row;
//                     for DMAX >= 16 followed by the centres by axis,
//                     [DMAX][K padded to 4], for the streamed point path
//   PRODUCT_PEAK      [c_i^-2 (DMAX), w (DMAX)]   padded axes: c^-2 = 1, w = 0
//   OSCILLATORY       [2 pi u, 0, 0, 0, a (DMAX)]
//   MOROKOFF_CAFLISCH [(1+1/d)^d, 1/d, 0, 0]
//   MAP_DENSITY       [edges (d*(G'+1))]
// FP64 Gaussian sum: the point and the centres are scaled by sqrt(32 / ln2) / s, so that a peak's squared scaled
// distance y gives its term e^(-r^2 / 2s^2) = 2^(-y/64) (exp2_64ths); the map table carries the scale
__host__ __device__ inline double gauss_scale64(double s) { return 0x1.b2da4e9808a53p+2 / fabs(s); }

template <int ID, typename T, int DMAX>
__device__ void prep_params(const double* __restrict__ raw, int np, int d, T* out) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if constexpr (ID == VEGAS_GAUSS_SUM) {
    const int K = (np - 3) / d;
    if constexpr (DMAX >= 16) {
      const int KP = gauss_kp(K);
      for (int i = tid; i < DMAX * KP; i += nt) {
        const int k = i / KP, q = i - k * KP;
        out[4 + K * DMAX + i] = (T)((k < d && q < K) ? raw[3 + q * d + k] : 0.0);
      }
    }
    // FP32 with four axes: the scale sigma = sqrt(log2(e) / (2 s^2)) in slot 3 and the centres times sigma, so
    // that a peak's term is 2^-(sum of squared scaled distances); FP64: sigma = gauss_scale64(s), the term
    // 2^(-y/64)
    constexpr bool kScaled = (sizeof(T) == 4 && DMAX == 4) || sizeof(T) == 8;
    const double sigma = sizeof(T) == 8 ? gauss_scale64(raw[1])
                         : kScaled      ? sqrt(0.5 * 1.4426950408889634) / fabs(raw[1])
                                        : 1.0;
    for (int i = tid; i < 4 + K * DMAX; i += nt) {
      double v = 0.0;
      if (i == 0) v = raw[0];
      else if (i == 1) v = (sizeof(T) == 8 ? -1.0 : -1.4426950408889634) / (2.0 * raw[1] * raw[1]);
      else if (i == 2) v = (double)K;
      else if (i == 3) v = kScaled ? sigma : 0.0;
      else if (i >= 4) {
        const int e = i - 4;
        int k = e / DMAX, j = e - k * DMAX;
        if (sizeof(T) == 4 && DMAX == 4 && e < (K & ~1) * DMAX) {  // the paired peaks
          const int r = e & (2 * DMAX - 1);
          k = 2 * (e / (2 * DMAX)) + (r & 1);
          j = 2 * (r >> 2) + ((r >> 1) & 1);
        }
        v = j < d ? raw[3 + k * d + j] * sigma : 0.0;
      }
      out[i] = (T)v;
    }
  } else if constexpr (ID == VEGAS_PRODUCT_PEAK) {
    for (int i = tid; i < 2 * DMAX; i += nt) {
      const int j = i % DMAX;
      double v = i < DMAX ? 1.0 : 0.0;  // padded axes: c^-2 = 1, w = 0
      if (j < d) v = i < DMAX ? 1.0 / (raw[j] * raw[j]) : raw[d + j];
      out[i] = (T)v;
    }
  } else if constexpr (ID == VEGAS_OSCILLATORY) {
    for (int i = tid; i < 4 + DMAX; i += nt) {
      double v = 0.0;
      if (i == 0) v = 6.283185307179586 * raw[0];
      else if (i >= 4 && i - 4 < d) v = raw[1 + (i - 4)];
      out[i] = (T)v;
    }
  } else if constexpr (ID == VEGAS_MOROKOFF_CAFLISCH) {
    if (tid == 0) {
      out[0] = (T)pow(1.0 + 1.0 / d, (double)d);
      out[1] = (T)(1.0 / d);
      out[2] = out[3] = T(0);
    }
  } else if constexpr (ID == VEGAS_MAP_DENSITY) {
    for (int i = tid; i < np; i += nt) out[i] = (T)raw[i];
  }
}

// 2^x with the special-function unit (ex2.approx.ftz: about 2 ulp, results
// below 2^-126 flush to zero)
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// log2 with the special-function unit, for the FP32 form's allocation
// weight: the counts are a reproducible function of the weight's bits, so the
// weight itself only has to be deterministic.
__device__ __forceinline__ float log2_fast(float x) { return __log2f(x); }

// Packed FP32 pairs (sm_100-family f32x2 arithmetic): one instruction does two
// independent IEEE single operations with round-to-nearest.  Each lane
// rounds as the scalar operation would.  The fill is issue-bound, so this
// halves the issue cost of the paired arithmetic.
__device__ __forceinline__ uint64_t pk2(float lo, float hi) {
  return ((uint64_t)__float_as_uint(hi) << 32) | __float_as_uint(lo);
}
__device__ __forceinline__ float lo2(uint64_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float hi2(uint64_t v) { return __uint_as_float((uint32_t)(v >> 32)); }
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// One padded row of DMAX parameters from 16-byte aligned shared memory, as
// 16-byte vector loads.
template <typename T, int DMAX>
__device__ __forceinline__ void load_row(const T* __restrict__ p, T (&out)[DMAX]) {
  if constexpr (sizeof(T) == 4 && DMAX % 4 == 0) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int i = 0; i < DMAX / 4; ++i) {
      const float4 v = q[i];
      out[4 * i] = v.x;
      out[4 * i + 1] = v.y;
      out[4 * i + 2] = v.z;
      out[4 * i + 3] = v.w;
    }
  } else if constexpr (sizeof(T) == 8 && DMAX % 2 == 0) {
    const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
    for (int i = 0; i < DMAX / 2; ++i) {
      const double2 v = q[i];
      out[2 * i] = v.x;
      out[2 * i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < DMAX; ++i) out[i] = p[i];
  }
}

// f(x) with the derived parameters p (shared memory) and the scalars s0, s1,
// K loaded into registers once per thread.
template <int ID, typename T, int DMAX>
__device__ __forceinline__ T integrand(const T (&x)[DMAX], int d, const T* __restrict__ p, int np, T s0, T s1,
                                       int K) {
  if constexpr (ID == VEGAS_GAUSS_SUM && sizeof(T) == 4 && DMAX == 4) {
    // FP32, four axes: two peaks a step, each packed operation doing one axis of both, one packed accumulate a
    // pair.  Point and centres are scaled by sigma (slot 3), so a peak's term is 2^-r with r its squared scaled
    // distance.  The 1000-Gaussian ridge, 5e6 evaluations: fill 2.33 ms with pairs of axes, 2.21 with pairs of
    // peaks, 2.12 scaled, 1.96 with four pairs a loop step (1.95 with eight)
    const float sg = p[3];
    const float y0 = x[0] * sg, y1 = x[1] * sg, y2 = x[2] * sg, y3 = x[3] * sg;
    const uint64_t x0 = pk2(y0, y0), x1 = pk2(y1, y1), x2 = pk2(y2, y2), x3 = pk2(y3, y3);
    const float4* mu = reinterpret_cast<const float4*>(p + 4);
    uint64_t acc2 = 0ull;  // (+0, +0)
    int k = 0;
#pragma unroll 4
    for (; k + 1 < K; k += 2, mu += 2) {
      const float4 ma = mu[0], mb = mu[1];
      const uint64_t d0 = sub2(x0, pk2(ma.x, ma.y)), d1 = sub2(x1, pk2(ma.z, ma.w));
      const uint64_t d2 = sub2(x2, pk2(mb.x, mb.y)), d3 = sub2(x3, pk2(mb.z, mb.w));
      uint64_t r2 = mul2(d0, d0);
      r2 = fma2(d1, d1, r2);
      r2 = fma2(d2, d2, r2);
      r2 = fma2(d3, d3, r2);
      acc2 = add2(acc2, pk2(ex2_approx(-lo2(r2)), ex2_approx(-hi2(r2))));
    }
    float acc = lo2(acc2) + hi2(acc2);
    if (k < K) {  // an odd last peak, stored as a row
      const float4 m = *reinterpret_cast<const float4*>(p + 4 + 4 * k);
      const float e0 = y0 - m.x, e1 = y1 - m.y, e2 = y2 - m.z, e3 = y3 - m.w;
      acc += ex2_approx(-fmaf(e3, e3, fmaf(e2, e2, fmaf(e1, e1, e0 * e0))));
    }
    return s0 * acc;
  } else if constexpr (ID == VEGAS_GAUSS_SUM && sizeof(T) == 4 && DMAX % 4 == 0) {
    // FP32: the squared distance in packed pairs of axes, then one exp2 per peak
    uint64_t xp[DMAX / 2];
#pragma unroll
    for (int i = 0; i < DMAX / 2; ++i) xp[i] = pk2(x[2 * i], x[2 * i + 1]);
    const float4* mu = reinterpret_cast<const float4*>(p + 4);
    float acc = 0.0f;
#pragma unroll 2
    for (int k = 0; k < K; ++k, mu += DMAX / 4) {
      uint64_t r2 = 0ull;  // (+0, +0)
#pragma unroll
      for (int i = 0; i < DMAX / 4; ++i) {
        const float4 m = mu[i];
        const uint64_t d0 = sub2(xp[2 * i], pk2(m.x, m.y));
        r2 = fma2(d0, d0, r2);
        const uint64_t d1 = sub2(xp[2 * i + 1], pk2(m.z, m.w));
        r2 = fma2(d1, d1, r2);
      }
      acc += ex2_approx((lo2(r2) + hi2(r2)) * s1);
    }
    return s0 * acc;
  } else if constexpr (ID == VEGAS_GAUSS_SUM) {
    const T* mu = p + 4;
    T acc = T(0);
    for (int k = 0; k < K; ++k, mu += DMAX) {
      T m[DMAX];
      load_row<T, DMAX>(mu, m);
      T r2 = T(0);
#pragma unroll
      for (int j = 0; j < DMAX; ++j) {
        const T dx = x[j] - m[j];  // padded axes hold x = mu = 0
        r2 = fma(dx, dx, r2);
      }
      if constexpr (sizeof(T) == 8) acc += exp2_64ths(-r2);  // point and centres scaled: r2 = 64 log2(e) r^2/2s^2
      else acc += ex2_approx(r2 * s1);
    }
    return s0 * acc;
  } else if constexpr (ID == VEGAS_PRODUCT_PEAK && sizeof(T) == 4 && DMAX % 4 == 0) {
    // FP32: denominators of two axes per packed operation, one division per four axes
    float r = 1.0f;
#pragma unroll
    for (int g = 0; g < DMAX / 4; ++g) {
      const float4 c2 = reinterpret_cast<const float4*>(p)[g];
      const float4 w = reinterpret_cast<const float4*>(p + DMAX)[g];
      const uint64_t d0 = sub2(pk2(x[4 * g], x[4 * g + 1]), pk2(w.x, w.y));
      const uint64_t d1 = sub2(pk2(x[4 * g + 2], x[4 * g + 3]), pk2(w.z, w.w));
      const uint64_t e0 = fma2(d0, d0, pk2(c2.x, c2.y)), e1 = fma2(d1, d1, pk2(c2.z, c2.w));
      const uint64_t e = mul2(e0, e1);  // padded axes: x = w = 0 and c^-2 = 1, a factor of 1
      r = r / (lo2(e) * hi2(e));
    }
    return r;
  } else if constexpr (ID == VEGAS_PRODUCT_PEAK) {
    // product of the denominators in groups of four, one division per group
    T r = T(1), den = T(1);
#pragma unroll
    for (int j = 0; j < DMAX; ++j) {
      if (j < d) {
        const T dx = x[j] - p[DMAX + j];
        den *= fma(dx, dx, p[j]);
      }
      if ((j & 3) == 3 || j == DMAX - 1) {
        r = r / den;
        den = T(1);
      }
    }
    return r;
  } else if constexpr (ID == VEGAS_OSCILLATORY) {
    T arg = s0;
#pragma unroll
    for (int j = 0; j < DMAX; ++j) arg = fma(p[4 + j], x[j], arg);
    return cos(arg);
  } else if constexpr (ID == VEGAS_SIN_EXP) {
    if constexpr (sizeof(T) == 8) return sin(x[0]) + exp(x[1 % DMAX]);
    else return sinf(x[0]) + expf(x[1 % DMAX]);
  } else if constexpr (ID == VEGAS_LINEAR) {
    T s = T(0);
#pragma unroll
    for (int j = 0; j < DMAX; ++j) s += x[j];
    return s;
  } else if constexpr (ID == VEGAS_COSINE) {
    T r = T(1);
#pragma unroll
    for (int j = 0; j < DMAX; ++j)
      if (j < d) r *= cos(x[j]);
    return r;
  } else if constexpr (ID == VEGAS_EXPONENTIAL) {
    T s = T(0);
#pragma unroll
    for (int j = 0; j < DMAX; ++j) s = fma(x[j], x[j], s);
    if constexpr (sizeof(T) == 8) return exp(s);
    else return expf(s);
  } else if constexpr (ID == VEGAS_ROOS_ARNOLD) {
    T r = T(1);
#pragma unroll
    for (int j = 0; j < DMAX; ++j)
      if (j < d) r *= fabs(fma(T(4), x[j], T(-2)));
    return r;
  } else if constexpr (ID == VEGAS_MOROKOFF_CAFLISCH) {
    T r = s0;
#pragma unroll
    for (int j = 0; j < DMAX; ++j)
      if (j < d) r *= pow(x[j], s1);
    return r;
  } else {  // VEGAS_MAP_DENSITY
    const int G = np / d - 1;
    T r = T(1);
#pragma unroll
    for (int j = 0; j < DMAX; ++j) {
      if (j < d) {
        const T* e = p + j * (G + 1);
        int lo = 0, hi = G - 1;  // largest i in [0, G-1] with e[i] <= x
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (e[mid] <= x[j]) lo = mid;
          else hi = mid - 1;
        }
        r *= T(1) / (T(G) * (e[lo + 1] - e[lo]));
      }
    }
    return r;
  }
}

// Philox4x32-10 with the round keys precomputed on the host (kernel
// parameters): rk0[r] = key0 + r * 0x9E3779B9, rk1[r] = key1 + r * 0xBB67AE85.
__device__ __forceinline__ uint4 philox_rk(uint4 c, const uint32_t* rk0, const uint32_t* rk1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk0[round], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ rk1[round],
                   (uint32_t)p0);
  }
  return c;
}

// Two Philox4x32-10 blocks in lockstep.  The rounds of one block form a
// dependent chain; two independent chains interleaved halve its stalls.
__device__ __forceinline__ void philox_rk_x2(uint4& c, uint4& e, const uint32_t* rk0, const uint32_t* rk1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
    const uint64_t q0 = (uint64_t)0xD2511F53u * e.x, q1 = (uint64_t)0xCD9E8D57u * e.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk0[round], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ rk1[round],
                   (uint32_t)p0);
    e = make_uint4((uint32_t)(q1 >> 32) ^ e.y ^ rk0[round], (uint32_t)q1, (uint32_t)(q0 >> 32) ^ e.w ^ rk1[round],
                   (uint32_t)q0);
  }
}

// Coordinates c_k of cube h (axis 0 fastest), by multiplication with the
// magic reciprocals.  In the FP32 form they are kept as the high bits of a
// float in [2^23, 2^24): 0x4B000000 | c_k << b_k, with b_k fraction bits.
template <typename T, int DMAX, bool EXACT>
__device__ __forceinline__ void decode_cube(const FillArgs& a, uint32_t h, uint32_t (&cb)[DMAX]) {
  uint32_t rest = h;
#pragma unroll
  for (int k = 0; k < DMAX; ++k) {
    cb[k] = 0u;
    if (EXACT || k < a.d) {
      const uint32_t q = (uint32_t)(((uint64_t)rest * a.magic[k]) >> a.shift[k]);  // rest / s_k
      const uint32_t ck = rest - q * a.nstrat[k];
      rest = q;
      if constexpr (sizeof(T) == 8) cb[k] = ck;
      else cb[k] = 0x4B000000u | (ck << a.fbits[k]);
    }
  }
}

// Coordinates of cube h + 1 from those of cube h, in the encoding of
// decode_cube: one added to axis 0 and carried upwards (an odometer).  A
// thread's consecutive evaluations stay in a cube or move forward by whole
// cubes (one when every cube holds at least two evaluations, as the
// allocation guarantees), so after one full decode a step costs an add and a
// compare; the carry into axis k is taken once in s_0 ... s_{k-1} steps.
template <typename T, int DMAX, bool EXACT>
__device__ __forceinline__ void next_cube(const FillArgs& a, uint32_t (&cb)[DMAX]) {
#pragma unroll
  for (int k = 0; k < DMAX; ++k) {
    if (EXACT || k < a.d) {
      const uint32_t one = sizeof(T) == 8 ? 1u : (1u << a.fbits[k]);
      const uint32_t zero = sizeof(T) == 8 ? 0u : 0x4B000000u;
      cb[k] += one;
      if (cb[k] < zero + a.nstrat[k] * one) return;
      cb[k] = zero;
    }
  }
}

// RN(V) 2^-53 for a 64-bit integer V, by integer arithmetic: normalise, round the 64 bits to 53 (to nearest,
// ties to even) and assemble the exponent.  Equal to __ull2double_rn(V) * 2^-53, bit for bit (checked on the
// host against the IEEE conversion on 5e7 values with the ties and the zero); on GB300 the FP64 conversions
// take issue slots of the FP64 pipe, the integer operations do not (the d = 8 FP64 fill: 49.9 -> 44.8 ms with
// this and the floor below).
__device__ __forceinline__ double rn_u64_2m53(uint64_t V) {
  const int lz = __clzll(V);
  const uint64_t m = V << (lz & 63);
  uint64_t q = m >> 11;
  const uint32_t rem = (uint32_t)m & 0x7FFu;
  q += (uint64_t)((rem > 0x400u) | ((rem == 0x400u) & ((uint32_t)q & 1u)));
  const uint64_t db = ((uint64_t)(1033 - lz) << 52) + q - (1ull << 52);
  return __longlong_as_double(V ? (long long)db : 0ll);
}

// Point of evaluation j in the cube with coordinates cb: Philox words, the
// position z = (c + u) N_g / s_k, interval i = min(floor z, N_g - 1), the
// point x = e_i + (z - i) dx_i and the Jacobian J = prod N_g dx_i.
//   FP64: u has 53 bits; z = RN(RN(c + u) * g) in FP64.
//   FP32: v = c 2^b + (w >> (32 - b)) < 2^23, so c + u = v 2^-b is exact; the
//         float 2^23 + v is assembled from bits, and z = RN(v g 2^-b) is one
//         fused multiply-add with the exact constant -2^23 g 2^-b.
// Axes beyond d get x = 0 (the padded integrand parameters match).  J0 is the
// starting value of the Jacobian product: the value scale of the FP32 form.
template <typename T, int DMAX, bool EXACT>
__device__ __forceinline__ void make_point(const FillArgs& a, const uint32_t* __restrict__ rk0,
                                           const uint32_t* __restrict__ rk1, const uint32_t (&cb)[DMAX], int64_t j,
                                           const TabEntry<T>* __restrict__ tab, T (&x)[DMAX], int (&bin)[DMAX],
                                           T& J, T J0) {
  const int G = a.G;
  J = J0;
  uint4 r = make_uint4(0u, 0u, 0u, 0u);
  const uint32_t jlo = (uint32_t)j, jhi = (uint32_t)((uint64_t)j >> 32);
  // FP32 with exactly 8 axes: both blocks of the point at once
  constexpr bool kPair = sizeof(T) == 4 && EXACT && DMAX == 8;
  uint4 ra = make_uint4(jlo, jhi, a.iter, a.pid << 16), rb = make_uint4(jlo, jhi, a.iter, (a.pid << 16) | 1u);
  if constexpr (kPair) philox_rk_x2(ra, rb, rk0, rk1);
#pragma unroll
  for (int k = 0; k < DMAX; ++k) {
    x[k] = T(0);
    bin[k] = 0;
    if (EXACT || k < a.d) {
      int i;
      T dz;
      if constexpr (sizeof(T) == 8) {
        if ((k & 1) == 0) r = philox_rk(make_uint4(jlo, jhi, a.iter, (a.pid << 16) | (uint32_t)(k >> 1)), rk0, rk1);
        const uint32_t whi = (k & 1) ? r.z : r.x, wlo = (k & 1) ? r.w : r.y;
        const uint64_t bits = (((uint64_t)whi << 32) | wlo) >> 11;
        double z;
        if (cb[k] < 2048u) {
          // c + u = (c 2^53 + bits) 2^-53 with the integer exact in 64 bits: rounding it to 53 bits and scaling
          // by 2^-53 gives RN(c + u), so z = RN(RN(c + u) N_g / s)
          z = __dmul_rn(rn_u64_2m53(((uint64_t)cb[k] << 53) | bits), a.gz64[k]);
        } else {
          const double u = __dmul_rn(__ull2double_rn(bits), 0x1p-53);
          z = __dmul_rn(__dadd_rn((double)cb[k], u), a.gz64[k]);
        }
        // floor of z from its bits (0 <= z < 2^21): exponent e, the integer part of the mantissa, and the
        // double floor(z) with the fraction bits cleared; integer operations instead of two conversions
        const uint32_t zh = (uint32_t)__double2hiint(z);
        const int e = (int)(zh >> 20) - 1023;
        const bool ge1 = e >= 0;
        const int sh = ge1 ? 20 - e : 0;  // 8 .. 20 for 1 <= z < 8192
        int iz = ge1 ? (int)(((zh & 0xFFFFFu) | 0x100000u) >> sh) : 0;
        double fl = __hiloint2double(ge1 ? (int)(zh & (0xFFFFFFFFu << sh)) : 0, 0);
        if (iz > G - 1) {
          iz = G - 1;
          fl = (double)(G - 1);
        }
        i = iz;
        dz = z - fl;  // exact
      } else {
        if constexpr (kPair) r = k < 4 ? ra : rb;
        else if ((k & 3) == 0) r = philox_rk(make_uint4(jlo, jhi, a.iter, (a.pid << 16) | (uint32_t)(k >> 2)), rk0, rk1);
        const uint32_t w = (k & 3) == 0 ? r.x : (k & 3) == 1 ? r.y : (k & 3) == 2 ? r.z : r.w;
        const float big = __uint_as_float(cb[k] | (w >> (32 - a.fbits[k])));  // 2^23 + v
        const float z = fmaf(big, a.gzb32[k], a.gzn32[k]);                     // RN(v g 2^-b)
        i = (int)z;  // z >= 0: truncation is floor
        i = i < G - 1 ? i : G - 1;
        dz = z - (float)i;  // exact
      }
      const TabEntry<T> te = tab[VG_IDX(k * G + i, a.d * G, a.flags, 1)];
      x[k] = fma(dz, te.dx, te.e);
      J = J * te.jk;
      bin[k] = i;
    }
  }
}

// ---------------------------------------------------------------------------
// Streamed FP32 point path for wide maps (DMAX >= 16).  The array path holds
// the cube digits, the coordinates and the intervals of all axes in registers
// (172 and 254 registers a thread at 16 and 32 axes).  The streamed path makes
// the point four axes at a time (one Philox call) and folds every coordinate
// into the integrand's running sums or products at once, so a thread holds
// only those: it fits in 64 registers.  The cube digits come packed, 8 bits
// an axis (every s_k <= 256), and the intervals go straight to the packed
// words of the two-phase histogram.  Families: the Gaussian sum with at most
// kStreamMaxPeaks peaks, and every family whose value is a sum or a product
// over the axes.
// ---------------------------------------------------------------------------
constexpr int kStreamMaxPeaks = 8;

// Slot of tile evaluation jl in the per-evaluation arrays written by one
// thread and read back by the same thread (map weights, packed intervals).
// Thread t owns evaluations S t .. S t + S - 1 (S = 2^spt_log2 a thread), so
// storing them at jl would put the lanes of a warp S (or S * words) apart and
// make them collide on a few shared-memory banks; slot (jl mod S) * 256 + jl / S
// puts them on consecutive words.  The packed intervals add word w * tile.
__device__ __forceinline__ int tix(int jl, int spt_log2) {
  return ((jl & ((1 << spt_log2) - 1)) << 8) | (jl >> spt_log2);
}

__host__ __device__ inline bool stream_family(int integrand, int K) {
  switch (integrand) {
    case VEGAS_GAUSS_SUM: return K <= kStreamMaxPeaks;
    case VEGAS_PRODUCT_PEAK:
    case VEGAS_OSCILLATORY:
    case VEGAS_LINEAR:
    case VEGAS_COSINE:
    case VEGAS_EXPONENTIAL:
    case VEGAS_ROOS_ARNOLD:
    case VEGAS_MOROKOFF_CAFLISCH:
    case kIntegrandTabulated:
    case kIntegrandPoints: return true;
    default: return false;
  }
}

// digits c_k of cube h, 8 bits each, four axes a word
template <int DMAX>
__device__ __forceinline__ void decode_packed(const FillArgs& a, uint32_t h, uint32_t (&cw)[DMAX / 4]) {
  uint32_t rest = h;
#pragma unroll
  for (int g = 0; g < DMAX / 4; ++g) {
    uint32_t w = 0u;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = 4 * g + q;
      if (k < a.d) {
        const uint32_t qq = (uint32_t)(((uint64_t)rest * a.magic[k]) >> a.shift[k]);
        w |= (rest - qq * a.nstrat[k]) << (8 * q);
        rest = qq;
      }
    }
    cw[g] = w;
  }
}

// Point j of the cube with digits cw, its Jacobian J (from J0) and f there.
// binw_col receives the packed intervals (4 or 2 axes a word, word w at
// binw_col[w * tile], tile = 2^a.tile_log2); xout, if not NULL,
// the coordinates.
template <int ID, int DMAX>
__device__ __forceinline__ float stream_point_eval(const FillArgs& a, const uint32_t* __restrict__ rk0,
                                                   const uint32_t* __restrict__ rk1, const uint32_t (&cw)[DMAX / 4],
                                                   int64_t j, const TabEntry<float>* __restrict__ tab,
                                                   const float* __restrict__ prm, float s0, float s1, int K,
                                                   float& J, uint32_t* __restrict__ binw_col,
                                                   float* __restrict__ xout) {
  const int d = a.d, G = a.G;
  const uint32_t jlo = (uint32_t)j, jhi = (uint32_t)((uint64_t)j >> 32);
  float r2[kStreamMaxPeaks];
#pragma unroll
  for (int q = 0; q < kStreamMaxPeaks; ++q) r2[q] = 0.0f;
  float acc = (ID == VEGAS_OSCILLATORY) ? s0 : 0.0f;
  float prod = 1.0f;
  const int KP = gauss_kp(K);
  const float* muT = prm + 4 + K * DMAX;
  const int ng = (d + 3) >> 2;
#pragma unroll 1
  for (int g = 0; g < ng; ++g) {
    const uint4 r = philox_rk(make_uint4(jlo, jhi, a.iter, (a.pid << 16) | (uint32_t)g), rk0, rk1);
    uint32_t word = 0u, w16a = 0u, w16b = 0u;
    float den = 1.0f;
    float xv[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    uint32_t dig = 0u;
#pragma unroll
    for (int gg = 0; gg < DMAX / 4; ++gg)
      if (gg == g) dig = cw[gg];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = 4 * g + q;
      if (k < d) {
        const uint32_t w = q == 0 ? r.x : q == 1 ? r.y : q == 2 ? r.z : r.w;
        const uint32_t fb = a.fbits[k];
        const float big = __uint_as_float(0x4B000000u | (((dig >> (8 * q)) & 255u) << fb) | (w >> (32 - fb)));
        const float z = fmaf(big, a.gzb32[k], a.gzn32[k]);
        int i = (int)z;
        i = i < G - 1 ? i : G - 1;
        const float dz = z - (float)i;
        const TabEntry<float> te = tab[VG_IDX(k * G + i, a.d * G, a.flags, 2)];
        const float x = fmaf(dz, te.dx, te.e);
        J = J * te.jk;
        word |= (uint32_t)i << (8 * q);
        if (q < 2) w16a |= (uint32_t)i << (16 * q);
        else w16b |= (uint32_t)i << (16 * (q - 2));
        xv[q] = x;
        if constexpr (ID == VEGAS_GAUSS_SUM) {
          const float4* m4 = reinterpret_cast<const float4*>(muT + k * KP);
#pragma unroll
          for (int p4 = 0; p4 < kStreamMaxPeaks / 4; ++p4) {
            if (4 * p4 < KP) {
              const float4 m = m4[p4];
              const float e0 = x - m.x, e1 = x - m.y, e2 = x - m.z, e3 = x - m.w;
              r2[4 * p4] = fmaf(e0, e0, r2[4 * p4]);
              r2[4 * p4 + 1] = fmaf(e1, e1, r2[4 * p4 + 1]);
              r2[4 * p4 + 2] = fmaf(e2, e2, r2[4 * p4 + 2]);
              r2[4 * p4 + 3] = fmaf(e3, e3, r2[4 * p4 + 3]);
            }
          }
        } else if constexpr (ID == VEGAS_PRODUCT_PEAK) {
          const float e = x - prm[DMAX + k];
          den *= fmaf(e, e, prm[k]);
        } else if constexpr (ID == VEGAS_OSCILLATORY) {
          acc = fmaf(prm[4 + k], x, acc);
        } else if constexpr (ID == VEGAS_LINEAR) {
          acc += x;
        } else if constexpr (ID == VEGAS_COSINE) {
          prod *= cosf(x);
        } else if constexpr (ID == VEGAS_EXPONENTIAL) {
          acc = fmaf(x, x, acc);
        } else if constexpr (ID == VEGAS_ROOS_ARNOLD) {
          prod *= fabsf(fmaf(4.0f, x, -2.0f));
        } else if constexpr (ID == VEGAS_MOROKOFF_CAFLISCH) {
          prod *= powf(x, s1);
        }
      }
    }
    if (xout) {  // the point's four coordinates: one 16-byte store when rows are 16-byte aligned
      if ((d & 3) == 0) {
        *reinterpret_cast<float4*>(xout + 4 * g) = make_float4(xv[0], xv[1], xv[2], xv[3]);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (4 * g + q < d) xout[4 * g + q] = xv[q];
      }
    }
    if (binw_col) {
      if (a.bin_shift == 3) {
        binw_col[(g << a.tile_log2)] = word;
      } else {
        binw_col[(2 * g) << a.tile_log2] = w16a;
        if (4 * g + 2 < d) binw_col[(2 * g + 1) << a.tile_log2] = w16b;
      }
    }
    if constexpr (ID == VEGAS_PRODUCT_PEAK) prod = prod / den;  // one division per four axes
  }
  if constexpr (ID == VEGAS_GAUSS_SUM) {
    float sum = 0.0f;
#pragma unroll
    for (int q = 0; q < kStreamMaxPeaks; ++q)
      if (q < K) sum += ex2_approx(r2[q] * s1);
    return s0 * sum;
  } else if constexpr (ID == VEGAS_OSCILLATORY) {
    return cosf(acc);
  } else if constexpr (ID == VEGAS_LINEAR) {
    return acc;
  } else if constexpr (ID == VEGAS_EXPONENTIAL) {
    return expf(acc);
  } else if constexpr (ID == VEGAS_MOROKOFF_CAFLISCH) {
    return s0 * prod;
  } else {  // PRODUCT_PEAK, COSINE, ROOS_ARNOLD; tabulated and points: unused
    return prod;
  }
}

// Asynchronous 8-byte global -> shared copies (cp.async, no registers held):
// the single-integral fill loads the next tile's cube offsets while it
// computes the current one.
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Shared-memory views of the fill and the per-thread running state; one tile
// of evaluations is processed by fill_tile, which both the single-integral and
// the batched kernels call.
template <typename T>
struct FillShared {
  TabEntry<T>* tab;
  T* hist_s;          // direct mode: shared histogram of T
  uint32_t* hist_u;   // two-phase: fixed-point tile histogram
  ff* hist_acc;       // two-phase: float-float CTA histogram (acc32 == 0)
  float* hist_accf;   // two-phase: FP32 CTA histogram (acc32 == 1), the same bytes
  uint32_t* binw;     // two-phase: intervals of an evaluation, 4 or 2 per word
  float* wv_s;        // two-phase: map weight of every evaluation
  T* prm;
  int* off_r;         // cube offsets relative to the tile, clamped to +-2^30
  int64_t* raw_off;   // prefetched global offsets of the cubes a tile can meet (single-integral fill)
  T* invn;
  T* vals;
  int* longlist;
  int* startc;        // cube of every thread's first evaluation
  int* misc;          // [0] long count, [1] cubes in tile; single-integral fill: [2] first cube and [3] cubes
                     // that the next tile can meet, whose offsets are being prefetched
  float* wmax;        // [8] per-warp max of the map weight
  double* red;
};

template <typename T>
__device__ __forceinline__ FillShared<T> fill_shared(unsigned char* smem, const FillArgs& a, bool table_in_smem) {
  FillShared<T> S;
  S.tab = table_in_smem ? (TabEntry<T>*)(smem + a.sm_table) : (TabEntry<T>*)a.gtable;
  S.hist_s = (T*)(smem + a.sm_hist);
  S.hist_u = (uint32_t*)(smem + a.sm_hist);
  S.hist_acc = (ff*)(smem + a.sm_hacc);
  S.hist_accf = (float*)(smem + a.sm_hacc);
  S.binw = (uint32_t*)(smem + a.sm_bins);
  S.wv_s = (float*)(smem + a.sm_wv);
  S.prm = (T*)(smem + a.sm_params);
  S.off_r = (int*)(smem + a.sm_off);
  S.raw_off = (int64_t*)(smem + a.sm_raw);
  S.invn = (T*)(smem + a.sm_invn);
  S.vals = (T*)(smem + a.sm_vals);
  S.longlist = (int*)(smem + a.sm_long);
  S.startc = (int*)(smem + a.sm_start);
  S.misc = (int*)(smem + a.sm_misc);
  S.wmax = (float*)(smem + a.sm_misc + 16);
  S.red = (double*)(smem + a.sm_misc + 64);
  return S;
}

template <typename T>
struct FillState {
  Acc<T> acc_i, acc_v;
  float lmax = -__builtin_huge_valf();
  bool bad = false;
  float inv_scale = 0.0f;  // two-phase: 1/scale of the tile histogram waiting to be folded
  int vexp = 0;            // FP32: the evaluations carry J f 2^-vexp
  T J0 = T(1);             // 2^-vexp
};

// Power-of-two value scale of the FP32 form.  Cube sums of (J f)^2 must stay
// in FP32 range; a product peak in d = 12 reaches |f| = prod c_i^2 ~ 1e28.
// From a bound B of |f| (prod c_i^2 for PRODUCT_PEAK, |A| K for GAUSS_SUM),
// e = floor(log2(B) / 2), so the scaled peak value is about sqrt(B).  The
// scaling is exact, so it changes no rounding until the FP64 outputs, where
// 2^e (sums of J f) and 2^2e (sums of its square) are multiplied back.  Host
// and device compute it the same way: products of frexp mantissas.
__host__ __device__ inline int value_exponent(int integrand, int d, const double* raw, int np) {
  double m = 1.0;
  int E = 0, k = 0;
  if (integrand == VEGAS_PRODUCT_PEAK && np >= d) {
    for (int i = 0; i < d; ++i) {
      m *= frexp(fabs(raw[i]), &k);
      E += k;
      m = frexp(m, &k);
      E += k;
    }
    E = 2 * E;  // B = (prod c_i)^2 = m^2 2^(2E) with m in [0.5, 1)
    m = frexp(m * m, &k);
    E += k;
  } else if (integrand == VEGAS_GAUSS_SUM && np >= 3) {
    m = frexp(fabs(raw[0]) * raw[2], &E);
  } else {
    return 0;
  }
  if (!(m > 0.0) || !(m < 1.0)) return 0;  // a zero, infinite or NaN bound: no scale
  const int e = (E - 1) >> 1;              // B in [2^(E-1), 2^E)
  return e < 0 ? 0 : (e > 120 ? 120 : e);
}

// map table {xs e, xs dx, N_g dx} from the FP64 edges (xs: the point's scale, 1 but for the FP64 Gaussian sum),
// and zeroed histograms
template <typename T>
__device__ __forceinline__ void fill_prologue(const FillArgs& a, const FillShared<T>& S, int d, bool table_in_smem,
                                              double xs) {
  const int G = a.G, dG = d * G, tid = threadIdx.x;
  if (table_in_smem) {
    for (int b = tid; b < dG; b += kFillThreads) {
      const int k = b / G, i = b - k * G;
      const double e0 = a.edges[k * (G + 1) + i], e1 = a.edges[k * (G + 1) + i + 1];
      const double dx = __dsub_rn(e1, e0), jk = __dmul_rn((double)G, dx);
      S.tab[b] = TabEntry<T>{(T)(e0 * xs), (T)(dx * xs), (T)jk, T(0)};
    }
  }
  if (a.hist_mode == kHistShared)
    for (int b = tid; b < (dG << a.hist_rep_log2); b += kFillThreads) S.hist_s[b] = T(0);
  if (a.hist_mode == kHistTwoPhase)
    for (int b = tid; b < dG; b += kFillThreads) {
      S.hist_u[b] = 0u;
      if (a.acc32) S.hist_accf[b] = 0.0f;
      else S.hist_acc[b] = ff{0.0f, 0.0f};
    }
}

// One tile of 2^a.tile_log2 evaluations of integral a (tile index local to a).  rk0 /
// rk1: the Philox round keys (kernel parameters, so that they are
// constant-bank operands).  STREAM: the streamed point path (FP32, DMAX >= 16,
// two-phase histogram, s_k <= 256).
// TLC: the tile's log2 at compile time (the exact-d kernels are built for both sizes), 0 to read a.tile_log2.
template <int ID, typename T, int DMAX, bool EXACT, bool STREAM = false, bool PREFETCH = false, int TLC = 0>
__device__ __forceinline__ void fill_tile(const FillArgs& a, const uint32_t* __restrict__ rk0,
                                          const uint32_t* __restrict__ rk1, const FillShared<T>& S,
                                          FillState<T>& st, int tile, T ps0, T ps1, int pK, double* hist_g,
                                          int next_tile = 0) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int d = EXACT ? DMAX : a.d, G = a.G, dG = d * a.G;
  const bool two_phase = a.hist_mode == kHistTwoPhase;
  // intervals per packed word: 4 (8 bits) or 2 (16 bits); the exact-d path runs with N_g <= 256 only
  const int bpw = EXACT ? 4 : (32 >> a.bin_shift);
  const int nw = (d + bpw - 1) / bpw;
  TabEntry<T>* tab = S.tab;
  T* hist_s = S.hist_s;
  uint32_t* hist_u = S.hist_u;
  ff* hist_acc = S.hist_acc;
  uint32_t* binw = S.binw;
  float* wv_s = S.wv_s;
  T* prm = S.prm;
  int* off_r = S.off_r;
  T* invn = S.invn;
  T* vals = S.vals;
  int* longlist = S.longlist;
  int* startc = S.startc;
  int* misc = S.misc;
  float* wmax = S.wmax;
  auto& acc_i = st.acc_i;
  auto& acc_v = st.acc_v;
  float& lmax = st.lmax;
  bool& bad = st.bad;
  float& inv_scale = st.inv_scale;
  const int TL = TLC ? TLC : a.tile_log2, tileN = 1 << TL, spt_log2 = TL - 8, spt = 1 << spt_log2;
  const int maxc = tile_max_cubes(tileN);
  const int64_t j0 = (int64_t)tile << TL;
  const int len = (int)min((int64_t)tileN, a.neval - j0);
  constexpr int kRelCap = 1 << 30;
  // first cube of the tile and the number of cubes it can meet (up to the
  // next tile's first cube); with PREFETCH the previous tile left them, and
  // the cubes' global offsets, in shared memory
  int h0, ncand;
  int nh0 = 0, nend = 0;
  if constexpr (PREFETCH) {
    h0 = misc[2];
    ncand = misc[3];
    if (next_tile < a.ntiles) {  // bounds of the next tile, needed once this tile's prologue is done
      nh0 = a.tile_first[next_tile];
      nend = next_tile + 1 < a.ntiles ? a.tile_first[next_tile + 1] : a.NH - 1;
    }
  } else {
    h0 = a.tile_first[tile];
    ncand = min(maxc, (tile + 1 < a.ntiles ? a.tile_first[tile + 1] : a.NH - 1) - h0 + 1);
  }

  // ---- fold the previous tile's fixed-point histogram ----
  if (two_phase && inv_scale > 0.0f) {
    for (int b = tid; b < dG; b += kFillThreads) {
      const uint32_t q = hist_u[b];
      if (q) {
        if (a.acc32) S.hist_accf[b] += __fmul_rn((float)q, inv_scale);
        else hist_acc[b] = ff_add(hist_acc[b], __fmul_rn((float)q, inv_scale));
        hist_u[b] = 0u;
      }
    }
  }
  // ---- offsets of the cubes the tile can meet (up to the next tile's first cube), relative to the tile
  // and clamped to +-2^30; n_h is the difference of neighbours ----
  if constexpr (PREFETCH) {
    // one pass over the prefetched offsets: relative offsets, 1/n_h and the
    // start-cube entries of the threads whose first evaluation a cube holds
    const int64_t* raw = S.raw_off;
    for (int c = tid; c <= ncand; c += kFillThreads) {
      const int64_t g0 = raw[c], rel0 = g0 - j0;
      const int o0 = rel0 < -kRelCap ? -kRelCap : (rel0 > kRelCap ? kRelCap : (int)rel0);
      off_r[c] = o0;
      if (c < ncand) {
        const int64_t g1 = raw[c + 1], rel1 = g1 - j0;
        const int o1 = rel1 < -kRelCap ? -kRelCap : (rel1 > kRelCap ? kRelCap : (int)rel1);
        const int r0 = max(o0, 0), r1 = min(o1, len);
        T inv = T(0);
        if (r0 < r1) {
          const int64_t n = (o0 > -kRelCap && o1 < kRelCap) ? (int64_t)(o1 - o0) : g1 - g0;
          if constexpr (sizeof(T) == 8) inv = 1.0 / (double)n;
          else inv = __fdividef(1.0f, (float)n);
          for (int t = (r0 + spt - 1) >> spt_log2; (t << spt_log2) < r1; ++t)
            startc[VG_IDX(t, kFillThreads, a.flags, 20)] = c;
          if (r1 == len) misc[1] = c + 1;  // cubes met by the tile
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
    // the offsets of the next tile go to the same buffer, read by now, while
    // this tile computes; they are complete before the barrier after phase A
    if (next_tile < a.ntiles) {
      const int nc = min(maxc, nend - nh0 + 1);
      for (int c = tid; c <= nc; c += kFillThreads) cp_async8(S.raw_off + c, a.offsets + (int64_t)nh0 + c);
      cp_async_commit();
      if (tid == 0) {
        misc[2] = nh0;
        misc[3] = nc;
      }
    }
  } else {
  for (int c = tid; c <= ncand; c += kFillThreads) {
    const int64_t rel = a.offsets[(int64_t)h0 + c] - j0;  // h0 + c <= NH
    off_r[c] = rel < -kRelCap ? -kRelCap : (rel > kRelCap ? kRelCap : (int)rel);
  }
  if (tid == 0) {
    misc[0] = 0;
    a.carries[2 * tile] = Carry{-1, 0, 0.0, 0.0};
    a.carries[2 * tile + 1] = Carry{-1, 0, 0.0, 0.0};
  }
  __syncthreads();
  // 1/n_h of every cube the tile meets; every cube tells the threads whose first evaluation it holds
  for (int c = tid; c < ncand; c += kFillThreads) {
    const int o0 = off_r[c], o1 = off_r[c + 1];
    const int r0 = max(o0, 0), r1 = min(o1, len);
    T inv = T(0);
    if (r0 < r1) {
      // a cube longer than 2^30 (clamped ends) takes its count from the global offsets
      const int64_t n = (o0 > -kRelCap && o1 < kRelCap)
                            ? (int64_t)(o1 - o0)
                            : a.offsets[(int64_t)h0 + c + 1] - a.offsets[(int64_t)h0 + c];
      if constexpr (sizeof(T) == 8) inv = 1.0 / (double)n;
      else inv = __fdividef(1.0f, (float)n);
      for (int t = (r0 + spt - 1) >> spt_log2; (t << spt_log2) < r1; ++t)
        startc[VG_IDX(t, kFillThreads, a.flags, 21)] = c;
      if (r1 == len) misc[1] = c + 1;  // cubes met by the tile
    }
    invn[c] = inv;
  }
  __syncthreads();
  }

  // ---- phase A: point, map, integrand, J f; map weights ----
  const int jl0 = tid << spt_log2;
  float my_max = 0.0f;
  if constexpr (STREAM) {
    static_assert(sizeof(T) == 4 && DMAX >= 16, "the streamed path is FP32 and wide");
    if (jl0 < len) {
      int c = startc[tid];
      int c_decoded = -1;
      uint32_t cw[DMAX / 4];
#pragma unroll 1
      for (int s = 0; s < spt; ++s) {
        const int jl = jl0 + s;
        if (jl < len) {
          while (off_r[VG_IDX(c + 1, maxc + 1, a.flags, 3)] <= jl) ++c;
          if (c != c_decoded) {
            decode_packed<DMAX>(a, (uint32_t)(h0 + c), cw);
            c_decoded = c;
          }
          float J = st.J0;
          float* xo = (ID == kIntegrandPoints) ? a.points_out + (j0 + jl) * d : nullptr;
          float f = stream_point_eval<ID, DMAX>(a, rk0, rk1, cw, j0 + jl, tab, prm, ps0, ps1, pK, J,
                                                binw + tix(jl, spt_log2), xo);
          if constexpr (ID == kIntegrandPoints) continue;
          if constexpr (ID == kIntegrandTabulated) f = a.values[j0 + jl];
          if (!isfinite(f)) bad = true;
          const float v = J * f;
          vals[VG_IDX(jl, tileN, a.flags, 4)] = v;
          if constexpr (ID == kIntegrandTabulated) {
            const int64_t j = j0 + jl;
            if (a.train_w && j % a.train_stride == 0)
              a.train_w[j / a.train_stride] = powf(fabsf(v) * (float)invn[c], a.train_power);
          }
          const float wv = v * v * (float)invn[VG_IDX(c, maxc, a.flags, 5)];
          if (!(STREAM && a.wv_recompute)) wv_s[tix(jl, spt_log2)] = wv;  // else phase B recomputes it
          my_max = fmaxf(my_max, wv);
        }
      }
    }
  } else if (jl0 < len) {
    int c = startc[tid];
    uint32_t cb[DMAX];
    decode_cube<T, DMAX, EXACT>(a, (uint32_t)(h0 + c), cb);
#pragma unroll 1
    for (int s = 0; s < spt; ++s) {
      const int jl = jl0 + s;
      if (jl < len) {
        while (off_r[VG_IDX(c + 1, maxc + 1, a.flags, 6)] <= jl) {
          ++c;
          next_cube<T, DMAX, EXACT>(a, cb);
        }
        T x[DMAX];
        int bin[DMAX];
        T J;
        make_point<T, DMAX, EXACT>(a, rk0, rk1, cb, j0 + jl, tab, x, bin, J, st.J0);
        if constexpr (ID == kIntegrandPoints) {  // the points only, for an outside evaluation
          float* xo = a.points_out + (j0 + jl) * d;
          if ((d & 3) == 0) {  // 16-byte aligned rows
#pragma unroll
            for (int k = 0; k < DMAX; k += 4)
              if (k < d)
                *reinterpret_cast<float4*>(xo + k) =
                    make_float4((float)x[k], (float)x[k + 1], (float)x[k + 2], (float)x[k + 3]);
          } else {
#pragma unroll
            for (int k = 0; k < DMAX; ++k)
              if (k < d) xo[k] = (float)x[k];
          }
          continue;
        }
        T f;
        if constexpr (ID == kIntegrandTabulated) f = (T)a.values[j0 + jl];
        else f = integrand<ID, T, DMAX>(x, d, prm, a.np_derived, ps0, ps1, pK);
        if (!isfinite(f)) bad = true;
        const T v = J * f;
        vals[VG_IDX(jl, tileN, a.flags, 7)] = v;
        if constexpr (ID == kIntegrandTabulated) {
          // training weights (|J f| / n_h)^p of every train_stride-th evaluation
          const int64_t j = j0 + jl;
          if (a.train_w && j % a.train_stride == 0)
            a.train_w[j / a.train_stride] = powf(fabsf((float)v) * (float)invn[c], a.train_power);
        }
        const T wv = v * v * invn[VG_IDX(c, maxc, a.flags, 8)];
        if (two_phase) {
          wv_s[tix(jl, spt_log2)] = (float)wv;
          my_max = fmaxf(my_max, (float)wv);
          if (bpw == 4) {
#pragma unroll
            for (int w = 0; w < (DMAX + 3) / 4; ++w) {
              if (4 * w < d) {
                // intervals below 256: byte 0 of each, four to a word
                const uint32_t b0 = (uint32_t)bin[4 * w];
                const uint32_t b1 = 4 * w + 1 < DMAX ? (uint32_t)bin[4 * w + 1] : 0u;
                const uint32_t b2 = 4 * w + 2 < DMAX ? (uint32_t)bin[4 * w + 2] : 0u;
                const uint32_t b3 = 4 * w + 3 < DMAX ? (uint32_t)bin[4 * w + 3] : 0u;
                const uint32_t word = __byte_perm(__byte_perm(b0, b1, 0x0040u), __byte_perm(b2, b3, 0x0040u), 0x5410u);
                binw[(w << TL) + tix(jl, spt_log2)] = word;
              }
            }
          } else {
#pragma unroll
            for (int w = 0; w < (DMAX + 1) / 2; ++w) {
              if (2 * w < d) {
                uint32_t word = (uint32_t)bin[2 * w];
                if (2 * w + 1 < DMAX) word |= (uint32_t)bin[2 * w + 1] << 16;
                binw[(w << TL) + tix(jl, spt_log2)] = word;
              }
            }
          }
        } else {
#pragma unroll
          for (int k = 0; k < DMAX; ++k) {
            if (k < d) {
              if (a.hist_mode == kHistShared)
                atomicAdd(hist_s + VG_IDX(((k * G + bin[k]) << a.hist_rep_log2) + (lane & ((1 << a.hist_rep_log2) - 1)),
                                          dG << a.hist_rep_log2, a.flags, 9),
                          wv);
              else atomicAdd(hist_g + VG_IDX(k * G + bin[k], dG, a.flags, 10), (double)wv);
            }
          }
        }
      }
    }
  }
  if (two_phase) {
    for (int o = 16; o > 0; o >>= 1) my_max = fmaxf(my_max, __shfl_xor_sync(0xffffffffu, my_max, o));
    if (lane == 0) wmax[warp] = my_max;
  }
  if constexpr (PREFETCH) cp_async_wait_all();
  __syncthreads();
  if constexpr (ID == kIntegrandPoints) return;

  // ---- phase B (two-phase histogram): fixed-point shared integer atomics ----
  if (two_phase) {
    float tmax = 0.0f;
#pragma unroll
    for (int w = 0; w < kFillThreads / 32; ++w) tmax = fmaxf(tmax, wmax[w]);
    if (tmax > 0.0f && isfinite(tmax)) {
      // tmax < 2^et and a bin gets at most 2^TL weights of the tile, so with
      // scale = 2^(31 - TL - et) every bin total stays below 2^31 (plus the
      // rounding of 2^TL values)
      int et;
      frexpf(tmax, &et);
      const int se = min(31 - TL - et, 126);
      const float scale = ldexpf(1.0f, se);
      inv_scale = ldexpf(1.0f, -se);
      if (jl0 < len) {
        int c = startc[tid];  // the evaluation's cube, for a weight recomputed from its value
#pragma unroll 1
        for (int s = 0; s < spt; ++s) {
          const int jl = jl0 + s;
          if (jl < len) {
            float wv;
            if (STREAM && a.wv_recompute) {  // the single fill's streamed layout has no weight slots
              while (off_r[VG_IDX(c + 1, maxc + 1, a.flags, 23)] <= jl) ++c;
              const float v = vals[VG_IDX(jl, tileN, a.flags, 24)];
              wv = (float)(v * v * (float)invn[VG_IDX(c, maxc, a.flags, 25)]);
            } else {
              wv = wv_s[tix(jl, spt_log2)];
            }
            const uint32_t q = (uint32_t)__float2uint_rn(wv * scale);
            if (q) {
              if (bpw == 4) {
                for (int w = 0; w < nw; ++w) {
                  const uint32_t word = binw[(w << TL) + tix(jl, spt_log2)];
                  const int kk = 4 * w;
#pragma unroll
                  for (int b = 0; b < 4; ++b)
                    if (kk + b < d)
                      atomicAdd(hist_u + VG_IDX((kk + b) * G + ((word >> (8 * b)) & 255u), dG, a.flags, 11), q);
                }
              } else {
                for (int w = 0; w < nw; ++w) {
                  const uint32_t word = binw[(w << TL) + tix(jl, spt_log2)];
                  const int kk = 2 * w;
                  atomicAdd(hist_u + VG_IDX(kk * G + (word & 0xFFFFu), dG, a.flags, 12), q);
                  if (kk + 1 < d) atomicAdd(hist_u + VG_IDX((kk + 1) * G + (word >> 16), dG, a.flags, 13), q);
                }
              }
            }
          }
        }
      }
    } else {
      inv_scale = 0.0f;
    }
  }

  // ---- cube statistics ----
  const int ncub = misc[1];
  // one cube segment done: a cube inside the tile is final, one crossing an
  // edge becomes a Carry for the fix-up kernel
  auto finish = [&](int c, int L, auto mean, T m2) {
    const int r0 = off_r[c], r1 = off_r[c + 1];
    const bool before = r0 < 0, after = r1 > len;
    const int h = h0 + c;
    if (before || after) {
      a.carries[VG_IDX(2 * tile + (before ? 0 : 1), 2 * a.ntiles, a.flags, 14)] = Carry{h, L, to_double(mean), (double)m2};
      return;
    }
    const int n = r1 - r0;
    float ell;
    acc_i.add(mean);
    if constexpr (sizeof(T) == 8) {
      // sigma_h^2 = M2 / (n - 1) divided exactly (it decides the counts); sigma_h^2 / n with the tile's 1/n
      const double var = m2 / (double)(n - 1);
      acc_v.add(var * invn[c]);
      // the FP64 form keeps the reproducible log2, so that the counts of a
      // free-running FP64 run follow the CPU reference bit for bit
      ell = __fmul_rn(a.half_beta, log2r(var));
    } else {
      const float nf = (float)n;
      acc_v.add(__fdividef(m2, nf * (nf - 1.0f)));
      ell = a.half_beta * (log2_fast(__fdividef(m2, nf - 1.0f)) + (float)(2 * st.vexp));
    }
    a.ell[VG_IDX(h, a.NH, a.flags, 15)] = ell;
    lmax = fmaxf(lmax, ell);
    if (a.cube_mean) {
      a.cube_mean[VG_IDX(h, a.NH, a.flags, 16)] = ldexp(to_double(mean), st.vexp);
      a.cube_m2[VG_IDX(h, a.NH, a.flags, 17)] = ldexp((double)m2, 2 * st.vexp);
    }
  };

  bool had_long = false;
  for (int c = tid; c < ncub; c += kFillThreads) {
    const int r0 = max(off_r[c], 0), r1 = min(off_r[c + 1], len);
    const int L = r1 - r0;
    if (L > kLongSegment) {
      longlist[VG_IDX(atomicAdd(&misc[0], 1), tile_max_long(tileN), a.flags, 22)] = c;
      had_long = true;
      continue;
    }
    // one pass over the segment, shifted by its first value: mean = v0 + s/L,
    // M2 = q - s^2/L with s, q the sums of (v - v0) and (v - v0)^2; the shift
    // keeps q within (L + 1) M2, so the cancellation costs a few ulps
    const T v0 = vals[VG_IDX(r0, tileN, a.flags, 18)];
    T sd = T(0), qd = T(0);
    for (int r = r0 + 1; r < r1; ++r) {
      const T dv = vals[VG_IDX(r, tileN, a.flags, 19)] - v0;
      sd += dv;
      qd = fma(dv, dv, qd);
    }
    if constexpr (sizeof(T) == 8) {
      // a cube inside the tile has L = n_h: its 1/n_h is the tile's
      const double sl = (off_r[c] >= 0 && off_r[c + 1] <= len) ? sd * invn[c] : sd / (double)L;
      finish(c, L, v0 + sl, fmax(fma(-sd, sl, qd), 0.0));
    } else {
      const float sl = __fdividef(sd, (float)L);
      // mean = v0 + sl as a normalised float-float (TwoSum), so that the
      // low words summed into the iteration estimate stay rounding errors
      finish(c, L, ff_add(ff{v0, 0.0f}, sl), fmaxf(fmaf(-sd, sl, qd), 0.0f));
    }
  }
  // the long segments, if the tile has any, one warp each; without them the
  // single-integral fill ends the tile at this barrier
  if constexpr (PREFETCH) {
    if (!__syncthreads_or(had_long)) return;
  } else {
    (void)had_long;
    __syncthreads();
  }
  const int nlong = misc[0];
  for (int e = warp; e < nlong; e += kFillThreads / 32) {
    const int c = longlist[e];
    const int r0 = max(off_r[c], 0), r1 = min(off_r[c + 1], len);
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

// ---------------------------------------------------------------------------
// Cubes that cross tile edges.  A cube that starts in tile t and ends in tile
// t_end leaves an "after" record in slot 2t+1 of tile t and a "before" record
// in slot 2u of every later tile u <= t_end.  Before the fix-up merges them,
// the before records are reduced from the right within blocks of
// kCarryBlock consecutive tiles: slot 2u then holds the merge of u up to the
// end of its run of same-cube records inside u's block.  The fix-up reads one
// record per block, so a cube spanning T tiles costs T / kCarryBlock steps
// instead of T.  The merge is Chan et al.'s pairwise update of
// (count, mean, M2), which is associative up to rounding.
// ---------------------------------------------------------------------------
constexpr int kCarryBlock = 256;

__device__ __forceinline__ void chan_merge(double& cnt, double& mean, double& m2, double nb, double mb, double qb) {
  const double nt = cnt + nb, delta = mb - mean;
  mean += delta * nb / nt;
  m2 += qb + delta * delta * cnt * nb / nt;
  cnt = nt;
}

// One thread per tile, blockDim.x == kCarryBlock.  rec: the tile's before
// record (h < 0: none); joins: the record continues the previous tile's run
// (same integral and cube, both present).  Returns the run's suffix merge.
__device__ __forceinline__ Carry carry_suffix(Carry rec, bool joins) {
  __shared__ int seg[kCarryBlock];
  __shared__ int wtot[kCarryBlock / 32];
  __shared__ double sc[2][kCarryBlock], sm[2][kCarryBlock], sq[2][kCarryBlock];
  const int u = threadIdx.x, lane = u & 31, w = u >> 5;
  // segment ids: inclusive scan of the run heads
  int head = (u == 0 || !joins) ? 1 : 0;
  int x = head;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wtot[w] = x;
  __syncthreads();
  for (int k = 0; k < w; ++k) x += wtot[k];
  seg[u] = x;
  sc[0][u] = rec.h >= 0 ? (double)rec.cnt : 0.0;
  sm[0][u] = rec.mean;
  sq[0][u] = rec.m2;
  __syncthreads();
  int cur = 0;
#pragma unroll 1
  for (int o = 1; o < kCarryBlock; o <<= 1) {
    double c = sc[cur][u], m = sm[cur][u], q = sq[cur][u];
    if (rec.h >= 0 && u + o < kCarryBlock && seg[u + o] == seg[u]) chan_merge(c, m, q, sc[cur][u + o], sm[cur][u + o], sq[cur][u + o]);
    sc[cur ^ 1][u] = c;
    sm[cur ^ 1][u] = m;
    sq[cur ^ 1][u] = q;
    cur ^= 1;
    __syncthreads();
  }
  if (rec.h >= 0) {
    rec.cnt = (int32_t)sc[cur][u];
    rec.mean = sm[cur][u];
    rec.m2 = sq[cur][u];
  }
  return rec;
}

// Fill of one integral: a persistent grid walks the tiles round-robin.
// EXACT: d == DMAX and the map table is in shared memory, so the per-axis
// bounds checks vanish and the table reads are shared-memory loads.  The FP32
// form with d <= 8 asks for 4 resident CTAs (at most 64 registers): measured
// 7 % faster than 3 CTAs with more registers.  Wider or FP64 forms would spill.
template <int ID, typename T, int DMAX, bool EXACT, bool STREAM = false, int TLC = 0>
__global__ void __launch_bounds__(kFillThreads, (sizeof(T) == 4 && (DMAX <= 8 || STREAM)) ? 4 : (sizeof(T) == 8 && EXACT) ? 2 : 1)
    fill_kernel(const __grid_constant__ FillArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31;
  const int d = EXACT ? DMAX : a.d, dG = d * a.G;
  const bool table_in_smem = EXACT || a.table_smem;
  const FillShared<T> S = fill_shared<T>(smem, a, table_in_smem);
  double* hist_g = a.hist_part + (size_t)blockIdx.x * dG;
  double xs = 1.0;  // the FP64 Gaussian sum takes its point scaled (gauss_scale64)
  if constexpr (ID == VEGAS_GAUSS_SUM && sizeof(T) == 8) xs = gauss_scale64(a.params_raw[1]);
  fill_prologue<T>(a, S, d, table_in_smem, xs);
  prep_params<ID, T, DMAX>(a.params_raw, a.np_raw, d, S.prm);
  // the exact-d FP32 kernels (d = 4 or 8) and the streamed ones do without the prefetch buffer, which buys a
  // fourth resident CTA (d = 8 ridge: 2.09 ms at 3 CTAs with the buffer, 1.99 ms at 4 without; d = 30 streamed,
  // with no weight slots either: 61.6 -> 56.8 ms an iteration); the host leaves the buffer out of exactly these
  // layouts.  The general FP32 kernels keep it (d = 8, N_g = 1024: 4-26 % faster with it)
  constexpr bool kPrefetch = !(sizeof(T) == 4 && ((DMAX <= 8 && EXACT) || STREAM));
  if (kPrefetch && blockIdx.x < a.ntiles) {  // the first tile's cube offsets; later tiles' come during the tile before
    const int t = blockIdx.x, fh0 = a.tile_first[t];
    const int nc = min(tile_max_cubes(1 << (TLC ? TLC : a.tile_log2)), (t + 1 < a.ntiles ? a.tile_first[t + 1] : a.NH - 1) - fh0 + 1);
    for (int c = tid; c <= nc; c += kFillThreads) cp_async8(S.raw_off + c, a.offsets + (int64_t)fh0 + c);
    cp_async_commit();
    if (tid == 0) {
      S.misc[2] = fh0;
      S.misc[3] = nc;
    }
    cp_async_wait_all();
  }
  __syncthreads();
  const T ps0 = S.prm[0], ps1 = S.prm[1];
  const int pK = (ID == VEGAS_GAUSS_SUM) ? (int)S.prm[2] : 0;
  FillState<T> st;
  if constexpr (sizeof(T) == 4) {
    st.vexp = a.vexp ? *a.vexp : 0;
    st.J0 = ldexpf(1.0f, -st.vexp);
  }
  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x)
    fill_tile<ID, T, DMAX, EXACT, STREAM, kPrefetch, TLC>(a, a.rk0, a.rk1, S, st, tile, ps0, ps1, pK, hist_g,
                                                 tile + gridDim.x);
  if constexpr (ID == kIntegrandPoints) return;

  // ---- epilogue: CTA partial sums, max weight, flags, histogram ----
  const double si = block_sum(st.acc_i.value(), S.red);
  const double sv = block_sum(st.acc_v.value(), S.red);
  if (tid == 0) {
    a.cta_part[2 * blockIdx.x] = si;
    a.cta_part[2 * blockIdx.x + 1] = sv;
  }
  float lmax = st.lmax;
  for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  if (lane == 0) atomicMax(a.ellmax_key, float_key(lmax));
  if (__syncthreads_or(st.bad) && tid == 0) atomicOr(a.flags, 1);
  if (a.hist_mode == kHistShared)
    for (int b = tid; b < dG; b += kFillThreads) {
      double t = 0.0;
      for (int c = 0; c < (1 << a.hist_rep_log2); ++c) t += (double)S.hist_s[(b << a.hist_rep_log2) + c];
      hist_g[b] = t;
    }
  if (a.hist_mode == kHistTwoPhase) {
    for (int b = tid; b < dG; b += kFillThreads) {
      const float pend = st.inv_scale > 0.0f ? __fmul_rn((float)S.hist_u[b], st.inv_scale) : 0.0f;
      if (a.acc32) {
        hist_g[b] = (double)S.hist_accf[b] + (double)pend;
      } else {
        ff acc = S.hist_acc[b];
        if (st.inv_scale > 0.0f) acc = ff_add(acc, pend);
        hist_g[b] = ff_to_double(acc);
      }
    }
  }
}

}  // namespace vg
