// vegas_device.cuh -- device helpers of the GB300 VEGAS+ kernels.
//
// Philox4x32-10 point draws, the reproducible FP32 log2/exp2 of the allocation
// weights, float-float accumulation, and the integrand families.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/vegas.h"

namespace vg {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Each round takes the two
// 32x32->64 products of counter words 0 and 2 with the round multipliers.  The
// high halves are xor-ed with words 1 and 3 and the round key; the key grows
// by the Weyl increments between rounds.  Ten rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// ---------------------------------------------------------------------------
// Reproducible FP32 log2 / exp2 of the allocation weights.  The allocation
// turns real weights into integer counts, so it is written as a fixed sequence
// of single IEEE operations (no contraction; the _rn intrinsics are never
// fused).  The results are therefore the same on any IEEE machine:
//   log2 x = e + (2/ln 2) atanh t,  t = (m-1)/(m+1),  m in (1/sqrt2, sqrt2];
//            atanh t ~ t (1 + t^2/3 + t^4/5 + t^6/7 + t^8/9), |t| < 0.172.
//   2^y    = 2^n e^(r ln 2), n = rint y, |r| <= 1/2; Taylor series to degree 7.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float log2r_mant(float m, int e) {
  const float kThird = 0x1.555556p-2f, kFifth = 0x1.99999ap-3f, kSeventh = 0x1.24924ap-3f,
              kNinth = 0x1.c71c72p-4f, kLog2e = 0x1.715476p+0f, kSqrt2 = 0x1.6a09e6p+0f;
  if (m > kSqrt2) {
    m = __fmul_rn(m, 0.5f);
    e += 1;
  }
  const float t = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
  const float t2 = __fmul_rn(t, t);
  float p = kNinth;
  p = __fadd_rn(__fmul_rn(p, t2), kSeventh);
  p = __fadd_rn(__fmul_rn(p, t2), kFifth);
  p = __fadd_rn(__fmul_rn(p, t2), kThird);
  p = __fadd_rn(__fmul_rn(p, t2), 1.0f);
  const float s = __fmul_rn(__fmul_rn(t, p), 2.0f);
  return __fadd_rn((float)e, __fmul_rn(s, kLog2e));
}

// x >= 0 in double: -inf for 0, NaN for negative / non-finite input.
__device__ __forceinline__ float log2r(double x) {
  if (x == 0.0) return -__int_as_float(0x7f800000);
  if (!(x > 0.0) || isinf(x)) return __int_as_float(0x7fc00000);
  int e;
  const double m2 = frexp(x, &e);          // exact: x = m2 2^e, m2 in [0.5, 1)
  const float m = __double2float_rn(m2 * 2.0);  // in [1, 2], one rounding
  return log2r_mant(m, e - 1);
}

__device__ __forceinline__ float log2r(float x) {
  if (x == 0.0f) return -__int_as_float(0x7f800000);
  if (!(x > 0.0f) || isinf(x)) return __int_as_float(0x7fc00000);
  int e;
  const float m2 = frexpf(x, &e);  // exact
  return log2r_mant(__fmul_rn(m2, 2.0f), e - 1);
}

// 2^y for y <= 0 (y < -30 gives 0)
__device__ __forceinline__ float exp2r(float y) {
  const float kLn2 = 0x1.62e430p-1f;
  if (y < -30.0f) return 0.0f;
  const float n = rintf(y);
  const float r = __fsub_rn(y, n);
  const float s = __fmul_rn(r, kLn2);
  float p = 0x1.a01a02p-13f;                          // 1/7!
  p = __fadd_rn(__fmul_rn(p, s), 0x1.6c16c2p-10f);    // 1/6!
  p = __fadd_rn(__fmul_rn(p, s), 0x1.111112p-7f);     // 1/5!
  p = __fadd_rn(__fmul_rn(p, s), 0x1.555556p-5f);     // 1/4!
  p = __fadd_rn(__fmul_rn(p, s), 0x1.555556p-3f);     // 1/3!
  p = __fadd_rn(__fmul_rn(p, s), 0x1p-1f);            // 1/2!
  p = __fadd_rn(__fmul_rn(p, s), 1.0f);
  p = __fadd_rn(__fmul_rn(p, s), 1.0f);
  const float scale = __int_as_float((127 + (int)n) << 23);  // 2^n exactly, n in [-30, 0]
  return __fmul_rn(p, scale);
}

// quantised allocation weight q = rint(2^24 2^(ell - ell_max)), 0 for ell = -inf
__device__ __forceinline__ uint32_t quant_weight(float ell, float ell_max) {
  if (isinf(ell) && ell < 0.0f) return 0u;
  const float w = exp2r(__fsub_rn(ell, ell_max));
  return (uint32_t)rintf(__fmul_rn(w, 16777216.0f));
}

// order-preserving int key of a float, for atomicMax on floats
__device__ __forceinline__ int float_key(float f) {
  int b = __float_as_int(f);
  return b >= 0 ? b : (b ^ 0x7fffffff);
}
__device__ __forceinline__ float key_float(int k) { return __int_as_float(k >= 0 ? k : (k ^ 0x7fffffff)); }

// ---------------------------------------------------------------------------
// float-float accumulation (Knuth TwoSum): hi + lo carries ~48 bits
// ---------------------------------------------------------------------------
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff ff_add(ff a, float b) {
  const float s = __fadd_rn(a.hi, b);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff{s, __fadd_rn(a.lo, err)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff r = ff_add(a, b.hi);
  r.lo = __fadd_rn(r.lo, b.lo);
  return r;
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// ---------------------------------------------------------------------------
// Integrands.  Parameters are "derived": the fill prologue turns the caller's
// params into the form below, in the precision T of the evaluation, and stages
// them in shared memory.
//   GAUSS_SUM         [A, c, K, mu(K*d)]  with c = -1/(2 s^2) (FP64, for exp)
//                                         or c = -log2(e)/(2 s^2) (FP32, for exp2)
//   PRODUCT_PEAK      [c_i^-2 (d), w (d)]
//   OSCILLATORY       [2 pi u, a (d)]
//   MOROKOFF_CAFLISCH [(1+1/d)^d, 1/d]
//   MAP_DENSITY       [edges (d*(G'+1))]
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T vexp(T x);
template <>
__device__ __forceinline__ double vexp<double>(double x) { return exp(x); }
template <>
__device__ __forceinline__ float vexp<float>(float x) { return expf(x); }

template <int ID, typename T, int DMAX>
__device__ __forceinline__ T integrand(const T (&x)[DMAX], int d, const T* __restrict__ p, int np) {
  if constexpr (ID == VEGAS_GAUSS_SUM) {
    const T A = p[0], c = p[1];
    const int K = (int)p[2];
    const T* mu = p + 3;
    T acc = T(0);
    for (int k = 0; k < K; ++k) {
      T r2 = T(0);
#pragma unroll
      for (int j = 0; j < DMAX; ++j) {
        if (j < d) {
          const T dx = x[j] - mu[j];
          r2 = fma(dx, dx, r2);
        }
      }
      mu += d;
      if constexpr (sizeof(T) == 8) acc += exp(r2 * c);
      else acc += exp2f(r2 * c);
    }
    return A * acc;
  } else if constexpr (ID == VEGAS_PRODUCT_PEAK) {
    // product of the denominators in groups of four, one division per group
    T r = T(1);
    T den = T(1);
#pragma unroll
    for (int j = 0; j < DMAX; ++j) {
      if (j < d) {
        const T dx = x[j] - p[d + j];
        den *= fma(dx, dx, p[j]);
      }
      if ((j & 3) == 3 || j == DMAX - 1) {
        r = r / den;
        den = T(1);
      }
    }
    return r;
  } else if constexpr (ID == VEGAS_OSCILLATORY) {
    T arg = p[0];
#pragma unroll
    for (int j = 0; j < DMAX; ++j)
      if (j < d) arg = fma(p[1 + j], x[j], arg);
    return cos(arg);
  } else if constexpr (ID == VEGAS_SIN_EXP) {
    return sin(x[0]) + vexp<T>(x[1 % DMAX]);
  } else if constexpr (ID == VEGAS_LINEAR) {
    T s = T(0);
#pragma unroll
    for (int j = 0; j < DMAX; ++j)
      if (j < d) s += x[j];
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
    for (int j = 0; j < DMAX; ++j)
      if (j < d) s = fma(x[j], x[j], s);
    return vexp<T>(s);
  } else if constexpr (ID == VEGAS_ROOS_ARNOLD) {
    T r = T(1);
#pragma unroll
    for (int j = 0; j < DMAX; ++j)
      if (j < d) r *= fabs(fma(T(4), x[j], T(-2)));
    return r;
  } else if constexpr (ID == VEGAS_MOROKOFF_CAFLISCH) {
    T r = p[0];
#pragma unroll
    for (int j = 0; j < DMAX; ++j)
      if (j < d) r *= pow(x[j], p[1]);
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

}  // namespace vg
