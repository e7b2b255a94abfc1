// vegas_device.cuh -- device helpers of the GB300 VEGAS+ kernels.
//
// Philox4x32-10 point draws, the reproducible FP32 log2/exp2 of the allocation
// weights, float-float accumulation, the integrand families and the FP64 exp
// of the FP64 form's Gaussian integrand.
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

// ---------------------------------------------------------------------------
// e^x in FP64 by Tang's table-driven method (P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point
// arithmetic", ACM TOMS 15(2), 1989) with 64 table entries:
//   x = n ln2/64 + r, n = rint(64 x / ln2), |r| <= ln2/128 (+ rounding),
//   e^x = 2^(n >> 6) 2^((n & 63)/64) e^r,
// e^r - 1 by its Taylor polynomial to degree 5, whose truncation is below
// r^6/720 < 4e-17 relative.  n comes from one fused multiply-add against
// 1.5 2^52 (its low word); r from a two-part ln2/64 whose first part has 36
// significant bits, so n ln2_hi/64 and x - n ln2_hi/64 are exact for |x| < 2^10.
// The result is within about one ulp of e^x.  Ten FP64 operations; the rest
// (table index, exponent) is integer work.  Below x = -745.2 the result is 0
// (e^x is below half the smallest subnormal); from -745.2 to -707.6 the scale
// takes one more multiply, which rounds to the subnormal result; above 707.6
// and for NaN the library exp() runs.
__device__ const double kExp2Table64[64] = {
    // 2^(j/64), j = 0..63, each rounded to the nearest double (from a 60-digit decimal evaluation)
    0x1.0000000000000p+0, 0x1.02c9a3e778061p+0, 0x1.059b0d3158574p+0, 0x1.0874518759bc8p+0,
    0x1.0b5586cf9890fp+0, 0x1.0e3ec32d3d1a2p+0, 0x1.11301d0125b51p+0, 0x1.1429aaea92de0p+0,
    0x1.172b83c7d517bp+0, 0x1.1a35beb6fcb75p+0, 0x1.1d4873168b9aap+0, 0x1.2063b88628cd6p+0,
    0x1.2387a6e756238p+0, 0x1.26b4565e27cddp+0, 0x1.29e9df51fdee1p+0, 0x1.2d285a6e4030bp+0,
    0x1.306fe0a31b715p+0, 0x1.33c08b26416ffp+0, 0x1.371a7373aa9cbp+0, 0x1.3a7db34e59ff7p+0,
    0x1.3dea64c123422p+0, 0x1.4160a21f72e2ap+0, 0x1.44e086061892dp+0, 0x1.486a2b5c13cd0p+0,
    0x1.4bfdad5362a27p+0, 0x1.4f9b2769d2ca7p+0, 0x1.5342b569d4f82p+0, 0x1.56f4736b527dap+0,
    0x1.5ab07dd485429p+0, 0x1.5e76f15ad2148p+0, 0x1.6247eb03a5585p+0, 0x1.6623882552225p+0,
    0x1.6a09e667f3bcdp+0, 0x1.6dfb23c651a2fp+0, 0x1.71f75e8ec5f74p+0, 0x1.75feb564267c9p+0,
    0x1.7a11473eb0187p+0, 0x1.7e2f336cf4e62p+0, 0x1.82589994cce13p+0, 0x1.868d99b4492edp+0,
    0x1.8ace5422aa0dbp+0, 0x1.8f1ae99157736p+0, 0x1.93737b0cdc5e5p+0, 0x1.97d829fde4e50p+0,
    0x1.9c49182a3f090p+0, 0x1.a0c667b5de565p+0, 0x1.a5503b23e255dp+0, 0x1.a9e6b5579fdbfp+0,
    0x1.ae89f995ad3adp+0, 0x1.b33a2b84f15fbp+0, 0x1.b7f76f2fb5e47p+0, 0x1.bcc1e904bc1d2p+0,
    0x1.c199bdd85529cp+0, 0x1.c67f12e57d14bp+0, 0x1.cb720dcef9069p+0, 0x1.d072d4a07897cp+0,
    0x1.d5818dcfba487p+0, 0x1.da9e603db3285p+0, 0x1.dfc97337b9b5fp+0, 0x1.e502ee78b3ff6p+0,
    0x1.ea4afa2a490dap+0, 0x1.efa1bee615a27p+0, 0x1.f50765b6e4540p+0, 0x1.fa7c1819e90d8p+0};

__device__ __forceinline__ double exp_table64(double x) {
  constexpr double kInvL = 0x1.71547652b82fep+6;  // 64 / ln2
  constexpr double kL1 = 0x1.62e42fefa0000p-7;    // ln2 / 64, first 36 bits
  constexpr double kL2 = 0x1.cf79abc9e3b3ap-46;   // ln2 / 64 - kL1
  constexpr double kShift = 0x1.8p52;
  const double t = fma(x, kInvL, kShift);
  const int n = __double2loint(t);  // the low word of 1.5 2^52 + n is n
  const double nd = t - kShift;
  double r = fma(-nd, kL1, x);
  r = fma(-nd, kL2, r);
  const double r2 = r * r;
  double q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  q = fma(q, r, 1.0 / 6.0);
  q = fma(q, r, 0.5);
  const double p = fma(q, r2, r);  // e^r - 1
  const double T = __ldg(&kExp2Table64[n & 63]);
  const double y = fma(T, p, T);  // in [1, 2)
  const int m = n >> 6;
  // |x| < 707.6: 2^m (|m| <= 1021) is a normal scale; add it to the exponent field
  if ((__double2hiint(x) & 0x7FFFFFFF) >= 0x40861CCC) {  // |x| >= 707.6, or NaN
    if (x < -745.2) return 0.0;
    if (!(x < 0.0)) return exp(x);  // NaN, or above the normal range
    // -745.2 <= x <= -707.6: m in [-1076, -1021].  y 2^(m + 64) is normal (an exponent add); the exact scale
    // 2^-64 then rounds once, to the subnormal result
    return __hiloint2double(__double2hiint(y) + ((m + 64) << 20), __double2loint(y)) * 0x1p-64;
  }
  return __hiloint2double(__double2hiint(y) + (m << 20), __double2loint(y));
}

// 2^(y/64) by the same 64-entry table, for arguments already in units of ln2/64 (the FP64 Gaussian sum scales its
// point and centres so that the squared distance is this argument: no multiply before the reduction).  n = the
// integer nearest y (from adding 1.5 2^52, its low word), f = y - n in [-1/2, 1/2] (exact), and
// 2^(f/64) - 1 = e^(f c) - 1 with c = ln2/64 as a degree-5 polynomial in f whose coefficients are c^k/k!
// (|f c| <= ln2/128: truncation below 4e-17).  The result 2^(n>>6) 2^((n&63)/64) (1 + p) is within about one ulp
// of 2^(y/64).  Nine FP64 operations (three adds, five FMAs, one multiply) against the ten of exp_table64 and the
// multiply that would form its argument.  Below y = -68800 the result is 0 (2^(y/64) is below half the smallest
// subnormal); from -68800 to -65344 one more multiply rounds to the subnormal result; from 65344 up and for NaN
// the library exp2() runs.
__device__ __forceinline__ double exp2_64ths(double y) {
  constexpr double kShift = 0x1.8p52;
  constexpr double kC1 = 0x1.62e42fefa39efp-7;   // c = ln2 / 64
  constexpr double kC2 = 0x1.ebfbdff82c58fp-15;  // c^2 / 2
  constexpr double kC3 = 0x1.c6b08d704a0c0p-23;  // c^3 / 6
  constexpr double kC4 = 0x1.3b2ab6fba4e77p-31;  // c^4 / 24
  constexpr double kC5 = 0x1.5d87fe78a6731p-40;  // c^5 / 120
  const double t = y + kShift;
  const int n = __double2loint(t);
  const double f = y - (t - kShift);
  double q = fma(f, kC5, kC4);
  q = fma(q, f, kC3);
  q = fma(q, f, kC2);
  q = fma(q, f, kC1);
  const double p = q * f;  // 2^(f/64) - 1
  const double T = __ldg(&kExp2Table64[n & 63]);
  const double r = fma(T, p, T);
  const int m = n >> 6;
  if ((__double2hiint(y) & 0x7FFFFFFF) >= 0x40EFE800) {  // |y| >= 65344, or NaN
    if (y < -68800.0) return 0.0;
    if (!(y < 0.0)) return exp2(y * 0x1p-6);  // NaN, or above the normal range
    // m in [-1075, -1021]: r 2^(m + 64) is normal; the exact scale 2^-64 then rounds once, to the subnormal result
    return __hiloint2double(__double2hiint(r) + ((m + 64) << 20), __double2loint(r)) * 0x1p-64;
  }
  return __hiloint2double(__double2hiint(r) + (m << 20), __double2loint(r));
}

// ---------------------------------------------------------------------------
// Bounds-checking builds (nvcc -DVEGAS_BOUNDS_CHECK; build_lib.build(check=True)), the substitute for a memory
// sanitizer: every index that the fill derives from data (an interval from a point, a cube from the offsets, a
// slot of the tile's shared arrays, a histogram bin) goes through VG_IDX.  An index outside [0, n) sets bit 3 and
// the site number (bits 8-15) in the caller's device flag word and is replaced by 0, so that no access leaves its
// array; the handle then reports VEGAS_ECUDA.  Ordinary builds compile VG_IDX to the index itself.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long checked_index(long long i, long long n, int* flags, int site) {
  if (i >= 0 && i < n) return i;
  if (flags) atomicOr(flags, 8 | (site << 8));
  return 0;
}
#ifdef VEGAS_BOUNDS_CHECK
#define VG_IDX(i, n, flags, site) (vg::checked_index((long long)(i), (long long)(n), (flags), (site)))
#else
#define VG_IDX(i, n, flags, site) (i)
#endif

}  // namespace vg
