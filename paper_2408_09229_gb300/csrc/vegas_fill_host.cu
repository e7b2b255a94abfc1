// vegas_fill_host.cu -- vegas_fill: scratch layout, the tile-to-cube search,
// the fix-up of cubes that cross tile edges, the fixed-order reductions of
// the iteration sums and of the map weights, and the launch sequence
// (Algorithm 1 "fill weights" with Algorithm 2 inside).
#include <algorithm>
#include <cmath>

#include "vegas_device.cuh"
#include "vegas_fill.cuh"
#include "vegas_internal.h"

namespace vg {

int dmax_for(int d) { return d <= 4 ? 4 : d <= 8 ? 8 : d <= 16 ? 16 : 32; }

// Number of derived parameters the fill stages, or -1 when the caller's
// parameter count does not fit the family (layouts in vegas.h).
int derived_param_count(int integrand, int d, const double* host_params, int64_t np) {
  switch (integrand) {
    case VEGAS_GAUSS_SUM:
      if (np < 3 + d || (np - 3) % d != 0) return -1;
      if (host_params && (int64_t)host_params[2] * d + 3 != np) return -1;
      return (int)np;
    case VEGAS_PRODUCT_PEAK: return np == 2 * d ? (int)np : -1;
    case VEGAS_OSCILLATORY: return np == 1 + d ? (int)np : -1;
    case VEGAS_SIN_EXP: return (d == 2 && np == 0) ? 0 : -1;
    case VEGAS_LINEAR:
    case VEGAS_COSINE:
    case VEGAS_EXPONENTIAL:
    case VEGAS_ROOS_ARNOLD: return np == 0 ? 0 : -1;
    case VEGAS_MOROKOFF_CAFLISCH: return np == 0 ? 2 : -1;
    case VEGAS_MAP_DENSITY: return (np % d == 0 && np / d >= 2) ? (int)np : -1;
    case kIntegrandTabulated:
    case kIntegrandPoints: return np == 0 ? 0 : -1;
    default: return -1;
  }
}

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct ScratchLayout {
  size_t tile_first, carries, cta_part, fix_part, hist_part, gtable, ellmax, total;
  int ntiles, grid_max, nfix;
};

int num_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

ScratchLayout scratch_layout(int d, int G, int64_t neval, int sms) {
  ScratchLayout L{};
  // sized for the smallest tile (the most tiles), whichever tile a launch takes
  L.ntiles = (int)((neval + (1 << kTileLog2Min) - 1) >> kTileLog2Min);
  L.grid_max = std::max(1, std::min(L.ntiles, 8 * std::max(sms, 1)));
  L.nfix = (L.ntiles + 255) / 256;
  size_t off = 0;
  L.tile_first = off; off = align_up(off + sizeof(int32_t) * L.ntiles);
  L.carries = off;    off = align_up(off + sizeof(Carry) * 2 * (size_t)L.ntiles);
  L.cta_part = off;   off = align_up(off + sizeof(double) * 2 * (size_t)L.grid_max);
  L.fix_part = off;   off = align_up(off + sizeof(double) * 2 * (size_t)L.nfix);
  L.hist_part = off;  off = align_up(off + sizeof(double) * (size_t)L.grid_max * d * G);
  L.gtable = off;     off = align_up(off + sizeof(TabEntry<double>) * (size_t)d * G);
  L.ellmax = off;     off = align_up(off + 16);  // max-ell key at +0, FP32 value scale exponent at +4
  L.total = off;
  return L;
}

// magic multiplier for n / s with n < 2^31 (Granlund & Montgomery, PLDI'94,
// Thm 4.2): l = ceil(log2 s), m = ceil(2^(31+l) / s), n / s = (n m) >> (31+l)
void magic_div(uint32_t s, uint32_t& m, uint32_t& shift) {
  uint32_t l = 0;
  while ((uint64_t(1) << l) < s) ++l;
  m = (uint32_t)(((uint64_t(1) << (31 + l)) + s - 1) / s);
  shift = 31 + l;
}

// Shared-memory regions of the fill kernel.  The map-weight histogram goes to
// shared memory when it fits the budget.  FP32 with N_g <= 256 uses the
// two-phase fixed-point form; otherwise the histogram is of the evaluation
// type.  When the histogram does not fit, a per-CTA global histogram takes
// FP64 atomic adds.  The map table goes to shared memory when it also fits;
// otherwise the kernel reads it from global memory.
int smem_layout(FillArgs& a, size_t tsz, int nprm, bool fp32, bool table_ok = true, bool prefetch = true,
                bool streamed = false) {
  const int dG = a.d * a.G;
  // shared-memory regions start on 128-byte boundaries (the widest access is a 32-byte FP64 table entry)
  auto al = [](size_t x) { return (x + 127) / 128 * 128; };
  const int tile = 1 << a.tile_log2, maxc = tile_max_cubes(tile);
  // the buffer of the next tile's global offsets, filled by cp.async during a tile (single-integral fill)
  const size_t raw = prefetch ? al(sizeof(int64_t) * (maxc + 1)) : 0;
  const size_t base = al(nprm * tsz) + al(sizeof(int) * (maxc + 1)) +
                      raw +
                      al(tsz * maxc) + al(tsz * tile) +
                      al(sizeof(int) * tile_max_long(tile)) + al(sizeof(int) * kFillThreads) +
                      al(64 + 8 * 32);
  const size_t budget = 160 * 1024;
  const size_t table = al((size_t)dG * 4 * tsz);
  // two-phase: interval indices packed 8 bits (N_g <= 256) or 16 bits wide
  a.bin_shift = a.G <= 256 ? 3 : 4;
  const int per_word = 32 >> a.bin_shift;
  const size_t bin_words = (size_t)tile * 4 * ((a.d + per_word - 1) / per_word);
  // the streamed path recomputes each evaluation's weight in phase B (no weight slots) and accumulates the CTA
  // histogram in FP32: the smaller layout holds a fourth resident CTA at d = 30
  const size_t wv_bytes = streamed ? 0 : al(sizeof(float) * tile);
  a.wv_recompute = streamed ? 1 : 0;
  const size_t two_phase_ff = al((size_t)dG * 4) + al((size_t)dG * 8) + al(bin_words) + wv_bytes;
  const size_t two_phase_32 = al((size_t)dG * 4) + al((size_t)dG * 4) + al(bin_words) + wv_bytes;
  const size_t shared_hist = al((size_t)dG * tsz);
  size_t hist;
  a.acc32 = 0;
  // the two-phase form folds all d N_g intervals of the CTA histogram once per
  // tile: measured faster than shared FP32 atomics for
  // N_g <= 256 and for d N_g <= 2048, slower beyond (d = 8, N_g = 1024: 2.3x)
  const bool two_phase_ok = fp32 && (a.G <= 256 || dG <= 2048);
  if (two_phase_ok && !streamed && base + two_phase_ff <= budget) {
    a.hist_mode = kHistTwoPhase;
    hist = two_phase_ff;
  } else if (two_phase_ok && base + two_phase_32 <= budget) {
    a.hist_mode = kHistTwoPhase;
    a.acc32 = 1;
    hist = two_phase_32;
  } else if (base + shared_hist <= budget) {
    a.hist_mode = kHistShared;
    hist = shared_hist;
    // FP64 atomic adds into shared memory are slow when lanes of a warp hit one address, and they do on the
    // slow axes, where a warp's evaluations share the cube coordinate: up to 16 copies of the histogram (at
    // most 64 KB), lane l adding into copy l mod copies, summed in copy order at the end of the CTA (d = 8,
    // N_g = 50: 57.0 ms with one copy, 51.0 with 8, 50.0 with 16)
    a.hist_rep_log2 = 0;
    if (!fp32)
      while (a.hist_rep_log2 < 4 && ((size_t)dG * tsz << (a.hist_rep_log2 + 1)) <= 64 * 1024 &&
             base + al((size_t)dG * tsz << (a.hist_rep_log2 + 1)) <= budget)
        ++a.hist_rep_log2;
    hist = al((size_t)dG * tsz << a.hist_rep_log2);
  } else {
    a.hist_mode = kHistGlobal;
    hist = 0;
  }
  a.table_smem = table_ok && base + hist + table <= budget;
  size_t off = 0;
  a.sm_table = (int)off;  off += a.table_smem ? table : 0;
  a.sm_hist = (int)off;
  if (a.hist_mode == kHistTwoPhase) {
    off += al((size_t)dG * 4);
    a.sm_hacc = (int)off; off += al((size_t)dG * (a.acc32 ? 4 : 8));
    a.sm_bins = (int)off; off += al(bin_words);
    a.sm_wv = (int)off;   off += wv_bytes;
  } else {
    off += a.hist_mode == kHistShared ? hist : 0;
    a.sm_hacc = a.sm_bins = a.sm_wv = (int)off;
  }
  a.sm_params = (int)off; off += al(nprm * tsz);
  a.sm_off = (int)off;    off += al(sizeof(int) * (maxc + 1));
  a.sm_raw = (int)off;    off += raw;
  a.sm_invn = (int)off;   off += al(tsz * maxc);
  a.sm_vals = (int)off;   off += al(tsz * tile);
  a.sm_long = (int)off;   off += al(sizeof(int) * tile_max_long(tile));
  a.sm_start = (int)off;  off += al(sizeof(int) * kFillThreads);
  a.sm_misc = (int)off;   off += al(64 + 8 * 32);
  a.sm_total = (int)off;
  return off <= 227 * 1024 ? VEGAS_OK : VEGAS_EINVAL;
}

}  // namespace

// Per-axis constants (magic reciprocals, z scales, FP32 fraction bits), the
// Philox round keys and the shared-memory layout of a.  a.d, a.G, a.key0 and
// a.key1 must be set.
int fill_args_axes(FillArgs& a, const int32_t* nstrat, int precision, int nprm, bool prefetch, bool streamed) {
  const int G = a.G;
  for (int k = 0; k < a.d; ++k) {
    a.nstrat[k] = (uint32_t)nstrat[k];
    magic_div(a.nstrat[k], a.magic[k], a.shift[k]);
    // z = (c + u) * N_g / s_k: the scale rounded once, in each precision
    a.gz64[k] = (double)G / (double)nstrat[k];
    uint32_t l = 0;
    while ((1u << l) < (uint32_t)nstrat[k]) ++l;
    a.fbits[k] = 23u - l;
    volatile float gf = (float)G, sf = (float)nstrat[k];
    const float g32 = gf / sf;
    a.gzb32[k] = std::ldexp(g32, -(int)a.fbits[k]);
    a.gzn32[k] = -8388608.0f * a.gzb32[k];
  }
  for (int r = 0; r < 10; ++r) {
    a.rk0[r] = a.key0 + (uint32_t)r * 0x9E3779B9u;
    a.rk1[r] = a.key1 + (uint32_t)r * 0xBB67AE85u;
  }
  const size_t tsz = precision == VEGAS_FP64 ? sizeof(double) : sizeof(float);
  return smem_layout(a, tsz, nprm, precision == VEGAS_FP32, true, prefetch, streamed);
}

namespace {

// first cube of every tile: largest h with offsets[h] <= tile * 2^tile_log2; thread
// 0 also resets the max-ell key and writes the FP32 value scale exponent
__global__ void tile_first_kernel(const int64_t* __restrict__ offsets, int NH, int ntiles, int tile_log2, int32_t* tile_first,
                                  int* ellmax_key, int* vexp, int fp32, int integrand, int d,
                                  const double* __restrict__ params, int np) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) {
    *ellmax_key = float_key(-__int_as_float(0x7f800000));
    *vexp = fp32 ? value_exponent(integrand, d, params, np) : 0;
  }
  if (t >= ntiles) return;
  const int64_t j0 = (int64_t)t << tile_log2;
  int lo = 0, hi = NH - 1;
  while (lo < hi) {
    const int mid = (int)(((int64_t)lo + hi + 1) >> 1);
    if (offsets[mid] <= j0) lo = mid;
    else hi = mid - 1;
  }
  tile_first[t] = lo;
}

template <typename T>
// gauss_params: the FP64 Gaussian sum's parameters [A, s, ...], whose point scale gauss_scale64(s) the table
// carries (the fill kernel's prologue does the same), else null
__global__ void table_kernel(const double* __restrict__ edges, int d, int G, TabEntry<T>* tab,
                             const double* __restrict__ gauss_params) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= d * G) return;
  const double xs = gauss_params ? gauss_scale64(gauss_params[1]) : 1.0;
  const int k = b / G, i = b - k * G;
  const double e0 = edges[k * (G + 1) + i], e1 = edges[k * (G + 1) + i + 1];
  const double dx = __dsub_rn(e1, e0), jk = __dmul_rn((double)G, dx);
  tab[b] = TabEntry<T>{(T)(e0 * xs), (T)(dx * xs), (T)jk, T(0)};
}

// Runs of "before" records reduced from the right within blocks of
// kCarryBlock tiles (carry_suffix); one thread per tile.
__global__ void __launch_bounds__(kCarryBlock) carry_scan_kernel(const __grid_constant__ FillArgs a) {
  const int u = blockIdx.x * kCarryBlock + threadIdx.x;
  Carry rec{-1, 0, 0.0, 0.0};
  bool joins = false;
  if (u < a.ntiles) {
    rec = a.carries[2 * u];
    if (rec.h >= 0 && threadIdx.x > 0) joins = a.carries[2 * (u - 1)].h == rec.h;
  }
  rec = carry_suffix(rec, joins);
  if (u < a.ntiles && rec.h >= 0) a.carries[2 * u] = rec;
}

// Merge the parts of every cube that crosses a tile edge.  Thread t owns the
// cube that starts in tile t and ends after it (slot 2t+1); the later parts
// are the "starts before" slots 2u of tiles u > t, pre-reduced per block of
// kCarryBlock tiles, so the walk reads one record per block.
__global__ void fixup_kernel(const __grid_constant__ FillArgs a, double* fix_part) {
  __shared__ double red[32];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double ai = 0.0, av = 0.0;
  float lmax = -__int_as_float(0x7f800000);
  bool broken = false;
  const int e = a.vexp ? *a.vexp : 0;
  if (t < a.ntiles) {
    const Carry r = a.carries[2 * t + 1];
    if (r.h >= 0) {
      const int h = r.h;
      const int64_t n = a.offsets[h + 1] - a.offsets[h];
      double cnt = r.cnt, mean = r.mean, m2 = r.m2;
      for (int u = t + 1; cnt < (double)n && u < a.ntiles; u = (u / kCarryBlock + 1) * kCarryBlock) {
        const Carry q = a.carries[2 * u];
        if (q.h != h) {
          broken = true;
          break;
        }
        chan_merge(cnt, mean, m2, q.cnt, q.mean, q.m2);
      }
      if (cnt != (double)n) broken = true;
      ai = mean;
      av = m2 / ((double)n * (double)(n - 1));
      float l2 = log2r(m2 / (double)(n - 1));
      if (e != 0) l2 += (float)(2 * e);  // the FP32 value scale
      const float ell = __fmul_rn(a.half_beta, l2);
      a.ell[h] = ell;
      lmax = ell;
      if (a.cube_mean) {
        a.cube_mean[h] = ldexp(mean, e);
        a.cube_m2[h] = ldexp(m2, 2 * e);
      }
    }
  }
  const double si = block_sum(ai, red);
  const double sv = block_sum(av, red);
  if (threadIdx.x == 0) {
    fix_part[2 * blockIdx.x] = si;
    fix_part[2 * blockIdx.x + 1] = sv;
  }
  for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  if ((threadIdx.x & 31) == 0) atomicMax(a.ellmax_key, float_key(lmax));
  if (broken) atomicOr(a.flags, 2);
}

// (I_t, sigma_t^2) = (sum mean_h / N_h, sum M2_h/(n_h(n_h-1)) / N_h^2), Eqs. (5)-(6);
// the sums carry the FP32 value scale 2^-vexp, multiplied back here
__global__ void results_kernel(const double* __restrict__ cta_part, int ncta, const double* __restrict__ fix_part,
                               int nfix, int NH, const int* __restrict__ vexp, double* result) {
  __shared__ double red[32];
  double si = 0.0, sv = 0.0;
  for (int i = threadIdx.x; i < ncta; i += blockDim.x) {
    si += cta_part[2 * i];
    sv += cta_part[2 * i + 1];
  }
  for (int i = threadIdx.x; i < nfix; i += blockDim.x) {
    si += fix_part[2 * i];
    sv += fix_part[2 * i + 1];
  }
  si = block_sum(si, red);
  sv = block_sum(sv, red);
  if (threadIdx.x == 0) {
    const int e = *vexp;
    result[0] = ldexp(si / (double)NH, e);
    result[1] = ldexp(sv / ((double)NH * (double)NH), 2 * e);
  }
}

// map weights: sum the per-CTA histograms.  A block owns 32 bins (one per
// lane); its 8 warps take every 8th CTA, and the 8 warp sums are added in
// warp order, so the order is fixed.
__global__ void __launch_bounds__(256) bins_kernel(const double* __restrict__ hist_part, int ncta, int dG,
                                                   const int* __restrict__ vexp, double* bins) {
  __shared__ double part[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int b = blockIdx.x * 32 + lane;
  double s = 0.0;
  if (b < dG)
    for (int c = w; c < ncta; c += 8) s += hist_part[(size_t)c * dG + b];
  part[w][lane] = s;
  __syncthreads();
  if (w == 0 && b < dG) {
    double t = 0.0;
    for (int k = 0; k < 8; ++k) t += part[k][lane];
    bins[b] = ldexp(t, 2 * *vexp);
  }
}


}  // namespace
}  // namespace vg

using namespace vg;

extern "C" size_t vegas_fill_scratch_bytes(const vegas_geometry* g, int64_t neval) {
  if (!g || g->dim < 1 || g->dim > kMaxDim || g->nbins < 2 || g->nbins > kMaxBins || neval < 1) return 0;
  return scratch_layout(g->dim, g->nbins, neval, num_sms()).total;
}

namespace vg {
// One plan per tile size: the shared-memory layout, the kernel it selects and its resident CTAs per SM.  A
// launch takes the larger tile (fewer tile prologues and barriers) unless that loses the exact-d path or a
// resident CTA, as the staging grows with the tile (d = 8: 2048 at 4 CTAs an SM; d = 12 to 30, streamed: 1024).
namespace {
int plan_one(const FillArgs& base, const int32_t* nstrat, int precision, int integrand, int64_t nparams, int nprm,
             int tile_log2, FillPlan& p) {
  const int d = base.d, G = base.G, dmax = dmax_for(d);
  const bool internal = integrand == kIntegrandTabulated || integrand == kIntegrandPoints;
  p.a = base;
  p.a.tile_log2 = tile_log2;
  p.a.ntiles = (int)((base.neval + (int64_t(1) << tile_log2) - 1) >> tile_log2);
  // the prefetch buffer: every kernel but the exact-d FP32 ones and the streamed ones (the kernel's own rule); first
  // laid out without it for FP32 with DMAX <= 8, where the exact-d path may apply
  if (fill_args_axes(p.a, nstrat, precision, nprm, !(precision == VEGAS_FP32 && dmax <= 8)) != VEGAS_OK)
    return VEGAS_EINVAL;
  p.exact = d == dmax && (dmax == 4 || dmax == 8) && p.a.table_smem && !internal && G <= 256;
  // the general FP32 kernels with DMAX <= 8 take the prefetch buffer (only the exact-d ones go without): lay out
  // again with it; the larger layout cannot make the exact-d path possible
  if (!p.exact && precision == VEGAS_FP32 && dmax <= 8 &&
      fill_args_axes(p.a, nstrat, precision, nprm, true) != VEGAS_OK)
    return VEGAS_EINVAL;
  // the streamed point path: FP32, 16 or 32 axes, two-phase histogram, at most 256 strata an axis
  p.streamed = precision == VEGAS_FP32 && dmax >= 16 && p.a.hist_mode == kHistTwoPhase &&
               stream_family(integrand, integrand == VEGAS_GAUSS_SUM ? (int)((nparams - 3) / d) : 0);
  for (int k = 0; k < d && p.streamed; ++k) p.streamed = nstrat[k] <= 256;
  // the streamed kernels' own layout: no prefetch buffer, no weight slots, an FP32 CTA histogram (their rule).
  // It is smaller than the layout above, so the two-phase histogram still fits; were it not, the general kernel runs
  if (p.streamed) {
    FillArgs b = p.a;
    if (fill_args_axes(b, nstrat, precision, nprm, false, true) == VEGAS_OK && b.hist_mode == kHistTwoPhase)
      p.a = b;
    else
      p.streamed = false;
  }
  // the streamed path takes its map table from global memory (read through L1) when that frees enough
  // shared memory for one more resident CTA: d = 30, 1e8 evaluations, 3 CTAs an SM instead of 2,
  // 16.5 -> 14.6 ms (its lookups are random either way; the table stays in L1)
  if (p.streamed && p.a.table_smem) {
    FillArgs b = p.a;
    smem_layout(b, sizeof(float), nprm, true, false, false, true);
    if (b.hist_mode == p.a.hist_mode &&
        fill_occupancy_f32_stream(integrand, dmax, tile_log2, b.sm_total) >
            fill_occupancy_f32_stream(integrand, dmax, tile_log2, p.a.sm_total))
      p.a = b;
  }
  // the general FP32 kernels, too, read the map table from global memory (through L1) when that gives more
  // resident CTAs: the 1000-Gaussian ridge in d = 4 with N_g = 1024 held 2 CTAs an SM with its 64 KB table in
  // shared memory
  if (!p.exact && !p.streamed && precision == VEGAS_FP32 && p.a.table_smem) {
    FillArgs b = p.a;
    smem_layout(b, sizeof(float), nprm, true, false, true, false);
    if (fill_occupancy_f32(integrand, dmax, tile_log2, b.sm_total) >
        fill_occupancy_f32(integrand, dmax, tile_log2, p.a.sm_total))
      p.a = b;
  }
  const int sm = p.a.sm_total;
  const int tl = tile_log2;
  p.per_sm = precision == VEGAS_FP64
                 ? (p.exact ? fill_occupancy_f64_exact(integrand, dmax, tl, sm) : fill_occupancy_f64(integrand, dmax, tl, sm))
                 : (p.exact      ? fill_occupancy_f32_exact(integrand, dmax, tl, sm)
                    : p.streamed ? fill_occupancy_f32_stream(integrand, dmax, tl, sm)
                                 : fill_occupancy_f32(integrand, dmax, tl, sm));
  return p.per_sm > 0 ? VEGAS_OK : VEGAS_ECUDA;
}
}  // namespace

int fill_plan(const FillArgs& base, const int32_t* nstrat, int precision, int integrand, int64_t nparams, int nprm,
              FillPlan& out, int tile_log2) {
  if (tile_log2 != 0) {
    if (tile_log2 < kTileLog2Min || tile_log2 > kTileLog2Max) return VEGAS_EINVAL;
    return plan_one(base, nstrat, precision, integrand, nparams, nprm, tile_log2, out);
  }
  FillPlan big, small;
  const int rbig = plan_one(base, nstrat, precision, integrand, nparams, nprm, kTileLog2Max, big);
  const int rsmall = plan_one(base, nstrat, precision, integrand, nparams, nprm, kTileLog2Min, small);
  if (rbig != VEGAS_OK && rsmall != VEGAS_OK) return rsmall;
  const bool take_big = rbig == VEGAS_OK && (rsmall != VEGAS_OK || (big.exact && !small.exact) ||
                                             (big.exact == small.exact && big.per_sm >= small.per_sm));
  out = take_big ? big : small;
  return VEGAS_OK;
}

int fill_impl(const vegas_geometry* g, int precision, int integrand, const double* d_params, int64_t nparams,
              int64_t neval, uint64_t seed, int32_t iteration, uint32_t problem_id, double beta,
              const double* d_edges, const int64_t* d_offsets, float* d_ell, double* d_bins, double* d_result,
              double* d_cube_mean, double* d_cube_m2, int* d_flags, void* d_scratch, size_t scratch_bytes,
              void* stream, cudaEvent_t ev_before, cudaEvent_t ev_after, const FillExtra* extra) {
  const bool internal = integrand == kIntegrandTabulated || integrand == kIntegrandPoints;
  if (internal) {
    if (precision != VEGAS_FP32 || !extra) return VEGAS_EINVAL;
    if (integrand == kIntegrandTabulated && (!extra->values || (extra->train_w && extra->train_stride < 1)))
      return VEGAS_EINVAL;
    if (integrand == kIntegrandPoints && !extra->points) return VEGAS_EINVAL;
  }
  if (!g || !g->nstrat || g->dim < 1 || g->dim > kMaxDim || g->nbins < 2 || g->nbins > kMaxBins)
    return VEGAS_EINVAL;
  if (precision != VEGAS_FP64 && precision != VEGAS_FP32) return VEGAS_EINVAL;
  if (!d_edges || !d_offsets || !d_ell || !d_bins || !d_result || !d_flags || !d_scratch) return VEGAS_EINVAL;
  if ((d_cube_mean == nullptr) != (d_cube_m2 == nullptr)) return VEGAS_EINVAL;
  if (nparams > 0 && !d_params) return VEGAS_EINVAL;
  if (!(beta >= 0.0 && beta <= 1.0) || iteration < 0 || problem_id > 0xFFFFu) return VEGAS_EINVAL;
  const int d = g->dim, G = g->nbins;
  int64_t NH = 1;
  for (int k = 0; k < d; ++k) {
    if (g->nstrat[k] < 1) return VEGAS_EINVAL;
    if (precision == VEGAS_FP32 && g->nstrat[k] > 65536) return VEGAS_EINVAL;
    NH *= g->nstrat[k];
    if (NH >= (int64_t(1) << 31)) return VEGAS_EINVAL;
  }
  if (neval < 2 * NH || neval > kMaxEval) return VEGAS_EINVAL;
  const int npd = derived_param_count(integrand, d, nullptr, nparams);
  if (npd < 0) return VEGAS_EINVAL;
  const int dmax = dmax_for(d);
  const int nprm = derived_smem_count(integrand, d, dmax, (int)nparams);
  if (nprm > kMaxDerivedParams) return VEGAS_EINVAL;

  const int sms = num_sms();
  if (sms <= 0) return VEGAS_ECUDA;
  const ScratchLayout L = scratch_layout(d, G, neval, sms);
  if (scratch_bytes < L.total) return VEGAS_ENOSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* sc = (unsigned char*)d_scratch;

  FillArgs a{};
  a.d = d;
  a.G = G;
  a.NH = (int)NH;
  a.neval = neval;
  a.key0 = (uint32_t)seed;
  a.key1 = (uint32_t)(seed >> 32);
  a.iter = (uint32_t)iteration;
  a.pid = problem_id;
  a.half_beta = (float)beta * 0.5f;
  a.np_derived = npd;
  a.iid = integrand;
  a.edges = d_edges;
  a.offsets = d_offsets;
  a.tile_first = (const int32_t*)(sc + L.tile_first);
  a.params_raw = d_params;
  a.np_raw = (int)nparams;
  a.ell = d_ell;
  a.cube_mean = d_cube_mean;
  a.cube_m2 = d_cube_m2;
  a.flags = d_flags;
  a.ellmax_key = (int*)(sc + L.ellmax);
  a.carries = (Carry*)(sc + L.carries);
  a.cta_part = (double*)(sc + L.cta_part);
  a.hist_part = (double*)(sc + L.hist_part);
  a.gtable = sc + L.gtable;
  a.vexp = (const int*)(sc + L.ellmax + 4);
  if (extra) {
    a.values = extra->values;
    a.points_out = extra->points;
    a.train_w = extra->train_w;
    a.train_stride = extra->train_stride > 0 ? extra->train_stride : 1;
    a.train_power = extra->train_power;
  }
  FillPlan P;
  const int rp = fill_plan(a, g->nstrat, precision, integrand, nparams, nprm, P, g->tile_log2);
  if (rp != VEGAS_OK) return rp;
  a = P.a;
  const bool exact = P.exact, streamed = P.streamed;
  const int per_sm = P.per_sm;
  const int nfix = (a.ntiles + 255) / 256;
  const int grid = std::max(1, std::min(std::min(L.grid_max, per_sm * sms), a.ntiles));

  tile_first_kernel<<<(a.ntiles + 255) / 256, 256, 0, s>>>(d_offsets, a.NH, a.ntiles, a.tile_log2,
                                                            (int32_t*)(sc + L.tile_first),
                                                            a.ellmax_key, (int*)a.vexp, precision == VEGAS_FP32,
                                                            integrand, d, d_params, (int)nparams);
  VG_CHECK(cudaGetLastError());
  if (a.hist_mode == kHistGlobal)
    VG_CHECK(cudaMemsetAsync(a.hist_part, 0, sizeof(double) * (size_t)grid * d * G, s));
  if (!a.table_smem) {
    const int n = d * G;
    if (precision == VEGAS_FP64)
      table_kernel<double><<<(n + 255) / 256, 256, 0, s>>>(d_edges, d, G, (TabEntry<double>*)a.gtable,
                                                          integrand == VEGAS_GAUSS_SUM ? d_params : nullptr);
    else
      table_kernel<float><<<(n + 255) / 256, 256, 0, s>>>(d_edges, d, G, (TabEntry<float>*)a.gtable, nullptr);
    VG_CHECK(cudaGetLastError());
  }
  if (ev_before) VG_CHECK(cudaEventRecord(ev_before, s));
  const int rc = precision == VEGAS_FP64
                     ? (exact ? launch_fill_f64_exact(integrand, dmax, a, grid, s) : launch_fill_f64(integrand, dmax, a, grid, s))
                     : (exact    ? launch_fill_f32_exact(integrand, dmax, a, grid, s)
                        : streamed ? launch_fill_f32_stream(integrand, dmax, a, grid, s)
                                 : launch_fill_f32(integrand, dmax, a, grid, s));
  if (rc != VEGAS_OK) return rc;
  if (ev_after) VG_CHECK(cudaEventRecord(ev_after, s));
  if (integrand == kIntegrandPoints) return VEGAS_OK;  // no sums: the points are the output
  double* fix_part = (double*)(sc + L.fix_part);
  carry_scan_kernel<<<nfix, kCarryBlock, 0, s>>>(a);
  VG_CHECK(cudaGetLastError());
  fixup_kernel<<<nfix, 256, 0, s>>>(a, fix_part);
  VG_CHECK(cudaGetLastError());
  results_kernel<<<1, 256, 0, s>>>(a.cta_part, grid, fix_part, nfix, a.NH, a.vexp, d_result);
  VG_CHECK(cudaGetLastError());
  bins_kernel<<<(d * G + 31) / 32, 256, 0, s>>>(a.hist_part, grid, d * G, a.vexp, d_bins);
  VG_CHECK(cudaGetLastError());
  return VEGAS_OK;
}
}  // namespace vg

extern "C" int vegas_fill(const vegas_geometry* g, int precision, int integrand, const double* d_params,
                          int64_t nparams, int64_t neval, uint64_t seed, int32_t iteration, uint32_t problem_id,
                          double beta, const double* d_edges, const int64_t* d_offsets, float* d_ell,
                          double* d_bins, double* d_result, double* d_cube_mean, double* d_cube_m2, int* d_flags,
                          void* d_scratch, size_t scratch_bytes, void* stream) {
  return fill_impl(g, precision, integrand, d_params, nparams, neval, seed, iteration, problem_id, beta, d_edges,
                   d_offsets, d_ell, d_bins, d_result, d_cube_mean, d_cube_m2, d_flags, d_scratch, scratch_bytes,
                   stream, nullptr, nullptr);
}


namespace vg {
const int* fill_ellmax_key(const vegas_geometry* g, int64_t neval, const void* d_scratch) {
  const ScratchLayout L = scratch_layout(g->dim, g->nbins, neval, num_sms());
  return (const int*)((const unsigned char*)d_scratch + L.ellmax);
}
}  // namespace vg
