// vegas_map.cuh -- device code of the map refinement (adjustWeights +
// updateMap of Algorithm 1 in cuVegas; Sec. 2.1.1, refinement with damping
// alpha), shared by the single-integral entry point and the batched driver.
#pragma once
#include <cmath>

#include "vegas_device.cuh"

namespace vg {

// One CTA per axis.  Smooth the weights (7,1)/8 - (1,6,1)/8 - (1,7)/8,
// normalise to r_i, damp m_i = ((1 - r_i)/ln(1/r_i))^alpha, then place edge j
// where the cumulative damped weight reaches j * sum(m) / N_g.  The weight is
// uniform inside each old interval.
// w: the axis's weights; ei / eo: its old and new edges (may not alias);
// sh: 2G doubles of shared memory.  Called by a whole CTA.
__device__ __forceinline__ void refine_axis_body(int G, double alpha, const double* __restrict__ w,
                                                 const double* __restrict__ ei, double* __restrict__ eo, double* sh) {
  double* m = sh;          // [G] smoothed weights, then damped weights
  double* P = sh + G;      // [G] inclusive prefix of m
  __shared__ double red[32];
  __shared__ int flags[2];  // [0] bad weight, [1] some positive weight
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) flags[0] = flags[1] = 0;
  __syncthreads();
  for (int i = tid; i < G; i += nt) {
    const double v = w[i];
    if (!isfinite(v) || v < 0.0) flags[0] = 1;
    if (v > 0.0) flags[1] = 1;
  }
  __syncthreads();
  if (flags[0] || !flags[1] || alpha == 0.0) {
    for (int i = tid; i <= G; i += nt) eo[i] = ei[i];
    return;
  }
  // smoothing
  for (int i = tid; i < G; i += nt) {
    double s;
    if (i == 0) s = (7.0 * w[0] + w[1]) / 8.0;
    else if (i == G - 1) s = (w[G - 2] + 7.0 * w[G - 1]) / 8.0;
    else s = (w[i - 1] + 6.0 * w[i] + w[i + 1]) / 8.0;
    m[i] = s;
  }
  __syncthreads();
  double part = 0.0;
  for (int i = tid; i < G; i += nt) part += m[i];
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((tid & 31) == 0) red[tid >> 5] = part;
  __syncthreads();
  if (tid == 0) {
    double S = 0.0;
    for (int i = 0; i < nt / 32; ++i) S += red[i];
    red[31] = S;
  }
  __syncthreads();
  const double S = red[31];
  // normalise and damp
  for (int i = tid; i < G; i += nt) {
    const double r = m[i] / S;
    m[i] = r <= 0.0 ? 0.0 : r >= 1.0 ? 1.0 : pow((1.0 - r) / log(1.0 / r), alpha);
  }
  __syncthreads();
  // inclusive prefix of m: each thread a contiguous chunk, then the chunk sums
  const int chunk = (G + nt - 1) / nt;
  const int c0 = tid * chunk, c1 = min(G, c0 + chunk);
  double run = 0.0;
  for (int i = c0; i < c1; ++i) {
    run += m[i];
    P[i] = run;
  }
  double x = run;
  const int lane = tid & 31, wid = tid >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) red[wid] = x;
  __syncthreads();
  double before = x - run;
  for (int q = 0; q < wid; ++q) before += red[q];
  for (int i = c0; i < c1; ++i) P[i] += before;
  __syncthreads();
  const double total = P[G - 1];
  const double step = total / G;
  // new inner edges
  for (int j = 1 + tid; j < G; j += nt) {
    const double target = j * step;
    int lo = 0, hi = G - 1;  // smallest i with P[i] > target, at most G-1
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (P[mid] > target) hi = mid;
      else lo = mid + 1;
    }
    const int i = lo;
    const double acc = i > 0 ? P[i - 1] : 0.0;
    double frac = m[i] > 0.0 ? (target - acc) / m[i] : 0.0;
    frac = frac < 0.0 ? 0.0 : (frac > 1.0 ? 1.0 : frac);
    eo[j] = ei[i] + frac * (ei[i + 1] - ei[i]);
  }
  if (tid == 0) {
    eo[0] = ei[0];
    eo[G] = ei[G];
  }
  __syncthreads();
  // strictly increasing inner edges, below the last edge
  if (tid == 0) {
    for (int j = 1; j < G; ++j)
      if (!(eo[j] > eo[j - 1])) eo[j] = nextafter(eo[j - 1], INFINITY);
    for (int j = G - 1; j >= 1; --j)
      if (!(eo[j] < eo[j + 1])) eo[j] = nextafter(eo[j + 1], -INFINITY);
  }
}

// Eqs. (8)-(9) over iterations t >= skip; iterations with sigma_t = 0 give
// their mean exactly with sigma 0.  out = {estimate, sigma, chi2/dof, n_used}.
// lagged: iteration t is weighted by 1/sigma_{t-1}^2, the variance estimate of
// the iteration before it (its own for t = 0 or when sigma_{t-1} = 0).  Those
// samples are independent of iteration t's, so the weight carries no
// information about I_t and the weighted mean stays unbiased when I_t and
// sigma_t are correlated (heavy-tailed weights: a run that misses the tail is
// low in both).  The variance of a mean with such weights is
// sum w_t^2 sigma_t^2 / (sum w_t)^2; with equal sigma both forms reduce to the
// plain mean and sigma / sqrt(n).
__device__ __forceinline__ void combine_dev(const double* est, const double* sig, int n, int skip, double* out,
                                            bool lagged = false) {
  if (skip < 0) skip = 0;
  const int used = n - skip;
  if (used <= 0) {
    out[0] = out[1] = out[2] = nan("");
    out[3] = 0.0;
    return;
  }
  int nzero = 0;
  double zsum = 0.0;
  for (int t = skip; t < n; ++t)
    if (sig[t] == 0.0) {
      ++nzero;
      zsum += est[t];
    }
  if (nzero > 0) {
    const double mean = zsum / nzero;
    bool agree = true;
    for (int t = skip; t < n; ++t)
      if (sig[t] == 0.0 && est[t] != mean) agree = false;
    out[0] = mean;
    out[1] = 0.0;
    out[2] = agree ? 0.0 : INFINITY;
    out[3] = used;
    return;
  }
  double wsum = 0.0, wisum = 0.0, w2var = 0.0;
  for (int t = skip; t < n; ++t) {
    const double sw = (lagged && t > 0 && sig[t - 1] > 0.0) ? sig[t - 1] : sig[t];
    const double w = 1.0 / (sw * sw);
    wsum += w;
    wisum += w * est[t];
    w2var += w * w * sig[t] * sig[t];
  }
  const double mean = wisum / wsum;
  double chi2 = 0.0;
  for (int t = skip; t < n; ++t) {
    const double dv = est[t] - mean;
    chi2 += dv * dv / (sig[t] * sig[t]);
  }
  out[0] = mean;
  out[1] = lagged ? sqrt(w2var) / wsum : sqrt(1.0 / wsum);
  out[2] = used > 1 ? chi2 / (used - 1) : 0.0;
  out[3] = used;
}

// combine_dev over one block of kCombineThreads threads, for the handle, which
// combines after every iteration: iteration t is summed by thread
// (t - skip) mod kCombineThreads and the partial sums meet in a fixed tree, so
// the result is deterministic and a call costs O(n / kCombineThreads) instead
// of O(n) on one thread (a 6000-iteration run spent most of its time there).
constexpr int kCombineThreads = 256;

__device__ __forceinline__ double combine_tree_sum(double v, double* buf) {
  const int tid = threadIdx.x;
  buf[tid] = v;
  __syncthreads();
#pragma unroll 1
  for (int s = kCombineThreads / 2; s > 0; s >>= 1) {
    if (tid < s) buf[tid] += buf[tid + s];
    __syncthreads();
  }
  const double r = buf[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ void combine_block(const double* est, const double* sig, int n, int skip, double* out,
                                              bool lagged) {
  __shared__ double buf[kCombineThreads];
  const int tid = threadIdx.x;
  if (skip < 0) skip = 0;
  const int used = n - skip;
  if (used <= 0) {
    if (tid == 0) {
      out[0] = out[1] = out[2] = nan("");
      out[3] = 0.0;
    }
    return;
  }
  double nz = 0.0, zs = 0.0, ws = 0.0, wi = 0.0, w2 = 0.0;
  for (int t = skip + tid; t < n; t += kCombineThreads) {
    if (sig[t] == 0.0) {
      nz += 1.0;
      zs += est[t];
      continue;
    }
    const double sw = (lagged && t > 0 && sig[t - 1] > 0.0) ? sig[t - 1] : sig[t];
    const double w = 1.0 / (sw * sw);
    ws += w;
    wi += w * est[t];
    w2 += w * w * sig[t] * sig[t];
  }
  const double nzero = combine_tree_sum(nz, buf);
  if (nzero > 0.0) {  // exact iterations: their mean, sigma 0
    const double mean = combine_tree_sum(zs, buf) / nzero;
    int bad = 0;
    for (int t = skip + tid; t < n; t += kCombineThreads)
      if (sig[t] == 0.0 && est[t] != mean) bad = 1;
    const int any_bad = __syncthreads_or(bad);
    if (tid == 0) {
      out[0] = mean;
      out[1] = 0.0;
      out[2] = any_bad ? INFINITY : 0.0;
      out[3] = used;
    }
    return;
  }
  const double wsum = combine_tree_sum(ws, buf);
  const double wisum = combine_tree_sum(wi, buf);
  const double w2var = combine_tree_sum(w2, buf);
  const double mean = wisum / wsum;
  double c2 = 0.0;
  for (int t = skip + tid; t < n; t += kCombineThreads) {
    const double dv = est[t] - mean;
    c2 += dv * dv / (sig[t] * sig[t]);
  }
  const double chi2 = combine_tree_sum(c2, buf);
  if (tid == 0) {
    out[0] = mean;
    out[1] = lagged ? sqrt(w2var) / wsum : sqrt(1.0 / wsum);
    out[2] = used > 1 ? chi2 / (used - 1) : 0.0;
    out[3] = used;
  }
}

}  // namespace vg
