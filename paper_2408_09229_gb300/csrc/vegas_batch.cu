// vegas_batch.cu -- the batched form of the iteration loop (Algorithm 1 of
// cuVegas, once per integral of the batch): buffers, the per-iteration
// kernels over the work of every running integral, graph capture and replay,
// the launch-shape tuner, and the C ABI of vegas_batch_*.
//
// One iteration of the batch is a captured graph of:
//   memset     map weights of every integral to zero
//   plan       prefix sums of the tiles and allocation blocks of the running
//              integrals; zero the iteration sums and the work counter
//   bsum       allocation pass 1 (block sums of the quantised weights)
//   scan       allocation pass 2 (one CTA per integral)
//   offsets    allocation pass 3 (counts n_h as offsets, Sec. 2.1.2)
//   tile_first first cube of every tile; reset the max-ell keys
//   fill       Algorithm 2 over all tiles (vegas_batch_fill.cuh)
//   carry_scan runs of tile records of cubes that span tiles, pre-reduced
//   fixup      cubes that cross tile edges
//   refine     the map of every running integral, in place (Sec. 2.1.1)
//   finish     record (I_t, sigma_t), Eqs. (8)-(9), the rtol test, and the
//              count of integrals still running
// The host replays the graph and reads that count after each iteration.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "vegas_alloc.cuh"
#include "vegas_batch.cuh"
#include "vegas_device.cuh"
#include "vegas_fill.cuh"
#include "vegas_internal.h"
#include "vegas_map.cuh"

namespace vg {
namespace {

// ---------------------------------------------------------------------------
// device kernels of one batch iteration
// ---------------------------------------------------------------------------

// exclusive prefix sums over the running integrals of their tiles and
// allocation blocks; one CTA of 1024 threads, 4 integrals a thread
__global__ void __launch_bounds__(1024) batch_plan_kernel(const __grid_constant__ BatchLaunch L) {
  __shared__ int64_t wt[2][32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  int64_t nt[4], nb[4], st = 0, sb = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int p = 4 * tid + i;
    const bool on = p < L.P && L.ctl[p].active;
    nt[i] = on ? L.prob[p].a.ntiles : 0;
    nb[i] = on ? L.prob[p].nblocks : 0;
    st += nt[i];
    sb += nb[i];
  }
  int64_t xt = st, xb = sb;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t yt = __shfl_up_sync(0xffffffffu, xt, o), yb = __shfl_up_sync(0xffffffffu, xb, o);
    if (lane >= o) {
      xt += yt;
      xb += yb;
    }
  }
  if (lane == 31) {
    wt[0][w] = xt;
    wt[1][w] = xb;
  }
  __syncthreads();
  int64_t bt = xt - st, bb = xb - sb;
  for (int k = 0; k < w; ++k) {
    bt += wt[0][k];
    bb += wt[1][k];
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int p = 4 * tid + i;
    if (p < L.P) {
      L.act_tile[p] = (int32_t)bt;
      L.act_blk[p] = bb;
    }
    if (p == L.P - 1) {
      L.act_tile[L.P] = (int32_t)(bt + nt[i]);
      L.act_blk[L.P] = bb + nb[i];
    }
    bt += nt[i];
    bb += nb[i];
  }
  for (int i = tid; i < 2 * L.P; i += blockDim.x) L.acc[i] = 0.0;
  if (tid == 0) {
    L.counter[0] = 0u;
    L.counter[1] = 0u;
  }
}

// the tile prefix of each fill group: block g sums the tiles of the running integrals of group g (the other
// integrals count 0, so a search in the prefix skips them), 4 integrals a thread (P <= 4096); zeroes the group's
// work counter
__global__ void __launch_bounds__(1024) batch_group_plan_kernel(const __grid_constant__ BatchLaunch L) {
  __shared__ int64_t wt[32];
  const int g = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  int32_t* pre = L.grp_tile + (size_t)g * (L.P + 1);
  int64_t nt[4], st = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int p = 4 * tid + i;
    const bool on = p < L.P && L.ctl[p].active && L.prob[p].group == g;
    nt[i] = on ? L.prob[p].a.ntiles : 0;
    st += nt[i];
  }
  int64_t xt = st;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t yt = __shfl_up_sync(0xffffffffu, xt, o);
    if (lane >= o) xt += yt;
  }
  if (lane == 31) wt[w] = xt;
  __syncthreads();
  int64_t bt = xt - st;
  for (int k = 0; k < w; ++k) bt += wt[k];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int p = 4 * tid + i;
    if (p < L.P) pre[p] = (int32_t)bt;
    if (p == L.P - 1) pre[L.P] = (int32_t)(bt + nt[i]);
    bt += nt[i];
  }
  if (tid == 0) L.counter[2 + g] = 0u;
}

__global__ void __launch_bounds__(kAllocThreads) batch_bsum_kernel(const __grid_constant__ BatchLaunch L) {
  const int64_t blk = blockIdx.x;
  if (blk >= L.act_blk[L.P]) return;
  const int p = batch_find(L.act_blk, L.P, blk);
  if (L.ctl[p].uniform) return;
  const BatchProblem& q = L.prob[p];
  block_sum_body(q.a.ell, q.a.NH, L.key + p, 0, q.bsum, blk - L.act_blk[p]);
}

__global__ void __launch_bounds__(1024) batch_scan_kernel(const __grid_constant__ BatchLaunch L) {
  const int p = blockIdx.x;
  if (!L.ctl[p].active || L.ctl[p].uniform) return;
  block_scan_body(L.prob[p].bsum, L.prob[p].nblocks);
}

__global__ void __launch_bounds__(kAllocThreads) batch_offsets_kernel(const __grid_constant__ BatchLaunch L) {
  const int64_t blk = blockIdx.x;
  if (blk >= L.act_blk[L.P]) return;
  const int p = batch_find(L.act_blk, L.P, blk);
  const BatchProblem& q = L.prob[p];
  offsets_body(q.a.ell, q.a.NH, q.a.neval, L.key + p, L.ctl[p].uniform, q.bsum, const_cast<int64_t*>(q.a.offsets),
               blk - L.act_blk[p]);
}

// first cube of every tile of the running integrals; the max-ell keys start
// over for the fill (the offsets pass above has read them)
__global__ void batch_tile_first_kernel(const __grid_constant__ BatchLaunch L) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  if (gt >= L.act_tile[L.P]) return;
  const int p = batch_find(L.act_tile, L.P, gt);
  const int t = gt - L.act_tile[p];
  const FillArgs& a = L.prob[p].a;
  if (t == 0) L.key[p] = float_key(-__int_as_float(0x7f800000));
  const int64_t j0 = (int64_t)t << a.tile_log2;
  int lo = 0, hi = a.NH - 1;
  while (lo < hi) {
    const int mid = (int)(((int64_t)lo + hi + 1) >> 1);
    if (a.offsets[mid] <= j0) lo = mid;
    else hi = mid - 1;
  }
  const_cast<int32_t*>(a.tile_first)[t] = lo;
}

// runs of "before" records reduced from the right within blocks of
// kCarryBlock consecutive tiles of the work list (carry_suffix)
__global__ void __launch_bounds__(kCarryBlock) batch_carry_scan_kernel(const __grid_constant__ BatchLaunch L) {
  const int gt = blockIdx.x * kCarryBlock + threadIdx.x;
  Carry rec{-1, 0, 0.0, 0.0};
  bool joins = false;
  Carry* car = nullptr;
  int t = 0;
  if (gt < L.act_tile[L.P]) {
    const int p = batch_find(L.act_tile, L.P, gt);
    t = gt - L.act_tile[p];
    car = L.prob[p].a.carries;
    rec = car[2 * t];
    if (rec.h >= 0 && threadIdx.x > 0 && t > 0) joins = car[2 * (t - 1)].h == rec.h;
  }
  rec = carry_suffix(rec, joins);
  if (car && rec.h >= 0) car[2 * t] = rec;
}

// cubes that cross tile edges (the single-integral fix-up, per integral of
// the batch); the walk reads one pre-reduced record per block of the work
// list; the sums go to the integral's accumulators, one atomic add per warp
// when the warp's tiles share their integral
__global__ void __launch_bounds__(256) batch_fixup_kernel(const __grid_constant__ BatchLaunch L) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  double ai = 0.0, av = 0.0;
  float lmax = -__int_as_float(0x7f800000);
  bool broken = false, have = false;
  int p = -1;
  if (gt < L.act_tile[L.P]) {
    p = batch_find(L.act_tile, L.P, gt);
    const int t = gt - L.act_tile[p];
    const FillArgs& a = L.prob[p].a;
    const Carry r = a.carries[2 * t + 1];
    if (r.h >= 0) {
      have = true;
      const int h = r.h;
      const int64_t n = a.offsets[h + 1] - a.offsets[h];
      double cnt = r.cnt, mean = r.mean, m2 = r.m2;
      const int base = L.act_tile[p];
      for (int u = t + 1; cnt < (double)n && u < a.ntiles;
           u = ((base + u) / kCarryBlock + 1) * kCarryBlock - base) {
        const Carry c = a.carries[2 * u];
        if (c.h != h) {
          broken = true;
          break;
        }
        chan_merge(cnt, mean, m2, c.cnt, c.mean, c.m2);
      }
      if (cnt != (double)n) broken = true;
      ai = mean;
      av = m2 / ((double)n * (double)(n - 1));
      float l2 = log2r(m2 / (double)(n - 1));
      const int e = a.vexp ? *a.vexp : 0;
      if (e != 0) l2 += (float)(2 * e);  // the FP32 value scale
      const float ell = __fmul_rn(a.half_beta, l2);
      a.ell[h] = ell;
      lmax = ell;
    }
  }
  const int p0 = __shfl_sync(0xffffffffu, p, 0);
  if (__all_sync(0xffffffffu, p == p0)) {
    ai = warp_sum(ai);
    av = warp_sum(av);
    for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    const bool any = __any_sync(0xffffffffu, have);
    if ((threadIdx.x & 31) == 0 && p0 >= 0 && any) {
      atomicAdd(L.acc + 2 * p0, ai);
      atomicAdd(L.acc + 2 * p0 + 1, av);
      atomicMax(L.key + p0, float_key(lmax));
    }
  } else if (have) {
    atomicAdd(L.acc + 2 * p, ai);
    atomicAdd(L.acc + 2 * p + 1, av);
    atomicMax(L.key + p, float_key(lmax));
  }
  if (broken) atomicOr(L.flags + p, 2);
}

// map refinement in place: block (p, k) refines axis k of integral p from a
// shared-memory copy of its edges
__global__ void __launch_bounds__(256) batch_refine_kernel(const __grid_constant__ BatchLaunch L) {
  extern __shared__ double rsh[];
  const int p = blockIdx.x, k = blockIdx.y;
  if (!L.ctl[p].active) return;
  const BatchProblem& q = L.prob[p];
  if (k >= q.a.d) return;
  const int G = L.G;
  double* e = const_cast<double*>(q.a.edges) + (size_t)k * (G + 1);
  double* ecopy = rsh + 2 * G;
  for (int i = threadIdx.x; i <= G; i += blockDim.x) ecopy[i] = e[i];
  __syncthreads();
  refine_axis_body(G, L.alpha, q.bins + (size_t)k * G, ecopy, e, rsh);
}

// (I_t, sigma_t^2) = (sum means / N_h, sum variances / N_h^2), Eqs. (5)-(6);
// record, combine (Eqs. (8)-(9)), advance the Philox iteration and stop the
// integral at the rtol target or on an error flag
__global__ void batch_finish_kernel(const __grid_constant__ BatchLaunch L, double beta, int it_cap) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= L.P) return;
  BatchCtl c = L.ctl[p];
  if (!c.active) return;
  BatchProblem& q = L.prob[p];
  const double NH = (double)q.a.NH;
  const int t = c.nrec;
  if (t >= it_cap) {  // the host sizes the record for every replay; never expected
    atomicOr(L.flags + p, 4);
    c.active = 0;
    L.ctl[p] = c;
    return;
  }
  const int e = q.a.vexp ? *q.a.vexp : 0;  // the sums carry the FP32 value scale 2^-e
  q.it_est[t] = ldexp(L.acc[2 * p] / NH, e);
  q.it_sig[t] = ldexp(sqrt(L.acc[2 * p + 1] / (NH * NH)), e);
  double* out = L.out + 4 * p;
  combine_dev(q.it_est, q.it_sig, t + 1, L.skip, out);
  c.nrec = t + 1;
  c.uniform = beta == 0.0 ? 1 : 0;
  q.a.iter += 1u;
  // the FP32 evaluation's sigma counts as at least its rounding floor (kFp32SigmaFloor)
  if (L.rtol > 0.0 && t + 1 > L.skip && fmax(out[1], kFp32SigmaFloor * fabs(out[0])) <= L.rtol * fabs(out[0])) {
    c.active = 0;
    c.converged = 1;
  }
  if (L.flags[p] != 0) c.active = 0;
  L.ctl[p] = c;
  if (c.active) atomicAdd(L.counter + 1, 1u);
}

// uniform maps, uniform counts, nothing recorded
__global__ void batch_reset_kernel(const __grid_constant__ BatchLaunch L) {
  const int p = blockIdx.x;
  BatchProblem& q = L.prob[p];
  const int G = L.G, d = q.a.d;
  double* e = const_cast<double*>(q.a.edges);
  for (int i = threadIdx.x; i < d * (G + 1); i += blockDim.x) {
    const int k = i / (G + 1), j = i - k * (G + 1);
    (void)k;
    e[i] = (double)j / (double)G;
  }
  if (threadIdx.x == 0) {
    L.ctl[p] = BatchCtl{1, 1, 0, 0};
    q.a.iter = 0u;
    L.flags[p] = 0;
    for (int i = 0; i < 4; ++i) L.out[4 * p + i] = 0.0;
  }
}

// start of an integrate call: every integral without an error runs again
__global__ void batch_activate_kernel(const __grid_constant__ BatchLaunch L) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= L.P) return;
  L.ctl[p].active = L.flags[p] == 0 ? 1 : 0;
  L.ctl[p].converged = 0;
}

// the per-integral iteration records moved to arrays of capacity cap
__global__ void batch_set_records_kernel(BatchProblem* prob, int P, double* est, double* sig, int cap) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  prob[p].it_est = est + (size_t)p * cap;
  prob[p].it_sig = sig + (size_t)p * cap;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

constexpr int kGroupDmax[3] = {4, 8, 16};

// 0.999 quantile of chi2_nu / nu (Wilson-Hilferty), the default bound of VEGAS_RESULT_CHI2_HIGH
double chi2_dof_quantile_999_batch(int nu) {
  const double z = 3.090232306167813;
  const double a = 2.0 / (9.0 * nu);
  const double c = 1.0 - a + z * std::sqrt(a);
  return c * c * c;
}

int num_sms_now() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

int default_nstrat_batch(int64_t neval, int d) {
  const int64_t half = neval / 2;
  int64_t s = 1;
  for (;;) {
    const int64_t cand = s + 1;
    int64_t prod = 1;
    bool over = false;
    for (int k = 0; k < d; ++k) {
      if (prod > half / cand) {
        over = true;
        break;
      }
      prod *= cand;
    }
    if (over || prod > half) break;
    s = cand;
  }
  return (int)std::min<int64_t>(s, 65536);
}

}  // namespace
// the fill of group g: family g / 3, width kGroupDmax[g % 3]
int launch_batch_fill(int variant, int group, const BatchLaunch& L, int grid, int smem, cudaStream_t s) {
  if (variant < 0 || variant >= kBatchVariants || group < 0 || group >= kBatchGroups) return VEGAS_EINVAL;
  const int dmax = kGroupDmax[group % 3];
  switch (group / 3) {
    case 0: return launch_batch_fill_gauss(variant, dmax, group, L, grid, smem, s);
    case 1: return launch_batch_fill_peak(variant, dmax, group, L, grid, smem, s);
    default: return launch_batch_fill_osc(variant, dmax, group, L, grid, smem, s);
  }
}

int batch_fill_occupancy(int variant, int group, int smem) {
  if (variant < 0 || variant >= kBatchVariants || group < 0 || group >= kBatchGroups) return 0;
  const int dmax = kGroupDmax[group % 3];
  switch (group / 3) {
    case 0: return batch_fill_occupancy_gauss(variant, dmax, smem);
    case 1: return batch_fill_occupancy_peak(variant, dmax, smem);
    default: return batch_fill_occupancy_osc(variant, dmax, smem);
  }
}

}  // namespace vg

using namespace vg;

struct HostProblem {
  int d, iid, nstrat, dmax, nprm, tile_log2;
  int64_t neval, NH, ntiles, nblocks;
  int64_t ntiles_cap;  // tiles at the smallest usable tile: the size of its tile arrays
  std::vector<double> params;
};

struct vegas_batch_s {
  int device = 0, P = 0, G = 0, sms = 0;
  double alpha = 0.5, beta = 0.75;
  uint64_t seed = 0;
  int skip = 0;
  cudaStream_t own_stream = nullptr, cap_stream = nullptr, user_stream = nullptr;
  bool has_user_stream = false;
  std::vector<HostProblem> hp;
  int64_t tiles_total = 0, blocks_total = 0;
  int maxd = 1, smem = 0;
  // the shared-memory layouts for tiles of 1024 and 2048 evaluations (layout_ok: it fits) and the tile in use
  FillArgs layout[2] = {};
  bool layout_ok[2] = {false, false};
  int tile_log2 = kTileLog2Max;
  double* d_bins = nullptr;  // all integrals' map weights, contiguous
  size_t bins_total = 0;
  // device memory: one arena, plus the iteration records
  unsigned char* arena = nullptr;
  BatchLaunch L{};
  double* d_it = nullptr;  // [2][P][it_cap]
  int it_cap = 0;
  int rec_bound = 0;  // upper bound of any integral's recorded iterations
  double chi2_bound = 0.0;  // <= 0: the 0.999 quantile of chi2_nu / nu
  // device memory hooks (NULL: cudaMalloc / cudaFree) and the sizes they were asked for
  vegas_alloc_fn al_alloc = nullptr;
  vegas_free_fn al_free = nullptr;
  void* al_ctx = nullptr;
  size_t arena_bytes = 0, it_bytes = 0;
  uint32_t* h_running = nullptr;  // pinned
  double* h_out = nullptr;        // pinned [P][4]
  BatchCtl* h_ctl = nullptr;      // pinned [P]
  int* h_flags = nullptr;         // pinned [P]
  // launch shape and graph
  int variant = 0, ctas_per_sm = 0, chunk = 4;
  int fill_grid[kBatchGroups] = {};        // 0: no integral of the group
  int64_t group_tiles[kBatchGroups] = {};  // tiles of each fill group (all integrals)
  cudaGraphExec_t exec = nullptr;
  bool graph_dirty = true;
  double graph_rtol = -1.0;
  int graph_skip = -1;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaStream_t stream() const { return has_user_stream ? user_stream : own_stream; }
};

namespace {

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DevGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

void* batch_alloc(vegas_batch_s* b, size_t bytes) {
  void* p = nullptr;
  if (b->al_alloc) {
    p = b->al_alloc(b->al_ctx, bytes, (void*)b->stream());
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  return p;
}

// the caller has synchronised the batch's stream (cudaFree also synchronises)
void batch_free(vegas_batch_s* b, void* p, size_t bytes) {
  if (!p) return;
  if (b->al_free) b->al_free(b->al_ctx, p, bytes, (void*)b->stream());
  else cudaFree(p);
}

void release(vegas_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  batch_free(b, b->arena, b->arena_bytes);
  batch_free(b, b->d_it, b->it_bytes);
  if (b->h_running) cudaFreeHost(b->h_running);
  if (b->h_out) cudaFreeHost(b->h_out);
  if (b->h_ctl) cudaFreeHost(b->h_ctl);
  if (b->h_flags) cudaFreeHost(b->h_flags);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->own_stream) cudaStreamDestroy(b->own_stream);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
}

// records of capacity cap for every integral, keeping what is recorded
int ensure_records(vegas_batch_s* b, int need) {
  if (need <= b->it_cap) return VEGAS_OK;
  const int cap = std::max(need, std::max(16, 2 * b->it_cap));
  const size_t nbytes = sizeof(double) * 2 * (size_t)b->P * cap;
  double* nd = (double*)batch_alloc(b, nbytes);
  if (!nd) return VEGAS_ENOMEM;
  cudaStream_t s = b->stream();
  if (b->d_it && b->it_cap > 0) {
    for (int half = 0; half < 2; ++half)
      VG_CHECK(cudaMemcpy2DAsync(nd + (size_t)half * b->P * cap, sizeof(double) * cap,
                                 b->d_it + (size_t)half * b->P * b->it_cap, sizeof(double) * b->it_cap,
                                 sizeof(double) * b->it_cap, b->P, cudaMemcpyDeviceToDevice, s));
  }
  batch_set_records_kernel<<<(b->P + 127) / 128, 128, 0, s>>>(b->L.prob, b->P, nd, nd + (size_t)b->P * cap, cap);
  VG_CHECK(cudaGetLastError());
  VG_CHECK(cudaStreamSynchronize(s));
  batch_free(b, b->d_it, b->it_bytes);
  b->d_it = nd;
  b->it_bytes = nbytes;
  b->it_cap = cap;
  b->graph_dirty = true;
  return VEGAS_OK;
}

// the kernels of one iteration, in stream order on s
int enqueue_iteration(vegas_batch_s* b, const BatchLaunch& L, cudaStream_t s) {
  const int P = b->P;
  VG_CHECK(cudaMemsetAsync(b->d_bins, 0, sizeof(double) * b->bins_total, s));
  batch_plan_kernel<<<1, 1024, 0, s>>>(L);
  VG_CHECK(cudaGetLastError());
  batch_group_plan_kernel<<<kBatchGroups, 1024, 0, s>>>(L);
  VG_CHECK(cudaGetLastError());
  const unsigned nb = (unsigned)std::max<int64_t>(1, b->blocks_total);
  batch_bsum_kernel<<<nb, kAllocThreads, 0, s>>>(L);
  VG_CHECK(cudaGetLastError());
  batch_scan_kernel<<<P, 1024, 0, s>>>(L);
  VG_CHECK(cudaGetLastError());
  batch_offsets_kernel<<<nb, kAllocThreads, 0, s>>>(L);
  VG_CHECK(cudaGetLastError());
  const unsigned ntb = (unsigned)((b->tiles_total + 255) / 256);
  batch_tile_first_kernel<<<ntb, 256, 0, s>>>(L);
  VG_CHECK(cudaGetLastError());
  for (int g = 0; g < kBatchGroups; ++g) {
    if (b->fill_grid[g] <= 0) continue;  // no integral of this group
    const int rc = launch_batch_fill(b->variant, g, L, b->fill_grid[g], b->smem, s);
    if (rc != VEGAS_OK) return rc;
  }
  batch_carry_scan_kernel<<<ntb, kCarryBlock, 0, s>>>(L);
  VG_CHECK(cudaGetLastError());
  batch_fixup_kernel<<<ntb, 256, 0, s>>>(L);
  VG_CHECK(cudaGetLastError());
  const size_t rsmem = sizeof(double) * (3 * (size_t)b->G + 1);
  batch_refine_kernel<<<dim3(P, b->maxd), 256, rsmem, s>>>(L);
  VG_CHECK(cudaGetLastError());
  batch_finish_kernel<<<(P + 127) / 128, 128, 0, s>>>(L, b->beta, b->it_cap);
  VG_CHECK(cudaGetLastError());
  return VEGAS_OK;
}

}  // namespace

namespace {

// capture one iteration on the batch's capture stream and instantiate it
int capture(vegas_batch_s* b, double rtol) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  BatchLaunch L = b->L;
  L.rtol = rtol;
  L.skip = b->skip;
  L.chunk_tiles = b->chunk;
  // each group's fill grid: resident CTAs per SM (sets the kernel's shared-memory attribute) times SMs, at most
  // the group's tiles; 0 for a group with no integral
  for (int g = 0; g < kBatchGroups; ++g) {
    b->fill_grid[g] = 0;
    if (b->group_tiles[g] == 0) continue;
    const int occ = batch_fill_occupancy(b->variant, g, b->smem);
    if (occ <= 0) return VEGAS_ECUDA;
    const int per_sm = b->ctas_per_sm > 0 ? std::min(b->ctas_per_sm, occ) : occ;
    b->fill_grid[g] = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * b->sms, b->group_tiles[g]));
  }
  cudaGraph_t g = nullptr;
  VG_CHECK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
  const int rc = enqueue_iteration(b, L, b->cap_stream);
  const cudaError_t ec = cudaStreamEndCapture(b->cap_stream, &g);
  if (rc != VEGAS_OK || ec != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc != VEGAS_OK ? rc : VEGAS_ECUDA;
  }
  const cudaError_t ei = cudaGraphInstantiate(&b->exec, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    b->exec = nullptr;
    return VEGAS_ECUDA;
  }
  b->graph_dirty = false;
  b->graph_rtol = rtol;
  b->graph_skip = b->skip;
  return VEGAS_OK;
}

int run_iterations(vegas_batch_s* b, int nitn, double rtol, int* nrun, float* ms) {
  cudaStream_t s = b->stream();
  int rc = ensure_records(b, b->rec_bound + nitn);
  if (rc != VEGAS_OK) return rc;
  if (b->graph_dirty || !b->exec || b->graph_rtol != rtol || b->graph_skip != b->skip) {
    if ((rc = capture(b, rtol)) != VEGAS_OK) return rc;
  }
  batch_activate_kernel<<<(b->P + 127) / 128, 128, 0, s>>>(b->L);
  VG_CHECK(cudaGetLastError());
  VG_CHECK(cudaEventRecord(b->ev0, s));
  int it = 0;
  for (; it < nitn; ++it) {
    VG_CHECK(cudaGraphLaunch(b->exec, s));
    b->rec_bound++;
    VG_CHECK(cudaMemcpyAsync(b->h_running, b->L.counter + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    VG_CHECK(cudaStreamSynchronize(s));
    if (*b->h_running == 0u) {
      ++it;
      break;
    }
  }
  VG_CHECK(cudaEventRecord(b->ev1, s));
  VG_CHECK(cudaEventSynchronize(b->ev1));
  if (ms) VG_CHECK(cudaEventElapsedTime(ms, b->ev0, b->ev1));
  if (nrun) *nrun = it;
  return VEGAS_OK;
}

int reset_batch(vegas_batch_s* b) {
  cudaStream_t s = b->stream();
  batch_reset_kernel<<<b->P, 256, 0, s>>>(b->L);
  VG_CHECK(cudaGetLastError());
  VG_CHECK(cudaStreamSynchronize(s));
  b->rec_bound = 0;
  return VEGAS_OK;
}

}  // namespace

extern "C" int vegas_batch_create(const vegas_problem* problems, int32_t nproblems, int32_t nbins, double alpha,
                                  double beta, uint64_t seed, vegas_batch* out) {
  return vegas_batch_create_ex(problems, nproblems, nbins, alpha, beta, seed, nullptr, nullptr, nullptr, out);
}

extern "C" int vegas_batch_create_ex(const vegas_problem* problems, int32_t nproblems, int32_t nbins, double alpha,
                                     double beta, uint64_t seed, vegas_alloc_fn alloc, vegas_free_fn free_fn,
                                     void* ctx, vegas_batch* out) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return VEGAS_EINVAL;
  if (!out || !problems || nproblems < 1 || nproblems > kBatchMaxProblems) return VEGAS_EINVAL;
  if (nbins < 2 || nbins > 256 || !(alpha >= 0.0) || !(beta >= 0.0 && beta <= 1.0)) return VEGAS_EINVAL;
  *out = nullptr;
  const int P = nproblems, G = nbins;
  std::vector<HostProblem> hp(P);
  int64_t tiles = 0, blocks = 0;
  int maxd = 1, nprm_max = 4;
  for (int p = 0; p < P; ++p) {
    const vegas_problem& q = problems[p];
    HostProblem& h = hp[p];
    if (q.dim < 1 || q.dim > kBatchMaxDim) return VEGAS_EINVAL;
    if (q.integrand != VEGAS_GAUSS_SUM && q.integrand != VEGAS_PRODUCT_PEAK && q.integrand != VEGAS_OSCILLATORY)
      return VEGAS_EINVAL;
    if (q.nparams < 0 || (q.nparams > 0 && !q.params)) return VEGAS_EINVAL;
    if (derived_param_count(q.integrand, q.dim, q.params, q.nparams) < 0) return VEGAS_EINVAL;
    if (q.neval < 2 || q.neval > kMaxEval) return VEGAS_EINVAL;
    h.d = q.dim;
    h.iid = q.integrand;
    h.neval = q.neval;
    h.nstrat = q.nstrat > 0 ? q.nstrat : default_nstrat_batch(q.neval, q.dim);
    if (h.nstrat > 65536) return VEGAS_EINVAL;
    int64_t NH = 1;
    for (int k = 0; k < h.d; ++k) {
      NH *= h.nstrat;
      if (NH >= (int64_t(1) << 31)) return VEGAS_EINVAL;
    }
    if (q.neval < 2 * NH) return VEGAS_EINVAL;
    h.NH = NH;
    h.nblocks = (NH + kBlockCubes - 1) / kBlockCubes;
    h.dmax = dmax_for(h.d);
    h.nprm = derived_smem_count(h.iid, h.d, h.dmax, (int)q.nparams);
    if (h.nprm > kMaxDerivedParams) return VEGAS_EINVAL;
    // integrals wider than 8 axes run the streamed point path
    if (h.dmax >= 16 && (h.nstrat > 256 || !stream_family(h.iid, h.iid == VEGAS_GAUSS_SUM ? (int)((q.nparams - 3) / h.d) : 0)))
      return VEGAS_EINVAL;
    h.params.assign(q.params, q.params + q.nparams);
    blocks += h.nblocks;
    maxd = std::max(maxd, h.d);
    nprm_max = std::max(nprm_max, h.nprm);
  }
  // one shared-memory layout for every integral: the widest map and parameter set, for each tile size whose
  // layout fits; the batch starts at 2048 evaluations where that fits (the 256-integral workload: 112 ms an
  // iteration against 123 with tiles of 1024), and vegas_batch_tune / vegas_batch_set_tile may change it
  FillArgs layouts[2] = {};
  bool ok[2] = {false, false};
  {
    std::vector<int32_t> ones(maxd, 1);
    for (int i = 0; i < 2; ++i) {
      FillArgs& l = layouts[i];
      l.d = maxd;
      l.G = G;
      l.tile_log2 = kTileLog2Min + i;
      ok[i] = fill_args_axes(l, ones.data(), VEGAS_FP32, nprm_max, false) == VEGAS_OK && l.table_smem &&
              l.hist_mode == kHistTwoPhase;
    }
    if (!ok[0] && !ok[1]) return VEGAS_EINVAL;
  }
  const int tile0 = ok[1] ? kTileLog2Max : kTileLog2Min, tile_min = ok[0] ? kTileLog2Min : kTileLog2Max;
  int64_t tiles_cap = 0;
  for (HostProblem& h : hp) {
    h.tile_log2 = tile0;
    h.ntiles = (h.neval + (int64_t(1) << tile0) - 1) >> tile0;
    h.ntiles_cap = (h.neval + (int64_t(1) << tile_min) - 1) >> tile_min;
    tiles += h.ntiles;
    tiles_cap += h.ntiles_cap;
  }
  if (tiles_cap >= (int64_t(1) << 31) || blocks >= (int64_t(1) << 31)) return VEGAS_EINVAL;
  const FillArgs& layout = layouts[tile0 - kTileLog2Min];

  vegas_batch_s* b = new (std::nothrow) vegas_batch_s;
  if (!b) return VEGAS_ENOMEM;
  b->P = P;
  b->G = G;
  b->alpha = alpha;
  b->beta = beta;
  b->seed = seed;
  b->al_alloc = alloc;
  b->al_free = free_fn;
  b->al_ctx = ctx;
  b->hp = std::move(hp);
  b->tiles_total = tiles;
  b->blocks_total = blocks;
  b->maxd = maxd;
  b->smem = layout.sm_total;
  b->tile_log2 = tile0;
  for (int i = 0; i < 2; ++i) {
    b->layout[i] = layouts[i];
    b->layout_ok[i] = ok[i];
  }
  auto fail = [&](int rc) {
    release(b);
    delete b;
    return rc;
  };
  if (cudaGetDevice(&b->device) != cudaSuccess) return fail(VEGAS_ECUDA);
  b->sms = num_sms_now();
  if (b->sms <= 0) return fail(VEGAS_ECUDA);
  if (cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess)
    return fail(VEGAS_ECUDA);

  // arena layout
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align256(off + bytes);
    return at;
  };
  const size_t o_prob = take(sizeof(BatchProblem) * P), o_ctl = take(sizeof(BatchCtl) * P),
               o_act_tile = take(sizeof(int32_t) * (P + 1)), o_act_blk = take(sizeof(int64_t) * (P + 1)),
               o_grp_tile = take(sizeof(int32_t) * kBatchGroups * (P + 1)),
               o_counter = take(sizeof(uint32_t) * (2 + kBatchGroups)), o_acc = take(sizeof(double) * 2 * P),
               o_key = take(sizeof(int) * P), o_flags = take(sizeof(int) * P), o_out = take(sizeof(double) * 4 * P),
               o_vexp = take(sizeof(int) * P);
  std::vector<size_t> o_edges(P), o_bins(P), o_params(P), o_offsets(P), o_ell(P), o_tf(P), o_car(P), o_bsum(P);
  size_t bins_begin = off;
  for (int p = 0; p < P; ++p) o_bins[p] = off, off += sizeof(double) * (size_t)b->hp[p].d * G;
  b->bins_total = (off - bins_begin) / sizeof(double);
  off = align256(off);
  for (int p = 0; p < P; ++p) o_edges[p] = take(sizeof(double) * (size_t)b->hp[p].d * (G + 1));
  for (int p = 0; p < P; ++p) o_params[p] = take(sizeof(double) * std::max<size_t>(1, b->hp[p].params.size()));
  for (int p = 0; p < P; ++p) o_offsets[p] = take(sizeof(int64_t) * (size_t)(b->hp[p].NH + 1));
  for (int p = 0; p < P; ++p) o_ell[p] = take(sizeof(float) * (size_t)b->hp[p].NH);
  for (int p = 0; p < P; ++p) o_tf[p] = take(sizeof(int32_t) * (size_t)b->hp[p].ntiles_cap);
  for (int p = 0; p < P; ++p) o_car[p] = take(sizeof(Carry) * 2 * (size_t)b->hp[p].ntiles_cap);
  for (int p = 0; p < P; ++p) o_bsum[p] = take(sizeof(uint64_t) * (size_t)(b->hp[p].nblocks + 1));
  b->arena = (unsigned char*)batch_alloc(b, off);
  if (!b->arena) return fail(VEGAS_ENOMEM);
  b->arena_bytes = off;
  unsigned char* A = b->arena;
  BatchLaunch& L = b->L;
  L.P = P;
  L.G = G;
  L.alpha = alpha;
  L.rtol = 0.0;
  L.skip = 0;
  L.chunk_tiles = b->chunk;
  L.prob = (BatchProblem*)(A + o_prob);
  L.ctl = (BatchCtl*)(A + o_ctl);
  L.act_tile = (int32_t*)(A + o_act_tile);
  L.act_blk = (int64_t*)(A + o_act_blk);
  L.grp_tile = (int32_t*)(A + o_grp_tile);
  L.counter = (uint32_t*)(A + o_counter);
  L.acc = (double*)(A + o_acc);
  L.key = (int*)(A + o_key);
  L.flags = (int*)(A + o_flags);
  L.out = (double*)(A + o_out);
  b->d_bins = (double*)(A + bins_begin);
  for (int r = 0; r < 10; ++r) {
    L.rk0[r] = (uint32_t)seed + (uint32_t)r * 0x9E3779B9u;
    L.rk1[r] = (uint32_t)(seed >> 32) + (uint32_t)r * 0xBB67AE85u;
  }

  std::vector<BatchProblem> host(P);
  std::vector<int> vexp(P, 0);
  for (int p = 0; p < P; ++p) {
    const HostProblem& h = b->hp[p];
    BatchProblem& q = host[p];
    memset(&q, 0, sizeof(q));
    FillArgs& a = q.a;
    a.d = h.d;
    a.G = G;
    a.NH = (int)h.NH;
    a.ntiles = (int)h.ntiles;
    a.tile_log2 = h.tile_log2;
    a.neval = h.neval;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.iter = 0u;
    a.pid = (uint32_t)p;
    a.half_beta = (float)beta * 0.5f;
    a.np_derived = (int)h.params.size();
    if (h.iid == VEGAS_GAUSS_SUM || h.iid == VEGAS_PRODUCT_PEAK || h.iid == VEGAS_OSCILLATORY)
      a.np_derived = derived_param_count(h.iid, h.d, nullptr, (int64_t)h.params.size());
    a.iid = h.iid;
    a.edges = (const double*)(A + o_edges[p]);
    a.offsets = (const int64_t*)(A + o_offsets[p]);
    a.tile_first = (const int32_t*)(A + o_tf[p]);
    a.params_raw = (const double*)(A + o_params[p]);
    a.np_raw = (int)h.params.size();
    a.ell = (float*)(A + o_ell[p]);
    a.cube_mean = nullptr;
    a.cube_m2 = nullptr;
    a.flags = L.flags + p;
    a.ellmax_key = L.key + p;
    a.carries = (Carry*)(A + o_car[p]);
    a.vexp = (const int*)(A + o_vexp) + p;
    vexp[p] = value_exponent(h.iid, h.d, h.params.data(), (int)h.params.size());
    std::vector<int32_t> ns(h.d, h.nstrat);
    if (fill_args_axes(a, ns.data(), VEGAS_FP32, nprm_max, false) != VEGAS_OK) return fail(VEGAS_EINVAL);
    a.table_smem = layout.table_smem;
    a.hist_mode = layout.hist_mode;
    a.acc32 = layout.acc32;  // the accumulator regions are the layout's
    a.wv_recompute = layout.wv_recompute;
    a.sm_table = layout.sm_table;
    a.sm_hist = layout.sm_hist;
    a.sm_hacc = layout.sm_hacc;
    a.sm_bins = layout.sm_bins;
    a.sm_wv = layout.sm_wv;
    a.sm_params = layout.sm_params;
    a.sm_off = layout.sm_off;
    a.sm_raw = layout.sm_raw;
    a.sm_invn = layout.sm_invn;
    a.sm_vals = layout.sm_vals;
    a.sm_long = layout.sm_long;
    a.sm_start = layout.sm_start;
    a.sm_misc = layout.sm_misc;
    a.sm_total = layout.sm_total;
    q.bins = (double*)(A + o_bins[p]);
    q.bsum = (uint64_t*)(A + o_bsum[p]);
    q.nblocks = h.nblocks;
    q.dmax = h.dmax;
    q.group = batch_group(h.iid, h.dmax);
    b->group_tiles[q.group] += h.ntiles;
    if (!h.params.empty() &&
        cudaMemcpy(A + o_params[p], h.params.data(), sizeof(double) * h.params.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess)
      return fail(VEGAS_ECUDA);
  }
  if (cudaMemcpy(L.prob, host.data(), sizeof(BatchProblem) * P, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(A + o_vexp, vexp.data(), sizeof(int) * P, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(VEGAS_ECUDA);
  if (cudaMallocHost((void**)&b->h_running, sizeof(uint32_t)) != cudaSuccess ||
      cudaMallocHost((void**)&b->h_out, sizeof(double) * 4 * P) != cudaSuccess ||
      cudaMallocHost((void**)&b->h_ctl, sizeof(BatchCtl) * P) != cudaSuccess ||
      cudaMallocHost((void**)&b->h_flags, sizeof(int) * P) != cudaSuccess)
    return fail(VEGAS_ENOMEM);
  int rc = ensure_records(b, 16);
  if (rc != VEGAS_OK) return fail(rc);
  if ((rc = reset_batch(b)) != VEGAS_OK) return fail(rc);
  *out = b;
  return VEGAS_OK;
}

extern "C" int vegas_batch_destroy(vegas_batch b) {
  if (!b) return VEGAS_EINVAL;
  DevGuard g(b->device);
  if (b->has_user_stream) cudaStreamSynchronize(b->user_stream);
  cudaStreamSynchronize(b->own_stream);
  release(b);
  delete b;
  return VEGAS_OK;
}

extern "C" int vegas_batch_set_stream(vegas_batch b, void* stream) {
  if (!b) return VEGAS_EINVAL;
  b->user_stream = (cudaStream_t)stream;
  b->has_user_stream = true;
  return VEGAS_OK;
}

extern "C" int vegas_batch_set_chi2_bound(vegas_batch b, double bound) {
  if (!b || std::isnan(bound)) return VEGAS_EINVAL;
  b->chi2_bound = bound > 0.0 ? bound : 0.0;
  return VEGAS_OK;
}

extern "C" int vegas_batch_set_skip(vegas_batch b, int32_t skip) {
  if (!b || skip < 0) return VEGAS_EINVAL;
  b->skip = skip;
  return VEGAS_OK;
}

namespace {

// every integral to tiles of 2^tile_log2 evaluations: the arguments' tile, tile count and shared-memory layout,
// the group tile counts, uploaded; the next iteration recaptures its graph
int apply_tile(vegas_batch_s* b, int tile_log2) {
  const int i = tile_log2 - kTileLog2Min;
  if (i < 0 || i > 1 || !b->layout_ok[i]) return VEGAS_EINVAL;
  const FillArgs& l = b->layout[i];
  cudaStream_t s = b->stream();
  VG_CHECK(cudaStreamSynchronize(s));
  // read back, change the tile fields only, write back: the device copy also holds what the device sets (the
  // Philox iteration of each integral, the pointers to its iteration records)
  std::vector<BatchProblem> prob(b->P);
  VG_CHECK(cudaMemcpy(prob.data(), b->L.prob, sizeof(BatchProblem) * b->P, cudaMemcpyDeviceToHost));
  int64_t tiles = 0;
  for (int g = 0; g < kBatchGroups; ++g) b->group_tiles[g] = 0;
  for (int p = 0; p < b->P; ++p) {
    HostProblem& h = b->hp[p];
    BatchProblem& q = prob[p];
    FillArgs& a = q.a;
    h.tile_log2 = tile_log2;
    h.ntiles = (h.neval + (int64_t(1) << tile_log2) - 1) >> tile_log2;
    a.tile_log2 = tile_log2;
    a.ntiles = (int)h.ntiles;
    a.table_smem = l.table_smem;
    a.hist_mode = l.hist_mode;
    a.acc32 = l.acc32;
    a.wv_recompute = l.wv_recompute;
    a.sm_table = l.sm_table;
    a.sm_hist = l.sm_hist;
    a.sm_hacc = l.sm_hacc;
    a.sm_bins = l.sm_bins;
    a.sm_wv = l.sm_wv;
    a.sm_params = l.sm_params;
    a.sm_off = l.sm_off;
    a.sm_raw = l.sm_raw;
    a.sm_invn = l.sm_invn;
    a.sm_vals = l.sm_vals;
    a.sm_long = l.sm_long;
    a.sm_start = l.sm_start;
    a.sm_misc = l.sm_misc;
    a.sm_total = l.sm_total;
    b->group_tiles[q.group] += h.ntiles;
    tiles += h.ntiles;
  }
  VG_CHECK(cudaMemcpy(b->L.prob, prob.data(), sizeof(BatchProblem) * b->P, cudaMemcpyHostToDevice));
  b->tiles_total = tiles;
  b->smem = l.sm_total;
  b->tile_log2 = tile_log2;
  b->graph_dirty = true;
  return VEGAS_OK;
}

}  // namespace

extern "C" int vegas_batch_set_tile(vegas_batch b, int32_t tile_log2) {
  if (!b) return VEGAS_EINVAL;
  DevGuard g(b->device);
  return apply_tile(b, tile_log2);
}

extern "C" int vegas_batch_set_launch(vegas_batch b, int32_t variant, int32_t ctas_per_sm, int32_t chunk_tiles) {
  if (!b || variant < 0 || variant >= kBatchVariants || chunk_tiles < 1 || chunk_tiles > 4096) return VEGAS_EINVAL;
  b->variant = variant;
  b->ctas_per_sm = ctas_per_sm > 0 ? ctas_per_sm : 0;
  b->chunk = chunk_tiles;
  b->graph_dirty = true;
  return VEGAS_OK;
}

extern "C" int vegas_batch_reset(vegas_batch b) {
  if (!b) return VEGAS_EINVAL;
  DevGuard g(b->device);
  return reset_batch(b);
}

extern "C" int vegas_batch_integrate(vegas_batch b, int32_t nitn, double rtol, vegas_problem_result* results,
                                     int32_t* nitn_run, float* ms) {
  if (!b || nitn < 1 || !(rtol >= 0.0)) return VEGAS_EINVAL;
  DevGuard g(b->device);
  clear_stale_error();
  int nrun = 0;
  int rc = run_iterations(b, nitn, rtol, &nrun, ms);
  if (rc != VEGAS_OK) return rc;
  if (nitn_run) *nitn_run = nrun;
  if (results) {
    cudaStream_t s = b->stream();
    VG_CHECK(cudaMemcpyAsync(b->h_out, b->L.out, sizeof(double) * 4 * b->P, cudaMemcpyDeviceToHost, s));
    VG_CHECK(cudaMemcpyAsync(b->h_ctl, b->L.ctl, sizeof(BatchCtl) * b->P, cudaMemcpyDeviceToHost, s));
    VG_CHECK(cudaMemcpyAsync(b->h_flags, b->L.flags, sizeof(int) * b->P, cudaMemcpyDeviceToHost, s));
    VG_CHECK(cudaStreamSynchronize(s));
    for (int p = 0; p < b->P; ++p) {
      vegas_problem_result& r = results[p];
      r.estimate = b->h_out[4 * p];
      r.sigma = b->h_out[4 * p + 1];
      r.chi2_dof = b->h_out[4 * p + 2];
      r.n_used = (int32_t)b->h_out[4 * p + 3];
      r.nitn_run = b->h_ctl[p].nrec;
      r.converged = b->h_ctl[p].converged;
      const int f = b->h_flags[p];
      r.status = (f & 14) ? VEGAS_ECUDA : (f & 1) ? VEGAS_ENONFINITE : VEGAS_OK;
      r.flags = 0;
      r.pad = 0;
      if (r.n_used >= 2) {
        const double bound = b->chi2_bound > 0.0 ? b->chi2_bound : chi2_dof_quantile_999_batch(r.n_used - 1);
        if (!(r.chi2_dof <= bound)) r.flags |= VEGAS_RESULT_CHI2_HIGH;
      }
      if (r.sigma < kFp32SigmaFloor * std::fabs(r.estimate)) r.flags |= VEGAS_RESULT_FP32_FLOOR;  // FP32 only
    }
  }
  return VEGAS_OK;
}

extern "C" int vegas_batch_tune(vegas_batch b, int32_t* variant, int32_t* ctas_per_sm, int32_t* chunk_tiles,
                                float* ms) {
  if (!b) return VEGAS_EINVAL;
  DevGuard g(b->device);
  const int chunks[3] = {1, 4, 16};
  float best = INFINITY;
  int bv = b->variant, bc = b->ctas_per_sm, bk = b->chunk, bt = b->tile_log2;
  for (int tl = kTileLog2Min; tl <= kTileLog2Max; ++tl) {
    if (!b->layout_ok[tl - kTileLog2Min]) continue;
    int rc = apply_tile(b, tl);
    if (rc != VEGAS_OK) return rc;
    for (int v = 0; v < kBatchVariants; ++v) {
      int occ = 0;  // the most resident CTAs of any present group's kernel (capture clamps each group to its own)
      for (int gr = 0; gr < kBatchGroups; ++gr)
        if (b->group_tiles[gr] > 0) occ = std::max(occ, batch_fill_occupancy(v, gr, b->smem));
      for (int c = 1; c <= occ; ++c) {
        for (int k : chunks) {
          if ((rc = vegas_batch_set_launch(b, v, c, k)) != VEGAS_OK) return rc;
          float t = INFINITY;
          for (int rep = 0; rep < 2; ++rep) {  // the first run captures the graph and warms up
            if ((rc = reset_batch(b)) != VEGAS_OK) return rc;
            float m = 0.0f;
            int n = 0;
            if ((rc = run_iterations(b, 1, 0.0, &n, &m)) != VEGAS_OK) return rc;
            if (rep > 0) t = m;
          }
          if (t < best) {
            best = t;
            bv = v;
            bc = c;
            bk = k;
            bt = tl;
          }
        }
      }
    }
  }
  int rc = apply_tile(b, bt);
  if (rc != VEGAS_OK) return rc;
  if ((rc = vegas_batch_set_launch(b, bv, bc, bk)) != VEGAS_OK) return rc;
  if ((rc = reset_batch(b)) != VEGAS_OK) return rc;
  if (variant) *variant = bv;
  if (ctas_per_sm) *ctas_per_sm = bc;
  if (chunk_tiles) *chunk_tiles = bk;
  if (ms) *ms = best;
  return VEGAS_OK;
}

extern "C" int vegas_batch_get(vegas_batch b, int32_t problem, int32_t what, void* host_out, int64_t count) {
  if (!b || problem < 0 || problem >= b->P || !host_out || count < 0) return VEGAS_EINVAL;
  DevGuard g(b->device);
  cudaStream_t s = b->stream();
  VG_CHECK(cudaStreamSynchronize(s));
  const HostProblem& h = b->hp[problem];
  BatchProblem q;
  VG_CHECK(cudaMemcpy(&q, b->L.prob + problem, sizeof(q), cudaMemcpyDeviceToHost));
  BatchCtl c;
  VG_CHECK(cudaMemcpy(&c, b->L.ctl + problem, sizeof(c), cudaMemcpyDeviceToHost));
  const void* src = nullptr;
  size_t elem = 0;
  int64_t n = 0;
  switch (what) {
    case VEGAS_BATCH_EDGES: src = q.a.edges; elem = sizeof(double); n = (int64_t)h.d * (b->G + 1); break;
    case VEGAS_BATCH_OFFSETS: src = q.a.offsets; elem = sizeof(int64_t); n = h.NH + 1; break;
    case VEGAS_BATCH_ELL: src = q.a.ell; elem = sizeof(float); n = h.NH; break;
    case VEGAS_BATCH_BINS: src = q.bins; elem = sizeof(double); n = (int64_t)h.d * b->G; break;
    case VEGAS_BATCH_ITER_EST: src = q.it_est; elem = sizeof(double); n = c.nrec; break;
    case VEGAS_BATCH_ITER_SIG: src = q.it_sig; elem = sizeof(double); n = c.nrec; break;
    case VEGAS_BATCH_INFO: {
      if (count < 4) return VEGAS_ENOSPACE;
      int64_t* o = (int64_t*)host_out;
      o[0] = h.d;
      o[1] = h.nstrat;
      o[2] = h.NH;
      o[3] = c.nrec;
      if (count >= 5) o[4] = h.tile_log2;
      return VEGAS_OK;
    }
    default: return VEGAS_EINVAL;
  }
  if (count < n) return VEGAS_ENOSPACE;
  if (n > 0) VG_CHECK(cudaMemcpy(host_out, src, elem * (size_t)n, cudaMemcpyDeviceToHost));
  return VEGAS_OK;
}
