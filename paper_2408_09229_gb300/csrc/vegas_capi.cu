// vegas_capi.cu -- the handle of the C ABI: buffers, the iteration loop of
// Algorithm 1 in cuVegas on one CUDA stream, timing events, checkpoints.
//
// One iteration on the handle's stream:
//   vegas_allocate  n_h from the last iteration's weights (uniform at first)
//   fill_impl       Algorithm 2 plus the cube fix-up and the reductions
//   vegas_refine    map refinement into the other edge buffer
//   record+combine  store (I_t, sigma_t) and the running Eqs. (8)-(9)
// No host round trip happens inside the loop unless an rtol target is set.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <new>
#include <unordered_map>
#include <vector>

#include "vegas_internal.h"

// One VEGAS+ state: the map, the stratification weights of the last
// iteration, the records of the current call and their combination.  The
// handle's result is arm 0; arm 1 is plain VEGAS+ run beside a learned
// proposal while the judge compares the two (vegas_set_flow_judge).
struct Arm {
  double* d_edges[2] = {nullptr, nullptr};
  int cur = 0;
  float* d_ell = nullptr;
  int64_t ell_cap = 0;
  bool ell_valid = false;
  const int* fill_key = nullptr;  // max-ell key left in the fill scratch by this arm's last fill, or NULL
  std::vector<int32_t> ell_nstrat;
  double* d_it_est = nullptr;
  double* d_it_sig = nullptr;
  int it_cap = 0;
  double* d_out = nullptr;  // [4] estimate, sigma, chi2/dof, n_used
};

enum { kJudgeOpen = 0, kJudgeFlowKept = 1, kJudgePlainWon = 2 };

struct vegas_s {
  int device = 0;
  int dim = 0, nbins = 0, nstrat_scalar = 0;
  double alpha = 0.5, beta = 0.75;
  std::vector<int32_t> nstrat_axes;  // empty: use nstrat_scalar / automatic
  int skip = 0, precision = VEGAS_FP64, weighting = VEGAS_WEIGHT_AUTO;
  double rtol = 0.0, chi2_bound = 0.0;
  cudaStream_t own_stream = nullptr, user_stream = nullptr;
  bool has_user_stream = false;
  // device memory: through the caller's hooks when set, else cudaMalloc / cudaFree; every live
  // allocation with its size
  vegas_alloc_fn al_alloc = nullptr;
  vegas_free_fn al_free = nullptr;
  void* al_ctx = nullptr;
  std::unordered_map<void*, size_t> live;
  // device buffers
  Arm arm[2];
  double* d_bins = nullptr;
  int64_t* d_offsets = nullptr;
  int64_t off_cap = 0;
  void* d_fill_scratch = nullptr;
  size_t fill_scratch_cap = 0;
  void* d_alloc_scratch = nullptr;
  size_t alloc_scratch_cap = 0;
  double* d_params = nullptr;
  int64_t params_cap = 0;
  double* d_result = nullptr;  // [2]
  int* d_flags = nullptr;
  double* h_out = nullptr;  // pinned [8]
  int64_t iter_counter = 0;
  // learned proposal: the flow's parameters (NULL: off), Adam state, the
  // per-evaluation buffers and the training schedule
  float* d_flow = nullptr;
  float *d_flow_m = nullptr, *d_flow_v = nullptr, *d_flow_g = nullptr, *d_flow_loss = nullptr;
  int64_t flow_np = 0;
  int flow_step = 0, flow_train_iters = 0, flow_train_steps = 0, flow_train_samples = 0, flow_trained = 0;
  int flow_batch = 4096;
  float flow_lr = 1e-3f, flow_temper = 1.0f, flow_floor = 0.0f;
  float *d_X = nullptr, *d_logdet = nullptr, *d_values = nullptr;
  int64_t x_cap = 0, ld_cap = 0, val_cap = 0;
  float *d_train_x = nullptr, *d_train_w = nullptr;
  int64_t tx_cap = 0, tw_cap = 0;
  void* d_grad_scratch = nullptr;
  size_t grad_scratch_cap = 0;
  // exploration: the adapted maps [S][d][G+1] and the samples' mixture density
  double* d_explore = nullptr;
  int64_t explore_cap = 0;
  // the judge of the learned proposal: window (0: off), state, paired iterations since the flow was
  // set, and sigma_t^2 x iteration time of each form over the paired iterations after training
  int judge_window = 0, judge_state = kJudgeOpen;
  int64_t judge_pairs = 0;
  std::vector<double> judge_vt[2];
  double judge_ratio = 0.0;
  // timing
  std::vector<cudaEvent_t> ev;  // 6 per iteration: start, fill start, fill end, end, arm-0 end, arm-1 end
  int last_nrun = 0;
  cudaStream_t stream() const { return has_user_stream ? user_stream : own_stream; }
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int now = -1;
    if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
  }
};

void* dalloc(vegas_s* h, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 1;
  if (h->al_alloc) {
    p = h->al_alloc(h->al_ctx, bytes, (void*)h->stream());
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) h->live[p] = bytes;
  return p;
}

// give back a buffer; the caller has synchronised the handle's stream (cudaFree also synchronises)
void dfree(vegas_s* h, void* p) {
  if (!p) return;
  auto it = h->live.find(p);
  const size_t bytes = it == h->live.end() ? 0 : it->second;
  if (it != h->live.end()) h->live.erase(it);
  if (h->al_free) h->al_free(h->al_ctx, p, bytes, (void*)h->stream());
  else cudaFree(p);
}

template <typename T>
void dfree_ptr(vegas_s* h, T*& p) {
  dfree(h, (void*)p);
  p = nullptr;
}

template <typename T>
int grow(vegas_s* h, T*& p, int64_t& cap, int64_t need) {
  if (need <= cap && p) return VEGAS_OK;
  if (p) {
    cudaStreamSynchronize(h->stream());
    dfree_ptr(h, p);
  }
  cap = 0;
  p = (T*)dalloc(h, sizeof(T) * (size_t)need);
  if (!p) return VEGAS_ENOMEM;
  cap = need;
  return VEGAS_OK;
}

int grow_bytes(vegas_s* h, void*& p, size_t& cap, size_t need) {
  if (need <= cap && p) return VEGAS_OK;
  if (p) {
    cudaStreamSynchronize(h->stream());
    dfree_ptr(h, p);
  }
  cap = 0;
  p = dalloc(h, need);
  if (!p) return VEGAS_ENOMEM;
  cap = need;
  return VEGAS_OK;
}

// the record arrays of an arm, for nitn iterations (contents not kept)
int grow_records(vegas_s* h, Arm& A, int nitn) {
  if (A.it_cap >= nitn && A.d_it_est && A.d_it_sig) return VEGAS_OK;
  if (A.d_it_est || A.d_it_sig) cudaStreamSynchronize(h->stream());
  dfree_ptr(h, A.d_it_est);
  dfree_ptr(h, A.d_it_sig);
  A.it_cap = 0;
  A.d_it_est = (double*)dalloc(h, sizeof(double) * nitn);
  A.d_it_sig = (double*)dalloc(h, sizeof(double) * nitn);
  if (!A.d_it_est || !A.d_it_sig) return VEGAS_ENOMEM;
  A.it_cap = nitn;
  return VEGAS_OK;
}

// every device pointer the handle holds, for moving them to another allocator
std::vector<void**> device_fields(vegas_s* h) {
  std::vector<void**> f;
  for (Arm& A : h->arm)
    for (double** p : {&A.d_edges[0], &A.d_edges[1], &A.d_it_est, &A.d_it_sig, &A.d_out}) f.push_back((void**)p);
  for (Arm& A : h->arm) f.push_back((void**)&A.d_ell);
  f.push_back((void**)&h->d_bins);
  f.push_back((void**)&h->d_offsets);
  f.push_back(&h->d_fill_scratch);
  f.push_back(&h->d_alloc_scratch);
  f.push_back((void**)&h->d_params);
  f.push_back((void**)&h->d_result);
  f.push_back((void**)&h->d_flags);
  for (float** p : {&h->d_flow, &h->d_flow_m, &h->d_flow_v, &h->d_flow_g, &h->d_flow_loss, &h->d_X, &h->d_logdet,
                    &h->d_values, &h->d_train_x, &h->d_train_w})
    f.push_back((void**)p);
  f.push_back(&h->d_grad_scratch);
  f.push_back((void**)&h->d_explore);
  return f;
}

// 0.999 quantile of chi2_nu / nu by the Wilson-Hilferty approximation: chi2_nu / nu is close to the cube of a
// normal variable of mean 1 - 2/(9 nu) and variance 2/(9 nu)
double chi2_dof_quantile_999(int nu) {
  const double z = 3.090232306167813;  // 0.999 quantile of the standard normal
  const double a = 2.0 / (9.0 * nu);
  const double c = 1.0 - a + z * std::sqrt(a);
  return c * c * c;
}

int upload_uniform_edges(vegas_s* h, Arm& A) {
  const int G = h->nbins;
  std::vector<double> e((size_t)h->dim * (G + 1));
  for (int k = 0; k < h->dim; ++k)
    for (int i = 0; i <= G; ++i) e[(size_t)k * (G + 1) + i] = (double)i / (double)G;
  A.cur = 0;
  A.ell_valid = false;
  A.fill_key = nullptr;
  VG_CHECK(cudaMemcpy(A.d_edges[0], e.data(), sizeof(double) * e.size(), cudaMemcpyHostToDevice));
  return VEGAS_OK;
}

// the judge starts over: plain VEGAS+ from the uniform map, no decision yet
void judge_reset(vegas_s* h) {
  h->judge_state = kJudgeOpen;
  h->judge_pairs = 0;
  h->judge_vt[0].clear();
  h->judge_vt[1].clear();
  h->judge_ratio = 0.0;
  h->arm[1].ell_valid = false;
  h->arm[1].fill_key = nullptr;
  h->arm[1].cur = 0;
}

// largest s with s^d <= neval / 2, at least 1
int default_nstrat(int64_t neval, int d) {
  const int64_t half = neval / 2;
  int64_t s = 1;
  for (;;) {
    const int64_t cand = s + 1;
    int64_t p = 1;
    bool over = false;
    for (int k = 0; k < d; ++k) {
      if (p > half / cand) {
        over = true;
        break;
      }
      p *= cand;
    }
    if (over || p > half) break;
    s = cand;
  }
  return (int)s;
}

// offsets [n + 1] and an arm's allocation weights [n]; contents are not kept
int ensure_cubes(vegas_s* h, Arm& A, int64_t n) {
  int rc = grow(h, h->d_offsets, h->off_cap, n + 1);
  if (rc != VEGAS_OK) return rc;
  if (A.ell_cap >= n && A.d_ell) return VEGAS_OK;
  A.ell_valid = false;
  A.fill_key = nullptr;
  return grow(h, A.d_ell, A.ell_cap, n);
}

void release(vegas_s* h) {
  for (void** f : device_fields(h)) {
    dfree(h, *f);
    *f = nullptr;
  }
  if (h->h_out) cudaFreeHost(h->h_out);
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
}

}  // namespace

extern "C" int vegas_create(int dim, int nbins, int nstrat, double alpha, double beta, vegas_handle* out) {
  if (!out) return VEGAS_EINVAL;
  *out = nullptr;
  if (dim < 1 || dim > vg::kMaxDim || nbins < 2 || nbins > vg::kMaxBins || !(alpha >= 0.0) || !std::isfinite(alpha) ||
      !(beta >= 0.0 && beta <= 1.0))
    return VEGAS_EINVAL;
  vegas_s* h = new (std::nothrow) vegas_s();
  if (!h) return VEGAS_ENOMEM;
  h->dim = dim;
  h->nbins = nbins;
  h->nstrat_scalar = nstrat;
  h->alpha = alpha;
  h->beta = beta;
  int rc = VEGAS_OK;
  if (cudaGetDevice(&h->device) != cudaSuccess) rc = VEGAS_ECUDA;
  const size_t ne = (size_t)dim * (nbins + 1), nb = (size_t)dim * nbins;
  if (rc == VEGAS_OK && cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess)
    rc = VEGAS_ECUDA;
  Arm& A = h->arm[0];
  if (rc == VEGAS_OK &&
      (!(A.d_edges[0] = (double*)dalloc(h, sizeof(double) * ne)) ||
       !(A.d_edges[1] = (double*)dalloc(h, sizeof(double) * ne)) ||
       !(A.d_out = (double*)dalloc(h, sizeof(double) * 4)) || !(h->d_bins = (double*)dalloc(h, sizeof(double) * nb)) ||
       !(h->d_result = (double*)dalloc(h, sizeof(double) * 2)) || !(h->d_flags = (int*)dalloc(h, sizeof(int))) ||
       cudaMallocHost((void**)&h->h_out, sizeof(double) * 8) != cudaSuccess))
    rc = VEGAS_ENOMEM;
  if (rc == VEGAS_OK) rc = upload_uniform_edges(h, A);
  if (rc == VEGAS_OK && cudaMemset(h->d_flags, 0, sizeof(int)) != cudaSuccess) rc = VEGAS_ECUDA;
  if (rc != VEGAS_OK) {
    cudaGetLastError();
    release(h);
    delete h;
    return rc;
  }
  *out = h;
  return VEGAS_OK;
}

extern "C" int vegas_destroy(vegas_handle h) {
  if (!h) return VEGAS_OK;
  DeviceGuard g(h->device);
  cudaStreamSynchronize(h->stream());
  release(h);
  delete h;
  return VEGAS_OK;
}

extern "C" int vegas_set_allocator(vegas_handle h, vegas_alloc_fn alloc, vegas_free_fn free_fn, void* ctx) {
  if (!h || (alloc == nullptr) != (free_fn == nullptr)) return VEGAS_EINVAL;
  DeviceGuard g(h->device);
  cudaStream_t s = h->stream();
  VG_CHECK(cudaStreamSynchronize(s));
  // new memory for every buffer first, so that a failure leaves the handle as it was
  const std::vector<void**> fields = device_fields(h);
  std::vector<void*> fresh(fields.size(), nullptr);
  std::vector<size_t> bytes(fields.size(), 0);
  auto give_back = [&]() {
    for (size_t i = 0; i < fields.size(); ++i)
      if (fresh[i]) {
        if (free_fn) free_fn(ctx, fresh[i], bytes[i], (void*)s);
        else cudaFree(fresh[i]);
      }
  };
  for (size_t i = 0; i < fields.size(); ++i) {
    void* p = *fields[i];
    if (!p) continue;
    auto it = h->live.find(p);
    bytes[i] = it == h->live.end() ? 0 : it->second;
    if (bytes[i] == 0) {
      give_back();
      return VEGAS_ECUDA;  // a buffer the handle does not know: internal error
    }
    if (alloc) {
      fresh[i] = alloc(ctx, bytes[i], (void*)s);
    } else if (cudaMalloc(&fresh[i], bytes[i]) != cudaSuccess) {
      cudaGetLastError();
      fresh[i] = nullptr;
    }
    if (!fresh[i]) {
      give_back();
      return VEGAS_ENOMEM;
    }
  }
  for (size_t i = 0; i < fields.size(); ++i)
    if (fresh[i] && cudaMemcpyAsync(fresh[i], *fields[i], bytes[i], cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
      cudaStreamSynchronize(s);
      give_back();
      return VEGAS_ECUDA;
    }
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    give_back();
    return VEGAS_ECUDA;
  }
  for (size_t i = 0; i < fields.size(); ++i)
    if (fresh[i]) dfree(h, *fields[i]);  // to the allocator that supplied it
  h->al_alloc = alloc;
  h->al_free = free_fn;
  h->al_ctx = ctx;
  for (size_t i = 0; i < fields.size(); ++i)
    if (fresh[i]) {
      *fields[i] = fresh[i];
      h->live[fresh[i]] = bytes[i];
    }
  // the max-ell keys pointed into the old fill scratch
  h->arm[0].fill_key = h->arm[1].fill_key = nullptr;
  return VEGAS_OK;
}

extern "C" int vegas_set_chi2_bound(vegas_handle h, double bound) {
  if (!h || std::isnan(bound)) return VEGAS_EINVAL;
  h->chi2_bound = bound > 0.0 ? bound : 0.0;
  return VEGAS_OK;
}

extern "C" int vegas_set_nstrat_axes(vegas_handle h, const int32_t* nstrat, int dim) {
  if (!h || !nstrat || dim != h->dim) return VEGAS_EINVAL;
  int64_t nh = 1;
  for (int k = 0; k < dim; ++k) {
    if (nstrat[k] < 1) return VEGAS_EINVAL;
    nh *= nstrat[k];
    if (nh >= (int64_t(1) << 31)) return VEGAS_EINVAL;
  }
  h->nstrat_axes.assign(nstrat, nstrat + dim);
  return VEGAS_OK;
}

extern "C" int vegas_set_weighting(vegas_handle h, int weighting) {
  if (!h || weighting < VEGAS_WEIGHT_AUTO || weighting > VEGAS_WEIGHT_LAGGED) return VEGAS_EINVAL;
  h->weighting = weighting;
  return VEGAS_OK;
}

extern "C" int vegas_set_skip(vegas_handle h, int skip) {
  if (!h || skip < 0) return VEGAS_EINVAL;
  h->skip = skip;
  return VEGAS_OK;
}

extern "C" int vegas_set_precision(vegas_handle h, int precision) {
  if (!h || (precision != VEGAS_FP64 && precision != VEGAS_FP32)) return VEGAS_EINVAL;
  h->precision = precision;
  return VEGAS_OK;
}

extern "C" int vegas_set_stream(vegas_handle h, void* stream) {
  if (!h) return VEGAS_EINVAL;
  h->has_user_stream = stream != nullptr;
  h->user_stream = (cudaStream_t)stream;
  return VEGAS_OK;
}

extern "C" int vegas_set_rtol(vegas_handle h, double rtol) {
  if (!h || !(rtol >= 0.0)) return VEGAS_EINVAL;
  h->rtol = rtol;
  return VEGAS_OK;
}

extern "C" int vegas_reset_map(vegas_handle h) {
  if (!h) return VEGAS_EINVAL;
  DeviceGuard g(h->device);
  VG_CHECK(cudaStreamSynchronize(h->stream()));
  h->iter_counter = 0;
  judge_reset(h);
  return upload_uniform_edges(h, h->arm[0]);
}

extern "C" int vegas_set_flow_judge(vegas_handle h, int32_t window) {
  if (!h || window < 0 || window > 1024) return VEGAS_EINVAL;
  h->judge_window = window;
  judge_reset(h);
  return VEGAS_OK;
}

namespace {

// Minimum paired iterations before the judge decides, so that plain VEGAS+'s own map has adapted.
constexpr int kJudgeMinAdapt = 5;

struct IterationPlan {
  const vegas_geometry* geo;
  const int32_t* ns;
  int64_t NH, neval, nparams, train_stride, n_train, train_rows;
  int integrand;
  uint64_t seed;
};

// One iteration of Algorithm 1 for arm a on the handle's stream: allocation from the arm's weights, the fill
// (with the learned proposal when with_flow), the map refinement and the record of (I_t, sigma_t) with the
// running combination.  Training steps follow when train.
int run_arm(vegas_s* h, int a, int it, bool with_flow, bool train, bool paired, const IterationPlan& P,
            cudaEvent_t ev_fill0, cudaEvent_t ev_fill1) {
  Arm& A = h->arm[a];
  cudaStream_t s = h->stream();
  const int d = h->dim, G = h->nbins;
  const bool uniform = !(A.ell_valid && A.ell_nstrat.size() == (size_t)d &&
                         std::equal(A.ell_nstrat.begin(), A.ell_nstrat.end(), P.ns));
  // the fill scratch's max-ell key belongs to the last fill, which was the other arm's when two alternate
  const int* key = paired ? nullptr : A.fill_key;
  int rc = vg::allocate_impl(A.d_ell, P.NH, P.neval, (uniform || h->beta == 0.0) ? 1 : 0, h->d_offsets,
                             h->d_alloc_scratch, h->alloc_scratch_cap, s, key);
  if (rc != VEGAS_OK) return rc;
  const uint32_t pid = (uint32_t)a;  // the plain arm draws with problem id 1: independent of arm 0's points
  if (with_flow) {
    // points x' of the VEGAS+ map, x = F(x') and |det dF/dx'|, then g = f(x) |det| tabulated by evaluation
    vg::FillExtra ex_points{nullptr, h->d_X, nullptr, 0, 1.0f};
    rc = vg::fill_impl(P.geo, VEGAS_FP32, vg::kIntegrandPoints, nullptr, 0, P.neval, P.seed, (int32_t)h->iter_counter,
                       pid, h->beta, A.d_edges[A.cur], h->d_offsets, A.d_ell, h->d_bins, h->d_result, nullptr, nullptr,
                       h->d_flags, h->d_fill_scratch, h->fill_scratch_cap, s, nullptr, nullptr, &ex_points);
    if (rc != VEGAS_OK) return rc;
    if ((rc = vg::flow_apply(d, VEGAS_FLOW_SAMPLE, h->d_flow, h->d_X, h->d_X, h->d_logdet, P.neval, s)) != VEGAS_OK)
      return rc;
    if ((rc = vg::flow_eval(P.integrand, d, h->d_params, P.nparams, h->d_X, h->d_logdet, h->d_values, P.neval, s)) !=
        VEGAS_OK)
      return rc;
    // the temper exponent ramps linearly to 1 over the training iterations: broad targets first
    const float power =
        h->flow_train_iters > 1
            ? h->flow_temper + (1.0f - h->flow_temper) * (float)h->flow_trained / (float)(h->flow_train_iters - 1)
            : 1.0f;
    vg::FillExtra ex_tab{h->d_values, nullptr, train ? h->d_train_w + P.train_rows : nullptr, (int)P.train_stride,
                         power};
    rc = vg::fill_impl(P.geo, VEGAS_FP32, vg::kIntegrandTabulated, nullptr, 0, P.neval, P.seed,
                       (int32_t)h->iter_counter, pid, h->beta, A.d_edges[A.cur], h->d_offsets, A.d_ell, h->d_bins,
                       h->d_result, nullptr, nullptr, h->d_flags, h->d_fill_scratch, h->fill_scratch_cap, s, ev_fill0,
                       ev_fill1, &ex_tab);
  } else {
    rc = vg::fill_impl(P.geo, h->precision, P.integrand, h->d_params, P.nparams, P.neval, P.seed,
                       (int32_t)h->iter_counter, pid, h->beta, A.d_edges[A.cur], h->d_offsets, A.d_ell, h->d_bins,
                       h->d_result, nullptr, nullptr, h->d_flags, h->d_fill_scratch, h->fill_scratch_cap, s, ev_fill0,
                       ev_fill1);
  }
  if (rc != VEGAS_OK) return rc;
  A.fill_key = vg::fill_ellmax_key(P.geo, P.neval, h->d_fill_scratch);
  rc = vegas_refine(d, G, h->alpha, h->d_bins, A.d_edges[A.cur], A.d_edges[1 - A.cur], s);
  if (rc != VEGAS_OK) return rc;
  A.cur = 1 - A.cur;
  A.ell_valid = true;
  A.ell_nstrat.assign(P.ns, P.ns + d);
  const bool lagged = h->weighting == VEGAS_WEIGHT_LAGGED || (h->weighting == VEGAS_WEIGHT_AUTO && with_flow);
  rc = vg::launch_record_combine(h->d_result, it, A.d_it_est, A.d_it_sig, h->skip, A.d_out, lagged, s);
  if (rc != VEGAS_OK) return rc;
  if (train) {
    // Adam steps on the weighted samples of this iteration (x = F(x'), weight |J f| / n_h), with uniform
    // points of the floor mixed in
    double* wsum = (double*)(h->d_train_w + ((P.train_rows + P.n_train + 1) & ~(int64_t)1));
    if ((rc = vg::flow_gather(h->d_X, d, P.train_stride, P.n_train, h->d_train_w + P.train_rows, h->flow_floor, P.seed,
                              (uint32_t)h->iter_counter, wsum, h->d_train_x, h->d_train_w, s)) != VEGAS_OK)
      return rc;
    // minibatches: consecutive windows of the training set, cycling
    const int64_t nb = std::min<int64_t>(P.train_rows, h->flow_batch);
    for (int k = 0; k < h->flow_train_steps; ++k) {
      const int64_t off = ((int64_t)k * nb) % (P.train_rows - nb + 1);
      rc = vegas_flow_grad(d, h->d_flow, h->d_train_x + off * d, h->d_train_w + off, nb, h->d_flow_g, h->d_flow_loss,
                           h->d_grad_scratch, h->grad_scratch_cap, s);
      if (rc != VEGAS_OK) return rc;
      rc = vegas_flow_adam(h->flow_np, h->d_flow, h->d_flow_g, h->d_flow_m, h->d_flow_v, ++h->flow_step, h->flow_lr,
                           0.9f, 0.999f, 1e-8f, s);
      if (rc != VEGAS_OK) return rc;
    }
    h->flow_trained++;
  }
  return VEGAS_OK;
}

double median(std::vector<double> v) {
  std::sort(v.begin(), v.end());
  const size_t n = v.size();
  return n % 2 ? v[n / 2] : 0.5 * (v[n / 2 - 1] + v[n / 2]);
}

// plain VEGAS+ won: its state and records become arm 0, the learned proposal stops
void judge_switch_to_plain(vegas_s* h) {
  std::swap(h->arm[0], h->arm[1]);
  h->judge_state = kJudgePlainWon;
}

}  // namespace

extern "C" int vegas_integrate(vegas_handle h, int integrand, const double* params, int64_t nparams, int64_t neval,
                               int nitn, uint64_t seed, vegas_result* out) {
  if (!h || !out || nitn < 1 || nparams < 0 || (nparams > 0 && !params)) return VEGAS_EINVAL;
  const int d = h->dim, G = h->nbins;
  const int npd = vg::derived_param_count(integrand, d, params, nparams);
  if (npd < 0 || npd > vg::kMaxDerivedParams) return VEGAS_EINVAL;
  if (neval < 2 || neval > vg::kMaxEval) return VEGAS_EINVAL;
  // strata
  std::vector<int32_t> ns(d);
  if (!h->nstrat_axes.empty()) {
    ns = h->nstrat_axes;
  } else {
    int sk = h->nstrat_scalar > 0 ? h->nstrat_scalar : default_nstrat(neval, d);
    if (h->precision == VEGAS_FP32 && h->nstrat_scalar <= 0 && sk > 65536) sk = 65536;
    for (int k = 0; k < d; ++k) ns[k] = sk;
  }
  int64_t NH = 1;
  for (int k = 0; k < d; ++k) {
    if (h->precision == VEGAS_FP32 && ns[k] > 65536) return VEGAS_EINVAL;
    NH *= ns[k];
    if (NH >= (int64_t(1) << 31)) return VEGAS_EINVAL;
  }
  if (neval < 2 * NH) return VEGAS_EINVAL;
  const bool flow = h->d_flow != nullptr && h->judge_state != kJudgePlainWon;
  if (flow && h->precision != VEGAS_FP32) return VEGAS_EINVAL;
  // plain VEGAS+ runs beside the learned proposal until the judge decides
  bool paired = flow && h->judge_window > 0 && h->judge_state == kJudgeOpen;

  DeviceGuard guard(h->device);
  vg::clear_stale_error();
  cudaStream_t s = h->stream();
  const vegas_geometry geo{d, G, ns.data(), 0, 0};
  int rc;
  if ((rc = ensure_cubes(h, h->arm[0], NH)) != VEGAS_OK) return rc;
  const size_t fill_need = vegas_fill_scratch_bytes(&geo, neval);
  const size_t alloc_need = vegas_allocate_scratch_bytes(NH);
  if (fill_need == 0 || alloc_need == 0) return VEGAS_EINVAL;
  if (fill_need > h->fill_scratch_cap) h->arm[0].fill_key = h->arm[1].fill_key = nullptr;  // the scratch moves
  if ((rc = grow_bytes(h, h->d_fill_scratch, h->fill_scratch_cap, fill_need)) != VEGAS_OK) return rc;
  if ((rc = grow_bytes(h, h->d_alloc_scratch, h->alloc_scratch_cap, alloc_need)) != VEGAS_OK) return rc;
  if (nparams > 0 && (rc = grow(h, h->d_params, h->params_cap, nparams)) != VEGAS_OK) return rc;
  if ((rc = grow_records(h, h->arm[0], nitn)) != VEGAS_OK) return rc;
  if (paired) {
    Arm& B = h->arm[1];
    const size_t ne = (size_t)d * (G + 1);
    if (!B.d_edges[0]) {
      B.ell_valid = false;
      if (!(B.d_edges[0] = (double*)dalloc(h, sizeof(double) * ne)) ||
          !(B.d_edges[1] = (double*)dalloc(h, sizeof(double) * ne)) ||
          !(B.d_out = (double*)dalloc(h, sizeof(double) * 4))) {  // all or nothing
        dfree_ptr(h, B.d_edges[0]);
        dfree_ptr(h, B.d_edges[1]);
        dfree_ptr(h, B.d_out);
        return VEGAS_ENOMEM;
      }
    }
    if (!B.ell_valid && (rc = upload_uniform_edges(h, B)) != VEGAS_OK) return rc;
    if ((rc = ensure_cubes(h, B, NH)) != VEGAS_OK) return rc;
    if ((rc = grow_records(h, B, nitn)) != VEGAS_OK) return rc;
  }
  while ((int)h->ev.size() < 6 * nitn) {
    cudaEvent_t e;
    VG_CHECK(cudaEventCreate(&e));
    h->ev.push_back(e);
  }
  if (nparams > 0)
    VG_CHECK(cudaMemcpyAsync(h->d_params, params, sizeof(double) * (size_t)nparams, cudaMemcpyHostToDevice, s));
  VG_CHECK(cudaMemsetAsync(h->d_flags, 0, sizeof(int), s));

  // learned proposal: per-evaluation buffers and the training sample
  IterationPlan P{&geo, ns.data(), NH, neval, nparams, 1, 0, 0, integrand, seed};
  if (flow) {
    if ((rc = grow(h, h->d_X, h->x_cap, neval * d)) != VEGAS_OK ||
        (rc = grow(h, h->d_logdet, h->ld_cap, neval)) != VEGAS_OK ||
        (rc = grow(h, h->d_values, h->val_cap, neval)) != VEGAS_OK)
      return rc;
    if (h->flow_train_iters > h->flow_trained && h->flow_train_samples > 0 && h->flow_train_steps > 0) {
      P.train_stride = std::max<int64_t>(1, neval / h->flow_train_samples);
      P.n_train = (neval + P.train_stride - 1) / P.train_stride;
      P.train_rows = vg::flow_train_rows(P.n_train, h->flow_floor);
      // d_train_w: the training set's weights [train_rows], the fill's raw weights [n_train], their sum (a double)
      if ((rc = grow(h, h->d_train_x, h->tx_cap, P.train_rows * d)) != VEGAS_OK ||
          (rc = grow(h, h->d_train_w, h->tw_cap, P.train_rows + P.n_train + 4)) != VEGAS_OK)
        return rc;
      const size_t gs = vegas_flow_grad_scratch_bytes(d, std::min<int64_t>(P.train_rows, h->flow_batch));
      if (gs == 0) return VEGAS_EINVAL;
      if ((rc = grow_bytes(h, h->d_grad_scratch, h->grad_scratch_cap, gs)) != VEGAS_OK) return rc;
    } else if (h->flow_train_iters > h->flow_trained) {
      h->flow_trained = h->flow_train_iters;  // nothing to train with
    }
  }

  int nrun = 0, njudge = 0, flags = 0;
  bool flow_now = flow;
  for (int it = 0; it < nitn; ++it) {
    cudaEvent_t* e = &h->ev[6 * it];
    VG_CHECK(cudaEventRecord(e[0], s));
    const bool train = flow_now && h->flow_trained < h->flow_train_iters;
    const bool trained_before = h->flow_trained >= h->flow_train_iters;
    if ((rc = run_arm(h, 0, it, flow_now, train, paired, P, e[1], e[2])) != VEGAS_OK) return rc;
    VG_CHECK(cudaEventRecord(e[4], s));
    if (paired) {
      if ((rc = run_arm(h, 1, it, false, false, true, P, nullptr, nullptr)) != VEGAS_OK) return rc;
      VG_CHECK(cudaEventRecord(e[5], s));
      ++njudge;
      ++h->judge_pairs;
    }
    VG_CHECK(cudaEventRecord(e[3], s));
    h->iter_counter++;
    nrun = it + 1;
    if (paired) {
      if (trained_before) {
        // sigma_t^2 x device time of each form on this iteration (training steps excluded: none ran)
        double sig[2];
        VG_CHECK(cudaMemcpyAsync(&h->h_out[0], h->arm[0].d_it_sig + it, sizeof(double), cudaMemcpyDeviceToHost, s));
        VG_CHECK(cudaMemcpyAsync(&h->h_out[1], h->arm[1].d_it_sig + it, sizeof(double), cudaMemcpyDeviceToHost, s));
        VG_CHECK(cudaStreamSynchronize(s));
        sig[0] = h->h_out[0];
        sig[1] = h->h_out[1];
        float t0 = 0.0f, t1 = 0.0f;
        VG_CHECK(cudaEventElapsedTime(&t0, e[0], e[4]));
        VG_CHECK(cudaEventElapsedTime(&t1, e[4], e[5]));
        h->judge_vt[0].push_back(sig[0] * sig[0] * (double)t0);
        h->judge_vt[1].push_back(sig[1] * sig[1] * (double)t1);
      }
      const int w = h->judge_window;
      if ((int)h->judge_vt[0].size() >= w && h->judge_pairs >= kJudgeMinAdapt + w) {
        const std::vector<double> f(h->judge_vt[0].end() - w, h->judge_vt[0].end());
        const std::vector<double> q(h->judge_vt[1].end() - w, h->judge_vt[1].end());
        h->judge_ratio = median(q) / median(f);
        if (h->judge_ratio > 1.0) {  // NaN or a tie: plain VEGAS+, the fallback
          h->judge_state = kJudgeFlowKept;
          flags |= VEGAS_RESULT_FLOW_KEPT;
        } else {
          judge_switch_to_plain(h);
          flags |= VEGAS_RESULT_FLOW_OFF;
          flow_now = false;
        }
        paired = false;
      }
    }
    if (h->rtol > 0.0 && it + 1 > h->skip) {
      VG_CHECK(cudaMemcpyAsync(h->h_out, h->arm[0].d_out, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
      if (paired)
        VG_CHECK(cudaMemcpyAsync(h->h_out + 4, h->arm[1].d_out, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
      VG_CHECK(cudaStreamSynchronize(s));
      // the FP32 form's sigma counts as at least its rounding floor
      const double fl = h->precision == VEGAS_FP32 ? vg::kFp32SigmaFloor : 0.0;
      const double r0 = std::max(h->h_out[1] / std::fabs(h->h_out[0]), fl);
      const double r1 = paired ? std::max(h->h_out[5] / std::fabs(h->h_out[4]), fl) : INFINITY;
      if (r0 <= h->rtol || r1 <= h->rtol) {
        if (paired) {  // the first form to reach the target is the result
          if (r1 < r0) {
            judge_switch_to_plain(h);
            flags |= VEGAS_RESULT_FLOW_OFF;
          } else {
            h->judge_state = kJudgeFlowKept;
            flags |= VEGAS_RESULT_FLOW_KEPT;
          }
        }
        break;
      }
    }
  }
  h->last_nrun = nrun;
  // results to the host
  const Arm& A = h->arm[0];
  int dflags = 0;
  VG_CHECK(cudaMemcpyAsync(h->h_out, A.d_out, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
  if (out->it_est && out->it_cap > 0)
    VG_CHECK(cudaMemcpyAsync(out->it_est, A.d_it_est, sizeof(double) * (size_t)std::min(nrun, (int)out->it_cap),
                             cudaMemcpyDeviceToHost, s));
  if (out->it_sigma && out->it_cap > 0)
    VG_CHECK(cudaMemcpyAsync(out->it_sigma, A.d_it_sig, sizeof(double) * (size_t)std::min(nrun, (int)out->it_cap),
                             cudaMemcpyDeviceToHost, s));
  VG_CHECK(cudaMemcpyAsync(&dflags, h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  VG_CHECK(cudaStreamSynchronize(s));
  out->estimate = h->h_out[0];
  out->sigma = h->h_out[1];
  out->chi2_dof = h->h_out[2];
  out->n_used = (int32_t)h->h_out[3];
  out->nitn_run = nrun;
  out->nitn_judge = njudge;
  out->neval_total = neval * (int64_t)(nrun + njudge);
  out->judge_ratio = (flags & (VEGAS_RESULT_FLOW_OFF | VEGAS_RESULT_FLOW_KEPT)) ? h->judge_ratio : 0.0;
  if (out->n_used >= 2) {
    const double bound = h->chi2_bound > 0.0 ? h->chi2_bound : chi2_dof_quantile_999(out->n_used - 1);
    if (!(out->chi2_dof <= bound)) flags |= VEGAS_RESULT_CHI2_HIGH;
  }
  if (h->precision == VEGAS_FP32 && out->sigma < vg::kFp32SigmaFloor * std::fabs(out->estimate))
    flags |= VEGAS_RESULT_FP32_FLOOR;
  out->flags = flags;
  // a cube crossing tiles was not reassembled, or (bounds-checking builds) an index check failed: internal error
  if (dflags & (2 | 8)) return VEGAS_ECUDA;
  if (flow && (rc = vg::flow_tc_status(true)) != VEGAS_OK) return rc;
  if (flow && (rc = vg::flow_grad_tc_status(true)) != VEGAS_OK) return rc;
  return (dflags & 1) ? VEGAS_ENONFINITE : VEGAS_OK;
}

extern "C" int vegas_get_timings(vegas_handle h, float* iter_ms, float* fill_ms, int cap, int* n) {
  if (!h || cap < 0) return VEGAS_EINVAL;
  DeviceGuard g(h->device);
  VG_CHECK(cudaStreamSynchronize(h->stream()));
  const int m = std::min(cap, h->last_nrun);
  for (int i = 0; i < m; ++i) {
    if (iter_ms) VG_CHECK(cudaEventElapsedTime(&iter_ms[i], h->ev[6 * i], h->ev[6 * i + 3]));
    if (fill_ms) VG_CHECK(cudaEventElapsedTime(&fill_ms[i], h->ev[6 * i + 1], h->ev[6 * i + 2]));
  }
  if (n) *n = h->last_nrun;
  return VEGAS_OK;
}

namespace {
struct StateHeader {
  char magic[8];
  uint32_t version;
  int32_t dim, nbins, ell_valid;
  int64_t ncubes, iter_counter;
  int32_t nstrat[vg::kMaxDim];
};
constexpr char kMagic[8] = {'V', 'E', 'G', 'A', 'S', 'G', 'B', '3'};
}  // namespace

extern "C" int vegas_get_state(vegas_handle h, void* buf, size_t* bytes) {
  if (!h || !bytes) return VEGAS_EINVAL;
  const Arm& A = h->arm[0];
  const size_t ne = (size_t)h->dim * (h->nbins + 1);
  int64_t nc = 0;
  if (A.ell_valid) {
    nc = 1;
    for (int32_t s : A.ell_nstrat) nc *= s;
  }
  const size_t need = sizeof(StateHeader) + sizeof(double) * ne + sizeof(float) * (size_t)nc;
  if (!buf) {
    *bytes = need;
    return VEGAS_OK;
  }
  if (*bytes < need) return VEGAS_ENOSPACE;
  DeviceGuard g(h->device);
  VG_CHECK(cudaStreamSynchronize(h->stream()));
  StateHeader hd{};
  std::memcpy(hd.magic, kMagic, 8);
  hd.version = 1;
  hd.dim = h->dim;
  hd.nbins = h->nbins;
  hd.ell_valid = A.ell_valid ? 1 : 0;
  hd.ncubes = nc;
  hd.iter_counter = h->iter_counter;
  for (int k = 0; k < h->dim && A.ell_valid; ++k) hd.nstrat[k] = A.ell_nstrat[k];
  unsigned char* p = (unsigned char*)buf;
  std::memcpy(p, &hd, sizeof hd);
  VG_CHECK(cudaMemcpy(p + sizeof hd, A.d_edges[A.cur], sizeof(double) * ne, cudaMemcpyDeviceToHost));
  if (nc > 0)
    VG_CHECK(cudaMemcpy(p + sizeof hd + sizeof(double) * ne, A.d_ell, sizeof(float) * (size_t)nc,
                        cudaMemcpyDeviceToHost));
  *bytes = need;
  return VEGAS_OK;
}

extern "C" int vegas_set_state(vegas_handle h, const void* buf, size_t bytes) {
  if (!h || !buf) return VEGAS_EINVAL;
  if (bytes < sizeof(StateHeader)) return VEGAS_ESTATE;
  StateHeader hd;
  std::memcpy(&hd, buf, sizeof hd);
  if (std::memcmp(hd.magic, kMagic, 8) != 0 || hd.version != 1 || hd.dim != h->dim || hd.nbins != h->nbins)
    return VEGAS_ESTATE;
  const size_t ne = (size_t)h->dim * (h->nbins + 1);
  int64_t nc = 0;
  if (hd.ell_valid) {
    nc = 1;
    for (int k = 0; k < hd.dim; ++k) {
      if (hd.nstrat[k] < 1) return VEGAS_ESTATE;
      nc *= hd.nstrat[k];
    }
    if (nc != hd.ncubes) return VEGAS_ESTATE;
  }
  if (bytes < sizeof hd + sizeof(double) * ne + sizeof(float) * (size_t)nc) return VEGAS_ESTATE;
  DeviceGuard g(h->device);
  VG_CHECK(cudaStreamSynchronize(h->stream()));
  const unsigned char* p = (const unsigned char*)buf;
  Arm& A = h->arm[0];
  A.cur = 0;
  VG_CHECK(cudaMemcpy(A.d_edges[0], p + sizeof hd, sizeof(double) * ne, cudaMemcpyHostToDevice));
  A.ell_valid = false;
  A.fill_key = nullptr;
  if (nc > 0) {
    const int rc = ensure_cubes(h, A, nc);
    if (rc != VEGAS_OK) return rc;
    VG_CHECK(cudaMemcpy(A.d_ell, p + sizeof hd + sizeof(double) * ne, sizeof(float) * (size_t)nc,
                        cudaMemcpyHostToDevice));
    A.ell_valid = true;
    A.ell_nstrat.assign(hd.nstrat, hd.nstrat + hd.dim);
  }
  h->iter_counter = hd.iter_counter;
  judge_reset(h);
  return VEGAS_OK;
}

extern "C" int vegas_get_edges(vegas_handle h, double* edges, size_t count) {
  if (!h || !edges || count < (size_t)h->dim * (h->nbins + 1)) return VEGAS_EINVAL;
  DeviceGuard g(h->device);
  VG_CHECK(cudaStreamSynchronize(h->stream()));
  VG_CHECK(cudaMemcpy(edges, h->arm[0].d_edges[h->arm[0].cur], sizeof(double) * (size_t)h->dim * (h->nbins + 1),
                      cudaMemcpyDeviceToHost));
  return VEGAS_OK;
}

extern "C" const char* vegas_strerror(int status) {
  switch (status) {
    case VEGAS_OK: return "ok";
    case VEGAS_EINVAL: return "invalid argument";
    case VEGAS_ENOMEM: return "out of memory";
    case VEGAS_ECUDA: return "CUDA error";
    case VEGAS_ENONFINITE: return "integrand returned a non-finite value";
    case VEGAS_ETIMEOUT: return "bounded device wait timed out";
    case VEGAS_ESTATE: return "state blob does not match the handle";
    case VEGAS_ENOSPACE: return "scratch or output buffer too small";
    default: return "unknown status";
  }
}

// ---------------------------------------------------------------------------
// learned proposal
// ---------------------------------------------------------------------------
extern "C" int vegas_set_flow(vegas_handle h, const float* params, int64_t nparams) {
  if (!h) return VEGAS_EINVAL;
  DeviceGuard g(h->device);
  VG_CHECK(cudaStreamSynchronize(h->stream()));
  judge_reset(h);
  if (!params) {
    for (float** p : {&h->d_flow, &h->d_flow_m, &h->d_flow_v, &h->d_flow_g, &h->d_flow_loss}) dfree_ptr(h, *p);
    h->flow_np = 0;
    return VEGAS_OK;
  }
  if (h->dim < 2 || h->dim > 32 || nparams != vegas_flow_param_count(h->dim)) return VEGAS_EINVAL;
  if (!h->d_flow) {
    const size_t b = sizeof(float) * (size_t)nparams;
    bool ok = true;
    for (float** p : {&h->d_flow, &h->d_flow_m, &h->d_flow_v, &h->d_flow_g}) ok = ok && (*p = (float*)dalloc(h, b));
    ok = ok && (h->d_flow_loss = (float*)dalloc(h, sizeof(float)));
    if (!ok) {  // all or nothing: the flow stays off
      for (float** p : {&h->d_flow, &h->d_flow_m, &h->d_flow_v, &h->d_flow_g, &h->d_flow_loss}) dfree_ptr(h, *p);
      h->flow_np = 0;
      return VEGAS_ENOMEM;
    }
  }
  h->flow_np = nparams;
  VG_CHECK(cudaMemcpy(h->d_flow, params, sizeof(float) * (size_t)nparams, cudaMemcpyHostToDevice));
  VG_CHECK(cudaMemset(h->d_flow_m, 0, sizeof(float) * (size_t)nparams));
  VG_CHECK(cudaMemset(h->d_flow_v, 0, sizeof(float) * (size_t)nparams));
  VG_CHECK(cudaMemset(h->d_flow_loss, 0, sizeof(float)));
  h->flow_step = 0;
  return VEGAS_OK;
}

extern "C" int vegas_set_flow_training(vegas_handle h, int32_t iterations, int32_t steps_per_iteration,
                                       int32_t samples, int32_t batch, float lr, float temper, float floor) {
  if (!h || iterations < 0 || steps_per_iteration < 0 || samples < 0 || batch < 1 || !(lr > 0.0f) ||
      !(temper > 0.0f && temper <= 1.0f) || !(floor >= 0.0f))
    return VEGAS_EINVAL;
  h->flow_floor = floor;
  h->flow_batch = batch;
  h->flow_temper = temper;
  h->flow_train_iters = iterations;
  h->flow_train_steps = steps_per_iteration;
  h->flow_train_samples = samples;
  h->flow_lr = lr;
  h->flow_trained = 0;
  return VEGAS_OK;
}

extern "C" int vegas_flow_explore(vegas_handle h, int32_t integrand, const double* params, int64_t nparams,
                                  int64_t neval, int32_t iterations, int32_t nmaps, int64_t samples_per_map,
                                  int32_t steps, int32_t batch, float lr, float floor, int32_t rounds,
                                  uint64_t seed) {
  if (!h || !h->d_flow || h->precision != VEGAS_FP32 || iterations < 1 || nmaps < 1 || rounds < 1 || rounds > 16 ||
      nmaps > vg::kMaxExploreMaps || samples_per_map < 1 || samples_per_map > vg::kMaxEval / nmaps || steps < 0 ||
      batch < 1 || !(lr > 0.0f) || !(floor >= 0.0f) || integrand == VEGAS_MAP_DENSITY)
    return VEGAS_EINVAL;
  const int d = h->dim, G = h->nbins;
  const int64_t m = (int64_t)nmaps * samples_per_map;
  if (m * d > vg::kMaxEval || vg::derived_param_count(integrand, d, params, nparams) < 0) return VEGAS_EINVAL;
  DeviceGuard guard(h->device);
  cudaStream_t s = h->stream();
  const int64_t ne = (int64_t)d * (G + 1);
  int rc;
  if ((rc = grow(h, h->d_explore, h->explore_cap, nmaps * ne + m)) != VEGAS_OK) return rc;
  double* maps = h->d_explore;
  double* q = h->d_explore + nmaps * ne;
  // 1. nmaps maps, each adapted from the uniform map by plain VEGAS+ with seed + k (the flow set aside meanwhile)
  float* flow = h->d_flow;
  h->d_flow = nullptr;
  vegas_result r{};
  for (int k = 0; k < nmaps && rc == VEGAS_OK; ++k) {
    if ((rc = vegas_reset_map(h)) != VEGAS_OK) break;
    if ((rc = vegas_integrate(h, integrand, params, nparams, neval, iterations, seed + (uint64_t)k, &r)) != VEGAS_OK)
      break;
    const Arm& A = h->arm[0];
    if (cudaMemcpyAsync(maps + k * ne, A.d_edges[A.cur], sizeof(double) * (size_t)ne, cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
      rc = VEGAS_ECUDA;
  }
  h->d_flow = flow;
  if (rc != VEGAS_OK) return rc;
  // 2. their pooled samples, the integrand there (the parameters are on the device since the last iteration) and
  // the balance-heuristic weights; the training set with the floor's uniform rows
  const int64_t rows = vg::flow_train_rows(m, floor);
  const int64_t nb = std::min<int64_t>(rows, batch);
  const size_t gs = vegas_flow_grad_scratch_bytes(d, nb);
  if (gs == 0) return VEGAS_EINVAL;
  if ((rc = grow(h, h->d_X, h->x_cap, m * d)) != VEGAS_OK || (rc = grow(h, h->d_logdet, h->ld_cap, m)) != VEGAS_OK ||
      (rc = grow(h, h->d_values, h->val_cap, m)) != VEGAS_OK ||
      (rc = grow(h, h->d_train_x, h->tx_cap, rows * d)) != VEGAS_OK ||
      (rc = grow(h, h->d_train_w, h->tw_cap, rows + m + 4)) != VEGAS_OK ||
      (rc = grow_bytes(h, h->d_grad_scratch, h->grad_scratch_cap, gs)) != VEGAS_OK)
    return rc;
  VG_CHECK(cudaMemsetAsync(h->d_logdet, 0, sizeof(float) * (size_t)m, s));
  if ((rc = vg::explore_points(d, G, nmaps, maps, m, seed, h->d_X, q, s)) != VEGAS_OK) return rc;
  if ((rc = vg::flow_eval(integrand, d, h->d_params, nparams, h->d_X, h->d_logdet, h->d_values, m, s)) != VEGAS_OK)
    return rc;
  float* wraw = h->d_train_w + rows;
  if ((rc = vg::explore_weights(h->d_values, q, m, wraw, s)) != VEGAS_OK) return rc;
  double* wsum = (double*)(h->d_train_w + ((rows + m + 1) & ~(int64_t)1));
  if ((rc = vg::flow_gather(h->d_X, d, 1, m, wraw, floor, seed, 0x45585052u, wsum, h->d_train_x, h->d_train_w, s)) !=
      VEGAS_OK)
    return rc;
  for (int round = 0; round < rounds; ++round) {
    if (round > 0) {
      // a later round's pool: m samples of the flow itself, x = F(u) with u uniform (the uniform map's points, whose
      // density is 1), weighted |f(x)| |det dF/du|; fresh Adam moments
      if ((rc = vegas_reset_map(h)) != VEGAS_OK) return rc;
      const Arm& A = h->arm[0];
      if ((rc = vg::explore_points(d, G, 1, A.d_edges[A.cur], m, seed + 0x9E3779B97F4A7C15ull * (uint64_t)round,
                                   h->d_X, q, s)) != VEGAS_OK ||
          (rc = vg::flow_apply(d, VEGAS_FLOW_SAMPLE, h->d_flow, h->d_X, h->d_X, h->d_logdet, m, s)) != VEGAS_OK ||
          (rc = vg::flow_eval(integrand, d, h->d_params, nparams, h->d_X, h->d_logdet, h->d_values, m, s)) !=
              VEGAS_OK ||
          (rc = vg::explore_weights(h->d_values, q, m, wraw, s)) != VEGAS_OK ||
          (rc = vg::flow_gather(h->d_X, d, 1, m, wraw, floor, seed, 0x45585052u + (uint32_t)round, wsum,
                                h->d_train_x, h->d_train_w, s)) != VEGAS_OK)
        return rc;
      VG_CHECK(cudaMemsetAsync(h->d_flow_m, 0, sizeof(float) * (size_t)h->flow_np, s));
      VG_CHECK(cudaMemsetAsync(h->d_flow_v, 0, sizeof(float) * (size_t)h->flow_np, s));
      h->flow_step = 0;
    }
    // 3. Adam steps on consecutive windows of the training set, cycling (the samples of all maps interleave)
    for (int k = 0; k < steps; ++k) {
      const int64_t off = ((int64_t)k * nb) % (rows - nb + 1);
      if ((rc = vegas_flow_grad(d, h->d_flow, h->d_train_x + off * d, h->d_train_w + off, nb, h->d_flow_g,
                                h->d_flow_loss, h->d_grad_scratch, h->grad_scratch_cap, s)) != VEGAS_OK ||
          (rc = vegas_flow_adam(h->flow_np, h->d_flow, h->d_flow_g, h->d_flow_m, h->d_flow_v, ++h->flow_step, lr,
                                0.9f, 0.999f, 1e-8f, s)) != VEGAS_OK)
        return rc;
    }
  }
  // 4. a uniform map again, for the run under the trained flow; the bounded waits of the flow's kernels
  if ((rc = vegas_reset_map(h)) != VEGAS_OK) return rc;
  if ((rc = vg::flow_tc_status(true)) != VEGAS_OK) return rc;
  return vg::flow_grad_tc_status(true);
}

extern "C" int vegas_get_flow(vegas_handle h, float* params, int64_t nparams, float* last_loss) {
  if (!h || !h->d_flow || (params && nparams != h->flow_np)) return VEGAS_EINVAL;
  DeviceGuard g(h->device);
  VG_CHECK(cudaStreamSynchronize(h->stream()));
  if (params) VG_CHECK(cudaMemcpy(params, h->d_flow, sizeof(float) * (size_t)nparams, cudaMemcpyDeviceToHost));
  if (last_loss) VG_CHECK(cudaMemcpy(last_loss, h->d_flow_loss, sizeof(float), cudaMemcpyDeviceToHost));
  return VEGAS_OK;
}
