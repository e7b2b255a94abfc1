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
#include <new>
#include <vector>

#include "vegas_internal.h"

struct vegas_s {
  int device = 0;
  int dim = 0, nbins = 0, nstrat_scalar = 0;
  double alpha = 0.5, beta = 0.75;
  std::vector<int32_t> nstrat_axes;  // empty: use nstrat_scalar / automatic
  int skip = 0, precision = VEGAS_FP64, weighting = VEGAS_WEIGHT_AUTO;
  double rtol = 0.0;
  cudaStream_t own_stream = nullptr, user_stream = nullptr;
  bool has_user_stream = false;
  // device buffers
  double* d_edges[2] = {nullptr, nullptr};
  int cur = 0;
  double* d_bins = nullptr;
  int64_t* d_offsets = nullptr;
  float* d_ell = nullptr;
  int64_t cubes_cap = 0;
  void* d_fill_scratch = nullptr;
  size_t fill_scratch_cap = 0;
  void* d_alloc_scratch = nullptr;
  size_t alloc_scratch_cap = 0;
  double* d_params = nullptr;
  int64_t params_cap = 0;
  double* d_result = nullptr;  // [2]
  double* d_out = nullptr;     // [4]
  int* d_flags = nullptr;
  double* d_it_est = nullptr;
  double* d_it_sig = nullptr;
  int it_cap = 0;
  double* h_out = nullptr;  // pinned [4]
  // carried-over stratification
  bool ell_valid = false;
  const int* fill_key = nullptr;  // max-ell key left in the fill scratch by the last fill, or NULL
  std::vector<int32_t> ell_nstrat;
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
  // timing
  std::vector<cudaEvent_t> ev;  // 4 per iteration: start, fill start, fill end, end
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

template <typename T>
int grow(T*& p, int64_t& cap, int64_t need) {
  if (need <= cap && p) return VEGAS_OK;
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
  if (cudaMalloc((void**)&p, sizeof(T) * (size_t)need) != cudaSuccess) {
    cudaGetLastError();
    return VEGAS_ENOMEM;
  }
  cap = need;
  return VEGAS_OK;
}

int grow_bytes(void*& p, size_t& cap, size_t need) {
  if (need <= cap && p) return VEGAS_OK;
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
  if (cudaMalloc(&p, need) != cudaSuccess) {
    cudaGetLastError();
    return VEGAS_ENOMEM;
  }
  cap = need;
  return VEGAS_OK;
}

int upload_uniform_edges(vegas_s* h) {
  const int G = h->nbins;
  std::vector<double> e((size_t)h->dim * (G + 1));
  for (int k = 0; k < h->dim; ++k)
    for (int i = 0; i <= G; ++i) e[(size_t)k * (G + 1) + i] = (double)i / (double)G;
  h->cur = 0;
  VG_CHECK(cudaMemcpy(h->d_edges[0], e.data(), sizeof(double) * e.size(), cudaMemcpyHostToDevice));
  return VEGAS_OK;
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

// offsets [n] and allocation weights [n] grow together; contents are not kept
int ensure_cubes(vegas_s* h, int64_t n) {
  if (n <= h->cubes_cap && h->d_offsets && h->d_ell) return VEGAS_OK;
  cudaFree(h->d_offsets);
  cudaFree(h->d_ell);
  h->d_offsets = nullptr;
  h->d_ell = nullptr;
  h->cubes_cap = 0;
  h->ell_valid = false;
  if (cudaMalloc((void**)&h->d_offsets, sizeof(int64_t) * (size_t)n) != cudaSuccess ||
      cudaMalloc((void**)&h->d_ell, sizeof(float) * (size_t)n) != cudaSuccess) {
    cudaGetLastError();
    return VEGAS_ENOMEM;
  }
  h->cubes_cap = n;
  return VEGAS_OK;
}

void release(vegas_s* h) {
  cudaFree(h->d_edges[0]);
  cudaFree(h->d_edges[1]);
  cudaFree(h->d_bins);
  cudaFree(h->d_offsets);
  cudaFree(h->d_ell);
  cudaFree(h->d_fill_scratch);
  cudaFree(h->d_alloc_scratch);
  cudaFree(h->d_params);
  cudaFree(h->d_result);
  cudaFree(h->d_out);
  cudaFree(h->d_flags);
  cudaFree(h->d_it_est);
  cudaFree(h->d_it_sig);
  if (h->h_out) cudaFreeHost(h->h_out);
  for (float* p : {h->d_flow, h->d_flow_m, h->d_flow_v, h->d_flow_g, h->d_flow_loss, h->d_X, h->d_logdet,
                   h->d_values, h->d_train_x, h->d_train_w})
    cudaFree(p);
  cudaFree(h->d_grad_scratch);
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
  if (rc == VEGAS_OK &&
      (cudaMalloc((void**)&h->d_edges[0], sizeof(double) * ne) != cudaSuccess ||
       cudaMalloc((void**)&h->d_edges[1], sizeof(double) * ne) != cudaSuccess ||
       cudaMalloc((void**)&h->d_bins, sizeof(double) * nb) != cudaSuccess ||
       cudaMalloc((void**)&h->d_result, sizeof(double) * 2) != cudaSuccess ||
       cudaMalloc((void**)&h->d_out, sizeof(double) * 4) != cudaSuccess ||
       cudaMalloc((void**)&h->d_flags, sizeof(int)) != cudaSuccess ||
       cudaMallocHost((void**)&h->h_out, sizeof(double) * 4) != cudaSuccess))
    rc = VEGAS_ENOMEM;
  if (rc == VEGAS_OK) rc = upload_uniform_edges(h);
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
  h->ell_valid = false;
  h->fill_key = nullptr;
  h->iter_counter = 0;
  return upload_uniform_edges(h);
}

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
    int s = h->nstrat_scalar > 0 ? h->nstrat_scalar : default_nstrat(neval, d);
    if (h->precision == VEGAS_FP32 && h->nstrat_scalar <= 0 && s > 65536) s = 65536;
    for (int k = 0; k < d; ++k) ns[k] = s;
  }
  int64_t NH = 1;
  for (int k = 0; k < d; ++k) {
    if (h->precision == VEGAS_FP32 && ns[k] > 65536) return VEGAS_EINVAL;
    NH *= ns[k];
    if (NH >= (int64_t(1) << 31)) return VEGAS_EINVAL;
  }
  if (neval < 2 * NH) return VEGAS_EINVAL;

  DeviceGuard guard(h->device);
  cudaStream_t s = h->stream();
  const vegas_geometry geo{d, G, ns.data()};
  int rc;
  if ((rc = ensure_cubes(h, NH + 1)) != VEGAS_OK) return rc;
  const size_t fill_need = vegas_fill_scratch_bytes(&geo, neval);
  const size_t alloc_need = vegas_allocate_scratch_bytes(NH);
  if (fill_need == 0 || alloc_need == 0) return VEGAS_EINVAL;
  if (fill_need > h->fill_scratch_cap) h->fill_key = nullptr;  // the scratch is about to move
  if ((rc = grow_bytes(h->d_fill_scratch, h->fill_scratch_cap, fill_need)) != VEGAS_OK) return rc;
  if ((rc = grow_bytes(h->d_alloc_scratch, h->alloc_scratch_cap, alloc_need)) != VEGAS_OK) return rc;
  if (nparams > 0 && (rc = grow(h->d_params, h->params_cap, nparams)) != VEGAS_OK) return rc;
  if (h->it_cap < nitn) {
    cudaFree(h->d_it_est);
    cudaFree(h->d_it_sig);
    h->d_it_est = h->d_it_sig = nullptr;
    h->it_cap = 0;
    if (cudaMalloc((void**)&h->d_it_est, sizeof(double) * nitn) != cudaSuccess ||
        cudaMalloc((void**)&h->d_it_sig, sizeof(double) * nitn) != cudaSuccess)
      return VEGAS_ENOMEM;
    h->it_cap = nitn;
  }
  while ((int)h->ev.size() < 4 * nitn) {
    cudaEvent_t e;
    VG_CHECK(cudaEventCreate(&e));
    h->ev.push_back(e);
  }
  if (nparams > 0)
    VG_CHECK(cudaMemcpyAsync(h->d_params, params, sizeof(double) * (size_t)nparams, cudaMemcpyHostToDevice, s));
  VG_CHECK(cudaMemsetAsync(h->d_flags, 0, sizeof(int), s));

  // learned proposal: per-evaluation buffers and the training sample
  const bool flow = h->d_flow != nullptr;
  int64_t train_stride = 1, n_train = 0, train_rows = 0;
  if (flow) {
    if (h->precision != VEGAS_FP32) return VEGAS_EINVAL;
    if ((rc = grow(h->d_X, h->x_cap, neval * d)) != VEGAS_OK || (rc = grow(h->d_logdet, h->ld_cap, neval)) != VEGAS_OK ||
        (rc = grow(h->d_values, h->val_cap, neval)) != VEGAS_OK)
      return rc;
    if (h->flow_train_iters > h->flow_trained && h->flow_train_samples > 0 && h->flow_train_steps > 0) {
      train_stride = std::max<int64_t>(1, neval / h->flow_train_samples);
      n_train = (neval + train_stride - 1) / train_stride;
      train_rows = vg::flow_train_rows(n_train, h->flow_floor);
      // d_train_w: the training set's weights [train_rows], the fill's raw weights [n_train], their sum (a double)
      if ((rc = grow(h->d_train_x, h->tx_cap, train_rows * d)) != VEGAS_OK ||
          (rc = grow(h->d_train_w, h->tw_cap, train_rows + n_train + 4)) != VEGAS_OK)
        return rc;
      const size_t gs = vegas_flow_grad_scratch_bytes(d, std::min<int64_t>(train_rows, h->flow_batch));
      if (gs == 0) return VEGAS_EINVAL;
      if ((rc = grow_bytes(h->d_grad_scratch, h->grad_scratch_cap, gs)) != VEGAS_OK) return rc;
    } else if (h->flow_train_iters > h->flow_trained) {
      h->flow_trained = h->flow_train_iters;  // nothing to train with
    }
  }

  // the stratification of an earlier call carries over only on the same cubes
  bool uniform = !(h->ell_valid && h->ell_nstrat == ns);
  int nrun = 0;
  for (int it = 0; it < nitn; ++it) {
    cudaEvent_t* e = &h->ev[4 * it];
    VG_CHECK(cudaEventRecord(e[0], s));
    rc = vg::allocate_impl(h->d_ell, NH, neval, (uniform || h->beta == 0.0) ? 1 : 0, h->d_offsets,
                           h->d_alloc_scratch, h->alloc_scratch_cap, s, h->fill_key);
    if (rc != VEGAS_OK) return rc;
    const bool train = flow && h->flow_trained < h->flow_train_iters;
    if (flow) {
      // points x' of the VEGAS+ map, x = F(x') and |det dF/dx'|, then g = f(x) |det| tabulated by evaluation
      vg::FillExtra ex_points{nullptr, h->d_X, nullptr, 0, 1.0f};
      rc = vg::fill_impl(&geo, VEGAS_FP32, vg::kIntegrandPoints, nullptr, 0, neval, seed, (int32_t)h->iter_counter,
                         0u, h->beta, h->d_edges[h->cur], h->d_offsets, h->d_ell, h->d_bins, h->d_result, nullptr,
                         nullptr, h->d_flags, h->d_fill_scratch, h->fill_scratch_cap, s, nullptr, nullptr, &ex_points);
      if (rc != VEGAS_OK) return rc;
      if ((rc = vg::flow_apply(d, VEGAS_FLOW_SAMPLE, h->d_flow, h->d_X, h->d_X, h->d_logdet, neval, s)) != VEGAS_OK)
        return rc;
      if ((rc = vg::flow_eval(integrand, d, h->d_params, nparams, h->d_X, h->d_logdet, h->d_values, neval, s)) !=
          VEGAS_OK)
        return rc;
      // the temper exponent ramps linearly to 1 over the training iterations: broad targets first
      const float power =
          h->flow_train_iters > 1
              ? h->flow_temper + (1.0f - h->flow_temper) * (float)h->flow_trained / (float)(h->flow_train_iters - 1)
              : 1.0f;
      vg::FillExtra ex_tab{h->d_values, nullptr, train ? h->d_train_w + train_rows : nullptr, (int)train_stride,
                           power};
      rc = vg::fill_impl(&geo, VEGAS_FP32, vg::kIntegrandTabulated, nullptr, 0, neval, seed,
                         (int32_t)h->iter_counter, 0u, h->beta, h->d_edges[h->cur], h->d_offsets, h->d_ell, h->d_bins,
                         h->d_result, nullptr, nullptr, h->d_flags, h->d_fill_scratch, h->fill_scratch_cap, s, e[1],
                         e[2], &ex_tab);
    } else {
      rc = vg::fill_impl(&geo, h->precision, integrand, h->d_params, nparams, neval, seed, (int32_t)h->iter_counter,
                         0u, h->beta, h->d_edges[h->cur], h->d_offsets, h->d_ell, h->d_bins, h->d_result, nullptr,
                         nullptr, h->d_flags, h->d_fill_scratch, h->fill_scratch_cap, s, e[1], e[2]);
    }
    if (rc != VEGAS_OK) return rc;
    h->fill_key = vg::fill_ellmax_key(&geo, neval, h->d_fill_scratch);
    rc = vegas_refine(d, G, h->alpha, h->d_bins, h->d_edges[h->cur], h->d_edges[1 - h->cur], s);
    if (rc != VEGAS_OK) return rc;
    h->cur = 1 - h->cur;
    const bool lagged = h->weighting == VEGAS_WEIGHT_LAGGED || (h->weighting == VEGAS_WEIGHT_AUTO && flow);
    rc = vg::launch_record_combine(h->d_result, it, h->d_it_est, h->d_it_sig, h->skip, h->d_out, lagged, s);
    if (rc != VEGAS_OK) return rc;
    if (train) {
      // Adam steps on the weighted samples of this iteration (x = F(x'), weight |J f| / n_h), with uniform
      // points of the floor mixed in
      double* wsum = (double*)(h->d_train_w + ((train_rows + n_train + 1) & ~(int64_t)1));
      if ((rc = vg::flow_gather(h->d_X, d, train_stride, n_train, h->d_train_w + train_rows, h->flow_floor, seed,
                                (uint32_t)h->iter_counter, wsum, h->d_train_x, h->d_train_w, s)) != VEGAS_OK)
        return rc;
      // minibatches: consecutive windows of the training set, cycling
      const int64_t nb = std::min<int64_t>(train_rows, h->flow_batch);
      for (int k = 0; k < h->flow_train_steps; ++k) {
        const int64_t off = ((int64_t)k * nb) % (train_rows - nb + 1);
        rc = vegas_flow_grad(d, h->d_flow, h->d_train_x + off * d, h->d_train_w + off, nb, h->d_flow_g,
                             h->d_flow_loss, h->d_grad_scratch, h->grad_scratch_cap, s);
        if (rc != VEGAS_OK) return rc;
        rc = vegas_flow_adam(h->flow_np, h->d_flow, h->d_flow_g, h->d_flow_m, h->d_flow_v, ++h->flow_step, h->flow_lr,
                             0.9f, 0.999f, 1e-8f, s);
        if (rc != VEGAS_OK) return rc;
      }
      h->flow_trained++;
    }
    VG_CHECK(cudaEventRecord(e[3], s));
    h->iter_counter++;
    uniform = false;
    h->ell_valid = true;
    h->ell_nstrat = ns;
    nrun = it + 1;
    if (h->rtol > 0.0 && it + 1 > h->skip) {
      VG_CHECK(cudaMemcpyAsync(h->h_out, h->d_out, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
      VG_CHECK(cudaStreamSynchronize(s));
      if (h->h_out[1] <= h->rtol * std::fabs(h->h_out[0])) break;
    }
  }
  h->last_nrun = nrun;
  // results to the host
  int flags = 0;
  VG_CHECK(cudaMemcpyAsync(h->h_out, h->d_out, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
  if (out->it_est && out->it_cap > 0)
    VG_CHECK(cudaMemcpyAsync(out->it_est, h->d_it_est, sizeof(double) * (size_t)std::min(nrun, (int)out->it_cap),
                             cudaMemcpyDeviceToHost, s));
  if (out->it_sigma && out->it_cap > 0)
    VG_CHECK(cudaMemcpyAsync(out->it_sigma, h->d_it_sig, sizeof(double) * (size_t)std::min(nrun, (int)out->it_cap),
                             cudaMemcpyDeviceToHost, s));
  VG_CHECK(cudaMemcpyAsync(&flags, h->d_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  VG_CHECK(cudaStreamSynchronize(s));
  out->estimate = h->h_out[0];
  out->sigma = h->h_out[1];
  out->chi2_dof = h->h_out[2];
  out->n_used = (int32_t)h->h_out[3];
  out->nitn_run = nrun;
  out->neval_total = neval * (int64_t)nrun;
  if (flags & 2) return VEGAS_ECUDA;  // a cube crossing tiles was not reassembled: internal error
  if (flow && (rc = vg::flow_tc_status(true)) != VEGAS_OK) return rc;
  return (flags & 1) ? VEGAS_ENONFINITE : VEGAS_OK;
}

extern "C" int vegas_get_timings(vegas_handle h, float* iter_ms, float* fill_ms, int cap, int* n) {
  if (!h || cap < 0) return VEGAS_EINVAL;
  DeviceGuard g(h->device);
  VG_CHECK(cudaStreamSynchronize(h->stream()));
  const int m = std::min(cap, h->last_nrun);
  for (int i = 0; i < m; ++i) {
    if (iter_ms) VG_CHECK(cudaEventElapsedTime(&iter_ms[i], h->ev[4 * i], h->ev[4 * i + 3]));
    if (fill_ms) VG_CHECK(cudaEventElapsedTime(&fill_ms[i], h->ev[4 * i + 1], h->ev[4 * i + 2]));
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
  const size_t ne = (size_t)h->dim * (h->nbins + 1);
  int64_t nc = 0;
  if (h->ell_valid) {
    nc = 1;
    for (int32_t s : h->ell_nstrat) nc *= s;
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
  hd.ell_valid = h->ell_valid ? 1 : 0;
  hd.ncubes = nc;
  hd.iter_counter = h->iter_counter;
  for (int k = 0; k < h->dim && h->ell_valid; ++k) hd.nstrat[k] = h->ell_nstrat[k];
  unsigned char* p = (unsigned char*)buf;
  std::memcpy(p, &hd, sizeof hd);
  VG_CHECK(cudaMemcpy(p + sizeof hd, h->d_edges[h->cur], sizeof(double) * ne, cudaMemcpyDeviceToHost));
  if (nc > 0)
    VG_CHECK(cudaMemcpy(p + sizeof hd + sizeof(double) * ne, h->d_ell, sizeof(float) * (size_t)nc,
                        cudaMemcpyDeviceToHost));
  *bytes = need;
  return VEGAS_OK;
}

extern "C" int vegas_set_state(vegas_handle h, const void* buf, size_t bytes) {
  if (!h || !buf || bytes < sizeof(StateHeader)) return VEGAS_EINVAL;
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
  h->cur = 0;
  VG_CHECK(cudaMemcpy(h->d_edges[0], p + sizeof hd, sizeof(double) * ne, cudaMemcpyHostToDevice));
  h->ell_valid = false;
  h->fill_key = nullptr;
  if (nc > 0) {
    const int rc = ensure_cubes(h, nc + 1);
    if (rc != VEGAS_OK) return rc;
    VG_CHECK(cudaMemcpy(h->d_ell, p + sizeof hd + sizeof(double) * ne, sizeof(float) * (size_t)nc,
                        cudaMemcpyHostToDevice));
    h->ell_valid = true;
    h->ell_nstrat.assign(hd.nstrat, hd.nstrat + hd.dim);
  }
  h->iter_counter = hd.iter_counter;
  return VEGAS_OK;
}

extern "C" int vegas_get_edges(vegas_handle h, double* edges, size_t count) {
  if (!h || !edges || count < (size_t)h->dim * (h->nbins + 1)) return VEGAS_EINVAL;
  DeviceGuard g(h->device);
  VG_CHECK(cudaStreamSynchronize(h->stream()));
  VG_CHECK(cudaMemcpy(edges, h->d_edges[h->cur], sizeof(double) * (size_t)h->dim * (h->nbins + 1),
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
  if (!params) {
    for (float** p : {&h->d_flow, &h->d_flow_m, &h->d_flow_v, &h->d_flow_g, &h->d_flow_loss}) {
      cudaFree(*p);
      *p = nullptr;
    }
    h->flow_np = 0;
    return VEGAS_OK;
  }
  if (h->dim < 2 || h->dim > 32 || nparams != vegas_flow_param_count(h->dim)) return VEGAS_EINVAL;
  if (!h->d_flow) {
    const size_t b = sizeof(float) * (size_t)nparams;
    if (cudaMalloc((void**)&h->d_flow, b) != cudaSuccess || cudaMalloc((void**)&h->d_flow_m, b) != cudaSuccess ||
        cudaMalloc((void**)&h->d_flow_v, b) != cudaSuccess || cudaMalloc((void**)&h->d_flow_g, b) != cudaSuccess ||
        cudaMalloc((void**)&h->d_flow_loss, sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
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

extern "C" int vegas_get_flow(vegas_handle h, float* params, int64_t nparams, float* last_loss) {
  if (!h || !h->d_flow || (params && nparams != h->flow_np)) return VEGAS_EINVAL;
  DeviceGuard g(h->device);
  VG_CHECK(cudaStreamSynchronize(h->stream()));
  if (params) VG_CHECK(cudaMemcpy(params, h->d_flow, sizeof(float) * (size_t)nparams, cudaMemcpyDeviceToHost));
  if (last_loss) VG_CHECK(cudaMemcpy(last_loss, h->d_flow_loss, sizeof(float), cudaMemcpyDeviceToHost));
  return VEGAS_OK;
}
