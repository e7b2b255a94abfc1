/*
 * vegas.h -- C ABI of the GB300 (sm_103a) VEGAS+ iteration loop.
 *
 * The library computes the VEGAS+ method as described in cuVegas (Tolotti,
 * Jnini, Vella, Passerone, arXiv 2408.09229):
 *   Sec. 2.1.1  adaptive importance sampling.  Separable map with N_g
 *               intervals per axis; Eqs. (2)-(4): J(y) = N_g dx_{i(y)} and
 *               I_MC = (1/N_ev) sum J f.
 *   Sec. 2.1.2  adaptive stratified sampling.  Eqs. (5)-(7): I = sum dI_h and
 *               sigma^2 = sum sigma_h^2 / n_h, with n_h proportional to sigma_h
 *               damped by beta, and sum n_h = N_eval.
 *   Sec. 2.1.3  inverse-variance combination of iterations, Eqs. (8)-(9).
 *   Algorithm 1 iteration loop; Algorithm 2 vegasFill.
 *
 * Two levels of entry points:
 *   1. A handle (vegas_create / vegas_integrate / vegas_destroy, plus setters,
 *      state and timing queries).  It owns its device buffers and runs whole
 *      integrations.
 *   2. Step entry points (vegas_allocate, vegas_fill, vegas_refine,
 *      vegas_combine).  Each runs one row of the iteration on caller-owned
 *      device buffers.  They are stateless: the caller passes plain device
 *      pointers and sizes, plus a caller-owned device scratch area whose size
 *      the matching *_scratch_bytes query returns.
 *
 * Conventions for all entry points:
 *   - The domain is the unit cube [0,1]^d.
 *   - Device pointers are "d_*" and must point to memory of the current CUDA
 *     device.  Host pointers have no prefix.
 *   - "stream" is a cudaStream_t passed as void*.  NULL means the legacy
 *     default stream.
 *   - Step entry points are asynchronous on the stream.  They return after
 *     queuing their kernels and report launch errors only.  Errors found on
 *     the device (a non-finite integrand value) go to the caller's device flag.
 *   - Every entry point returns VEGAS_OK (0) or a negative status from the
 *     list below.  No C++ exception crosses the ABI.
 *   - Arrays are row-major.  The map edges are [d][N_g+1] and the map weights
 *     are [d][N_g].  Hypercube h has coordinates c_k = (h / prod_{l<k} s_l)
 *     mod s_k, so axis 0 varies fastest.
 * Limits: 1 <= d <= 32, 2 <= N_g <= 4096, N_h = prod s_k < 2^31,
 * 2 N_h <= N_eval < 2^31 evaluations per iteration.
 */
#ifndef VEGAS_GB300_H
#define VEGAS_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define VEGAS_API __attribute__((visibility("default")))
#else
#define VEGAS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define VEGAS_OK 0
#define VEGAS_EINVAL (-1)     /* an argument is out of range                   */
#define VEGAS_ENOMEM (-2)     /* a device or host allocation failed            */
#define VEGAS_ECUDA (-3)      /* a CUDA runtime call or kernel launch failed   */
#define VEGAS_ENONFINITE (-4) /* the integrand returned NaN or +-inf           */
#define VEGAS_ETIMEOUT (-5)   /* a bounded device wait ran out                 */
#define VEGAS_ESTATE (-6)     /* a state blob does not match this handle       */
#define VEGAS_ENOSPACE (-7)   /* the caller's scratch or array is too small    */

/* ---- integrand families (compiled in; the layout of params per family) --- */
enum vegas_integrand {
  VEGAS_GAUSS_SUM = 0,         /* A sum_k exp(-|x-mu_k|^2/(2 s^2)); params [A, s, K, mu(K*d)]     */
  VEGAS_PRODUCT_PEAK = 1,      /* prod_i 1/(c_i^-2 + (x_i-w_i)^2); params [c(d), w(d)]            */
  VEGAS_OSCILLATORY = 2,       /* cos(2 pi u + sum_i a_i x_i); params [u, a(d)]                   */
  VEGAS_SIN_EXP = 3,           /* Table 3 (1): sin x_1 + exp x_2 (d = 2); no params              */
  VEGAS_LINEAR = 4,            /* Table 3 (2): sum x_i                                          */
  VEGAS_COSINE = 5,            /* Table 3 (3): prod cos x_i                                     */
  VEGAS_EXPONENTIAL = 6,       /* Table 3 (4): exp(sum x_i^2)                                   */
  VEGAS_ROOS_ARNOLD = 7,       /* Table 3 (5): prod |4 x_i - 2|                                 */
  VEGAS_MOROKOFF_CAFLISCH = 8, /* Table 3 (6): (1+1/d)^d prod x_i^(1/d)                         */
  VEGAS_MAP_DENSITY = 9,       /* density of a fixed separable map; params = its edges [d][G+1] */
  VEGAS_N_INTEGRANDS = 10
};
/* Table 3 (7) Gaussian and (8) Ridge are VEGAS_GAUSS_SUM instances. */

/* ---- precision of the per-evaluation arithmetic -------------------------- */
enum vegas_precision {
  VEGAS_FP64 = 0, /* points, map, integrand, cube and map-weight sums in FP64          */
  VEGAS_FP32 = 1  /* points, map and integrand in FP32; compensated FP32 sums per
                     cube, FP64 across cubes, map refinement and combination in FP64 */
};

/* ---- how the iterations are combined (Sec. 2.1.3) ------------------------ */
enum vegas_weighting {
  VEGAS_WEIGHT_AUTO = 0,             /* handle default: LAGGED with a learned proposal, else INVERSE_VARIANCE */
  VEGAS_WEIGHT_INVERSE_VARIANCE = 1, /* Eqs. (8)-(9): weight 1/sigma_t^2                                      */
  VEGAS_WEIGHT_LAGGED = 2            /* weight 1/sigma_{t-1}^2 (own sigma for t = 0 or sigma_{t-1} = 0);
                                        sigma^2 = sum w_t^2 sigma_t^2 / (sum w_t)^2                            */
};

/* ======================================================================== */
/* Level 1: handle                                                          */
/* ======================================================================== */
typedef struct vegas_s *vegas_handle;

typedef struct {
  double estimate;      /* Eq. (8): weighted mean of the used iterations (vegas_set_weighting) */
  double sigma;         /* Eq. (9), or its form for lagged weights                             */
  double chi2_dof;      /* sum_t (I_t - I)^2 / sigma_t^2 / (n_used - 1); 0 for one iteration */
  int64_t neval_total;  /* evaluations made by this call                                    */
  int32_t nitn_run;     /* iterations run (fewer than asked when the rtol target was met)   */
  int32_t n_used;       /* iterations in the weighted mean (those with index >= skip)       */
  double *it_est;       /* caller-owned host array of it_cap entries, or NULL: I_t          */
  double *it_sigma;     /* caller-owned host array of it_cap entries, or NULL: sigma_t      */
  int32_t it_cap;
  int32_t flags;        /* VEGAS_RESULT_* bits (below)                                      */
  int32_t nitn_judge;   /* iterations of the other form run beside these for the judge of
                           the learned proposal (vegas_set_flow_judge); their evaluations
                           are in neval_total, their estimates are not in the result        */
  int32_t pad;
  double judge_ratio;   /* at the judge's decision: median over its window of
                           sigma_t^2 x iteration time of plain VEGAS+ divided by that of
                           the learned proposal (above 1: the learned proposal reaches a
                           given error sooner); 0 when no decision was made               */
} vegas_result;

/* vegas_result.flags */
#define VEGAS_RESULT_CHI2_HIGH 1 /* chi2/dof above the bound of vegas_set_chi2_bound: the combined
                                    iterations disagree beyond their sigmas (Sec. 2.1.3), so the
                                    estimate and sigma should not be trusted                      */
#define VEGAS_RESULT_FLOW_OFF 2  /* the judge turned the learned proposal off; the result is the
                                    plain VEGAS+ iterations run beside it                        */
#define VEGAS_RESULT_FLOW_KEPT 4 /* the judge compared the two and kept the learned proposal      */
#define VEGAS_RESULT_FP32_FLOOR 8 /* FP32 form: sigma is below 2^-20 |estimate|, the relative rounding
                                     bias the FP32 evaluation can carry (a few FP32 ulps of each value);
                                     the error of the estimate is then max(sigma, 2^-20 |estimate|),
                                     which is also what the rtol stop compares                        */

/* Device memory hooks (not in the paper, which allocates with cudaMalloc).
 * alloc returns `bytes` of device memory of the handle's device, aligned to at
 * least 256 bytes, or NULL when it cannot; the library then returns
 * VEGAS_ENOMEM from the call that asked and keeps its state as before the call.
 * free returns a pointer that alloc gave, with the same byte count.  `stream`
 * is the cudaStream_t (as void*) of the handle or batch: the library frees a
 * buffer only after synchronising that stream, and reads or writes a buffer
 * only on that stream, so a stream-ordered pool (for example a framework's
 * caching allocator) may hand the memory back at once.  ctx is passed
 * through unchanged. */
typedef void *(*vegas_alloc_fn)(void *ctx, size_t bytes, void *stream);
typedef void (*vegas_free_fn)(void *ctx, void *ptr, size_t bytes, void *stream);

/* Create a handle for dimension dim, N_g = nbins intervals per axis, nstrat
 * strata per axis (nstrat <= 0: chosen at each integrate call as the largest s
 * with s^d <= neval/2), map damping alpha >= 0 (Sec. 2.1.1) and stratification
 * damping beta in [0, 1] (Sec. 2.1.2).  The handle binds to the current CUDA
 * device.  It allocates the map buffers there and uploads the uniform map.  The
 * per-cube buffers and scratch are sized on the first integrate call.
 * Errors: EINVAL for an out-of-range argument or NULL out, ENOMEM, ECUDA. */
VEGAS_API int vegas_create(int dim, int nbins, int nstrat, double alpha, double beta, vegas_handle *out);

/* Release the handle and its device buffers (synchronises its stream).
 * NULL is accepted. */
VEGAS_API int vegas_destroy(vegas_handle h);

/* Per-axis strata s_k (dim entries, each >= 1).  This overrides the nstrat
 * given to vegas_create.  Errors: EINVAL. */
VEGAS_API int vegas_set_nstrat_axes(vegas_handle h, const int32_t *nstrat, int dim);
/* Iterations with index < skip are left out of the weighted mean (default 0). */
VEGAS_API int vegas_set_skip(vegas_handle h, int skip);
/* VEGAS_FP64 (default) or VEGAS_FP32. */
VEGAS_API int vegas_set_precision(vegas_handle h, int precision);
/* How vegas_integrate combines the iterations (enum vegas_weighting; default
 * VEGAS_WEIGHT_AUTO).  Not in the paper, which uses Eq. (8) throughout.  Eq. (8)
 * weights iteration t by its own 1/sigma_t^2, which is biased when I_t and
 * sigma_t are correlated: under the learned proposal the weight J f / q is
 * heavy-tailed, an iteration that misses the tail is low in both, and the
 * weighted mean leans low by many sigma over hundreds of iterations.  LAGGED
 * takes the weight from the previous iteration's independent samples, so it
 * does not depend on I_t.  Errors: EINVAL. */
VEGAS_API int vegas_set_weighting(vegas_handle h, int weighting);
/* Run on this cudaStream_t.  NULL restores the handle's own stream. */
VEGAS_API int vegas_set_stream(vegas_handle h, void *stream);
/* Stop an integrate call early once sigma/|estimate| <= rtol (0 disables the
 * check, which is the default).  The check reads the result to the host after
 * every iteration.  In the FP32 form sigma counts as at least 2^-20 |estimate|
 * (VEGAS_RESULT_FP32_FLOOR). */
VEGAS_API int vegas_set_rtol(vegas_handle h, double rtol);
/* Back to the uniform map and uniform allocation; iteration counter to 0. */
VEGAS_API int vegas_reset_map(vegas_handle h);
/* Route every device allocation of the handle through alloc / free (both
 * non-NULL), or back to cudaMalloc / cudaFree (both NULL).  Ownership: the
 * handle still owns its buffers and the adapted map; the hook only supplies
 * and takes back their memory.  The call moves the buffers the handle holds
 * into memory of the new allocator (the map, the stratification, the learned
 * proposal's parameters and Adam state are kept) and gives the old memory back
 * to the allocator that supplied it; set the hook before the first integrate
 * call to avoid copying the per-cube buffers.  Pinned host memory for results
 * stays with the CUDA runtime.  On failure the handle keeps its old allocator
 * and buffers.  Errors: EINVAL (only one of alloc, free given), ENOMEM, ECUDA. */
VEGAS_API int vegas_set_allocator(vegas_handle h, vegas_alloc_fn alloc, vegas_free_fn free, void *ctx);
/* chi2/dof above which vegas_integrate sets VEGAS_RESULT_CHI2_HIGH (Sec. 2.1.3:
 * chi2/dof near 1 means the iterations agree within their sigmas).  bound <= 0
 * (the default) takes the 0.999 quantile of chi2_nu / nu with nu = n_used - 1,
 * by the Wilson-Hilferty cube-root normal approximation:
 * (1 - 2/(9 nu) + 3.0902 sqrt(2/(9 nu)))^3, e.g. 11.1 at nu = 1, 3.1 at nu = 9,
 * 1.4 at nu = 100.  One used iteration never raises the flag.  Errors: EINVAL. */
VEGAS_API int vegas_set_chi2_bound(vegas_handle h, double bound);

/* Run nitn iterations of Algorithm 1 on integrand family `integrand` with the
 * host array params[nparams] (layout in enum vegas_integrand).  Each iteration
 * makes neval evaluations.  The map and the stratification carry over from
 * earlier calls on the same handle.  The stratification is reset to uniform
 * when the number of hypercubes changes.  Evaluation j of iteration t (the
 * handle's iteration counter) draws its point from Philox4x32-10 with key
 * seed and counter (j, t, block), so results do not depend on the launch
 * shape.  The call synchronises the stream and fills *out.
 * Errors: EINVAL (bad integrand id, parameter count, neval < 2 N_h or
 * neval >= 2^31), ENOMEM, ECUDA, ENONFINITE (the result is still filled in). */
VEGAS_API int vegas_integrate(vegas_handle h, int integrand, const double *params, int64_t nparams, int64_t neval,
                    int nitn, uint64_t seed, vegas_result *out);

/* Device time of each iteration (iter_ms) and of its fill kernel (fill_ms) in
 * the last integrate call, from CUDA events on the handle's stream.  At most
 * cap entries are written; *n gets the number of iterations run. */
VEGAS_API int vegas_get_timings(vegas_handle h, float *iter_ms, float *fill_ms, int cap, int *n);

/* Checkpoint: the map edges, the stratification weights of the last
 * iteration, the strata and the iteration counter, in a self-describing blob.
 * vegas_get_state with buf == NULL stores the size in *bytes. */
VEGAS_API int vegas_get_state(vegas_handle h, void *buf, size_t *bytes);
/* Restore a blob made by vegas_get_state on a handle with the same dim and
 * nbins.  Errors: ESTATE for a mismatch. */
VEGAS_API int vegas_set_state(vegas_handle h, const void *buf, size_t bytes);

/* Copy the current map edges [dim][nbins+1] to a host array. */
VEGAS_API int vegas_get_edges(vegas_handle h, double *edges, size_t count);

/* A static string for a status code. */
VEGAS_API const char *vegas_strerror(int status);

/* ======================================================================== */
/* Level 2: step entry points (one row of Algorithm 1 each)                  */
/* ======================================================================== */

/* Geometry shared by the step entry points.  Host struct, host pointer.
 * tile_log2 (vegas_fill only): 0 lets the library cut the evaluations into
 * tiles of 2048, or of 1024 where the larger tile would cost a resident CTA;
 * 10 or 11 fixes tiles of 2^tile_log2 evaluations (other values: EINVAL).  The
 * FP32 form folds its fixed-point map weights to FP32 once per tile, so its
 * map weights depend on the tiles at the level of FP32 rounding; fixing the
 * tile reproduces them bit for bit, for instance those of a batched run
 * (VEGAS_BATCH_INFO reports its tile). */
typedef struct {
  int32_t dim;           /* d                                    */
  int32_t nbins;         /* N_g                                  */
  const int32_t *nstrat; /* host array of d strata s_k           */
  int32_t tile_log2;     /* 0, 10 or 11 (see above)              */
  int32_t pad;
} vegas_geometry;

/* -- updateEvalsPerCube + mapEvalsToCubes (Algorithm 1; Sec. 2.1.2, Eq. (7)) --
 * From the per-cube weights d_ell[ncubes] (float, ell_h = (beta/2) log2 of the
 * cube's sample variance of J f, -inf for zero variance, as written by
 * vegas_fill), write d_offsets[ncubes+1] (int64): off_0 = 0, off_N = neval,
 * and n_h = off_{h+1} - off_h = 2 + a share of neval - 2 N_h proportional to
 * q_h = rint(2^24 2^(ell_h - max ell)).  The shares use cumulative rounding,
 * off_h = 2h + floor(R Q_h / Q), so sum n_h = neval exactly and every decision
 * is integer.  uniform != 0 (first iteration, beta = 0) ignores d_ell, which may
 * be NULL; so does the case where every ell is -inf.  d_scratch holds
 * vegas_allocate_scratch_bytes(ncubes) bytes.
 * Errors: EINVAL (neval < 2 ncubes, neval >= 2^31, ncubes >= 2^31), ENOSPACE. */
VEGAS_API size_t vegas_allocate_scratch_bytes(int64_t ncubes);
VEGAS_API int vegas_allocate(const float *d_ell, int64_t ncubes, int64_t neval, int uniform, int64_t *d_offsets,
                   void *d_scratch, size_t scratch_bytes, void *stream);

/* -- vegas_allocate_static: the allocation step without any allocation ----
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory.  Examples are code whose device memory is
 * owned by another allocator (a framework's caching pool that has reserved the
 * free memory, or a process held to a fixed budget), and latency-critical
 * loops, where cudaMalloc or cudaFree would synchronise the device or fail.
 * It computes exactly what vegas_allocate computes, with the same arguments
 * except the scratch area.  Its scratch is a fixed array of about 0.5 MiB in
 * device global memory, declared in the library.  Every GPU that loads the
 * library holds that array until the process exits.
 *   - Limit: ncubes <= VEGAS_ALLOCATE_STATIC_MAX_CUBES; larger sizes return
 *     VEGAS_ENOSPACE before anything runs.
 *   - Set-up: each call made outside stream capture looks up the array's
 *     device address with the device current (after cudaDeviceReset the next
 *     such call finds the new context's array).  A call on a capturing stream
 *     uses the address that the last call outside capture found, so make the
 *     first call on a device before any stream capture on it.
 *   - Sharing: every call on a device shares the one array, which keeps the
 *     contents of the last call.  Each call re-initialises what it reads, so
 *     sequential calls are independent.  Calls that overlap on the GPU
 *     (different streams, or host threads without ordering) race on the
 *     array and give wrong offsets.
 *   - Allocation: the entry point calls no cudaMalloc, cudaFree or other
 *     allocating routine.
 * Errors: EINVAL as vegas_allocate, ENOSPACE above the limit, ECUDA. */
#define VEGAS_ALLOCATE_STATIC_MAX_CUBES (1LL << 28)
VEGAS_API int vegas_allocate_static(const float *d_ell, int64_t ncubes, int64_t neval, int uniform,
                                    int64_t *d_offsets, void *stream);

/* -- vegasFill (Algorithm 2; Eqs. (3)-(6)) ----------------------------------
 * Evaluate the integrand at the neval points of iteration `iteration`.
 * Evaluation j lies in the cube h with off_h <= j < off_{h+1}.  Its point comes
 * from Philox4x32-10 (key seed, counter (j, iteration, problem_id<<16 | block))
 * and goes through the map d_edges[d][N_g+1] (FP64).  The outputs are:
 *   d_ell[ncubes]     per-cube allocation weight for vegas_allocate (beta used);
 *   d_bins[d*N_g]     map weights sum over the cube's evaluations of (J f)^2 / n_h
 *                     (FP64, overwritten);
 *   d_result[2]       (I_t, sigma_t^2) of this iteration, Eqs. (5)-(6), FP64;
 *   d_cube_mean, d_cube_m2 [ncubes]  per-cube mean and centred second moment
 *                     of J f (FP64), or NULL to skip them;
 *   d_flags           device int; bit 0 is set when an integrand value was not
 *                     finite (never cleared by the library).
 * d_params[nparams] is a device copy of the integrand parameters.
 * precision is VEGAS_FP64 or VEGAS_FP32.
 * d_scratch holds vegas_fill_scratch_bytes(geometry, neval) bytes.
 * Errors: EINVAL, ENOSPACE, ECUDA. */
VEGAS_API size_t vegas_fill_scratch_bytes(const vegas_geometry *g, int64_t neval);
VEGAS_API int vegas_fill(const vegas_geometry *g, int precision, int integrand, const double *d_params, int64_t nparams,
               int64_t neval, uint64_t seed, int32_t iteration, uint32_t problem_id, double beta,
               const double *d_edges, const int64_t *d_offsets, float *d_ell, double *d_bins, double *d_result,
               double *d_cube_mean, double *d_cube_m2, int *d_flags, void *d_scratch, size_t scratch_bytes,
               void *stream);

/* -- adjustWeights + updateMap (Algorithm 1; Sec. 2.1.1) ---------------------
 * Per axis: smooth the map weights d_bins[d][N_g] with neighbours (weights
 * (7,1)/8 at the ends, (1,6,1)/8 inside), normalise to r_i, damp to
 * m_i = ((1 - r_i)/ln(1/r_i))^alpha, and place the N_g - 1 inner edges so that
 * each new interval holds 1/N_g of sum m.  The weight is uniform inside each
 * old interval.  Writes d_edges_out[d][N_g+1].  An axis whose weights are all
 * zero or not finite, or alpha == 0, keeps its edges.  d_edges_in and
 * d_edges_out must not overlap.  Errors: EINVAL, ECUDA. */
VEGAS_API int vegas_refine(int32_t dim, int32_t nbins, double alpha, const double *d_bins, const double *d_edges_in,
                 double *d_edges_out, void *stream);

/* -- combineIterationsResults (Algorithm 1; Sec. 2.1.3, Eqs. (8)-(9)) -------
 * From d_it_est[n] and d_it_sigma[n] (device), combine the iterations
 * t >= skip.  Writes d_out[4] = {estimate, sigma, chi2/dof, n_used}.
 * Iterations with sigma_t = 0 give their mean exactly with sigma 0.
 * Errors: EINVAL, ECUDA. */
VEGAS_API int vegas_combine(const double *d_it_est, const double *d_it_sigma, int32_t n, int32_t skip, double *d_out,
                  void *stream);
/* vegas_combine with a choice of weights: VEGAS_WEIGHT_INVERSE_VARIANCE is
 * Eqs. (8)-(9), VEGAS_WEIGHT_LAGGED weights iteration t by 1/sigma_{t-1}^2 (see
 * enum vegas_weighting; not in the paper).  The chi2/dof is the same for both.
 * Same buffers and layout as vegas_combine.  Errors: EINVAL (also for
 * VEGAS_WEIGHT_AUTO), ECUDA. */
VEGAS_API int vegas_combine_weighted(const double *d_it_est, const double *d_it_sigma, int32_t n, int32_t skip,
                           int32_t weighting, double *d_out, void *stream);

/* ======================================================================== */
/* Level 3: a batch of independent integrals                                */
/* ======================================================================== */
/* The paper runs one integral per launch (Algorithm 1).  A batch runs the same
 * iteration for many independent integrals at once: each step of Algorithm 1
 * is one launch over the work of every integral still running, the fill is
 * one persistent launch over all their evaluation tiles (Algorithm 2 per
 * integral), and one iteration of the whole batch is replayed as a captured
 * CUDA graph.  Every integral keeps its own map (N_g intervals per axis, the
 * same N_g for the batch), its own strata and counts (Sec. 2.1.2) and its own
 * combination of iterations (Eqs. (8)-(9)).  Evaluation is FP32 (the
 * VEGAS_FP32 form); sums across cubes and everything after the fill are FP64.
 * Integral p draws its points with problem_id = p in the Philox counter, from
 * the batch's one seed, so its evaluations equal those of vegas_fill with
 * problem_id = p on the same map and counts.  Sums over CTAs are taken with
 * atomic adds, so results are reproducible to FP64 rounding, not bit for bit.
 * Limits: 1 <= nproblems <= 4096; per integral 1 <= dim <= 16 and the
 * families GAUSS_SUM, PRODUCT_PEAK, OSCILLATORY; 2 <= nbins <= 256; an
 * integral with more than 8 axes has at most 256 strata per axis and, for
 * GAUSS_SUM, at most 8 peaks. */
typedef struct vegas_batch_s *vegas_batch;

typedef struct {
  int32_t dim;           /* d of this integral, 1..16                                  */
  int32_t integrand;     /* VEGAS_GAUSS_SUM, VEGAS_PRODUCT_PEAK or VEGAS_OSCILLATORY   */
  const double *params;  /* host array, layout of the family (copied at create)         */
  int64_t nparams;
  int64_t neval;         /* evaluations per iteration, 2 N_h <= neval < 2^31            */
  int32_t nstrat;        /* strata per axis (<= 65536); <= 0: the largest s with
                            s^d <= neval/2                                              */
  int32_t pad;
} vegas_problem;

typedef struct {
  double estimate, sigma, chi2_dof; /* Eqs. (8)-(9) over the recorded iterations >= skip  */
  int32_t n_used;                   /* iterations in the weighted mean                    */
  int32_t nitn_run;                 /* iterations recorded since create or reset          */
  int32_t converged;                /* 1: sigma <= rtol |estimate| was reached            */
  int32_t status;                   /* VEGAS_OK, VEGAS_ENONFINITE, or VEGAS_ECUDA when a
                                       cube split across tiles was not reassembled        */
  int32_t flags;                    /* VEGAS_RESULT_CHI2_HIGH when chi2/dof is above the
                                       bound of vegas_batch_set_chi2_bound;
                                       VEGAS_RESULT_FP32_FLOOR when sigma is below the FP32
                                       evaluation's rounding floor (the batch's rtol test
                                       uses the floor too)                                */
  int32_t pad;
} vegas_problem_result;

/* Create a batch of nproblems integrals on the current CUDA device, with
 * N_g = nbins, map damping alpha >= 0, stratification damping beta in [0,1]
 * and one Philox seed.  Copies the parameters, sizes and allocates every
 * device buffer (per integral: map, counts, allocation weights, tile records)
 * and uploads uniform maps.  Errors: EINVAL (an argument or a problem out of
 * range; nothing is allocated), ENOMEM, ECUDA. */
VEGAS_API int vegas_batch_create(const vegas_problem *problems, int32_t nproblems, int32_t nbins, double alpha,
                                 double beta, uint64_t seed, vegas_batch *out);
/* vegas_batch_create with device memory from alloc / free (both non-NULL;
 * both NULL is vegas_batch_create).  Every device buffer of the batch (one
 * arena for all integrals and the iteration records, which grow with the
 * iterations run) comes from alloc and goes back through free when the batch
 * no longer needs it, under the rules given at vegas_alloc_fn.  The batch owns
 * the buffers until then.  A NULL from alloc at create returns ENOMEM with
 * nothing leaked; at vegas_batch_integrate it returns ENOMEM with the batch
 * unchanged.  Pinned host memory for results stays with the CUDA runtime.
 * Errors: as vegas_batch_create, and EINVAL when only one hook is given. */
VEGAS_API int vegas_batch_create_ex(const vegas_problem *problems, int32_t nproblems, int32_t nbins, double alpha,
                                    double beta, uint64_t seed, vegas_alloc_fn alloc, vegas_free_fn free, void *ctx,
                                    vegas_batch *out);
VEGAS_API int vegas_batch_destroy(vegas_batch b);
/* chi2/dof above which a result gets VEGAS_RESULT_CHI2_HIGH; bound <= 0 (the
 * default) is the 0.999 quantile rule of vegas_set_chi2_bound.  Errors: EINVAL. */
VEGAS_API int vegas_batch_set_chi2_bound(vegas_batch b, double bound);
/* Stream of later calls (NULL: the legacy default stream).  The graph is
 * captured on a stream of the batch's own and launched on this one. */
VEGAS_API int vegas_batch_set_stream(vegas_batch b, void *stream);
/* Iterations with index < skip stay out of the combination (default 0). */
VEGAS_API int vegas_batch_set_skip(vegas_batch b, int32_t skip);
/* Launch shape of the fill: variant 0 (the larger resident-CTA count per
 * width: 4, 3 or 2 CTAs of 256 threads for 4, 8 or 16 axes) or 1 (half of
 * that, twice the registers), ctas_per_sm (<= 0: as many as fit) and
 * chunk_tiles, the consecutive tiles a CTA takes from the work counter at a
 * time.  Errors: EINVAL. */
VEGAS_API int vegas_batch_set_launch(vegas_batch b, int32_t variant, int32_t ctas_per_sm, int32_t chunk_tiles);
/* Tiles of 2^tile_log2 evaluations (10 or 11) for every integral of the
 * batch: the shared-memory layout of the fill changes with the tile.  A batch
 * starts at 11 where its layout fits, else 10; VEGAS_BATCH_INFO reports it.
 * The FP32 map weights depend on the tiles at the level of FP32 rounding (see
 * vegas_geometry).  Errors: EINVAL (another value, or a layout that does not
 * fit), ECUDA. */
VEGAS_API int vegas_batch_set_tile(vegas_batch b, int32_t tile_log2);
/* Time one iteration of the batch under each candidate launch shape (each tile
 * size whose layout fits, both variants, every resident-CTA count, chunk_tiles
 * in {1, 4, 16}), keep the fastest, and reset the batch (vegas_batch_reset).
 * The chosen shape and its iteration time go to the non-NULL outputs (the tile
 * through VEGAS_BATCH_INFO).  Errors: ECUDA. */
VEGAS_API int vegas_batch_tune(vegas_batch b, int32_t *variant, int32_t *ctas_per_sm, int32_t *chunk_tiles,
                               float *ms);
/* Uniform maps, uniform counts, no recorded iterations, iteration counter 0. */
VEGAS_API int vegas_batch_reset(vegas_batch b);
/* Run up to nitn iterations.  Every integral without an error takes part
 * until its combined sigma <= rtol |estimate| (rtol > 0, checked after each
 * iteration with index >= skip); the call returns early when none is left.
 * results[nproblems] (host, may be NULL) receives each integral's combination
 * over all its recorded iterations; nitn_run the iterations run by this call;
 * ms the wall time of those iterations on the device (CUDA events).
 * Errors: EINVAL, ENOMEM, ECUDA. */
VEGAS_API int vegas_batch_integrate(vegas_batch b, int32_t nitn, double rtol, vegas_problem_result *results,
                                    int32_t *nitn_run, float *ms);
/* Copy one integral's state to the host.  what selects the array and count
 * is the capacity of host_out in elements:
 *   VEGAS_BATCH_EDGES    double [d][N_g+1]  the current map
 *   VEGAS_BATCH_OFFSETS  int64  [N_h+1]     offsets of the last allocation
 *   VEGAS_BATCH_ELL      float  [N_h]       allocation weights of the last fill
 *   VEGAS_BATCH_BINS     double [d][N_g]    map weights of the last fill
 *   VEGAS_BATCH_ITER_EST double [nitn_run]  I_t of every recorded iteration
 *   VEGAS_BATCH_ITER_SIG double [nitn_run]  sigma_t
 *   VEGAS_BATCH_INFO     int64  [4 or 5]    d, strata per axis, N_h, nitn_run, and with count >= 5
 *                                           log2 of the fill's tile (evaluations)
 * Errors: EINVAL (unknown what, problem out of range), ENOSPACE (count too
 * small), ECUDA. */
enum vegas_batch_field {
  VEGAS_BATCH_EDGES = 0,
  VEGAS_BATCH_OFFSETS = 1,
  VEGAS_BATCH_ELL = 2,
  VEGAS_BATCH_BINS = 3,
  VEGAS_BATCH_ITER_EST = 4,
  VEGAS_BATCH_ITER_SIG = 5,
  VEGAS_BATCH_INFO = 6
};
VEGAS_API int vegas_batch_get(vegas_batch b, int32_t problem, int32_t what, void *host_out, int64_t count);

/* ======================================================================== */
/* Level 4: the learned proposal (a coupling flow after the VEGAS map)      */
/* ======================================================================== */
/* The paper has no learned component.  The VEGAS+ map (Sec. 2.1.1) samples
 * x' = M(y); a flow F maps x' to the point x = F(x') where the integrand is
 * evaluated, and VEGAS+ integrates g(x') = f(F(x')) |det dF/dx'|, whose
 * integral over the unit cube is that of f.  F is 6 affine coupling layers
 * (RealNVP) between a logit (clamped to [-20, 20]) and a sigmoid; layer l
 * conditions on the axes k = l (mod 2) through an MLP a_l -> 64 -> 64 -> 2 b_l
 * with ReLU, whose outputs 2j and 2j+1 give s_j = 2 tanh(o_2j / 2) and t_j.
 * The normalising direction N = F^-1 moves z_B to z_B e^s + t; the sampling
 * direction F moves it to (z_B - t) e^-s.  The MLPs run on the tensor cores
 * with bf16 weights and activations and FP32 accumulation; the log-
 * determinant is that of the map actually applied, so g stays unbiased.
 *
 * Parameters: one FP32 vector of vegas_flow_param_count(dim) values; per layer
 * l = 0..5 in order W1 [64][a_l], b1 [64], W2 [64][64], b2 [64],
 * W3 [2 b_l][64], b3 [2 b_l], row-major, with a_l = ceil(d/2) for even l and
 * floor(d/2) for odd l, b_l = d - a_l.  2 <= dim <= 32. */
enum vegas_flow_direction {
  VEGAS_FLOW_NORMALISE = 0, /* x -> x' = F^-1(x), log|det dF^-1/dx|  */
  VEGAS_FLOW_SAMPLE = 1     /* x' -> x = F(x'),   log|det dF/dx'|   */
};
/* Number of parameters of the flow for dim, or 0 when dim is out of range. */
VEGAS_API int64_t vegas_flow_param_count(int32_t dim);
/* Apply the flow to n points d_x_in [n][dim] (device, FP32, in [0,1]) in the
 * given direction: d_x_out [n][dim] and d_logdet [n] (device).  d_x_out may
 * equal d_x_in.  Asynchronous on stream.  The GEMMs run as tcgen05 MMAs
 * (bf16 operands, FP32 accumulators in tensor memory); the biases enter the
 * accumulation in FP32.  Errors: EINVAL, ECUDA. */
VEGAS_API int vegas_flow_apply(int32_t dim, int32_t direction, const float *d_params, const float *d_x_in,
                               float *d_x_out, float *d_logdet, int64_t n, void *stream);
/* Synchronise stream and report whether a bounded device wait of an earlier
 * vegas_flow_apply ran out (VEGAS_ETIMEOUT; the points of the affected tiles
 * are then not written) or not (VEGAS_OK); clears the report.
 * Errors: ECUDA. */
VEGAS_API int vegas_flow_check(void *stream);
/* Self-test of that bounded wait, as the transform uses it: one CTA waits
 * `polls` polls (1 <= polls <= 2^24) on an mbarrier.  arrive = 0: nothing
 * arrives, the wait runs out and the call returns VEGAS_ETIMEOUT (the report
 * is cleared); arrive != 0: a thread arrives first, the call returns VEGAS_OK.
 * Synchronises stream.  Nothing faults or hangs either way.
 * Errors: EINVAL, ECUDA. */
VEGAS_API int vegas_flow_wait_selftest(int32_t polls, int32_t arrive, void *stream);
/* Training loss and gradient.  For samples d_x [n][dim] with weights
 * d_w [n] >= 0 of positive sum (|f| over the density that drew them, e.g.
 * |J f| of a VEGAS+ iteration), loss = - sum_i w_i log|det dF^-1/dx(x_i)| /
 * sum_i w_i, the weighted negative log-likelihood of the flow's density with
 * a uniform base (its minimiser makes that density proportional to |f|).
 * Writes d_grad [param_count] and, if not NULL, d_loss [1] (device).
 * Weights that are negative or not finite count as 0; with no positive weight
 * the gradient is 0 and the loss 0.
 * d_scratch holds vegas_flow_grad_scratch_bytes(dim, n) bytes.  The partial
 * gradients of blocks of 32 samples are summed in a fixed order.
 * Errors: EINVAL, ENOSPACE, ECUDA. */
VEGAS_API size_t vegas_flow_grad_scratch_bytes(int32_t dim, int64_t n);
VEGAS_API int vegas_flow_grad(int32_t dim, const float *d_params, const float *d_x, const float *d_w, int64_t n,
                              float *d_grad, float *d_loss, void *d_scratch, size_t scratch_bytes, void *stream);
/* One Adam step (Kingma and Ba) on d_params with d_grad, moments d_m, d_v
 * (device, zero before step 1), step counting from 1.  Errors: EINVAL, ECUDA. */
VEGAS_API int vegas_flow_adam(int64_t nparams, float *d_params, const float *d_grad, float *d_m, float *d_v,
                              int32_t step, float lr, float beta1, float beta2, float eps, void *stream);

/* The learned proposal on a handle.  vegas_set_flow with parameters (host,
 * vegas_flow_param_count(dim) values) turns it on: every later iteration of
 * vegas_integrate draws the VEGAS+ points x', maps them to x = F(x'),
 * evaluates f there and integrates g(x') = f(F(x')) |det dF/dx'| (FP32 form
 * only; 2 <= dim <= 32).  NULL turns it off.  The Adam moments start at zero.
 * vegas_set_flow_training: during the next `iterations` iterations, after each
 * one, run steps_per_iteration Adam steps (learning rate lr) on minibatches of
 * `batch` consecutive rows of a sample of that iteration: every k-th
 * evaluation, k = neval / samples, weighted by (|J f| / n_h)^p, with |J f| /
 * n_h its share of the estimate and p ramping linearly from temper (0 < temper
 * <= 1; below 1 the first targets are broader than |f|) to 1 over the
 * training iterations.  floor >= 0 mixes uniform points into the training
 * set, one row in four, each weighted floor * 3 * the mean sample weight: the
 * loss gains floor times the cross-entropy of the uniform density, whose
 * minimiser is the density (target + floor * its mean) / (1 + floor).  Its
 * log barrier keeps the flow's density off zero on every region of the cube,
 * including regions that the flow's own samples no longer reach.  0 turns it
 * off (the training set is the samples alone).  vegas_get_flow copies the current
 * parameters (nparams = the count, or params NULL) and the last training loss.
 * The checkpoint of vegas_get_state does not include the flow.  With a flow
 * on, the default weighting (VEGAS_WEIGHT_AUTO, vegas_set_weighting) combines
 * the iterations with lagged weights.
 * Errors: EINVAL, ENOMEM, ECUDA. */
VEGAS_API int vegas_set_flow(vegas_handle h, const float *params, int64_t nparams);
VEGAS_API int vegas_set_flow_training(vegas_handle h, int32_t iterations, int32_t steps_per_iteration,
                                      int32_t samples, int32_t batch, float lr, float temper, float floor);
VEGAS_API int vegas_get_flow(vegas_handle h, float *params, int64_t nparams, float *last_loss);
/* Exploration for the learned proposal (not in the paper).  A VEGAS+ map
 * (Sec. 2.1.1) adapted from the uniform map follows the peaks its first
 * samples favour; maps adapted with other seeds favour others.
 * vegas_flow_explore adapts nmaps maps (1..64) on the handle, map k by
 * `iterations` plain VEGAS+ iterations of `neval` evaluations from the
 * uniform map with seed + k (the handle's strata and FP32 form; the flow is
 * set aside meanwhile), pools samples_per_map samples of each into one
 * training set and trains the handle's flow on it: `steps` Adam steps
 * (learning rate lr) on windows of `batch` consecutive rows, with the floor's
 * uniform rows as in vegas_set_flow_training.  Sample r comes from map
 * r mod nmaps; its weight is |f(x)| / q(x) with q = (1/nmaps) sum_k q_k the
 * mixture of the maps' densities q_k = prod_a 1 / (N_g dx_a) (the balance
 * heuristic, Veach and Guibas 1995), so every peak that some map reaches
 * carries its own mass however many maps reach it.  Each of rounds - 1
 * further rounds (rounds 1..16) replaces the pool by nmaps * samples_per_map
 * samples of the flow itself, x = F(u) with u uniform, weighted
 * |f(x)| |det dF/du|, and runs `steps` more Adam steps from fresh moments:
 * the flow then covers every peak, so its own samples weigh them more evenly
 * than the maps' did.  The handle's map is the
 * uniform map again on return, its flow trained, its in-loop training
 * schedule unchanged.  Requires a flow (vegas_set_flow) and the FP32 form;
 * integrand and params as for vegas_integrate (not MAP_DENSITY).  Returns
 * after the device work is done.  Errors: EINVAL (no flow, FP64, arguments),
 * ENOMEM, ECUDA, ETIMEOUT (a bounded wait of the flow's kernels), and those of
 * vegas_integrate.
 *
 * vegas_explore_points is its sampling step: nmaps maps d_maps (device, FP64,
 * [nmaps][dim][nbins + 1], each axis's edges increasing from 0 to 1), and
 * m = nmaps * samples_per_map samples: sample r from map r mod nmaps, with
 * uniform numbers from Philox4x32-10, counter (r low, r high, 4 g, "EXPR"
 * = 0x45585052) for axes 4g..4g+3, key (seed low, seed high), y = (u + 1/2)
 * 2^-32, z = y nbins, i = min(floor z, nbins - 1), x = e_i + (z - i)(e_{i+1}
 * - e_i) in FP64.  Writes d_x [m][dim] (x rounded to FP32) and d_q [m] (FP64,
 * the mixture density at the FP64 x; the interval of x_a in a map is the j
 * with e_j <= x_a < e_{j+1}, clamped to [0, nbins - 1]).  Caller-owned device
 * buffers; asynchronous on stream.  Errors: EINVAL, ECUDA. */
VEGAS_API int vegas_flow_explore(vegas_handle h, int32_t integrand, const double *params, int64_t nparams,
                                 int64_t neval, int32_t iterations, int32_t nmaps, int64_t samples_per_map,
                                 int32_t steps, int32_t batch, float lr, float floor, int32_t rounds,
                                 uint64_t seed);
VEGAS_API int vegas_explore_points(int32_t dim, int32_t nbins, int32_t nmaps, const double *d_maps,
                                   int64_t samples_per_map, uint64_t seed, float *d_x, double *d_q, void *stream);
/* Plain VEGAS+ as the fallback and the judge of the learned proposal (not in
 * the paper, which has no learned component; the yardstick is its estimator,
 * Eq. (6) of Sec. 2.1.2).  window > 0 turns the judge on; it applies from the
 * next vegas_integrate call with a flow set and carries over between calls.
 * Beside every iteration of the learned proposal the handle then runs one
 * plain VEGAS+ iteration (FP32 form) with its own map and stratification,
 * drawing with Philox problem id 1 so that its points are independent of the
 * learned proposal's.  After the flow's training iterations, the handle records
 * for each form sigma_t^2 times the iteration's device time (CUDA events; no
 * training step runs in these iterations): the product is the variance of the
 * estimate per unit of device time, lower for the form that reaches a given
 * error sooner.  Once `window` such pairs exist, and at least 5 + window pairs
 * in all (so that the plain map has adapted), the form with the lower median
 * product over the last `window` pairs is kept: if plain VEGAS+ wins (a tie or
 * NaN counts for it), the learned proposal stops, the handle continues with
 * the plain form's map, stratification and iterations, and the result combines
 * the plain iterations (VEGAS_RESULT_FLOW_OFF); otherwise the plain form stops
 * and the result is the learned proposal's (VEGAS_RESULT_FLOW_KEPT).  Before
 * the decision, an rtol target (vegas_set_rtol) that either form reaches ends
 * the call with that form's result and decides the same way.  vegas_set_flow,
 * vegas_reset_map and vegas_set_state start the judge over.  window = 0 (the
 * default) turns it off.  Errors: EINVAL (window < 0 or > 1024). */
VEGAS_API int vegas_set_flow_judge(vegas_handle h, int32_t window);

/* ======================================================================== */
/* Measurement support                                                      */
/* ======================================================================== */
/* Measure issue rates of the arithmetic pipes on the current device with
 * dependent-chain microkernels (FP32 FMA, FP64 FMA, MUFU ex2, integer
 * multiply-high).  rates[4] receives operations per SM per clock, measured
 * with the device clock counter.  Used to state the roofline of the fill
 * kernel.  Errors: ECUDA. */
VEGAS_API int vegas_probe_pipes(double rates[4]);
/* Measured rate of 32-bit integer atomic adds to shared memory with every lane
 * of a warp on its own bank: lane operations per SM per clock on the current
 * device.  It is the denominator of the accumulation's roofline; the paper
 * accumulates with global atomicAdd instead (Sec. 3.3.3), this library with
 * the fixed-point shared histogram of the fill.  Same method as
 * vegas_probe_pipes (four blocks per SM, median block, SM cycle counter).
 * Errors: EINVAL, ENOMEM, ECUDA. */
VEGAS_API int vegas_probe_shared_atomics(double *rate);
/* Measured throughput of the FP64 exponential that the FP64 form's Gaussian
 * integrand evaluates once per peak and evaluation (2^(y/64) from a table of
 * 64 entries, after Tang 1989, on an argument already scaled to units of
 * ln2/64) (Table 3's Gaussian and Ridge;
 * the ridge workloads): calls per SM per clock on the current device, same
 * method as vegas_probe_pipes.  With the FP64 FMA rate it states the FP64 fill's
 * roofline: the time the FP64 pipe needs for the evaluation's FP64 operations
 * and exponentials against the kernel's measured time.  Errors: ENOMEM, ECUDA. */
VEGAS_API int vegas_probe_exp64(double *rate);
/* n arguments d_x (device, FP64) into d_y: which = 0 e^x by the table-driven
 * exponential, which = 1 e^x by the CUDA library's exp(), which = 2 2^(x/64) by
 * the table-driven exponential that the FP64 Gaussian sum evaluates; for tests
 * against the library and against correctly rounded values.
 * Asynchronous on stream.  Errors: EINVAL, ECUDA. */
VEGAS_API int vegas_exp64_eval(const double *d_x, double *d_y, int64_t n, int32_t which, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* VEGAS_GB300_H */
