/*
 * oracle_vegas.h -- plain, slow, single-threaded FP64 CPU oracle of the VEGAS+
 * iteration loop of cuVegas (Tolotti et al., arXiv 2408.09229).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link,
 * load or execute this code: only tests/, __graft_entry__.smoke() and the
 * CPU-baseline / reference leg of bench.py use it.  It shares no code, header,
 * table or constant generator with the CUDA library; the two are written
 * separately from the paper and from the same readings of it (numbered below).
 *
 * Every routine states the passage of the paper it follows:
 *   Sec. 2.1.1  adaptive importance sampling, Eqs. (2)-(4): the separable map,
 *               J(y) = N_g * dx_{i(y)}, I_MC = (1/N_ev) sum J f.
 *   Sec. 2.1.2  adaptive stratified sampling, Eqs. (5)-(7): I = sum dI_h,
 *               sigma^2 = sum sigma_h^2 / n_h, n_h ~ sigma_h (damped by beta),
 *               sum n_h = N_eval.
 *   Sec. 2.1.3  estimation aggregation, Eqs. (8)-(9): inverse-variance average.
 *   Algorithm 1 the iteration loop (reset, map evaluations to cubes, fill,
 *               update evals per cube, adjust weights, update map, results).
 *   Algorithm 2 vegasFill: per evaluation, cube -> point -> Jacobian ->
 *               integrand -> map weights and cube weights.
 *   Table 3     the paper's test integrands.
 * Where the paper is silent the oracle takes numbered readings (R1..R20, the
 * same list the kernels follow); each use below states its reading.
 *
 * Parity pins: every function here is pinned by tests/test_oracle_*.py against
 * closed forms, brute force, invariants or published known-answer values; see
 * the header comment of each test file.  No function is "parity unpinned".
 */
#ifndef ORACLE_VEGAS_H
#define ORACLE_VEGAS_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* integrand families (same numbering as the library's public enum; the value
 * list is an interface, not shared code) */
enum {
  ORC_GAUSS_SUM = 0,          /* A * sum_k exp(-|x-mu_k|^2 / (2 s^2)); p = [A, s, K, mu(K*d)] */
  ORC_PRODUCT_PEAK = 1,       /* prod_i 1/(c_i^-2 + (x_i-w_i)^2);      p = [c(d), w(d)]      */
  ORC_OSCILLATORY = 2,        /* cos(2 pi u + sum a_i x_i);            p = [u, a(d)]         */
  ORC_SIN_EXP = 3,            /* Table 3 (1): sin x1 + exp x2, d = 2                          */
  ORC_LINEAR = 4,             /* Table 3 (2): sum x_i                                         */
  ORC_COSINE = 5,             /* Table 3 (3): prod cos x_i                                    */
  ORC_EXPONENTIAL = 6,        /* Table 3 (4): exp(sum x_i^2)                                  */
  ORC_ROOS_ARNOLD = 7,        /* Table 3 (5): prod |4 x_i - 2|                                */
  ORC_MOROKOFF_CAFLISCH = 8,  /* Table 3 (6): (1+1/d)^d prod x_i^(1/d)                        */
  ORC_MAP_DENSITY = 9,        /* test integrand: density of a fixed separable map; p = edges  */
  ORC_N_INTEGRANDS = 10
};

/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11).
 * Reading R1: the paper draws with cuRAND XORWOW states (Sec. 3.3.2); a
 * counter-based generator makes every point independent of the launch shape. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* f(x) for one point, FP64.  Returns 0, or -1 for a bad id / parameter count. */
int orc_integrand(int id, int dim, const double *params, int64_t nparams,
                  const double *x, double *f);

/* Reproducible FP32 log2 / exp2 used by the allocation weights (reading R4). */
float orc_log2r(double x);
float orc_exp2r(float y);
/* ell_h = (beta/2) log2(var_h), var_h = M2_h / (n_h - 1) (reading R4, Sec. 2.1.2) */
float orc_cube_ell(double m2, int64_t n, double beta);
/* quantised allocation weight q_h = rint(2^24 * 2^(ell_h - ell_max)) */
uint32_t orc_quant_weight(float ell, float ell_max);

/* Sec. 2.1.2 + reading R5: sample offsets off_h (ncubes+1 entries, off_0 = 0,
 * off_ncubes = neval) of n_h = off_{h+1} - off_h.  ell == NULL or beta == 0
 * gives the uniform first-iteration allocation.  Returns 0 or -1 (EINVAL). */
int orc_allocate(const float *ell, int64_t ncubes, int64_t neval, double beta, int64_t *offsets);

/* Sec. 2.1.1 map refinement with damping alpha, readings R6-R8, one axis.
 * w[nbins] accumulated weights, e_in/e_out[nbins+1] edges.  Returns 1 when
 * the axis was left unchanged (zero or non-finite weights, alpha == 0). */
int orc_refine_axis(int nbins, double alpha, const double *w, const double *e_in, double *e_out);

/* Sec. 2.1.3 Eqs. (8)-(9), reading R9: out = {estimate, sigma, chi2/dof, n_used} */
void orc_combine(const double *it_est, const double *it_sig, int n, int skip, double out[4]);

/* Lagged weights, reading R20 (not in the paper): iteration t is weighted by
 * 1/sigma_{t-1}^2 (its own sigma_t for t = 0 or sigma_{t-1} = 0); estimate
 * sum w_t I_t / sum w_t, sigma sqrt(sum w_t^2 sigma_t^2) / sum w_t, chi2/dof
 * and the sigma_t = 0 rule as in orc_combine. */
void orc_combine_lagged(const double *it_est, const double *it_sig, int n, int skip, double out[4]);

/* configuration of one integral */
typedef struct {
  int dim;              /* d */
  int nbins;            /* N_g */
  const int *nstrat;    /* s_k, k < d; number of cubes N_h = prod s_k */
  double alpha, beta;
  int points_f32;       /* 0: 53-bit coordinates and FP64 z; 1: FP32 z from 23-bit exact c + u (R3);
                           FP32 mode needs nstrat <= 2^16 */
  uint32_t problem_id;  /* enters the Philox counter (R2) */
} orc_config;

int64_t orc_ncubes(const orc_config *cfg);
/* largest s with s^d <= neval/2, at least 1 (reading R10) */
int orc_default_nstrat(int64_t neval, int dim);

/* Algorithm 2 over samples j in [j_begin, j_end) of iteration t: per-cube
 * partial statistics over the samples of the range (cnt, mean, m2: two-pass),
 * and map weights bins[k*nbins+i] += (J f)^2 / n_h (reading R11).  bins must
 * be zeroed by the caller; cnt/mean/m2 are overwritten.  Returns 0, or -2 if
 * an integrand value was not finite. */
int orc_fill_range(const orc_config *cfg, int integrand, const double *params, int64_t nparams,
                   int64_t neval, int t, uint64_t seed, const double *edges, const int64_t *offsets,
                   int64_t j_begin, int64_t j_end, int64_t *cnt, double *mean, double *m2, double *bins);

/* Algorithm 2 restricted to the evaluations of one cube h, whose evaluations
 * are [off_h, off_h + n_h): mean and centred second moment of J f (two-pass),
 * for spot checks of a full-size run one cube at a time. */
int orc_cube_stats(const orc_config *cfg, int integrand, const double *params, int64_t nparams, int t,
                   uint64_t seed, const double *edges, int64_t h, int64_t off_h, int64_t n_h, double *mean,
                   double *m2);

/* Eqs. (5)-(6) with V_h = 1/N_h (reading R12): iteration estimate and variance
 * from complete per-cube statistics, plus ell_h for the next allocation. */
void orc_finish_cubes(const orc_config *cfg, const int64_t *offsets, const double *mean, const double *m2,
                      float *ell, double *it_est, double *it_var);

/* One whole iteration (Algorithm 1 body) from the given map and offsets.
 * Writes mean/m2/ell (ncubes), bins (d*nbins), the refined edges, the next
 * offsets and the iteration estimate / variance.  Returns 0 or a negative code. */
int orc_iteration(const orc_config *cfg, int integrand, const double *params, int64_t nparams,
                  int64_t neval, int t, uint64_t seed, const double *edges, const int64_t *offsets,
                  double *mean, double *m2, float *ell, double *bins, double *edges_next,
                  int64_t *offsets_next, double *it_est, double *it_var);

/* Algorithm 1: nitn iterations from the uniform map.  it_est/it_sig (nitn)
 * and edges_out (d*(nbins+1), may be NULL) are written; out as orc_combine. */
int orc_integrate(const orc_config *cfg, int integrand, const double *params, int64_t nparams,
                  int64_t neval, int nitn, int skip, uint64_t seed, double *it_est, double *it_sig,
                  double *edges_out, double out[4]);

#ifdef __cplusplus
}
#endif
#endif
