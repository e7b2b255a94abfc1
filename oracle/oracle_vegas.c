/*
 * oracle_vegas.c -- plain, slow, single-threaded FP64 CPU oracle of the VEGAS+
 * iteration loop (cuVegas, arXiv 2408.09229).  TEST INFRASTRUCTURE ONLY: see
 * oracle_vegas.h for who may use it and for the map of paper passages.
 *
 * Build: gcc -O2 -std=c11 -fPIC -shared -ffp-contract=off (no fast-math), so
 * that every float/double operation is one IEEE operation on x86-64 and Arm.
 */
#include "oracle_vegas.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from the definition in Salmon et al., "Parallel random     */
/* numbers: as easy as 1, 2, 3", SC'11: ten rounds of two 32x32->64 bit      */
/* multiplications whose high halves are xor-ed with the other counter words */
/* and the round key; the key is bumped by the Weyl constants between rounds */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u; /* round multipliers */
  const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u; /* key schedule */
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += weyl0;
      k1 += weyl1;
    }
    uint64_t prod0 = (uint64_t)mul0 * (uint64_t)x0;
    uint64_t prod1 = (uint64_t)mul1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------ */
/* Integrands (Table 3 of the paper, plus the ridge / product-peak /         */
/* oscillatory families of the synthetic workloads)                          */
/* ------------------------------------------------------------------------ */
static int expected_nparams(int id, int d, const double *p, int64_t np) {
  switch (id) {
    case ORC_GAUSS_SUM:
      if (np < 3) return -1;
      return 3 + (int64_t)p[2] * d == np ? 0 : -1;
    case ORC_PRODUCT_PEAK: return np == 2 * (int64_t)d ? 0 : -1;
    case ORC_OSCILLATORY: return np == 1 + (int64_t)d ? 0 : -1;
    case ORC_SIN_EXP: return d == 2 ? 0 : -1;
    case ORC_LINEAR: case ORC_COSINE: case ORC_EXPONENTIAL:
    case ORC_ROOS_ARNOLD: case ORC_MOROKOFF_CAFLISCH: return 0;
    case ORC_MAP_DENSITY:
      /* edges of a separable map with G bins per axis: d*(G+1) values, G >= 1 */
      if (np < 2 * (int64_t)d || np % d != 0) return -1;
      return 0;
    default: return -1;
  }
}

int orc_integrand(int id, int d, const double *p, int64_t np, const double *x, double *f) {
  if (expected_nparams(id, d, p, np) != 0) return -1;
  double r = 0.0;
  switch (id) {
    case ORC_GAUSS_SUM: {
      /* sum of K isotropic Gaussians with common width s and prefactor A */
      double A = p[0], s = p[1];
      int64_t K = (int64_t)p[2];
      const double *mu = p + 3;
      double acc = 0.0;
      for (int64_t k = 0; k < K; ++k) {
        double r2 = 0.0;
        for (int j = 0; j < d; ++j) {
          double dx = x[j] - mu[k * d + j];
          r2 += dx * dx;
        }
        acc += exp(-r2 / (2.0 * s * s));
      }
      r = A * acc;
      break;
    }
    case ORC_PRODUCT_PEAK: {
      const double *c = p, *w = p + d;
      r = 1.0;
      for (int j = 0; j < d; ++j) {
        double dx = x[j] - w[j];
        r *= 1.0 / (1.0 / (c[j] * c[j]) + dx * dx);
      }
      break;
    }
    case ORC_OSCILLATORY: {
      double arg = 2.0 * M_PI * p[0];
      for (int j = 0; j < d; ++j) arg += p[1 + j] * x[j];
      r = cos(arg);
      break;
    }
    case ORC_SIN_EXP: r = sin(x[0]) + exp(x[1]); break;
    case ORC_LINEAR:
      for (int j = 0; j < d; ++j) r += x[j];
      break;
    case ORC_COSINE:
      r = 1.0;
      for (int j = 0; j < d; ++j) r *= cos(x[j]);
      break;
    case ORC_EXPONENTIAL: {
      double s = 0.0;
      for (int j = 0; j < d; ++j) s += x[j] * x[j];
      r = exp(s);
      break;
    }
    case ORC_ROOS_ARNOLD:
      r = 1.0;
      for (int j = 0; j < d; ++j) r *= fabs(4.0 * x[j] - 2.0);
      break;
    case ORC_MOROKOFF_CAFLISCH:
      r = pow(1.0 + 1.0 / d, d);
      for (int j = 0; j < d; ++j) r *= pow(x[j], 1.0 / d);
      break;
    case ORC_MAP_DENSITY: {
      /* f(x) = prod_k 1/(G * dx_{k,i}) with i the interval of the reference
       * map that holds x_k: the density of that map, whose integral is 1 */
      int64_t G = np / d - 1;
      r = 1.0;
      for (int k = 0; k < d; ++k) {
        const double *e = p + (int64_t)k * (G + 1);
        int64_t i = 0;
        while (i < G - 1 && x[k] >= e[i + 1]) ++i;
        r *= 1.0 / ((double)G * (e[i + 1] - e[i]));
      }
      break;
    }
    default: return -1;
  }
  *f = r;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Reproducible FP32 log2 and exp2 (reading R4).  The allocation turns real  */
/* weights into integer sample counts; to make that integer decision the    */
/* same on every machine, the weight is computed by this fixed sequence of  */
/* single IEEE float operations (no fused multiply-add, no libm call).      */
/*   log2(x) = e + (2/ln 2) atanh(t),  t = (m-1)/(m+1),  m in (1/sqrt2, sqrt2] */
/*   atanh(t) = t (1 + t^2/3 + t^4/5 + t^6/7 + t^8/9) + O(t^11), |t| < 0.172   */
/*   2^y = 2^n e^(r ln 2), n = rint(y), |r| <= 1/2, Taylor to degree 7        */
/* ------------------------------------------------------------------------ */
static const float kThird = 0x1.555556p-2f, kFifth = 0x1.99999ap-3f, kSeventh = 0x1.24924ap-3f,
                   kNinth = 0x1.c71c72p-4f, kLog2e = 0x1.715476p+0f, kLn2 = 0x1.62e430p-1f,
                   kSqrt2 = 0x1.6a09e6p+0f;
static const float kInvFact[8] = {1.0f, 1.0f, 0x1p-1f, 0x1.555556p-3f, 0x1.555556p-5f,
                                  0x1.111112p-7f, 0x1.6c16c2p-10f, 0x1.a01a02p-13f};

/* volatile stores keep each float operation a separate, rounded IEEE op */
static float fadd(float a, float b) { volatile float r = a + b; return r; }
static float fsub(float a, float b) { volatile float r = a - b; return r; }
static float fmul(float a, float b) { volatile float r = a * b; return r; }
static float fdiv(float a, float b) { volatile float r = a / b; return r; }

float orc_log2r(double x) {
  if (x == 0.0) return -INFINITY;
  if (!(x > 0.0) || isinf(x)) return NAN;
  int e;
  double m2 = frexp(x, &e); /* x = m2 * 2^e, m2 in [0.5, 1) */
  float m = (float)(m2 * 2.0); /* in [1, 2], rounded to float */
  e -= 1;
  if (m > kSqrt2) {
    m = fmul(m, 0.5f);
    e += 1;
  }
  float t = fdiv(fsub(m, 1.0f), fadd(m, 1.0f));
  float t2 = fmul(t, t);
  float p = kNinth;
  p = fadd(fmul(p, t2), kSeventh);
  p = fadd(fmul(p, t2), kFifth);
  p = fadd(fmul(p, t2), kThird);
  p = fadd(fmul(p, t2), 1.0f);
  float s = fmul(fmul(t, p), 2.0f);
  return fadd((float)e, fmul(s, kLog2e));
}

float orc_exp2r(float y) {
  if (y > 0.0f || isnan(y)) return NAN;
  if (y < -30.0f) return 0.0f;
  float n = rintf(y);
  float r = fsub(y, n);
  float s = fmul(r, kLn2);
  float p = kInvFact[7];
  for (int k = 6; k >= 0; --k) p = fadd(fmul(p, s), kInvFact[k]);
  return fmul(p, ldexpf(1.0f, (int)n));
}

float orc_cube_ell(double m2, int64_t n, double beta) {
  /* sigma_h^beta = var_h^(beta/2), var_h the unbiased sample variance of Jf
   * in cube h (Sec. 2.1.2: n_h proportional to sigma_h(Jf), damped by beta) */
  double var = m2 / (double)(n - 1);
  float half_beta = fmul((float)beta, 0.5f);
  return fmul(half_beta, orc_log2r(var));
}

uint32_t orc_quant_weight(float ell, float ell_max) {
  if (isinf(ell) && ell < 0) return 0u;
  float y = fsub(ell, ell_max);
  float w = orc_exp2r(y);
  return (uint32_t)rintf(fmul(w, 16777216.0f));
}

/* ------------------------------------------------------------------------ */
/* Allocation of evaluations to hypercubes (Sec. 2.1.2, Eq. (7); reading R5) */
/* n_h = 2 + share of R = N_eval - 2 N_h proportional to q_h, by cumulative */
/* rounding: off_h = 2h + floor(R * Q_h / Q), Q_h = sum_{h'<h} q_h', Q = Q_N */
/* ------------------------------------------------------------------------ */
int orc_allocate(const float *ell, int64_t ncubes, int64_t neval, double beta, int64_t *offsets) {
  if (ncubes < 1 || neval < 2 * ncubes) return -1;
  const int64_t R = neval - 2 * ncubes;
  int uniform = (ell == NULL) || (beta == 0.0);
  float ell_max = -INFINITY;
  if (!uniform) {
    for (int64_t h = 0; h < ncubes; ++h) {
      if (isnan(ell[h]) || (isinf(ell[h]) && ell[h] > 0)) return -2;
      if (ell[h] > ell_max) ell_max = ell[h];
    }
    if (isinf(ell_max)) uniform = 1; /* every cube had zero variance */
  }
  uint64_t *q = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)ncubes);
  if (!q) return -3;
  unsigned __int128 Q = 0;
  for (int64_t h = 0; h < ncubes; ++h) {
    q[h] = uniform ? 1u : orc_quant_weight(ell[h], ell_max);
    Q += q[h];
  }
  unsigned __int128 Qh = 0;
  for (int64_t h = 0; h <= ncubes; ++h) {
    unsigned __int128 share = ((unsigned __int128)(uint64_t)R * Qh) / Q;
    offsets[h] = 2 * h + (int64_t)share;
    if (h < ncubes) Qh += q[h];
  }
  free(q);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Map refinement, one axis (Sec. 2.1.1 "refined through the iterations ... */
/* controlled by a damping parameter alpha"; Algorithm 1 adjustWeights and  */
/* updateMap; readings R6 smoothing, R7 damping, R8 edge recomputation)     */
/* ------------------------------------------------------------------------ */
int orc_refine_axis(int N, double alpha, const double *w, const double *e_in, double *e_out) {
  int unchanged = 0;
  double wsum = 0.0;
  for (int i = 0; i < N; ++i) {
    if (!isfinite(w[i]) || w[i] < 0.0) unchanged = 1;
    wsum += w[i];
  }
  if (!(wsum > 0.0) || !isfinite(wsum) || alpha == 0.0 || N < 2) unchanged = 1;
  if (unchanged) {
    for (int i = 0; i <= N; ++i) e_out[i] = e_in[i];
    return 1;
  }
  double *ws = (double *)malloc(sizeof(double) * (size_t)N);
  double *m = (double *)malloc(sizeof(double) * (size_t)N);
  /* R6: smoothing with neighbours, weights (7,1)/8 at the ends, (1,6,1)/8 inside */
  ws[0] = (7.0 * w[0] + w[1]) / 8.0;
  for (int i = 1; i < N - 1; ++i) ws[i] = (w[i - 1] + 6.0 * w[i] + w[i + 1]) / 8.0;
  ws[N - 1] = (w[N - 2] + 7.0 * w[N - 1]) / 8.0;
  double S = 0.0;
  for (int i = 0; i < N; ++i) S += ws[i];
  /* R7: normalise, then damp: m_i = ((1 - r_i) / ln(1/r_i))^alpha */
  for (int i = 0; i < N; ++i) {
    double r = ws[i] / S;
    if (r <= 0.0) m[i] = 0.0;
    else if (r >= 1.0) m[i] = 1.0;
    else m[i] = pow((1.0 - r) / log(1.0 / r), alpha);
  }
  /* R8: new edges split the cumulative damped weight into N equal parts;
   * inside old interval i the weight is uniform, so the edge is found by
   * linear interpolation across that interval */
  double total = 0.0;
  for (int i = 0; i < N; ++i) total += m[i];
  double step = total / N;
  e_out[0] = e_in[0];
  e_out[N] = e_in[N];
  int i = 0;
  double acc = 0.0; /* weight of old intervals 0..i-1 */
  for (int j = 1; j < N; ++j) {
    double target = j * step;
    while (i < N - 1 && acc + m[i] <= target) {
      acc += m[i];
      ++i;
    }
    double width = e_in[i + 1] - e_in[i];
    double frac = m[i] > 0.0 ? (target - acc) / m[i] : 0.0;
    if (frac < 0.0) frac = 0.0;
    if (frac > 1.0) frac = 1.0;
    e_out[j] = e_in[i] + frac * width;
  }
  /* interior edges strictly increasing and below the last edge */
  for (int j = 1; j < N; ++j) {
    if (!(e_out[j] > e_out[j - 1])) e_out[j] = nextafter(e_out[j - 1], INFINITY);
  }
  for (int j = N - 1; j >= 1; --j) {
    if (!(e_out[j] < e_out[j + 1])) e_out[j] = nextafter(e_out[j + 1], -INFINITY);
  }
  free(ws);
  free(m);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Estimation aggregation (Sec. 2.1.3, Eqs. (8)-(9); reading R9)             */
/* ------------------------------------------------------------------------ */
void orc_combine(const double *I, const double *sig, int n, int skip, double out[4]) {
  if (skip < 0) skip = 0;
  int used = n - skip;
  if (used <= 0) {
    out[0] = NAN; out[1] = NAN; out[2] = NAN; out[3] = 0;
    return;
  }
  int nzero = 0;
  double zsum = 0.0;
  for (int t = skip; t < n; ++t)
    if (sig[t] == 0.0) { ++nzero; zsum += I[t]; }
  if (nzero > 0) {
    double mean = zsum / nzero;
    int agree = 1;
    for (int t = skip; t < n; ++t)
      if (sig[t] == 0.0 && I[t] != mean) agree = 0;
    out[0] = mean; out[1] = 0.0; out[2] = agree ? 0.0 : INFINITY; out[3] = used;
    return;
  }
  double wsum = 0.0, wisum = 0.0;
  for (int t = skip; t < n; ++t) {
    double w = 1.0 / (sig[t] * sig[t]);
    wsum += w;
    wisum += w * I[t];
  }
  double est = wisum / wsum;
  double chi2 = 0.0;
  for (int t = skip; t < n; ++t) {
    double dv = I[t] - est;
    chi2 += dv * dv / (sig[t] * sig[t]);
  }
  out[0] = est;
  out[1] = sqrt(1.0 / wsum);
  out[2] = used > 1 ? chi2 / (used - 1) : 0.0;
  out[3] = used;
}

void orc_combine_lagged(const double *I, const double *sig, int n, int skip, double out[4]) {
  if (skip < 0) skip = 0;
  int used = n - skip;
  if (used <= 0) {
    orc_combine(I, sig, n, skip, out);
    return;
  }
  for (int t = skip; t < n; ++t)
    if (sig[t] == 0.0) { /* exact iterations: the same rule as Eq. (8)'s */
      orc_combine(I, sig, n, skip, out);
      return;
    }
  double wsum = 0.0, wisum = 0.0, w2var = 0.0;
  for (int t = skip; t < n; ++t) {
    double s = (t > 0 && sig[t - 1] > 0.0) ? sig[t - 1] : sig[t]; /* the previous iteration's sigma */
    double w = 1.0 / (s * s);
    wsum += w;
    wisum += w * I[t];
    w2var += w * w * sig[t] * sig[t]; /* variance of a mean with weights fixed apart from I_t */
  }
  double est = wisum / wsum;
  double chi2 = 0.0;
  for (int t = skip; t < n; ++t) {
    double dv = I[t] - est;
    chi2 += dv * dv / (sig[t] * sig[t]);
  }
  out[0] = est;
  out[1] = sqrt(w2var) / wsum;
  out[2] = used > 1 ? chi2 / (used - 1) : 0.0;
  out[3] = used;
}

/* ------------------------------------------------------------------------ */
/* Configuration helpers                                                     */
/* ------------------------------------------------------------------------ */
int64_t orc_ncubes(const orc_config *cfg) {
  int64_t n = 1;
  for (int k = 0; k < cfg->dim; ++k) n *= cfg->nstrat[k];
  return n;
}

int orc_default_nstrat(int64_t neval, int dim) {
  /* R10: about two evaluations per hypercube */
  int64_t half = neval / 2, s = 1;
  for (;;) {
    int64_t p = 1, cand = s + 1;
    int over = 0;
    for (int k = 0; k < dim; ++k) {
      if (p > half / cand) { over = 1; break; }
      p *= cand;
    }
    if (over || p > half) break;
    s = cand;
  }
  return (int)s;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2 (vegasFill) over a range of evaluation indices                */
/* ------------------------------------------------------------------------ */
static void point_coordinates_f64(const orc_config *cfg, uint64_t seed, int t, int64_t j, double *u) {
  /* R2: key = seed; counter = (j lo, j hi, t, problem<<16 | block); in FP64
   * mode coordinate k takes two words of block k/2 and keeps 53 bits */
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  for (int k = 0; k < cfg->dim; ++k) {
    if (k % 2 == 0) {
      uint32_t ctr[4] = {(uint32_t)j, (uint32_t)((uint64_t)j >> 32), (uint32_t)t,
                         (cfg->problem_id << 16) | (uint32_t)(k / 2)};
      orc_philox4x32_10(ctr, key, out);
    }
    uint64_t hi = out[2 * (k % 2)], lo = out[2 * (k % 2) + 1];
    uint64_t bits = ((hi << 32) | lo) >> 11;
    u[k] = (double)bits * 0x1p-53;
  }
}

/* R2/R3, FP32 mode: coordinate k takes word k%4 of block k/4.  With
 * b = 23 - ceil(log2 s_k) fraction bits, the integer v = c_k 2^b + (w >> (32-b))
 * is below 2^23, so c_k + u = v 2^-b is exact in float; the point is then
 * z = RN32((c_k + u) N_g/s_k).  Writes v as a float (exact). */
static int frac_bits(int s) {
  int l = 0;
  while ((1 << l) < s) ++l;
  return 23 - l;
}

static void point_words_f32(const orc_config *cfg, uint64_t seed, int t, int64_t j, const int *c, float *v) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  for (int k = 0; k < cfg->dim; ++k) {
    if (k % 4 == 0) {
      uint32_t ctr[4] = {(uint32_t)j, (uint32_t)((uint64_t)j >> 32), (uint32_t)t,
                         (cfg->problem_id << 16) | (uint32_t)(k / 4)};
      orc_philox4x32_10(ctr, key, out);
    }
    int b = frac_bits(cfg->nstrat[k]);
    uint32_t iv = ((uint32_t)c[k] << b) | (out[k % 4] >> (32 - b));
    v[k] = (float)iv;
  }
}

int orc_fill_range(const orc_config *cfg, int integrand, const double *params, int64_t nparams,
                   int64_t neval, int t, uint64_t seed, const double *edges, const int64_t *offsets,
                   int64_t j_begin, int64_t j_end, int64_t *cnt, double *mean, double *m2, double *bins) {
  const int d = cfg->dim, G = cfg->nbins;
  const int64_t NH = orc_ncubes(cfg);
  if (offsets[NH] != neval || j_begin < 0 || j_end > neval) return -1;
  /* per-axis derived values (R3) */
  double *gz = (double *)malloc(sizeof(double) * d);
  float *gz32 = (float *)malloc(sizeof(float) * d);
  double *width = (double *)malloc(sizeof(double) * (size_t)d * G);
  double *jac = (double *)malloc(sizeof(double) * (size_t)d * G);
  for (int k = 0; k < d; ++k) {
    gz[k] = (double)G / (double)cfg->nstrat[k];
    gz32[k] = ldexpf(fdiv((float)G, (float)cfg->nstrat[k]), -frac_bits(cfg->nstrat[k]));
    for (int i = 0; i < G; ++i) {
      const double *e = edges + (size_t)k * (G + 1);
      width[(size_t)k * G + i] = e[i + 1] - e[i];
      jac[(size_t)k * G + i] = (double)G * width[(size_t)k * G + i];
    }
  }
  int64_t maxn = 0;
  for (int64_t h = 0; h < NH; ++h)
    if (offsets[h + 1] - offsets[h] > maxn) maxn = offsets[h + 1] - offsets[h];
  double *buf = (double *)malloc(sizeof(double) * (size_t)(maxn > 0 ? maxn : 1));
  double *u = (double *)malloc(sizeof(double) * d);
  float *u32 = (float *)malloc(sizeof(float) * d);
  int *c = (int *)malloc(sizeof(int) * d);
  int *bin = (int *)malloc(sizeof(int) * d);
  double *x = (double *)malloc(sizeof(double) * d);
  int status = 0;

  for (int64_t h = 0; h < NH; ++h) {
    int64_t lo = offsets[h], hi = offsets[h + 1];
    int64_t n_h = hi - lo;
    int64_t a = lo > j_begin ? lo : j_begin, b = hi < j_end ? hi : j_end;
    cnt[h] = 0; mean[h] = 0.0; m2[h] = 0.0;
    if (a >= b) continue;
    /* cube coordinates, axis 0 fastest (R3) */
    int64_t rest = h;
    for (int k = 0; k < d; ++k) {
      c[k] = (int)(rest % cfg->nstrat[k]);
      rest /= cfg->nstrat[k];
    }
    int64_t m = 0;
    for (int64_t j = a; j < b; ++j) {
      /* getPoint: uniform point y in the cube, then the map x(y) (Eq. (3)) */
      double J = 1.0;
      if (cfg->points_f32) point_words_f32(cfg, seed, t, j, c, u32);
      else point_coordinates_f64(cfg, seed, t, j, u);
      for (int k = 0; k < d; ++k) {
        double z, dz;
        int i;
        if (cfg->points_f32) {
          float zf = fmul(u32[k], gz32[k]);
          i = (int)floorf(zf);
          if (i > G - 1) i = G - 1;
          dz = (double)fsub(zf, (float)i);
        } else {
          z = ((double)c[k] + u[k]) * gz[k];
          i = (int)floor(z);
          if (i > G - 1) i = G - 1;
          dz = z - (double)i;
        }
        bin[k] = i;
        x[k] = fma(dz, width[(size_t)k * G + i], edges[(size_t)k * (G + 1) + i]);
        J *= jac[(size_t)k * G + i];
      }
      double f;
      orc_integrand(integrand, d, params, nparams, x, &f);
      if (!isfinite(f)) status = -2;
      double v = J * f; /* Eq. (4): one term J(y) f(x(y)) */
      buf[m++] = v;
      /* map weights (R11) */
      double wv = v * v / (double)n_h;
      for (int k = 0; k < d; ++k) bins[(size_t)k * G + bin[k]] += wv;
    }
    /* cube weights: two-pass mean and centred second moment (R12) */
    double s = 0.0;
    for (int64_t r = 0; r < m; ++r) s += buf[r];
    double mu = s / (double)m;
    double q = 0.0;
    for (int64_t r = 0; r < m; ++r) q += (buf[r] - mu) * (buf[r] - mu);
    cnt[h] = m; mean[h] = mu; m2[h] = q;
  }
  free(gz); free(gz32); free(width); free(jac); free(buf); free(u); free(u32); free(c); free(bin); free(x);
  return status;
}

int orc_cube_stats(const orc_config *cfg, int integrand, const double *params, int64_t nparams, int t,
                   uint64_t seed, const double *edges, int64_t h, int64_t off_h, int64_t n_h, double *mean,
                   double *m2) {
  /* the same sample loop as orc_fill_range, on a two-cube offset table
   * that places cube h at its true evaluation indices */
  orc_config one = *cfg;
  const int64_t NH = orc_ncubes(cfg);
  if (h < 0 || h >= NH || n_h < 2) return -1;
  int64_t offs[2] = {off_h, off_h + n_h};
  const int d = cfg->dim, G = cfg->nbins;
  double *gz = (double *)malloc(sizeof(double) * d);
  float *gz32 = (float *)malloc(sizeof(float) * d);
  double *u = (double *)malloc(sizeof(double) * d);
  float *u32 = (float *)malloc(sizeof(float) * d);
  double *x = (double *)malloc(sizeof(double) * d);
  double *buf = (double *)malloc(sizeof(double) * (size_t)n_h);
  int *c = (int *)malloc(sizeof(int) * d);
  int64_t rest = h;
  for (int k = 0; k < d; ++k) {
    gz[k] = (double)G / (double)cfg->nstrat[k];
    gz32[k] = ldexpf(fdiv((float)G, (float)cfg->nstrat[k]), -frac_bits(cfg->nstrat[k]));
    c[k] = (int)(rest % cfg->nstrat[k]);
    rest /= cfg->nstrat[k];
  }
  int status = 0;
  for (int64_t j = offs[0]; j < offs[1]; ++j) {
    double J = 1.0;
    if (one.points_f32) point_words_f32(&one, seed, t, j, c, u32);
    else point_coordinates_f64(&one, seed, t, j, u);
    for (int k = 0; k < d; ++k) {
      const double *e = edges + (size_t)k * (G + 1);
      double dz;
      int i;
      if (one.points_f32) {
        float zf = fmul(u32[k], gz32[k]);
        i = (int)floorf(zf);
        if (i > G - 1) i = G - 1;
        dz = (double)fsub(zf, (float)i);
      } else {
        double z = ((double)c[k] + u[k]) * gz[k];
        i = (int)floor(z);
        if (i > G - 1) i = G - 1;
        dz = z - (double)i;
      }
      double width = e[i + 1] - e[i];
      x[k] = fma(dz, width, e[i]);
      J *= (double)G * width;
    }
    double f;
    orc_integrand(integrand, d, params, nparams, x, &f);
    if (!isfinite(f)) status = -2;
    buf[j - offs[0]] = J * f;
  }
  double s = 0.0;
  for (int64_t r = 0; r < n_h; ++r) s += buf[r];
  double mu = s / (double)n_h, q = 0.0;
  for (int64_t r = 0; r < n_h; ++r) q += (buf[r] - mu) * (buf[r] - mu);
  *mean = mu;
  *m2 = q;
  free(gz); free(gz32); free(u); free(u32); free(x); free(buf); free(c);
  return status;
}

void orc_finish_cubes(const orc_config *cfg, const int64_t *offsets, const double *mean, const double *m2,
                      float *ell, double *it_est, double *it_var) {
  /* Eqs. (5)-(6): I = sum_h V_h mean_h, sigma^2 = sum_h V_h^2 var_h / n_h, with
   * V_h = 1/N_h the y-space volume of a cube (R12) */
  const int64_t NH = orc_ncubes(cfg);
  double isum = 0.0, vsum = 0.0;
  for (int64_t h = 0; h < NH; ++h) {
    int64_t n = offsets[h + 1] - offsets[h];
    isum += mean[h];
    vsum += m2[h] / ((double)n * (double)(n - 1));
    if (ell) ell[h] = orc_cube_ell(m2[h], n, cfg->beta);
  }
  *it_est = isum / (double)NH;
  *it_var = vsum / ((double)NH * (double)NH);
}

int orc_iteration(const orc_config *cfg, int integrand, const double *params, int64_t nparams,
                  int64_t neval, int t, uint64_t seed, const double *edges, const int64_t *offsets,
                  double *mean, double *m2, float *ell, double *bins, double *edges_next,
                  int64_t *offsets_next, double *it_est, double *it_var) {
  const int d = cfg->dim, G = cfg->nbins;
  const int64_t NH = orc_ncubes(cfg);
  int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)NH);
  /* Algorithm 1: reset weights */
  memset(bins, 0, sizeof(double) * (size_t)d * G);
  /* Algorithm 1: fill (Algorithm 2) over all evaluations */
  int st = orc_fill_range(cfg, integrand, params, nparams, neval, t, seed, edges, offsets, 0, neval, cnt,
                          mean, m2, bins);
  free(cnt);
  if (st != 0 && st != -2) return st;
  /* Algorithm 1: computeResults and the stratification statistics */
  orc_finish_cubes(cfg, offsets, mean, m2, ell, it_est, it_var);
  /* Algorithm 1: updateEvalsPerCube */
  int a = orc_allocate(ell, NH, neval, cfg->beta, offsets_next);
  if (a != 0) return a == -2 ? -2 : -1;
  /* Algorithm 1: adjustWeights + updateMap, axis by axis */
  for (int k = 0; k < d; ++k)
    orc_refine_axis(G, cfg->alpha, bins + (size_t)k * G, edges + (size_t)k * (G + 1),
                    edges_next + (size_t)k * (G + 1));
  return st;
}

int orc_integrate(const orc_config *cfg, int integrand, const double *params, int64_t nparams,
                  int64_t neval, int nitn, int skip, uint64_t seed, double *it_est, double *it_sig,
                  double *edges_out, double out[4]) {
  const int d = cfg->dim, G = cfg->nbins;
  const int64_t NH = orc_ncubes(cfg);
  if (d < 1 || G < 2 || NH < 1 || neval < 2 * NH || nitn < 1) return -1;
  size_t ne = (size_t)d * (G + 1);
  double *e0 = (double *)malloc(sizeof(double) * ne), *e1 = (double *)malloc(sizeof(double) * ne);
  int64_t *o0 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(NH + 1));
  int64_t *o1 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(NH + 1));
  double *mean = (double *)malloc(sizeof(double) * (size_t)NH);
  double *m2 = (double *)malloc(sizeof(double) * (size_t)NH);
  float *ell = (float *)malloc(sizeof(float) * (size_t)NH);
  double *bins = (double *)malloc(sizeof(double) * (size_t)d * G);
  /* Algorithm 1 init: uniform map (Sec. 2.1.1) and uniform allocation */
  for (int k = 0; k < d; ++k)
    for (int i = 0; i <= G; ++i) e0[(size_t)k * (G + 1) + i] = (double)i / (double)G;
  orc_allocate(NULL, NH, neval, cfg->beta, o0);
  int status = 0;
  for (int t = 0; t < nitn; ++t) {
    double I, V;
    int st = orc_iteration(cfg, integrand, params, nparams, neval, t, seed, e0, o0, mean, m2, ell, bins, e1,
                           o1, &I, &V);
    if (st == -2) status = -2;
    else if (st != 0) { status = st; break; }
    it_est[t] = I;
    it_sig[t] = sqrt(V);
    double *te = e0; e0 = e1; e1 = te;
    int64_t *to = o0; o0 = o1; o1 = to;
  }
  if (status != -1 && status != -3) orc_combine(it_est, it_sig, nitn, skip, out);
  if (edges_out) memcpy(edges_out, e0, sizeof(double) * ne);
  free(e0); free(e1); free(o0); free(o1); free(mean); free(m2); free(ell); free(bins);
  return status;
}
