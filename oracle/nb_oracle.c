/*
 * Naive Bayes oracle: a plain, slow, FP64 CPU implementation of what the
 * GPU library computes.  TEST INFRASTRUCTURE ONLY: the tests, the smoke
 * check and the CPU-baseline leg of the benchmark call it; the product path
 * never does.  It shares no code, header or table with the CUDA library.
 *
 * Paper: Sahay & Chaudhari, "An Efficient Detection of Malware by Naive
 * Bayes Classifier Using GPGPU", Sec. 4.
 *   - Posterior (Sec. 4, the single display equation): under the naive
 *     independence assumption P(C | a_1..a_n) is proportional to
 *     P(C) * prod_j P(a_j | C); the evidence P(a_1..a_n) is the same for
 *     every class.  We work with its logarithm, the joint log score
 *     s_c = log P(C=c) + sum_j log P(a_j | c).
 *   - Decision rule (Sec. 4, text under the equation): the file is malware
 *     (class 1) when the malware posterior is the higher one, otherwise
 *     benign (class 0); a tie therefore goes to benign, generalised here to
 *     "the lowest class index among the maxima".
 *   - The features are opcode occurrence counts (Sec. 3), so the count
 *     model is the multinomial event model with Laplace smoothing alpha;
 *     real-valued features use Gaussian class-conditional densities.
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   - prior: empirical n_c / n unless the caller supplies log priors;
 *   - smoothing: theta_cj = (N_cj + alpha) / (N_c + alpha * F);
 *   - Gaussian variance: maximum likelihood (divide by n_c) plus
 *     eps = var_smoothing * max_j Var(x_.j) over all training rows;
 *   - the multinomial coefficient and the evidence are class-independent
 *     and dropped from s_c; the log posterior restores the normalisation.
 *
 * Every function sums over features with j ascending, one row at a time.
 * Rows may be split over threads (a static partition); each row's
 * arithmetic is identical whichever thread runs it.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL 1

static const double kPi = 3.14159265358979323846;

/* The second half of the multinomial fit, from exact counts:
 *   log theta_cj = log(N_cj + alpha) - log(N_c + alpha * F),  N_c = sum_j N_cj
 *   log pi_c     = log n_c - log n, or the supplied log prior.             */
int oracle_mn_finalize(const uint64_t* counts, const uint64_t* nc, int64_t n,
                       int32_t F, int32_t C, double alpha,
                       const double* log_prior, double* log_theta,
                       double* log_pi) {
  if (F < 1 || C < 2 || !(alpha >= 0.0)) return OR_EINVAL;
  for (int32_t c = 0; c < C; ++c) {
    uint64_t Nc = 0;
    for (int32_t j = 0; j < F; ++j) Nc += counts[(int64_t)c * F + j];
    double log_den = log((double)Nc + alpha * (double)F);
    for (int32_t j = 0; j < F; ++j) {
      double num = (double)counts[(int64_t)c * F + j] + alpha;
      log_theta[(int64_t)c * F + j] = log(num) - log_den;
    }
  }
  for (int32_t c = 0; c < C; ++c) {
    if (log_prior) {
      if (!isfinite(log_prior[c])) return OR_EINVAL;
      log_pi[c] = log_prior[c];
    } else {
      if (nc[c] == 0) return OR_EINVAL;
      log_pi[c] = log((double)nc[c]) - log((double)n);
    }
  }
  return OR_OK;
}

/* ---------------------------------------------------------------------------
 * Multinomial fit (Sec. 4: "trained the model" on per-class opcode counts).
 *   n_c    = #{i : y_i = c}
 *   N_cj   = sum over rows of class c of x_ij        (exact, uint64)
 *   N_c    = sum_j N_cj
 *   log theta_cj = log(N_cj + alpha) - log(N_c + alpha * F)
 *   log pi_c     = log n_c - log n, or the supplied log prior.
 * X holds integer-valued counts; a negative or fractional value is an error.
 * Returns OR_EINVAL on bad arguments or on a class with no training rows
 * while no prior is supplied.
 * ------------------------------------------------------------------------ */
int oracle_mn_fit(const double* X, int64_t n, int32_t F, const int32_t* y,
                  int32_t C, double alpha, const double* log_prior,
                  uint64_t* counts, uint64_t* nc, double* log_theta,
                  double* log_pi) {
  if (n < 0 || F < 1 || C < 2 || !(alpha >= 0.0)) return OR_EINVAL;
  memset(counts, 0, sizeof(uint64_t) * (size_t)C * (size_t)F);
  memset(nc, 0, sizeof(uint64_t) * (size_t)C);
  for (int64_t i = 0; i < n; ++i) {
    int32_t c = y[i];
    if (c < 0 || c >= C) return OR_EINVAL;
    nc[c] += 1;
    for (int32_t j = 0; j < F; ++j) {
      double v = X[i * (int64_t)F + j];
      if (!(v >= 0.0) || v != floor(v) || v > 9.0e15) return OR_EINVAL;
      counts[(int64_t)c * F + j] += (uint64_t)v;
    }
  }
  return oracle_mn_finalize(counts, nc, n, F, C, alpha, log_prior, log_theta,
                            log_pi);
}

/* ---------------------------------------------------------------------------
 * Gaussian fit (real-valued features; the paper names no variant).
 *   mu_cj  = (1/n_c) sum_{y_i=c} x_ij                     (pass 1)
 *   var_cj = (1/n_c) sum_{y_i=c} (x_ij - mu_cj)^2 + eps     (pass 2)
 *   eps    = var_smoothing * max_j Var_all(x_.j), Var_all over all n rows,
 *            also computed in two passes.
 * ------------------------------------------------------------------------ */
int oracle_gauss_fit(const double* X, int64_t n, int32_t F, const int32_t* y,
                     int32_t C, double var_smoothing, const double* log_prior,
                     uint64_t* nc, double* mu, double* var, double* log_pi) {
  if (n < 1 || F < 1 || C < 2 || !(var_smoothing >= 0.0)) return OR_EINVAL;
  memset(nc, 0, sizeof(uint64_t) * (size_t)C);
  memset(mu, 0, sizeof(double) * (size_t)C * (size_t)F);
  memset(var, 0, sizeof(double) * (size_t)C * (size_t)F);
  for (int64_t i = 0; i < n; ++i) {
    int32_t c = y[i];
    if (c < 0 || c >= C) return OR_EINVAL;
    nc[c] += 1;
  }
  for (int32_t c = 0; c < C; ++c)
    if (nc[c] == 0) return OR_EINVAL;
  /* pass 1: class means */
  for (int64_t i = 0; i < n; ++i)
    for (int32_t j = 0; j < F; ++j)
      mu[(int64_t)y[i] * F + j] += X[i * (int64_t)F + j];
  for (int32_t c = 0; c < C; ++c)
    for (int32_t j = 0; j < F; ++j) mu[(int64_t)c * F + j] /= (double)nc[c];
  /* pass 2: class variances about those means */
  for (int64_t i = 0; i < n; ++i)
    for (int32_t j = 0; j < F; ++j) {
      double dlt = X[i * (int64_t)F + j] - mu[(int64_t)y[i] * F + j];
      var[(int64_t)y[i] * F + j] += dlt * dlt;
    }
  for (int32_t c = 0; c < C; ++c)
    for (int32_t j = 0; j < F; ++j) var[(int64_t)c * F + j] /= (double)nc[c];
  /* eps from the largest whole-data feature variance */
  double max_var = 0.0;
  for (int32_t j = 0; j < F; ++j) {
    double m = 0.0;
    for (int64_t i = 0; i < n; ++i) m += X[i * (int64_t)F + j];
    m /= (double)n;
    double v = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      double dlt = X[i * (int64_t)F + j] - m;
      v += dlt * dlt;
    }
    v /= (double)n;
    if (v > max_var) max_var = v;
  }
  double eps = var_smoothing * max_var;
  for (int64_t k = 0; k < (int64_t)C * F; ++k) {
    var[k] += eps;
    if (!(var[k] > 0.0)) return OR_EINVAL; /* a constant feature, no smoothing */
  }
  for (int32_t c = 0; c < C; ++c) {
    if (log_prior) {
      if (!isfinite(log_prior[c])) return OR_EINVAL;
      log_pi[c] = log_prior[c];
    } else {
      log_pi[c] = log((double)nc[c]) - log((double)n);
    }
  }
  return OR_OK;
}

/* ---------------------------------------------------------------------------
 * Joint log scores, row by row.
 *   multinomial: s_c = log pi_c + sum_j x_j * log theta_cj
 *   Gaussian:    s_c = log pi_c - 1/2 sum_j [ log(2 pi var_cj)
 *                                            + (x_j - mu_cj)^2 / var_cj ]
 * ------------------------------------------------------------------------ */
typedef struct {
  int kind; /* 0 multinomial, 1 Gaussian */
  const double* X;
  int64_t r0, r1;
  int32_t F, C;
  const double* p0; /* log_theta or mu */
  const double* p1; /* NULL or var */
  const double* log_pi;
  double* s;
} joint_job;

static void joint_rows(const joint_job* jb) {
  const int32_t F = jb->F, C = jb->C;
  for (int64_t i = jb->r0; i < jb->r1; ++i) {
    const double* x = jb->X + i * (int64_t)F;
    for (int32_t c = 0; c < C; ++c) {
      double acc = 0.0;
      if (jb->kind == 0) {
        const double* lt = jb->p0 + (int64_t)c * F;
        for (int32_t j = 0; j < F; ++j) acc += x[j] * lt[j];
        jb->s[i * C + c] = jb->log_pi[c] + acc;
      } else {
        const double* m = jb->p0 + (int64_t)c * F;
        const double* v = jb->p1 + (int64_t)c * F;
        for (int32_t j = 0; j < F; ++j) {
          double dlt = x[j] - m[j];
          acc += log(2.0 * kPi * v[j]) + dlt * dlt / v[j];
        }
        jb->s[i * C + c] = jb->log_pi[c] - 0.5 * acc;
      }
    }
  }
}

static void* joint_thread(void* arg) {
  joint_rows((const joint_job*)arg);
  return NULL;
}

static void run_joint(joint_job proto, int64_t n, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if ((int64_t)nthreads > n) nthreads = n > 0 ? (int)n : 1;
  if (nthreads == 1) {
    proto.r0 = 0;
    proto.r1 = n;
    joint_rows(&proto);
    return;
  }
  pthread_t tid[256];
  joint_job jobs[256];
  int started[256];
  for (int t = 0; t < nthreads; ++t) {
    jobs[t] = proto;
    jobs[t].r0 = n * t / nthreads;
    jobs[t].r1 = n * (t + 1) / nthreads;
    started[t] = pthread_create(&tid[t], NULL, joint_thread, &jobs[t]) == 0;
    if (!started[t]) joint_rows(&jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t)
    if (started[t]) pthread_join(tid[t], NULL);
}

void oracle_mn_joint(const double* X, int64_t n, int32_t F, int32_t C,
                     const double* log_theta, const double* log_pi, double* s,
                     int nthreads) {
  joint_job jb = {0, X, 0, 0, F, C, log_theta, NULL, log_pi, s};
  run_joint(jb, n, nthreads);
}

void oracle_gauss_joint(const double* X, int64_t n, int32_t F, int32_t C,
                        const double* mu, const double* var,
                        const double* log_pi, double* s, int nthreads) {
  joint_job jb = {1, X, 0, 0, F, C, mu, var, log_pi, s};
  run_joint(jb, n, nthreads);
}

/* ---------------------------------------------------------------------------
 * Decision (Sec. 4 decision rule) and log posterior (Sec. 4 equation).
 *   label_i  = smallest c with s_ic = max_c s_ic
 *   margin_i = (largest s_ic) - (second largest s_ic)          (>= 0)
 *   lp_ic    = s_ic - (m + log sum_c exp(s_ic - m)),  m = max_c s_ic
 * ------------------------------------------------------------------------ */
void oracle_decide(const double* s, int64_t n, int32_t C, uint8_t* label,
                   double* margin, double* lp) {
  for (int64_t i = 0; i < n; ++i) {
    const double* si = s + i * C;
    int32_t best = 0;
    for (int32_t c = 1; c < C; ++c)
      if (si[c] > si[best]) best = c;
    double second = -INFINITY;
    for (int32_t c = 0; c < C; ++c)
      if (c != best && si[c] > second) second = si[c];
    label[i] = (uint8_t)best;
    margin[i] = si[best] - second;
    if (lp) {
      double m = si[best];
      double sum = 0.0;
      for (int32_t c = 0; c < C; ++c) sum += exp(si[c] - m);
      double lse = m + log(sum);
      for (int32_t c = 0; c < C; ++c) lp[i * C + c] = si[c] - lse;
    }
  }
}
