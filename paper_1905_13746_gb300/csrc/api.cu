// C-ABI entry points of nbgpu: argument checking, model lifetime, dispatch
// to the fit and score kernels.  No exception crosses this boundary; every
// failure returns an nb_status and leaves a message for nb_last_error().
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <new>

#include "internal.cuh"

namespace nbg {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

nb_status cuda_status(cudaError_t e, const char* what) {
  set_error("%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return NB_ENOMEM;
  return NB_ECUDA;
}

int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cached[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 1;
  }
  return cached[dev];
}

static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// carve every table of a model out of one device allocation
static nb_status alloc_model(nb_model* m) {
  const size_t C = m->C, F = m->F, Fp = m->F_pad;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  // counts, nc and the status word lie in this order, so that the multinomial
  // fit clears all three with one memset
  const size_t o_counts = take(sizeof(uint64_t) * C * F);
  const size_t o_nc = take(sizeof(uint64_t) * C);
  const size_t o_st = take(sizeof(int) * 4);
  const size_t o_p0 = take(sizeof(double) * C * F);
  const size_t o_p1 = take(m->kind == NB_GAUSSIAN ? sizeof(double) * C * F : 0);
  const size_t o_lpi = take(sizeof(double) * C);
  const size_t o_gc = take(sizeof(double) * C);
  const size_t o_fin = take(sizeof(unsigned long long) * 4);
  const size_t o_c2 = take(sizeof(C2Header));
  const size_t o_delta = take(sizeof(float) * Fp);
  const size_t o_dq = take(sizeof(int32_t) * Fp);
  const size_t o_limbs = take(7 * Fp);   // three limb planes + packed limb words
  const size_t o_il0 = take(sizeof(float) * Fp);
  const size_t o_il1 = take(sizeof(float) * Fp);
  const size_t o_il2 = take(sizeof(float) * Fp);
  const size_t o_w = take(sizeof(float) * C * Fp);
  const size_t o_bias = take(sizeof(float) * C);
  const size_t o_wmax = take(sizeof(float) * 4);
  const size_t o_gmu = take(m->kind == NB_GAUSSIAN ? sizeof(float) * gauss_cpad(C) * Fp : 0);
  const size_t o_giv = take(m->kind == NB_GAUSSIAN ? sizeof(float) * gauss_cpad(C) * Fp : 0);
  const size_t o_gk = take(sizeof(float) * 2 * C);
  const bool tc = tc_tables(m->kind, m->C, m->F);
  const size_t o_tcw = take(tc ? tc_w_bytes(m->C, m->F) : 0);
  const size_t o_tcq = take(tc ? sizeof(int32_t) * C * F : 0);
  const size_t o_tch = take(tc ? sizeof(TcHeader) : 0);
  const bool tg = tcg_tables(m->kind, m->C, m->F);
  const int F8 = (m->F + kTcgFS - 1) / kTcgFS * kTcgFS;
  const size_t o_tgw = take(tg ? tcg_w_bytes(m->C, m->F) : 0);
  const size_t o_tgk = take(tg ? sizeof(float) * C : 0);
  const size_t o_tgc = take(tg ? sizeof(float) * F8 : 0);
  const size_t o_tgb = take(tg ? sizeof(float) * F8 : 0);
  const size_t o_tga = take(tg ? sizeof(float) * F8 : 0);
  const size_t o_tgh = take(tg ? sizeof(TcgHeader) : 0);
  void* mem = nullptr;
  cudaError_t e = cudaMalloc(&mem, off);
  if (e != cudaSuccess) return cuda_status(e, "cudaMalloc(model)");
  m->mem = mem;
  m->mem_bytes = off;
  char* b = static_cast<char*>(mem);
  ModelDev& d = m->d;
  d.counts = reinterpret_cast<uint64_t*>(b + o_counts);
  d.nc = reinterpret_cast<uint64_t*>(b + o_nc);
  d.p0 = reinterpret_cast<double*>(b + o_p0);
  d.p1 = m->kind == NB_GAUSSIAN ? reinterpret_cast<double*>(b + o_p1) : nullptr;
  d.log_pi = reinterpret_cast<double*>(b + o_lpi);
  d.gconst = reinterpret_cast<double*>(b + o_gc);
  d.status = reinterpret_cast<int*>(b + o_st);
  d.sstatus = d.status + 1;   // outside the fit's clear of counts, nc and status
  d.fin = reinterpret_cast<unsigned long long*>(b + o_fin);
  d.c2 = reinterpret_cast<C2Header*>(b + o_c2);
  d.delta = reinterpret_cast<float*>(b + o_delta);
  d.delta_q = reinterpret_cast<int32_t*>(b + o_dq);
  d.limbs = reinterpret_cast<uint4*>(b + o_limbs);
  d.il[0] = reinterpret_cast<float4*>(b + o_il0);
  d.il[1] = reinterpret_cast<float4*>(b + o_il1);
  d.il[2] = reinterpret_cast<float4*>(b + o_il2);
  d.w = reinterpret_cast<float*>(b + o_w);
  d.bias = reinterpret_cast<float*>(b + o_bias);
  d.wmax = reinterpret_cast<float*>(b + o_wmax);
  d.g_mu = m->kind == NB_GAUSSIAN ? reinterpret_cast<float*>(b + o_gmu) : nullptr;
  d.g_ivar = m->kind == NB_GAUSSIAN ? reinterpret_cast<float*>(b + o_giv) : nullptr;
  d.g_const = reinterpret_cast<float*>(b + o_gk);
  d.tc_w = tc ? reinterpret_cast<uint8_t*>(b + o_tcw) : nullptr;
  d.tc_q = tc ? reinterpret_cast<int32_t*>(b + o_tcq) : nullptr;
  d.tc_hdr = tc ? reinterpret_cast<TcHeader*>(b + o_tch) : nullptr;
  if (tg) d.tc_w = reinterpret_cast<uint8_t*>(b + o_tgw);
  d.tcg_kc = tg ? reinterpret_cast<float*>(b + o_tgk) : nullptr;
  d.tcg_ctr = tg ? reinterpret_cast<float*>(b + o_tgc) : nullptr;
  d.tcg_bmax = tg ? reinterpret_cast<float*>(b + o_tgb) : nullptr;
  d.tcg_amax = tg ? reinterpret_cast<float*>(b + o_tga) : nullptr;
  d.tcg_hdr = tg ? reinterpret_cast<TcgHeader*>(b + o_tgh) : nullptr;
  return NB_OK;
}

nb_status status_from_word(int w) {
  if (w & ST_TIMEOUT) {
    set_error("a bounded device wait ran out");
    return NB_ETIMEOUT;
  }
  if (w & ST_BAD_LABEL) {
    set_error("invalid labels: a label outside [0, C) or a class without training rows");
    return NB_EINVAL;
  }
  if (w & ST_BAD_VALUE) {
    set_error("invalid feature values: counts must be non-negative integers below 2^24, "
              "Gaussian features finite");
    return NB_EINVAL;
  }
  if (w & ST_OVF_RANGE) {
    set_error("overflow list names a column outside [0, F)");
    return NB_EINVAL;
  }
  if (w & ST_BAD_TABLE) {
    set_error("non-finite parameter table (zero variance or an infinite log probability)");
    return NB_EINVAL;
  }
  return NB_OK;
}

}  // namespace nbg

using namespace nbg;

extern "C" const char* nb_last_error(void) { return g_err; }
extern "C" uint64_t nb_kernel_launches(void) { return g_launches.load(); }
extern "C" const char* nb_version(void) { return "nbgpu 0.1 (sm_103a)"; }

static nb_status check_fit_args(nb_kind kind, const void* X, nb_dtype dtype, int64_t n,
                                int32_t F, int64_t ld, const int32_t* y, int32_t C,
                                const nb_fit_opts* opts) {
  if (kind != NB_MULTINOMIAL && kind != NB_GAUSSIAN) {
    set_error("fit: unknown kind %d", (int)kind);
    return NB_EINVAL;
  }
  if (elem_size(dtype) == 0) {
    set_error("fit: unknown dtype %d", (int)dtype);
    return NB_EINVAL;
  }
  if (C < 2 || C > 255 || F < 1 || n < 0 || ld < F || n > 0x7FFFFFFFLL) {
    set_error("fit: need 2 <= C <= 255, F >= 1, 0 <= n < 2^31, ld >= F (got C=%d F=%d n=%lld "
              "ld=%lld)",
              C, F, (long long)n, (long long)ld);
    return NB_EINVAL;
  }
  if (n > 0 && (!X || !y)) {
    set_error("fit: X and y must be non-NULL when n > 0");
    return NB_EINVAL;
  }
  const double alpha = opts ? opts->alpha : 1.0;
  const double vs = opts ? opts->var_smoothing : 1e-9;
  const double* prior = opts ? opts->log_prior : nullptr;
  const nb_aux* aux = opts ? opts->aux : nullptr;
  if (kind == NB_MULTINOMIAL && !(alpha > 0.0)) {
    set_error("fit: multinomial smoothing alpha must be > 0");
    return NB_EINVAL;
  }
  if (kind == NB_GAUSSIAN) {
    if (dtype != NB_F32) {
      set_error("fit: Gaussian models take F32 features");
      return NB_EINVAL;
    }
    if (C > kTcMaxC) {
      set_error("fit: Gaussian models support C <= %d", kTcMaxC);
      return NB_EUNSUPPORTED;
    }
    if (n < 1 || !(vs >= 0.0)) {
      set_error("fit: Gaussian fit needs n >= 1 and var_smoothing >= 0");
      return NB_EINVAL;
    }
  }
  if (prior) {
    for (int c = 0; c < C; ++c)
      if (!(prior[c] > -1e300 && prior[c] < 1e300)) {
        set_error("fit: log priors must be finite");
        return NB_EINVAL;
      }
  } else if (n == 0) {
    set_error("fit: an empirical prior needs training rows");
    return NB_EINVAL;
  }
  if (dtype == NB_U8 && aux && aux->ovf_ptr && (!aux->ovf_col || !aux->ovf_add)) {
    set_error("fit: overflow list needs ovf_col and ovf_add");
    return NB_EINVAL;
  }
  return NB_OK;
}

// launch the fit of an allocated model; optionally wait and report bad data
static nb_status fit_into(nb_model* m, const void* X, nb_dtype dtype, int64_t n, int64_t ld,
                          const int32_t* y, const double* prior, const nb_aux* aux, int no_sync,
                          cudaStream_t st) {
  // the multinomial fit clears the status word together with its counts
  if (m->kind != NB_MULTINOMIAL)
    NB_TRY_CUDA(cudaMemsetAsync(m->d.status, 0, sizeof(int), st), "memset(status)");
  double* prior_dev = nullptr;
  if (prior) {
    // stage the host priors in the model's own log_pi slot
    NB_TRY_CUDA(cudaMemcpyAsync(m->d.log_pi, prior, sizeof(double) * m->C,
                                cudaMemcpyHostToDevice, st),
                "memcpy(log prior)");
    prior_dev = m->d.log_pi;
  }
  nb_status s;
  if (m->kind == NB_MULTINOMIAL)
    s = launch_fit_multinomial(m, X, dtype, n, ld, y, aux, prior_dev, st);
  else
    s = launch_fit_gaussian(m, static_cast<const float*>(X), n, ld, y, prior_dev, st);
  if (s != NB_OK) return s;
  if (!no_sync) {
    int w = 0;
    NB_TRY_CUDA(cudaMemcpyAsync(&w, m->d.status, sizeof(int), cudaMemcpyDeviceToHost, st),
                "memcpy(status)");
    NB_TRY_CUDA(cudaStreamSynchronize(st), "nb_fit sync");
    return status_from_word(w);
  }
  return NB_OK;
}

extern "C" nb_status nb_fit(nb_kind kind, const void* X, nb_dtype dtype, int64_t n, int32_t F,
                            int64_t ld, const int32_t* y, int32_t C, const nb_fit_opts* opts,
                            void* cuda_stream, nb_model** out) {
  if (!out) {
    set_error("nb_fit: out is NULL");
    return NB_EINVAL;
  }
  *out = nullptr;
  nb_status s = check_fit_args(kind, X, dtype, n, F, ld, y, C, opts);
  if (s != NB_OK) return s;
  const double alpha = opts ? opts->alpha : 1.0;
  const double vs = opts ? opts->var_smoothing : 1e-9;
  const double* prior = opts ? opts->log_prior : nullptr;
  const nb_aux* aux = opts ? opts->aux : nullptr;
  const int no_sync = opts ? opts->no_sync : 0;
  nb_model* m = new (std::nothrow) nb_model();
  if (!m) {
    set_error("nb_fit: out of host memory");
    return NB_ENOMEM;
  }
  m->kind = kind;
  m->C = C;
  m->F = F;
  m->F_pad = (F + 31) / 32 * 32;
  m->nvec8 = m->F_pad / 16;
  m->alpha = alpha;
  m->var_smoothing = vs;
  m->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaGetDevice(&m->device);
  s = alloc_model(m);
  if (s != NB_OK) {
    delete m;
    return s;
  }
  // a Gaussian model may later be re-fitted by nb_refit_gaussian_noalloc,
  // whose fixed scratch is committed on this device now, while allocating is
  // still allowed; if that fails here, that entry point's first call retries
  if (kind == NB_GAUSSIAN && noalloc_scratch_prepare() != NB_OK) cudaGetLastError();
  cudaError_t e = cudaMemsetAsync(m->mem, 0, m->mem_bytes, m->stream);
  if (e == cudaSuccess) s = fit_into(m, X, dtype, n, ld, y, prior, aux, no_sync, m->stream);
  else s = cuda_status(e, "memset(model)");
  if (s != NB_OK) {
    cudaStreamSynchronize(m->stream);
    cudaFree(m->mem);
    delete m;
    return s;
  }
  *out = m;
  return NB_OK;
}

extern "C" nb_status nb_refit(nb_model* m, const void* X, nb_dtype dtype, int64_t n, int64_t ld,
                              const int32_t* y, const nb_fit_opts* opts, void* cuda_stream) {
  if (!m) {
    set_error("nb_refit: NULL model");
    return NB_EINVAL;
  }
  nb_status s = check_fit_args(m->kind, X, dtype, n, m->F, ld, y, m->C, opts);
  if (s != NB_OK) return s;
  if (opts && m->kind == NB_MULTINOMIAL) m->alpha = opts->alpha;
  if (opts && m->kind == NB_GAUSSIAN) m->var_smoothing = opts->var_smoothing;
  m->stream = static_cast<cudaStream_t>(cuda_stream);
  return fit_into(m, X, dtype, n, ld, y, opts ? opts->log_prior : nullptr,
                  opts ? opts->aux : nullptr, opts ? opts->no_sync : 0, m->stream);
}

extern "C" nb_status nb_model_check(const nb_model* m) {
  if (!m) {
    set_error("nb_model_check: NULL model");
    return NB_EINVAL;
  }
  int w[2] = {0, 0};
  cudaError_t e =
      cudaMemcpyAsync(w, m->d.status, 2 * sizeof(int), cudaMemcpyDeviceToHost, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return cuda_status(e, "nb_model_check");
  // the scoring word is reported once: clear it (in stream order) when set
  if (w[1] != 0) {
    e = cudaMemsetAsync(m->d.sstatus, 0, sizeof(int), m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_status(e, "nb_model_check");
  }
  return status_from_word(w[0] | w[1]);
}

extern "C" nb_status nb_model_counts(const nb_model* m, uint64_t* host_counts, uint64_t* host_nc) {
  if (!m) {
    set_error("nb_model_counts: NULL model");
    return NB_EINVAL;
  }
  NB_TRY_CUDA(cudaStreamSynchronize(m->stream), "sync");
  if (host_counts) {
    if (m->kind != NB_MULTINOMIAL) {
      set_error("nb_model_counts: a Gaussian model has no counts");
      return NB_EINVAL;
    }
    NB_TRY_CUDA(cudaMemcpy(host_counts, m->d.counts, sizeof(uint64_t) * m->C * m->F,
                           cudaMemcpyDeviceToHost),
                "memcpy counts");
  }
  if (host_nc)
    NB_TRY_CUDA(cudaMemcpy(host_nc, m->d.nc, sizeof(uint64_t) * m->C, cudaMemcpyDeviceToHost),
                "memcpy nc");
  return NB_OK;
}

extern "C" nb_status nb_model_params(const nb_model* m, double* p0, double* p1, double* log_pi) {
  if (!m) {
    set_error("nb_model_params: NULL model");
    return NB_EINVAL;
  }
  NB_TRY_CUDA(cudaStreamSynchronize(m->stream), "sync");
  const size_t cf = (size_t)m->C * m->F;
  if (p0)
    NB_TRY_CUDA(cudaMemcpy(p0, m->d.p0, sizeof(double) * cf, cudaMemcpyDeviceToHost), "memcpy");
  if (p1) {
    if (m->kind != NB_GAUSSIAN) {
      set_error("nb_model_params: only Gaussian models have variances");
      return NB_EINVAL;
    }
    NB_TRY_CUDA(cudaMemcpy(p1, m->d.p1, sizeof(double) * cf, cudaMemcpyDeviceToHost), "memcpy");
  }
  if (log_pi)
    NB_TRY_CUDA(cudaMemcpy(log_pi, m->d.log_pi, sizeof(double) * m->C, cudaMemcpyDeviceToHost),
                "memcpy");
  return NB_OK;
}

extern "C" nb_status nb_model_info(const nb_model* m, int32_t* kind, int32_t* C, int32_t* F) {
  if (!m) {
    set_error("nb_model_info: NULL model");
    return NB_EINVAL;
  }
  if (kind) *kind = m->kind;
  if (C) *C = m->C;
  if (F) *F = m->F;
  return NB_OK;
}

extern "C" void nb_model_free(nb_model* m) {
  if (!m) return;
  cudaStreamSynchronize(m->stream);
  cudaFree(m->mem);
  delete m;
}

static nb_path score_path(const nb_model* m, const void* X, nb_dtype dtype, int64_t ld,
                          int recheck) {
  const bool aligned = ((reinterpret_cast<uintptr_t>(X) & 15) == 0) &&
                       ((ld * elem_size(dtype)) % 16 == 0);
  if (m->kind == NB_MULTINOMIAL && m->C == 2 && aligned) return NB_PATH_TWO_CLASS;
  if (tc_eligible(m, dtype, X, ld)) return NB_PATH_TENSOR;
  if (dtype == NB_F32 && tcg_eligible(m, X, ld, recheck)) return NB_PATH_TENSOR_GAUSS;
  return NB_PATH_GENERAL;
}

extern "C" int nb_score_path(const nb_model* m, const void* X, nb_dtype dtype, int64_t ld,
                             int recheck) {
  if (!m || recheck < NB_RECHECK_OFF || recheck > NB_RECHECK_LP) {
    set_error("nb_score_path: NULL model or unknown recheck mode");
    return -1;
  }
  return (int)score_path(m, X, dtype, ld, recheck);
}

extern "C" nb_status nb_score_group(const nb_model* m, const void* X, nb_dtype dtype, int64_t n,
                                    int64_t ld, uint8_t* label, float* margin, float* logpost,
                                    const nb_score_opts* opts, void* cuda_stream,
                                    int64_t* n_rechecked) {
  if (!m) {
    set_error("nb_score_group: NULL model");
    return NB_EINVAL;
  }
  if (elem_size(dtype) == 0) {
    set_error("nb_score_group: unknown dtype %d", (int)dtype);
    return NB_EINVAL;
  }
  if (n < 0 || (n > 0 && ld < m->F)) {
    set_error("nb_score_group: need n >= 0 and ld >= F (n=%lld ld=%lld F=%d)", (long long)n,
              (long long)ld, m->F);
    return NB_EINVAL;
  }
  if (n == 0) {
    if (n_rechecked)
      NB_TRY_CUDA(cudaMemsetAsync(n_rechecked, 0, sizeof(int64_t),
                                  static_cast<cudaStream_t>(cuda_stream)),
                  "memset");
    return NB_OK;
  }
  const int want_lp = opts ? opts->want_logpost : 0;
  const int recheck = opts ? (int)opts->recheck : (int)NB_RECHECK_LP;
  const nb_aux* aux = opts ? opts->aux : nullptr;
  if (recheck < NB_RECHECK_OFF || recheck > NB_RECHECK_LP) {
    set_error("nb_score_group: unknown recheck mode %d", recheck);
    return NB_EINVAL;
  }
  if (n > 0 && (!X || !label || !margin || (want_lp && !logpost))) {
    set_error("nb_score_group: X, label, margin (and logpost when requested) must be non-NULL");
    return NB_EINVAL;
  }
  if (dtype == NB_U8 && aux && aux->ovf_ptr && (!aux->ovf_col || !aux->ovf_add)) {
    set_error("nb_score_group: overflow list needs ovf_col and ovf_add");
    return NB_EINVAL;
  }
  if (m->kind == NB_GAUSSIAN && dtype != NB_F32) {
    set_error("nb_score_group: Gaussian models score F32 features");
    return NB_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (n_rechecked) NB_TRY_CUDA(cudaMemsetAsync(n_rechecked, 0, sizeof(int64_t), st), "memset");
  ScoreOut o{label, margin, logpost, n_rechecked, want_lp, recheck};
  nb_status s;
  switch (score_path(m, X, dtype, ld, recheck)) {
    case NB_PATH_TWO_CLASS:
      // the two-class scorers count the rows they mark, so the recheck can
      // skip its scan when there are none
      o.counted = n_rechecked != nullptr;
      s = launch_score2(m, X, dtype, n, ld, aux, o, st);
      break;
    case NB_PATH_TENSOR: s = launch_score_tc(m, X, dtype, n, ld, aux, o, st); break;
    case NB_PATH_TENSOR_GAUSS:
      s = launch_score_tcg(m, static_cast<const float*>(X), n, ld, o, st);
      break;
    default: s = launch_score_general(m, X, dtype, n, ld, aux, o, st); break;
  }
  if (s != NB_OK) return s;
  return launch_recheck(m, X, dtype, n, ld, aux, o, st);
}
