// Allocation-free Gaussian re-fit.
//
// nb_refit on a Gaussian model takes its per-chunk partial sums from
// stream-ordered scratch (cudaMallocAsync / cudaFreeAsync).  Some callers
// cannot allocate device memory at the point where they re-train: a thread
// bound to a fixed memory budget whose pool must not grow, code running
// between the instantiation and the replays of a CUDA graph, or an embedded
// runtime that forbids allocation after start-up.  nb_refit_gaussian_noalloc
// does the same work with the partials in a file-scope device array instead,
// so the call itself allocates nothing.
//
// The array holds kScratchDoubles doubles (8 MiB).  It lives in this file's
// own device module, which the CUDA runtime loads on a device when the
// library first asks for the array's address there (with lazy module loading,
// the default, not when the library is loaded): nb_fit asks when it creates a
// Gaussian model, and so does the first call of this entry point on a device
// where that has not happened.  From then on the 8 MiB stay committed on that
// device until the process exits.  The address is looked up once per device.
// All calls share the one array and each leaves its partials there: calls
// that overlap on the GPU (different streams, no ordering between them) race
// on it.  Every value a call reads from the array is first written by the
// same call, so nothing has to be cleared between calls.
#include <mutex>

#include "internal.cuh"

namespace nbg {

constexpr size_t kScratchDoubles = size_t(1) << 20;   // 8 MiB

static __device__ __align__(256) double g_refit_scratch[kScratchDoubles];

static std::mutex g_scratch_mu;
static double* g_scratch_ptr[64] = {nullptr};

// Device address of the array for the current device (looked up once).
static nb_status scratch_for_current_device(double** out) {
  int dev = 0;
  NB_TRY_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= 64) {
    set_error("nb_refit_gaussian_noalloc: device index %d out of range", dev);
    return NB_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    NB_TRY_CUDA(cudaGetSymbolAddress(&p, g_refit_scratch), "cudaGetSymbolAddress");
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return NB_OK;
}

nb_status noalloc_scratch_prepare() {
  double* p = nullptr;
  return scratch_for_current_device(&p);
}

}  // namespace nbg

using namespace nbg;

extern "C" nb_status nb_refit_gaussian_noalloc(nb_model* m, const float* X, int64_t n,
                                               int64_t ld, const int32_t* y,
                                               const nb_fit_opts* opts, void* cuda_stream) {
  if (!m || m->kind != NB_GAUSSIAN) {
    set_error("nb_refit_gaussian_noalloc: needs a Gaussian model");
    return NB_EINVAL;
  }
  const int C = m->C, F = m->F, S = C + 1;
  if (n < 1 || ld < F || !X || !y) {
    set_error("nb_refit_gaussian_noalloc: need n >= 1, ld >= F and non-NULL X, y");
    return NB_EINVAL;
  }
  const double vs = opts ? opts->var_smoothing : m->var_smoothing;
  const double* prior = opts ? opts->log_prior : nullptr;
  if (!(vs >= 0.0)) {
    set_error("nb_refit_gaussian_noalloc: var_smoothing must be >= 0");
    return NB_EINVAL;
  }
  if (prior)
    for (int c = 0; c < C; ++c)
      if (!(prior[c] > -1e300 && prior[c] < 1e300)) {
        set_error("nb_refit_gaussian_noalloc: log priors must be finite");
        return NB_EINVAL;
      }
  // the same row chunks as nb_refit, so the partial sums and their order match
  const int64_t chunk_rows = gauss_chunk_rows(n);
  const long long nchunk = (n + chunk_rows - 1) / chunk_rows;
  const size_t need = (size_t)nchunk * S * F + 2 * (size_t)F;
  if (need > kScratchDoubles) {
    set_error("nb_refit_gaussian_noalloc: ceil(n/%lld)*(C+1)*F + 2F = %zu doubles exceeds the "
              "fixed scratch of %zu doubles; use nb_refit",
              (long long)chunk_rows, need, kScratchDoubles);
    return NB_EINVAL;
  }
  double* scratch = nullptr;
  nb_status s = scratch_for_current_device(&scratch);
  if (s != NB_OK) return s;

  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  m->var_smoothing = vs;
  m->stream = st;
  ModelDev& d = m->d;
  double* partial = scratch;
  double* mu_all = partial + (size_t)nchunk * S * F;
  double* m2_all = mu_all + F;
  NB_TRY_CUDA(cudaMemsetAsync(d.status, 0, sizeof(int), st), "memset(status)");
  NB_TRY_CUDA(cudaMemsetAsync(d.nc, 0, sizeof(uint64_t) * C, st), "memset(nc)");
  if (prior)
    NB_TRY_CUDA(cudaMemcpyAsync(d.log_pi, prior, sizeof(double) * C, cudaMemcpyHostToDevice, st),
                "memcpy(log prior)");
  const int sms = num_sms();
  const long long g = (n + 255) / 256;
  count_launch();
  k_label_hist<<<(unsigned)(g < sms * 4 ? g : sms * 4), 256, 0, st>>>(
      y, n, C, reinterpret_cast<unsigned long long*>(d.nc), d.status);
  NB_TRY_CUDA(cudaGetLastError(), "k_label_hist");
  const int tile = gauss_tile(C);
  const int smem = (int)(sizeof(double) * 8 * S * tile);
  if (smem > kSmemOptIn)
    NB_TRY_CUDA(cudaFuncSetAttribute(k_gauss_partial, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     smem),
                "cudaFuncSetAttribute");
  const dim3 grid((unsigned)nchunk, (F + tile - 1) / tile);
  const int rb = (S * F + 255) / 256;
  for (int pass = 0; pass < 2; ++pass) {
    count_launch();
    k_gauss_partial<<<grid, 256, smem, st>>>(X, ld, n, F, C, y, pass, d.p0, mu_all, partial,
                                             chunk_rows, tile, d.status);
    NB_TRY_CUDA(cudaGetLastError(), "k_gauss_partial");
    count_launch();
    k_gauss_reduce<<<rb < 1024 ? rb : 1024, 256, 0, st>>>(
        partial, (int)nchunk, F, C, reinterpret_cast<unsigned long long*>(d.nc), n, pass, d.p0,
        mu_all, d.p1, m2_all);
    NB_TRY_CUDA(cudaGetLastError(), "k_gauss_reduce");
  }
  count_launch();
  k_gauss_finalize<<<1, 256, 0, st>>>(m2_all, F, m->F_pad, C, vs,
                                       reinterpret_cast<unsigned long long*>(d.nc), n,
                                       prior != nullptr, d.p0, d.p1, d.log_pi, d.gconst, d.g_mu,
                                       d.g_ivar, d.g_const, d.status);
  NB_TRY_CUDA(cudaGetLastError(), "k_gauss_finalize");
  if (d.tcg_kc) {
    s = launch_derive_tcg(m, st);
    if (s != NB_OK) return s;
  }
  if (!(opts && opts->no_sync)) {
    int w = 0;
    NB_TRY_CUDA(cudaMemcpyAsync(&w, d.status, sizeof(int), cudaMemcpyDeviceToHost, st),
                "memcpy(status)");
    NB_TRY_CUDA(cudaStreamSynchronize(st), "sync");
    return status_from_word(w);
  }
  return NB_OK;
}
