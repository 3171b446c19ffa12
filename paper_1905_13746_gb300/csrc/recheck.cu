// FP64 recheck of marked rows (the fast scorers mark a row by writing the
// reserved label 255 when their rigorous error bound cannot guarantee the
// FP64 decision, or the log posteriors to 1e-5).
//
// A warp scans 32 labels at a time; for every marked row the whole warp
// recomputes the joint log scores from the stored features and the FP64
// tables exactly as defined (Sec. 4):
//   multinomial  s_c = log pi_c + sum_j x_j log theta_cj
//   Gaussian     s_c = log pi_c - 1/2 sum_j [log(2 pi var_cj) + (x_j - mu_cj)^2 / var_cj]
// then the label (lowest index among the maxima), the top-2 margin and the
// log posteriors, in FP64, rounded to FP32 only for the outputs.
#include <cuda_fp16.h>
#include <math.h>

#include "device.cuh"
#include "internal.cuh"

namespace nbg {

struct RArgs {
  const char* X;
  int64_t ld;   // elements
  int64_t n;
  int F, C, kind, dtype;
  const int64_t* ovf_ptr;
  const uint16_t* ovf_col;
  const uint16_t* ovf_add;
  const int8_t* row_exp;
  const double* p0;       // log theta | mu
  const double* p1;       // var
  const double* log_pi;
  const double* gconst;
  uint8_t* label;
  float* margin;
  float* logpost;
  int want_lp;
  unsigned long long* n_rechecked;
};

__device__ __forceinline__ double load_x(const RArgs& a, const char* rp, int j, double scale) {
  switch (a.dtype) {
    case NB_F32: return (double)reinterpret_cast<const float*>(rp)[j];
    case NB_U16: return (double)reinterpret_cast<const uint16_t*>(rp)[j];
    case NB_U8: return (double)reinterpret_cast<const uint8_t*>(rp)[j];
    case NB_BF16: {
      const uint32_t b = reinterpret_cast<const uint16_t*>(rp)[j];
      return (double)__uint_as_float(b << 16);
    }
    default: {
      const uint16_t b = reinterpret_cast<const uint8_t*>(rp)[j];
      return (double)e4m3x2_to_f32(b).x * scale;
    }
  }
}

__global__ void __launch_bounds__(256) k_recheck(const RArgs a) {
  __shared__ double s_sh[8][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * 8;
  const int es = a.dtype == NB_F32 ? 4 : ((a.dtype == NB_U16 || a.dtype == NB_BF16) ? 2 : 1);
  unsigned long long cnt = 0;
  for (int64_t base = ((int64_t)blockIdx.x * 8 + warp) * 32; base < a.n; base += nwarps * 32) {
    const int64_t row = base + lane;
    const bool f = row < a.n && a.label[row] == kLabelRecheck;
    unsigned m = __ballot_sync(0xFFFFFFFFu, f);
    while (m) {
      const int src = __ffs(m) - 1;
      m &= m - 1;
      const int64_t r = base + src;
      const char* rp = a.X + r * a.ld * es;
      const double scale =
          (a.dtype == NB_FP8E4M3 && a.row_exp) ? ldexp(1.0, (int)a.row_exp[r]) : 1.0;
      for (int c = 0; c < a.C; ++c) {
        double acc = 0.0;
        if (a.kind == NB_MULTINOMIAL) {
          const double* lt = a.p0 + (int64_t)c * a.F;
          for (int j = lane; j < a.F; j += 32) acc = fma(load_x(a, rp, j, scale), lt[j], acc);
          if (a.dtype == NB_U8 && a.ovf_ptr) {
            for (int64_t k = a.ovf_ptr[r] + lane; k < a.ovf_ptr[r + 1]; k += 32) {
              const int j = a.ovf_col[k];
              if (j < a.F) acc = fma((double)a.ovf_add[k], lt[j], acc);
            }
          }
        } else {
          const double* mu = a.p0 + (int64_t)c * a.F;
          const double* var = a.p1 + (int64_t)c * a.F;
          for (int j = lane; j < a.F; j += 32) {
            const double dx = load_x(a, rp, j, scale) - mu[j];
            acc += dx * dx / var[j];
          }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, off);
        if (lane == 0)
          s_sh[warp][c] = a.kind == NB_MULTINOMIAL ? a.log_pi[c] + acc : a.gconst[c] - 0.5 * acc;
      }
      __syncwarp();
      if (lane == 0) {
        const double* s = s_sh[warp];
        int best = 0;
        for (int c = 1; c < a.C; ++c)
          if (s[c] > s[best]) best = c;
        double second = -INFINITY;
        for (int c = 0; c < a.C; ++c)
          if (c != best && s[c] > second) second = s[c];
        a.label[r] = (uint8_t)best;
        a.margin[r] = (float)(s[best] - second);
        if (a.want_lp) {
          double sum = 0.0;
          for (int c = 0; c < a.C; ++c) sum += exp(s[c] - s[best]);
          const double lse = s[best] + log(sum);
          for (int c = 0; c < a.C; ++c) a.logpost[r * a.C + c] = (float)(s[c] - lse);
        }
        ++cnt;
      }
      __syncwarp();
    }
  }
  if (lane == 0 && cnt && a.n_rechecked) atomicAdd(a.n_rechecked, cnt);
}

nb_status launch_recheck(const nb_model* m, const void* X, nb_dtype dt, int64_t n, int64_t ld,
                         const nb_aux* aux, const ScoreOut& o, cudaStream_t st) {
  if (n == 0 || o.recheck == NB_RECHECK_OFF) return NB_OK;
  RArgs a{};
  a.X = static_cast<const char*>(X);
  a.ld = ld;
  a.n = n;
  a.F = m->F;
  a.C = m->C;
  a.kind = m->kind;
  a.dtype = dt;
  a.ovf_ptr = aux ? aux->ovf_ptr : nullptr;
  a.ovf_col = aux ? aux->ovf_col : nullptr;
  a.ovf_add = aux ? aux->ovf_add : nullptr;
  a.row_exp = aux ? aux->row_exp : nullptr;
  a.p0 = m->d.p0;
  a.p1 = m->d.p1;
  a.log_pi = m->d.log_pi;
  a.gconst = m->d.gconst;
  a.label = o.label;
  a.margin = o.margin;
  a.logpost = o.logpost;
  a.want_lp = o.want_lp;
  a.n_rechecked = reinterpret_cast<unsigned long long*>(o.n_rechecked);
  const int64_t chunks = (n + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 8;
  count_launch();
  k_recheck<<<(unsigned)(chunks < cap ? chunks : cap), 256, 0, st>>>(a);
  NB_TRY_CUDA(cudaGetLastError(), "k_recheck launch");
  return NB_OK;
}

}  // namespace nbg
