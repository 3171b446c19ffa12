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
#include "seg.cuh"

namespace nbg {

// FP64 tables of one model
struct RModel {
  int kind, C;
  const double* p0;       // log theta | mu
  const double* p1;       // var
  const double* log_pi;
  const double* gconst;
};

// one stored matrix and its outputs
struct RView {
  const char* X;
  int64_t ld;   // elements
  int dtype, F;
  const int64_t* ovf_ptr;
  const uint16_t* ovf_col;
  const uint16_t* ovf_add;
  const int8_t* row_exp;
  uint8_t* label;
  float* margin;
  float* logpost;
  const int32_t* cols;   // feature j is stored column cols[j] (nullptr: column j)
};

__device__ __forceinline__ double load_x(int dtype, const char* rp, int j, double scale) {
  switch (dtype) {
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

// The whole warp recomputes row r of v with model md; lane 0 writes outputs.
// Each lane sums its features j = lane, lane + 32, ... in ascending order for
// eight classes at a time (the row's value loaded once for the eight, eight
// independent FMA chains); a zero count adds nothing to a multinomial score
// (log theta is finite for alpha > 0) and is skipped.  Per class the lane's
// sum and the butterfly over the lanes are those of one class at a time.
__device__ __forceinline__ void recheck_row(const RView& v, const RModel& md, int64_t r,
                                            int want_lp, double* s_sh) {
  const int lane = threadIdx.x & 31;
  const int es = v.dtype == NB_F32 ? 4 : ((v.dtype == NB_U16 || v.dtype == NB_BF16) ? 2 : 1);
  const char* rp = v.X + r * v.ld * es;
  const double scale =
      (v.dtype == NB_FP8E4M3 && v.row_exp) ? ldexp(1.0, (int)v.row_exp[r]) : 1.0;
  constexpr int CB = 8;
  for (int c0 = 0; c0 < md.C; c0 += CB) {
    const int nc = md.C - c0 < CB ? md.C - c0 : CB;
    double acc[CB];
#pragma unroll
    for (int k = 0; k < CB; ++k) acc[k] = 0.0;
    if (md.kind == NB_MULTINOMIAL) {
      const double* lt = md.p0 + (int64_t)c0 * v.F;
      for (int j = lane; j < v.F; j += 32) {
        const double x = load_x(v.dtype, rp, v.cols ? v.cols[j] : j, scale);
        if (x == 0.0) continue;
#pragma unroll
        for (int k = 0; k < CB; ++k)
          if (k < nc) acc[k] = fma(x, lt[(int64_t)k * v.F + j], acc[k]);
      }
      if (v.dtype == NB_U8 && v.ovf_ptr) {
        for (int64_t e = v.ovf_ptr[r] + lane; e < v.ovf_ptr[r + 1]; e += 32) {
          const int j = v.ovf_col[e];
          if (j >= v.F) continue;
          const double add = (double)v.ovf_add[e];
#pragma unroll
          for (int k = 0; k < CB; ++k)
            if (k < nc) acc[k] = fma(add, lt[(int64_t)k * v.F + j], acc[k]);
        }
      }
    } else {
      const double* mu = md.p0 + (int64_t)c0 * v.F;
      const double* var = md.p1 + (int64_t)c0 * v.F;
      for (int j = lane; j < v.F; j += 32) {
        const double x = load_x(v.dtype, rp, j, scale);
#pragma unroll
        for (int k = 0; k < CB; ++k) {
          if (k < nc) {
            const double dx = x - mu[(int64_t)k * v.F + j];
            acc[k] += dx * dx / var[(int64_t)k * v.F + j];
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < CB; ++k) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_xor_sync(0xFFFFFFFFu, acc[k], off);
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < CB; ++k) {
        const int c = c0 + k;
        if (k < nc)
          s_sh[c] = md.kind == NB_MULTINOMIAL ? md.log_pi[c] + acc[k] : md.gconst[c] - 0.5 * acc[k];
      }
    }
  }
  __syncwarp();
  if (lane == 0) {
    int best = 0;
    for (int c = 1; c < md.C; ++c)
      if (s_sh[c] > s_sh[best]) best = c;
    double second = -INFINITY;
    for (int c = 0; c < md.C; ++c)
      if (c != best && s_sh[c] > second) second = s_sh[c];
    v.label[r] = (uint8_t)best;
    v.margin[r] = (float)(s_sh[best] - second);
    if (want_lp) {
      double sum = 0.0;
      for (int c = 0; c < md.C; ++c) sum += exp(s_sh[c] - s_sh[best]);
      const double lse = s_sh[best] + log(sum);
      for (int c = 0; c < md.C; ++c) v.logpost[r * md.C + c] = (float)(s_sh[c] - lse);
    }
  }
  __syncwarp();
}

struct RArgs {
  RView v;
  RModel md;
  int64_t n;
  int want_lp;
  int counted;   // *n_rechecked already holds the marked rows (skip when 0, do not add)
  int rows;      // rows per warp chunk (a power of two <= 32)
  unsigned long long* n_rechecked;
};

__global__ void __launch_bounds__(256) k_recheck(const RArgs a) {
  __shared__ double s_sh[8][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  pdl_wait();   // the scorer's labels and mark count
  if (a.counted && *a.n_rechecked == 0ull) return;   // the scorer marked no row
  // a warp takes chunks of a.rows rows (lanes below a.rows read a label) and
  // recomputes the chunk's marked rows one after another; small calls use short
  // chunks, so that densely marked rows spread over many warps
  const int64_t nwarps = (int64_t)gridDim.x * 8;
  unsigned long long cnt = 0;
  for (int64_t base = ((int64_t)blockIdx.x * 8 + warp) * a.rows; base < a.n;
       base += nwarps * a.rows) {
    const int64_t row = base + lane;
    const bool f = lane < a.rows && row < a.n && a.v.label[row] == kLabelRecheck;
    unsigned m = __ballot_sync(0xFFFFFFFFu, f);
    while (m) {
      const int src = __ffs(m) - 1;
      m &= m - 1;
      recheck_row(a.v, a.md, base + src, a.want_lp, s_sh[warp]);
      ++cnt;
    }
  }
  if (lane == 0 && cnt && a.n_rechecked && !a.counted) atomicAdd(a.n_rechecked, cnt);
}

nb_status launch_recheck(const nb_model* m, const void* X, nb_dtype dt, int64_t n, int64_t ld,
                         const nb_aux* aux, const ScoreOut& o, cudaStream_t st) {
  // NB_RECHECK_OFF still recomputes the rows a scorer could not compute at all
  // (see NB_RECHECK_OFF in the header); in that mode nothing else is marked
  if (n == 0) return NB_OK;
  RArgs a{};
  a.v.X = static_cast<const char*>(X);
  a.v.ld = ld;
  a.v.dtype = dt;
  a.v.F = m->F;
  a.v.ovf_ptr = aux ? aux->ovf_ptr : nullptr;
  a.v.ovf_col = aux ? aux->ovf_col : nullptr;
  a.v.ovf_add = aux ? aux->ovf_add : nullptr;
  a.v.row_exp = aux ? aux->row_exp : nullptr;
  a.v.label = o.label;
  a.v.margin = o.margin;
  a.v.logpost = o.logpost;
  a.md = RModel{m->kind, m->C, m->d.p0, m->d.p1, m->d.log_pi, m->d.gconst};
  a.n = n;
  a.want_lp = o.want_lp;
  a.counted = o.counted ? 1 : 0;
  a.n_rechecked = reinterpret_cast<unsigned long long*>(o.n_rechecked);
  // rows per warp chunk: 32, halved while the call has fewer chunks than the
  // grid has warps (down to one row per warp)
  const int64_t cap = (int64_t)num_sms() * 8;   // blocks of 8 warps
  int rows = 32;
  while (rows > 1 && (n + rows - 1) / rows < cap * 8) rows >>= 1;
  a.rows = rows;
  const int64_t blocks = ((n + rows - 1) / rows + 7) / 8;
  count_launch();
  NB_TRY_CUDA(launch_pdl(k_recheck, dim3((unsigned)(blocks < cap ? blocks : cap)), dim3(256), 0,
                         st, a),
              "k_recheck launch");
  return NB_OK;
}

// ---------------------------------------------------------------------------
// segmented recheck: warps take contiguous ranges of 32-row chunks of a group
// list and walk its groups
// ---------------------------------------------------------------------------
struct RSegArgs {
  const SegGroup* groups;
  const SegHeader* hdr;
  RModel md[kSegMaxModels];
  int dtype, F, want_lp;
  unsigned long long* n_rechecked;
};

__global__ void __launch_bounds__(256) k_recheck_seg(const RSegArgs a) {
  __shared__ double s_sh[8][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n_groups = a.hdr->n_groups;
  const long long chunks = a.hdr->chunks;
  const long long W = (long long)gridDim.x * 8, w = (long long)blockIdx.x * 8 + warp;
  const long long c0 = chunks * w / W, c1 = chunks * (w + 1) / W;
  if (c0 >= c1 || n_groups == 0) return;
  const SegGroup* gr = a.groups;
  int g = seg_find(n_groups, c0, [gr](int i) { return gr[i].chunk0; });
  unsigned long long cnt = 0;
  for (long long c = c0; c < c1; ++c) {
    while (g + 1 < n_groups && gr[g + 1].chunk0 <= c) ++g;
    const SegGroup& G = gr[g];
    const long long base = (c - G.chunk0) * 32;
    const long long row = base + lane;
    const bool f = row < G.n && G.label[row] == kLabelRecheck;
    unsigned m = __ballot_sync(0xFFFFFFFFu, f);
    if (!m) continue;
    RView v;
    v.cols = nullptr;
    v.X = G.X;
    v.dtype = a.dtype;
    v.F = a.F;
    const int es = a.dtype == NB_F32 ? 4 : ((a.dtype == NB_U16 || a.dtype == NB_BF16) ? 2 : 1);
    v.ld = G.ld_bytes / es;
    v.ovf_ptr = G.ovf_ptr;
    v.ovf_col = G.ovf_col;
    v.ovf_add = G.ovf_add;
    v.row_exp = G.row_exp;
    v.label = G.label;
    v.margin = G.margin;
    v.logpost = G.logpost;
    while (m) {
      const int src = __ffs(m) - 1;
      m &= m - 1;
      recheck_row(v, a.md[G.model], base + src, a.want_lp, s_sh[warp]);
      ++cnt;
    }
  }
  if (lane == 0 && cnt && a.n_rechecked) atomicAdd(a.n_rechecked, cnt);
}

nb_status launch_recheck_seg(const SegGroup* groups, const SegHeader* hdr,
                             const nb_model* const* models, int n_models, nb_dtype dt, int F,
                             int want_lp, int64_t* n_rechecked, cudaStream_t st) {
  RSegArgs a{};
  a.groups = groups;
  a.hdr = hdr;
  for (int i = 0; i < n_models && i < kSegMaxModels; ++i) {
    const nb_model* m = models[i];
    a.md[i] = RModel{m->kind, m->C, m->d.p0, m->d.p1, m->d.log_pi, m->d.gconst};
  }
  a.dtype = dt;
  a.F = F;
  a.want_lp = want_lp;
  a.n_rechecked = reinterpret_cast<unsigned long long*>(n_rechecked);
  count_launch();
  k_recheck_seg<<<num_sms() * 4, 256, 0, st>>>(a);
  NB_TRY_CUDA(cudaGetLastError(), "k_recheck_seg launch");
  return NB_OK;
}

}  // namespace nbg

namespace nbg {

// ---------------------------------------------------------------------------
// group-wise recheck: rows in the files' order, each with the model of its
// size group and that model's opcode selection (feature t = column cols[t] of
// the full histogram), the arithmetic of recheck_row unchanged
// ---------------------------------------------------------------------------
struct RGwArgs {
  const unsigned char* X;
  int64_t ld;
  int64_t n;
  const int64_t* sizes;
  int64_t bin_bytes;
  int n_bins, k;
  const int32_t* model_of;   // size group -> model slot
  const int32_t* cols;       // n_models x k
  RModel md[kSegMaxModels];
  uint8_t* label;
  float* margin;
  float* logpost;
  int want_lp;
  int counted;   // *n_rechecked already holds the marked rows (skip when 0, do not add)
  unsigned long long* n_rechecked;
};

__global__ void __launch_bounds__(256) k_recheck_gw(const RGwArgs a) {
  __shared__ double s_sh[8][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  pdl_wait();   // the scorer's labels and mark count
  if (a.counted && *a.n_rechecked == 0ull) return;   // the scorer marked no row
  const int64_t nwarps = (int64_t)gridDim.x * 8;
  unsigned long long cnt = 0;
  for (int64_t base = ((int64_t)blockIdx.x * 8 + warp) * 32; base < a.n; base += nwarps * 32) {
    const int64_t row = base + lane;
    const bool f = row < a.n && a.label[row] == kLabelRecheck;
    unsigned m = __ballot_sync(0xFFFFFFFFu, f);
    while (m) {
      const int src = __ffs(m) - 1;
      m &= m - 1;
      const int64_t r = base + src;
      long long sz = a.sizes[r];
      sz = sz < 0 ? 0 : sz;
      long long bin = sz / a.bin_bytes;
      if (bin > a.n_bins - 1) bin = a.n_bins - 1;
      const int g = a.model_of[bin];
      RView v;
      v.X = reinterpret_cast<const char*>(a.X);
      v.ld = a.ld;
      v.dtype = NB_U8;
      v.F = a.k;
      v.ovf_ptr = nullptr;
      v.ovf_col = nullptr;
      v.ovf_add = nullptr;
      v.row_exp = nullptr;
      v.label = a.label;
      v.margin = a.margin;
      v.logpost = a.logpost;
      v.cols = a.cols + (int64_t)g * a.k;
      recheck_row(v, a.md[g], r, a.want_lp, s_sh[warp]);
      ++cnt;
    }
  }
  if (lane == 0 && cnt && a.n_rechecked && !a.counted) atomicAdd(a.n_rechecked, cnt);
}

nb_status launch_recheck_gw(const unsigned char* X, int64_t ld, int64_t n, const int64_t* sizes,
                            int64_t bin_bytes, int n_bins, int k, const int32_t* model_of,
                            const int32_t* cols, const nb_model* const* models, int n_models,
                            uint8_t* label, float* margin, float* logpost, int want_lp,
                            int64_t* n_rechecked, bool counted, cudaStream_t st) {
  if (n == 0) return NB_OK;
  RGwArgs a{};
  a.X = X;
  a.ld = ld;
  a.n = n;
  a.sizes = sizes;
  a.bin_bytes = bin_bytes;
  a.n_bins = n_bins;
  a.k = k;
  a.model_of = model_of;
  a.cols = cols;
  for (int i = 0; i < n_models && i < kSegMaxModels; ++i) {
    const nb_model* m = models[i];
    a.md[i] = RModel{m->kind, m->C, m->d.p0, m->d.p1, m->d.log_pi, m->d.gconst};
  }
  a.label = label;
  a.margin = margin;
  a.logpost = logpost;
  a.want_lp = want_lp;
  a.counted = counted ? 1 : 0;
  a.n_rechecked = reinterpret_cast<unsigned long long*>(n_rechecked);
  const int64_t chunks = (n + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 8;
  count_launch();
  NB_TRY_CUDA(launch_pdl(k_recheck_gw, dim3((unsigned)(chunks < cap ? chunks : cap)), dim3(256),
                         0, st, a),
              "k_recheck_gw launch");
  return NB_OK;
}

}  // namespace nbg
