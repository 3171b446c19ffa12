// Naive Bayes fit on the GPU (Sec. 4, "trained the model").
//
// Multinomial (count features, Sec. 3):
//   n_c  = #{i : y_i = c}                 label histogram
//   N_cj = sum_{i : y_i = c} x_ij          exact, uint64
//   log theta_cj = log(N_cj + alpha) - log(N_c + alpha F)       FP64
//   log pi_c = log n_c - log n  (or the supplied log prior)     FP64
// The count reduction first buckets the row indices by class, so that a warp
// sums runs of rows of one class in registers and adds each feature's total
// to N_cj with one 64-bit atomic per run; integer sums do not depend on the
// order of the additions, so the counts are exact and reproducible.
//
// Gaussian (real-valued features): per-class means and maximum-likelihood
// variances in FP64 by two passes (mean, then squared deviations about it),
// each pass as fixed per-chunk partial sums reduced in a fixed order, so the
// result is bit-reproducible.  eps = var_smoothing * max_j Var(x_.j).
#include <cuda_fp16.h>
#include <math.h>

#include "device.cuh"
#include "internal.cuh"

namespace nbg {

constexpr int kRunRows = 128;     // rows per class run (bounds the 16/32-bit sums)

// ---------------------------------------------------------------------------
// label histogram (+ validation)
// ---------------------------------------------------------------------------
__global__ void k_label_hist(const int32_t* y, int64_t n, int C, unsigned long long* nc,
                             int* status) {
  __shared__ unsigned int h[256];
  for (int c = threadIdx.x; c < C; c += blockDim.x) h[c] = 0;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = y[i];
    if (c < 0 || c >= C)
      atomicOr(status, ST_BAD_LABEL);
    else
      atomicAdd(&h[c], 1u);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x)
    if (h[c]) atomicAdd(&nc[c], (unsigned long long)h[c]);
}

// offsets of the class buckets and of their run items (one block)
__global__ void k_bucket_setup(const unsigned long long* nc, int C, long long* offs,
                               unsigned long long* cursor, long long* item_base) {
  if (threadIdx.x == 0) {
    long long o = 0, it = 0;
    for (int c = 0; c < C; ++c) {
      offs[c] = o;
      cursor[c] = (unsigned long long)o;
      item_base[c] = it;
      o += (long long)nc[c];
      it += ((long long)nc[c] + kRunRows - 1) / kRunRows;
    }
    offs[C] = o;
    item_base[C] = it;
  }
}

// scatter row indices into their class bucket (block-aggregated reservations)
__global__ void k_bucket_scatter(const int32_t* y, int64_t n, int C, unsigned long long* cursor,
                                 int32_t* idx) {
  __shared__ unsigned int cnt[256];
  __shared__ unsigned long long base[256];
  const int64_t chunk = (int64_t)blockDim.x * 16;
  for (int64_t c0 = (int64_t)blockIdx.x * chunk; c0 < n; c0 += (int64_t)gridDim.x * chunk) {
    for (int c = threadIdx.x; c < C; c += blockDim.x) cnt[c] = 0;
    __syncthreads();
    int mycls[16];
    unsigned int myrank[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int64_t i = c0 + (int64_t)k * blockDim.x + threadIdx.x;
      mycls[k] = -1;
      if (i < n) {
        const int c = y[i];
        if (c >= 0 && c < C) {
          mycls[k] = c;
          myrank[k] = atomicAdd(&cnt[c], 1u);
        }
      }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x)
      base[c] = cnt[c] ? atomicAdd(&cursor[c], (unsigned long long)cnt[c]) : 0ull;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int64_t i = c0 + (int64_t)k * blockDim.x + threadIdx.x;
      if (mycls[k] >= 0) idx[base[mycls[k]] + myrank[k]] = (int32_t)i;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// dense counts: one warp = one class run (<= kRunRows rows) x one 1 KB slab
// ---------------------------------------------------------------------------
struct CountArgs {
  const char* X;
  int64_t ld_bytes;
  int F;
  int nvec_row;
  int nslab;
  int C;
  const int32_t* idx;
  const long long* offs;
  const long long* item_base;
  const unsigned long long* nc;
  const int8_t* row_exp;
  unsigned long long* counts;
  int* status;
};

__device__ __forceinline__ int find_class(const long long* item_base, int C, long long t) {
  int lo = 0, hi = C;  // item_base[lo] <= t < item_base[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (item_base[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

template <int DT>
struct CountDec;

// u8: packed 16-bit lanes, even and odd bytes of each word
template <>
struct CountDec<NB_U8> {
  static constexpr int EPV = 16, NACC = 8;
  __device__ __forceinline__ static void add(const uint4& x, uint32_t* acc, int8_t, int*) {
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      acc[2 * k] += w[k] & 0x00FF00FFu;
      acc[2 * k + 1] += (w[k] >> 8) & 0x00FF00FFu;
    }
  }
  __device__ __forceinline__ static uint32_t get(const uint32_t* acc, int e) {
    const int k = e >> 2, b = e & 3;
    const uint32_t a = acc[2 * k + (b & 1)];
    return (b >> 1) ? (a >> 16) : (a & 0xFFFFu);
  }
};
template <>
struct CountDec<NB_U16> {
  static constexpr int EPV = 8, NACC = 8;
  __device__ __forceinline__ static void add(const uint4& x, uint32_t* acc, int8_t, int*) {
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      acc[2 * k] += w[k] & 0xFFFFu;
      acc[2 * k + 1] += w[k] >> 16;
    }
  }
  __device__ __forceinline__ static uint32_t get(const uint32_t* acc, int e) { return acc[e]; }
};

__device__ __forceinline__ uint32_t checked_count(float v, int* status) {
  if (!(v >= 0.f) || v != floorf(v) || v >= 16777216.f) {
    atomicOr(status, ST_BAD_VALUE);
    return 0u;
  }
  return (uint32_t)v;
}

template <>
struct CountDec<NB_F32> {
  static constexpr int EPV = 4, NACC = 4;
  __device__ __forceinline__ static void add(const uint4& x, uint32_t* acc, int8_t, int* st) {
    acc[0] += checked_count(__uint_as_float(x.x), st);
    acc[1] += checked_count(__uint_as_float(x.y), st);
    acc[2] += checked_count(__uint_as_float(x.z), st);
    acc[3] += checked_count(__uint_as_float(x.w), st);
  }
  __device__ __forceinline__ static uint32_t get(const uint32_t* acc, int e) { return acc[e]; }
};
template <>
struct CountDec<NB_BF16> {
  static constexpr int EPV = 8, NACC = 8;
  __device__ __forceinline__ static void add(const uint4& x, uint32_t* acc, int8_t, int* st) {
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      acc[2 * k] += checked_count(__uint_as_float(w[k] << 16), st);
      acc[2 * k + 1] += checked_count(__uint_as_float(w[k] & 0xFFFF0000u), st);
    }
  }
  __device__ __forceinline__ static uint32_t get(const uint32_t* acc, int e) { return acc[e]; }
};
template <>
struct CountDec<NB_FP8E4M3> {
  static constexpr int EPV = 16, NACC = 16;
  __device__ __forceinline__ static void add(const uint4& x, uint32_t* acc, int8_t e, int* st) {
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
    const float sc = exp2f((float)e);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 lo = e4m3x2_to_f32((uint16_t)(w[k] & 0xFFFFu));
      const float2 hi = e4m3x2_to_f32((uint16_t)(w[k] >> 16));
      acc[4 * k] += checked_count(lo.x * sc, st);
      acc[4 * k + 1] += checked_count(lo.y * sc, st);
      acc[4 * k + 2] += checked_count(hi.x * sc, st);
      acc[4 * k + 3] += checked_count(hi.y * sc, st);
    }
  }
  __device__ __forceinline__ static uint32_t get(const uint32_t* acc, int e) { return acc[e]; }
};

template <int DT>
__global__ void __launch_bounds__(256) k_counts(const CountArgs a, long long nwork) {
  using Dec = CountDec<DT>;
  constexpr int NV = 2;   // 16-byte vectors per lane per row -> 1 KB slab per warp
  const int lane = threadIdx.x & 31;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long wk = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); wk < nwork;
       wk += nwarps) {
    const long long item = wk / a.nslab;
    const int slab = (int)(wk % a.nslab);
    const int c = find_class(a.item_base, a.C, item);
    const long long p0 = a.offs[c] + (item - a.item_base[c]) * kRunRows;
    long long p1 = p0 + kRunRows;
    if (p1 > a.offs[c + 1]) p1 = a.offs[c + 1];
    uint32_t acc[NV][Dec::NACC];
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
      for (int e = 0; e < Dec::NACC; ++e) acc[k][e] = 0;
    int vv[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) vv[k] = slab * 32 * NV + k * 32 + lane;
    // the run's row indices, lane l holding positions p0 + l + 32 i
    const int cnt = (int)(p1 - p0);   // <= kRunRows
    int ridx[kRunRows / 32];
#pragma unroll
    for (int i = 0; i < kRunRows / 32; ++i) {
      const int q = lane + 32 * i;
      ridx[i] = q < cnt ? a.idx[p0 + q] : 0;
    }
    // zero the padding beyond F in a partial last vector (never counted)
    uint32_t wmask[NV][4];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const int base = vv[k] * Dec::EPV;
      const int esz = 16 / Dec::EPV;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int valid = (a.F - base) * esz - 4 * q;   // valid bytes in word q
        valid = valid < 0 ? 0 : (valid > 4 ? 4 : valid);
        wmask[k][q] = valid >= 4 ? 0xFFFFFFFFu : ((1u << (8 * valid)) - 1u);
      }
    }
    constexpr int U = 8;   // rows in flight per lane
    for (int r0 = 0; r0 < cnt; r0 += U) {
      uint4 x[U][NV];
      int8_t ex[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int r = r0 + u;
        const int src = r & 31, slot = r >> 5;
        int row = ridx[0];
#pragma unroll
        for (int i = 1; i < kRunRows / 32; ++i) row = slot == i ? ridx[i] : row;
        row = __shfl_sync(0xFFFFFFFFu, row, src);
        const char* rp = a.X + (int64_t)row * a.ld_bytes;
        ex[u] = (DT == NB_FP8E4M3 && a.row_exp && r < cnt) ? a.row_exp[row] : (int8_t)0;
#pragma unroll
        for (int k = 0; k < NV; ++k)
          x[u][k] = (r < cnt && vv[k] < a.nvec_row) ? ld_stream16(rp + (int64_t)vv[k] * 16)
                                                   : make_uint4(0, 0, 0, 0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          if (vv[k] < a.nvec_row && r0 + u < cnt) {
            x[u][k].x &= wmask[k][0];
            x[u][k].y &= wmask[k][1];
            x[u][k].z &= wmask[k][2];
            x[u][k].w &= wmask[k][3];
            Dec::add(x[u][k], acc[k], ex[u], a.status);
          }
        }
      }
    }
    unsigned long long* out = a.counts + (long long)c * a.F;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      if (vv[k] >= a.nvec_row) continue;
      const int base = vv[k] * Dec::EPV;
#pragma unroll
      for (int e = 0; e < Dec::EPV; ++e) {
        const uint32_t v = Dec::get(acc[k], e);
        if (v && base + e < a.F) atomicAdd(&out[base + e], (unsigned long long)v);
      }
    }
  }
}

// Any alignment: one thread per (class run, feature), scalar loads.
__device__ __forceinline__ uint32_t load_count(int dt, const char* rp, int j, int8_t e,
                                               int* status) {
  switch (dt) {
    case NB_U8: return reinterpret_cast<const uint8_t*>(rp)[j];
    case NB_U16: return reinterpret_cast<const uint16_t*>(rp)[j];
    case NB_F32: return checked_count(reinterpret_cast<const float*>(rp)[j], status);
    case NB_BF16:
      return checked_count(
          __uint_as_float((uint32_t)reinterpret_cast<const uint16_t*>(rp)[j] << 16), status);
    default:
      return checked_count(
          e4m3x2_to_f32((uint16_t)reinterpret_cast<const uint8_t*>(rp)[j]).x * exp2f((float)e),
          status);
  }
}

__global__ void k_counts_scalar(const CountArgs a, int dt, int esize, long long nwork) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nwork;
       t += (long long)gridDim.x * blockDim.x) {
    const long long item = t / a.F;
    const int j = (int)(t % a.F);
    const int c = find_class(a.item_base, a.C, item);
    const long long p0 = a.offs[c] + (item - a.item_base[c]) * kRunRows;
    long long p1 = p0 + kRunRows;
    if (p1 > a.offs[c + 1]) p1 = a.offs[c + 1];
    unsigned long long s = 0;
    for (long long p = p0; p < p1; ++p) {
      const int64_t row = a.idx[p];
      const int8_t e = (dt == NB_FP8E4M3 && a.row_exp) ? a.row_exp[row] : (int8_t)0;
      s += load_count(dt, a.X + row * a.ld_bytes, j, e, a.status);
    }
    if (s) atomicAdd(&a.counts[(long long)c * a.F + j], s);
  }
  (void)esize;
}

// overflow entries of u8 storage: (class, column) histogram, shared memory
// bins when C*F fits, else direct 64-bit atomics
__global__ void k_counts_ovf(const int64_t* ptr, const uint16_t* col, const uint16_t* add,
                             const int32_t* y, int64_t n, int F, int C, int use_smem,
                             unsigned long long* counts, int* status) {
  extern __shared__ unsigned int bins[];
  const int nb = use_smem ? C * F : 0;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) bins[k] = 0;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = y[i];
    if (c < 0 || c >= C) continue;
    for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
      const uint32_t j = col[k];
      if (j >= (uint32_t)F) {
        atomicOr(status, ST_OVF_RANGE);
        continue;
      }
      if (use_smem)
        atomicAdd(&bins[c * F + j], (unsigned int)add[k]);
      else
        atomicAdd(&counts[(int64_t)c * F + j], (unsigned long long)add[k]);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nb; k += blockDim.x)
    if (bins[k]) atomicAdd(&counts[k], (unsigned long long)bins[k]);
}

// ---------------------------------------------------------------------------
// FP64 finalize of the general-C tables
// ---------------------------------------------------------------------------
// General-C finish (Sec. 4 likelihoods, Laplace smoothing): block (c, t)
// writes log theta_cj for the kFinTile features of tile t.  Every block sums
// the class total N_c from the exact counts (they sit in L2) and one thread
// takes log(N_c + alpha F): FP64 is slow on this part, so the per-feature
// logs are spread over C * F / kFinTile blocks rather than C.
constexpr int kFinTile = 512;

__global__ void __launch_bounds__(256) k_finalize_mn(const unsigned long long* counts,
                                                     const unsigned long long* nc, int64_t n,
                                                     int F, double alpha, int prior_given,
                                                     double* log_theta, double* log_pi,
                                                     int* status) {
  const int c = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ unsigned long long part[8];
  __shared__ double log_den;
  unsigned long long s = 0;
  for (int j = tid; j < F; j += blockDim.x) s += counts[(int64_t)c * F + j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
  if (lane == 0) part[warp] = s;
  __syncthreads();
  if (tid == 0) {
    unsigned long long t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += part[k];
    log_den = log((double)t + alpha * (double)F);
    if (blockIdx.y == 0 && !prior_given) {
      if (nc[c] == 0) {
        atomicOr(status, ST_BAD_LABEL);
        log_pi[c] = 0.0;
      } else {
        log_pi[c] = log((double)nc[c]) - log((double)n);
      }
    }
  }
  __syncthreads();
  const int j0 = blockIdx.y * kFinTile;
  const int j1 = min(F, j0 + kFinTile);
  for (int j = j0 + tid; j < j1; j += blockDim.x)
    log_theta[(int64_t)c * F + j] = log((double)counts[(int64_t)c * F + j] + alpha) - log_den;
}

// two-class tables: Delta (FP64 -> FP32, fixed point + limbs), b, interleaved
// copies for the scorer's 16-byte vectors.  One block.
__global__ void __launch_bounds__(1024) k_derive_c2(const double* log_theta, const double* log_pi,
                                                    int F, int F_pad, int nvec8, C2Header* hdr,
                                                    float* delta, int32_t* delta_q, uint4* limbs,
                                                    float4* il4, float4* il8, float4* il16,
                                                    int* status) {
  __shared__ double red[1024];
  double mx = 0.0;
  for (int j = threadIdx.x; j < F; j += blockDim.x) {
    const double d = log_theta[F + j] - log_theta[j];
    mx = fmax(mx, fabs(d));
    if (!isfinite(d)) atomicOr(status, ST_BAD_TABLE);
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  const double maxabs64 = red[0];
  int S = 0;
  if (maxabs64 > 0.0) {
    int e;
    frexp(maxabs64, &e);   // maxabs64 < 2^e
    S = 22 - e;
  }
  const double scale = ldexp(1.0, S);
  float mx32 = 0.f;
  for (int j = threadIdx.x; j < F_pad; j += blockDim.x) {
    const double d = j < F ? log_theta[F + j] - log_theta[j] : 0.0;
    const float d32 = (float)d;
    mx32 = fmaxf(mx32, fabsf(d32));
    delta[j] = d32;
    const int32_t q = (int32_t)llrint(d * scale);   // |q| <= 2^22
    delta_q[j] = q;
    // balanced base-256 digits q = q2*65536 + q1*256 + q0, each in [-128, 127]
    const int32_t q0 = ((q + 128) & 255) - 128;
    const int32_t r1 = (q - q0) >> 8;
    const int32_t q1 = ((r1 + 128) & 255) - 128;
    const int32_t q2 = (r1 - q1) >> 8;
    // u8 vectors hold 16 features; limb L of vector v is slot L * nvec8 + v,
    // byte (j % 16) of it
    const int v = j >> 4, b = j & 15;
    unsigned char* L = reinterpret_cast<unsigned char*>(limbs);
    L[((size_t)0 * nvec8 + v) * 16 + b] = (unsigned char)(q0 & 255);
    L[((size_t)1 * nvec8 + v) * 16 + b] = (unsigned char)(q1 & 255);
    L[((size_t)2 * nvec8 + v) * 16 + b] = (unsigned char)(q2 & 255);
    // the same limbs packed into one word per feature (overflow entries)
    reinterpret_cast<uint32_t*>(L + (size_t)3 * F_pad)[j] =
        (uint32_t)(q0 & 255) | ((uint32_t)(q1 & 255) << 8) | ((uint32_t)(q2 & 255) << 16);
    // FP32 tables for 4 / 8 / 16 elements per vector: quad q of vector v is
    // slot q * (F_pad / EPV) + v
    {
      float* t = reinterpret_cast<float*>(il4);
      const int epv = 4, vv = j / epv, e = j % epv;
      t[((size_t)(e >> 2) * (F_pad / epv) + vv) * 4 + (e & 3)] = d32;
    }
    {
      float* t = reinterpret_cast<float*>(il8);
      const int epv = 8, vv = j / epv, e = j % epv;
      t[((size_t)(e >> 2) * (F_pad / epv) + vv) * 4 + (e & 3)] = d32;
    }
    {
      float* t = reinterpret_cast<float*>(il16);
      const int epv = 16, vv = j / epv, e = j % epv;
      t[((size_t)(e >> 2) * (F_pad / epv) + vv) * 4 + (e & 3)] = d32;
    }
  }
  __shared__ float redf[1024];
  redf[threadIdx.x] = mx32;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) redf[threadIdx.x] = fmaxf(redf[threadIdx.x], redf[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double b = log_pi[1] - log_pi[0];
    hdr->b = (float)b;
    hdr->b64 = b;
    hdr->maxabs = redf[0];
    hdr->S = S;
    hdr->inv_scale = (float)ldexp(1.0, -S);
    hdr->maxabs_q = (float)maxabs64;
    hdr->pad = 0;
  }
}

// Two-class finish of the fit in one launch (Sec. 4 likelihoods, Laplace
// smoothing).  FP64 is slow on this part and the kernel is one chain of
// latencies, so the work is spread thin and overlapped: a block of 4 kFinF
// threads owns kFinF features; half of its threads take one log(n_cj + alpha)
// each while the other half sum the class totals N_0, N_1 from the exact
// counts and take log(N_c + alpha F) (and, in block 0, log pi_c).  Then one
// thread per feature forms Delta = log theta_1 - log theta_0, its FP32 copies
// and the centred weights of the general-C tables (w_c = log theta_c - mean).
// The blocks' maxima of |Delta| meet in fin[], and the last block to finish
// derives the fixed-point scale S and writes the integer Delta and its limbs.
// fin[] (zero before the launch) is cleared again by that block.
constexpr int kFinF = 64;          // features per block
constexpr int kFinT = 4 * kFinF;   // threads per block

__global__ void __launch_bounds__(kFinT) k_fit_finish_c2(
    const unsigned long long* counts, const unsigned long long* nc, int64_t n, int F, int F_pad,
    int nvec8, double alpha, int prior_given, double* log_theta, double* log_pi, C2Header* hdr,
    float* delta, int32_t* delta_q, uint4* limbs, float4* il4, float4* il8, float4* il16,
    float* w, float* bias, float* wmax, unsigned long long* fin, int* status) {
  constexpr int NT = kFinT, NL = 2 * kFinF;   // NL threads take the per-feature logs
  __shared__ unsigned long long part[2][2];
  __shared__ double ld[2];
  __shared__ double lt[2][kFinF];
  __shared__ double dmax[kFinF / 32];
  __shared__ float fmax32[kFinF / 32], wm32[kFinF / 32];
  __shared__ int last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  pdl_wait();   // the counting kernels' totals
  double lc = 0.0;
  if (tid < NL) {
    const int c = tid / kFinF, j = blockIdx.x * kFinF + tid % kFinF;
    if (j < F) lc = log((double)counts[(int64_t)c * F + j] + alpha);
  } else {
    // two warps per class, each summing every other 32 features
    const int wt = warp - NL / 32, c = wt >> 1, h = wt & 1;
    unsigned long long t = 0;
#pragma unroll 8
    for (int j = 32 * h + lane; j < F; j += 64) t += counts[(int64_t)c * F + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) part[c][h] = t;
    // the summing warps only: named barrier 1
    asm volatile("bar.sync 1, %0;" ::"r"(NT - NL) : "memory");
    if (h == 0 && lane == 0) ld[c] = log((double)(part[c][0] + part[c][1]) + alpha * (double)F);
    if (h == 1 && lane == 0 && blockIdx.x == 0 && !prior_given) {
      if (nc[c] == 0) {
        atomicOr(status, ST_BAD_LABEL);
        log_pi[c] = 0.0;
      } else {
        log_pi[c] = log((double)nc[c]) - log((double)n);
      }
    }
  }
  __syncthreads();
  if (tid < NL) {
    const int c = tid / kFinF, jl = tid % kFinF;
    const int j = blockIdx.x * kFinF + jl;
    double v = 0.0;
    if (j < F) {
      v = lc - ld[c];
      log_theta[(int64_t)c * F + j] = v;
    }
    lt[c][jl] = v;
  }
  __syncthreads();
  if (tid < kFinF) {
    const int j = blockIdx.x * kFinF + tid;
    double ad = 0.0;
    float a32 = 0.f, aw = 0.f;
    if (j < F_pad) {
      double d = 0.0;
      float w0 = 0.f, w1 = 0.f;
      if (j < F) {
        const double lt0 = lt[0][tid], lt1 = lt[1][tid];
        d = lt1 - lt0;
        if (!isfinite(d)) atomicOr(status, ST_BAD_TABLE);
        const double m = (lt0 + lt1) / 2.0;
        w0 = (float)(lt0 - m);
        w1 = (float)(lt1 - m);
        ad = fabs(d);
      }
      const float d32 = (float)d;
      a32 = fabsf(d32);
      aw = fmaxf(fabsf(w0), fabsf(w1));
      delta[j] = d32;
      w[j] = w0;
      w[(int64_t)F_pad + j] = w1;
      // FP32 tables for 4 / 8 / 16 elements per vector: quad q of vector v is
      // slot q * (F_pad / EPV) + v
      {
        float* t = reinterpret_cast<float*>(il4);
        const int epv = 4, vv = j / epv, e = j % epv;
        t[((size_t)(e >> 2) * (F_pad / epv) + vv) * 4 + (e & 3)] = d32;
      }
      {
        float* t = reinterpret_cast<float*>(il8);
        const int epv = 8, vv = j / epv, e = j % epv;
        t[((size_t)(e >> 2) * (F_pad / epv) + vv) * 4 + (e & 3)] = d32;
      }
      {
        float* t = reinterpret_cast<float*>(il16);
        const int epv = 16, vv = j / epv, e = j % epv;
        t[((size_t)(e >> 2) * (F_pad / epv) + vv) * 4 + (e & 3)] = d32;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ad = fmax(ad, __shfl_down_sync(0xffffffffu, ad, o));
      a32 = fmaxf(a32, __shfl_down_sync(0xffffffffu, a32, o));
      aw = fmaxf(aw, __shfl_down_sync(0xffffffffu, aw, o));
    }
    if (lane == 0) {
      dmax[warp] = ad;
      fmax32[warp] = a32;
      wm32[warp] = aw;
    }
  }
  __syncthreads();
  if (tid == 0) {
    double ad = dmax[0];
    float a32 = fmax32[0], aw = wm32[0];
    for (int k = 1; k < kFinF / 32; ++k) {
      ad = fmax(ad, dmax[k]);
      a32 = fmaxf(a32, fmax32[k]);
      aw = fmaxf(aw, wm32[k]);
    }
    // non-negative floating-point values order like their bit patterns
    atomicMax(&fin[0], (unsigned long long)__double_as_longlong(ad));
    atomicMax(reinterpret_cast<unsigned int*>(&fin[1]), __float_as_uint(a32));
    atomicMax(reinterpret_cast<unsigned int*>(&fin[1]) + 1, __float_as_uint(aw));
    __threadfence();
    last = atomicAdd(&fin[2], 1ull) == (unsigned long long)(gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const double maxabs64 = __longlong_as_double((long long)atomicAdd(&fin[0], 0ull));
  const unsigned long long m1 = atomicAdd(&fin[1], 0ull);
  int S = 0;
  if (maxabs64 > 0.0) {
    int e;
    frexp(maxabs64, &e);   // maxabs64 < 2^e
    S = 22 - e;
  }
  const double scale = ldexp(1.0, S);
  // U features per thread at a time: their log theta loads all go out before
  // the byte stores of the limbs (which may alias them) hold the next ones up
  constexpr int U = 4;
  for (int base = 0; base < F_pad; base += U * NT) {
    double dd[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int jj = base + u * NT + tid;
      dd[u] = jj < F ? log_theta[(int64_t)F + jj] - log_theta[jj] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int jj = base + u * NT + tid;
      if (jj >= F_pad) continue;
      const int32_t q = (int32_t)llrint(dd[u] * scale);   // |q| <= 2^22
      delta_q[jj] = q;
      // balanced base-256 digits q = q2*65536 + q1*256 + q0, each in [-128, 127]
      const int32_t q0 = ((q + 128) & 255) - 128;
      const int32_t r1 = (q - q0) >> 8;
      const int32_t q1 = ((r1 + 128) & 255) - 128;
      const int32_t q2 = (r1 - q1) >> 8;
      // u8 vectors hold 16 features; limb L of vector v is slot L * nvec8 + v,
      // byte (jj % 16) of it
      const int v = jj >> 4, b = jj & 15;
      unsigned char* L = reinterpret_cast<unsigned char*>(limbs);
      L[((size_t)0 * nvec8 + v) * 16 + b] = (unsigned char)(q0 & 255);
      L[((size_t)1 * nvec8 + v) * 16 + b] = (unsigned char)(q1 & 255);
      L[((size_t)2 * nvec8 + v) * 16 + b] = (unsigned char)(q2 & 255);
      // the same limbs packed into one word per feature (overflow entries)
      reinterpret_cast<uint32_t*>(L + (size_t)3 * F_pad)[jj] =
          (uint32_t)(q0 & 255) | ((uint32_t)(q1 & 255) << 8) | ((uint32_t)(q2 & 255) << 16);
    }
  }
  if (tid < 2) bias[tid] = (float)log_pi[tid];
  if (tid == 0) {
    const double b = log_pi[1] - log_pi[0];
    hdr->b = (float)b;
    hdr->b64 = b;
    hdr->maxabs = __uint_as_float((unsigned int)(m1 & 0xFFFFFFFFull));
    hdr->S = S;
    hdr->inv_scale = (float)ldexp(1.0, -S);
    hdr->maxabs_q = (float)maxabs64;
    hdr->pad = 0;
    *wmax = __uint_as_float((unsigned int)(m1 >> 32));
    fin[0] = 0ull;
    fin[1] = 0ull;
    fin[2] = 0ull;
  }
}

// general-C tables: w_cj = log theta_cj - mean_c log theta_cj (FP32), bias_c =
// log pi_c (FP32), wmax = max |w|.  The class-independent shift cancels in
// the margin and the log posterior.
__global__ void k_derive_general(const double* log_theta, const double* log_pi, int C, int F,
                                 int F_pad, float* w, float* bias, float* wmax, int* status) {
  float mx = 0.f;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < F_pad; j += gridDim.x * blockDim.x) {
    if (j >= F) {
      for (int c = 0; c < C; ++c) w[(int64_t)c * F_pad + j] = 0.f;
      continue;
    }
    double m = 0.0;
    for (int c = 0; c < C; ++c) m += log_theta[(int64_t)c * F + j];
    m /= (double)C;
    for (int c = 0; c < C; ++c) {
      const double v = log_theta[(int64_t)c * F + j] - m;
      if (!isfinite(v)) atomicOr(status, ST_BAD_TABLE);
      const float v32 = (float)v;
      w[(int64_t)c * F_pad + j] = v32;
      mx = fmaxf(mx, fabsf(v32));
    }
  }
  // block max then one atomic (non-negative floats compare as ints)
  __shared__ float red[256];
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(reinterpret_cast<int*>(wmax), __float_as_int(red[0]));
  if (blockIdx.x == 0)
    for (int c = threadIdx.x; c < C; c += blockDim.x) bias[c] = (float)log_pi[c];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int DT>
static nb_status run_counts(const CountArgs& a, long long nwork, cudaStream_t st) {
  if (nwork <= 0) return NB_OK;
  int occ = 0;
  NB_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_counts<DT>, 256, 0),
              "occupancy");
  long long blocks = (nwork + 7) / 8;
  const long long cap = (long long)num_sms() * (occ > 0 ? occ : 1);
  if (blocks > cap) blocks = cap;
  count_launch();
  k_counts<DT><<<(unsigned)blocks, 256, 0, st>>>(a, nwork);
  NB_TRY_CUDA(cudaGetLastError(), "k_counts launch");
  return NB_OK;
}

nb_status launch_fit_multinomial(nb_model* m, const void* X, nb_dtype dt, int64_t n, int64_t ld,
                                 const int32_t* y, const nb_aux* aux,
                                 const double* log_prior_dev, cudaStream_t st) {
  const int C = m->C, F = m->F;
  ModelDev& d = m->d;
  // counts, nc and the status word follow one another in the model's
  // allocation: one clear for all three
  NB_TRY_CUDA(cudaMemsetAsync(d.counts, 0,
                              (size_t)(reinterpret_cast<char*>(d.status + 1) -
                                       reinterpret_cast<char*>(d.counts)),
                              st),
              "memset");
  if (log_prior_dev && log_prior_dev != d.log_pi)
    NB_TRY_CUDA(cudaMemcpyAsync(d.log_pi, log_prior_dev, sizeof(double) * C,
                                cudaMemcpyDeviceToDevice, st),
                "memcpy prior");
  const int sms = num_sms();
  nb_status piped = NB_EUNSUPPORTED;
  if (C == 2 && m->tile.variant != NB_VARIANT_REGISTER)
    piped = launch_fit2_pipe(m, X, dt, n, ld, y, aux, st);
  if (piped != NB_OK && piped != NB_EUNSUPPORTED) return piped;
  if (n > 0 && piped != NB_OK) {
    const long long g = (n + 255) / 256;
    const unsigned hb = (unsigned)(g < sms * 4 ? g : sms * 4);
    count_launch();
    k_label_hist<<<hb, 256, 0, st>>>(y, n, C, reinterpret_cast<unsigned long long*>(d.nc),
                                     d.status);
    NB_TRY_CUDA(cudaGetLastError(), "k_label_hist");

    // scratch: offsets, cursors, run bases, bucketed row indices
    const size_t small = sizeof(long long) * (size_t)(C + 1) * 3;
    void* scratch = nullptr;
    NB_TRY_CUDA(cudaMallocAsync(&scratch, small + sizeof(int32_t) * (size_t)n, st),
                "cudaMallocAsync(fit scratch)");
    long long* offs = static_cast<long long*>(scratch);
    unsigned long long* cursor = reinterpret_cast<unsigned long long*>(offs + (C + 1));
    long long* item_base = offs + 2 * (C + 1);
    int32_t* idx = reinterpret_cast<int32_t*>(static_cast<char*>(scratch) + small);
    count_launch();
    k_bucket_setup<<<1, 32, 0, st>>>(reinterpret_cast<unsigned long long*>(d.nc), C, offs, cursor,
                                     item_base);
    const long long sb = (n + 256 * 16 - 1) / (256 * 16);
    count_launch();
    k_bucket_scatter<<<(unsigned)(sb < sms * 4 ? sb : sms * 4), 256, 0, st>>>(y, n, C, cursor,
                                                                              idx);
    NB_TRY_CUDA(cudaGetLastError(), "k_bucket_scatter");

    const int es = elem_size(dt);
    CountArgs a{};
    a.X = static_cast<const char*>(X);
    a.ld_bytes = ld * es;
    a.F = F;
    a.nvec_row = (F * es + 15) / 16;
    a.nslab = (a.nvec_row + 63) / 64;
    a.C = C;
    a.idx = idx;
    a.offs = offs;
    a.item_base = item_base;
    a.nc = reinterpret_cast<unsigned long long*>(d.nc);
    a.row_exp = aux ? aux->row_exp : nullptr;
    a.counts = reinterpret_cast<unsigned long long*>(d.counts);
    a.status = d.status;
    // upper bound on run items: n / kRunRows + C (exact count lives on the device)
    const long long items = (n + kRunRows - 1) / kRunRows + C;
    const long long nwork = items * a.nslab;
    // the kernel reads item_base[C] to skip work items past the end
    nb_status s = NB_OK;
    const bool aligned = ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && (a.ld_bytes % 16 == 0);
    if (!aligned) {
      const long long nw = items * F;
      const long long b = (nw + 255) / 256;
      count_launch();
      k_counts_scalar<<<(unsigned)(b < sms * 8 ? b : sms * 8), 256, 0, st>>>(a, dt, es, nw);
      const cudaError_t le = cudaGetLastError();
      s = le == cudaSuccess ? NB_OK : cuda_status(le, "k_counts_scalar");
    } else switch (dt) {
      case NB_U8: s = run_counts<NB_U8>(a, nwork, st); break;
      case NB_U16: s = run_counts<NB_U16>(a, nwork, st); break;
      case NB_F32: s = run_counts<NB_F32>(a, nwork, st); break;
      case NB_BF16: s = run_counts<NB_BF16>(a, nwork, st); break;
      case NB_FP8E4M3: s = run_counts<NB_FP8E4M3>(a, nwork, st); break;
    }
    if (s != NB_OK) {
      cudaFreeAsync(scratch, st);
      return s;
    }
    NB_TRY_CUDA(cudaFreeAsync(scratch, st), "cudaFreeAsync(fit scratch)");
    if (dt == NB_U8 && aux && aux->ovf_ptr) {
      const size_t bins = sizeof(unsigned int) * (size_t)C * F;
      const int use_smem = bins <= 96 * 1024;
      const int smem = use_smem ? (int)bins : 0;
      if (smem > kSmemOptIn)
        NB_TRY_CUDA(cudaFuncSetAttribute(k_counts_ovf, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem),
                    "cudaFuncSetAttribute");
      // shared 32-bit bins: at most 32,768 rows per block (adds are < 2^16)
      const long long ob = (n + 255) / 256;
      long long grid = ob < sms * 2 ? ob : sms * 2;
      if (use_smem && grid < (n + 32767) / 32768) grid = (n + 32767) / 32768;
      count_launch();
      k_counts_ovf<<<(unsigned)grid, 256, smem, st>>>(
          aux->ovf_ptr, aux->ovf_col, aux->ovf_add, y, n, F, C, use_smem,
          reinterpret_cast<unsigned long long*>(d.counts), d.status);
      NB_TRY_CUDA(cudaGetLastError(), "k_counts_ovf");
    }
  }
  if (C == 2) {
    count_launch();
    NB_TRY_CUDA(launch_pdl(k_fit_finish_c2, dim3((m->F_pad + kFinF - 1) / kFinF), dim3(kFinT),
                           0, st, reinterpret_cast<const unsigned long long*>(d.counts),
                           reinterpret_cast<const unsigned long long*>(d.nc), (int64_t)n, F,
                           m->F_pad, m->nvec8, m->alpha, (int)(log_prior_dev != nullptr), d.p0,
                           d.log_pi, d.c2, d.delta, d.delta_q, d.limbs, d.il[0], d.il[1],
                           d.il[2], d.w, d.bias, d.wmax, d.fin, d.status),
                "k_fit_finish_c2");
    return NB_OK;
  }
  count_launch();
  k_finalize_mn<<<dim3(C, (F + kFinTile - 1) / kFinTile), 256, 0, st>>>(
      reinterpret_cast<unsigned long long*>(d.counts), reinterpret_cast<unsigned long long*>(d.nc),
      n, F, m->alpha, log_prior_dev != nullptr, d.p0, d.log_pi, d.status);
  NB_TRY_CUDA(cudaGetLastError(), "k_finalize_mn");
  if (C == 2) {
    count_launch();
    k_derive_c2<<<1, 1024, 0, st>>>(d.p0, d.log_pi, F, m->F_pad, m->nvec8, d.c2, d.delta,
                                    d.delta_q, d.limbs, d.il[0], d.il[1], d.il[2], d.status);
    NB_TRY_CUDA(cudaGetLastError(), "k_derive_c2");
  }
  NB_TRY_CUDA(cudaMemsetAsync(d.wmax, 0, sizeof(float), st), "memset");
  {
    const int blocks = (m->F_pad + 255) / 256;
    count_launch();
    k_derive_general<<<blocks < 1024 ? blocks : 1024, 256, 0, st>>>(
        d.p0, d.log_pi, C, F, m->F_pad, d.w, d.bias, d.wmax, d.status);
    NB_TRY_CUDA(cudaGetLastError(), "k_derive_general");
  }
  if (d.tc_w) return launch_derive_tc(m, st);
  return NB_OK;
}

// ---------------------------------------------------------------------------
// Gaussian fit
// ---------------------------------------------------------------------------

// pass 0: sums of x; pass 1: sums of (x - mean)^2.  Slot C = all rows.
__global__ void __launch_bounds__(256) k_gauss_partial(const float* X, int64_t ld, int64_t n,
                                                       int F, int C, const int32_t* y, int pass,
                                                       const double* mu_c, const double* mu_all,
                                                       double* partial, int64_t chunk_rows,
                                                       int tile, int* status) {
  // partial layout: [chunk][slot 0..C][F]
  extern __shared__ double acc[];   // [8 warps][C+1][tile]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j0 = blockIdx.y * tile;
  const int64_t r0 = (int64_t)blockIdx.x * chunk_rows;
  int64_t r1 = r0 + chunk_rows;
  if (r1 > n) r1 = n;
  const int S = C + 1;
  for (int k = threadIdx.x; k < 8 * S * tile; k += blockDim.x) acc[k] = 0.0;
  __syncthreads();
  double* my = acc + (size_t)warp * S * tile;
  for (int64_t i = r0 + warp; i < r1; i += 8) {
    const int c = y[i];
    if (c < 0 || c >= C) {
      if (lane == 0) atomicOr(status, ST_BAD_LABEL);
      continue;
    }
    for (int jj = lane; jj < tile; jj += 32) {
      const int j = j0 + jj;
      if (j >= F) break;
      const double x = (double)X[i * ld + j];
      if (!isfinite(x)) atomicOr(status, ST_BAD_VALUE);
      if (pass == 0) {
        my[c * tile + jj] += x;
        my[C * tile + jj] += x;
      } else {
        const double dc = x - mu_c[(int64_t)c * F + j];
        const double da = x - mu_all[j];
        my[c * tile + jj] += dc * dc;
        my[C * tile + jj] += da * da;
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < S * tile; k += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += acc[(size_t)w * S * tile + k];
    const int slot = k / tile, jj = k % tile, j = j0 + jj;
    if (j < F) partial[((int64_t)blockIdx.x * S + slot) * F + j] = s;
  }
}

// sum the per-chunk partials in chunk order; pass 0 -> means, pass 1 -> variances
__global__ void k_gauss_reduce(const double* partial, int nchunk, int F, int C,
                               const unsigned long long* nc, int64_t n, int pass, double* mu_c,
                               double* mu_all, double* m2_c, double* m2_all) {
  const int S = C + 1;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < S * F; k += gridDim.x * blockDim.x) {
    const int slot = k / F, j = k % F;
    double s = 0.0;
    for (int ch = 0; ch < nchunk; ++ch) s += partial[((int64_t)ch * S + slot) * F + j];
    const double cnt = slot < C ? (double)nc[slot] : (double)n;
    const double v = cnt > 0 ? s / cnt : 0.0;
    if (pass == 0) {
      if (slot < C) mu_c[(int64_t)slot * F + j] = v; else mu_all[j] = v;
    } else {
      if (slot < C) m2_c[(int64_t)slot * F + j] = v; else m2_all[j] = v;
    }
  }
}

// var += eps, log prior, Gaussian constants and FP32 tables.  One block of
// 256 threads; reductions by warp shuffles and one pass over the warp results.
__global__ void __launch_bounds__(256) k_gauss_finalize(
    const double* m2_all, int F, int F_pad, int C, double var_smoothing,
    const unsigned long long* nc, int64_t n, int prior_given, const double* mu, double* var,
    double* log_pi, double* gconst, float* g_mu, float* g_ivar, float* g_const, int* status) {
  __shared__ double red[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double mx = 0.0;
  for (int j = threadIdx.x; j < F; j += blockDim.x) mx = fmax(mx, m2_all[j]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, off));
  if (lane == 0) red[warp] = mx;
  __syncthreads();
  double gm = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) gm = fmax(gm, red[w]);
  const double eps = var_smoothing * gm;
  __syncthreads();
  // the FP32 tables feature-major, gauss_cpad(C) classes per feature
  const int CP = gauss_cpad(C);
  for (int k = threadIdx.x; k < CP * F_pad; k += blockDim.x) {
    const int j = k / CP, c = k % CP;
    if (j >= F || c >= C) {
      g_mu[k] = 0.f;
      g_ivar[k] = 0.f;
      continue;
    }
    double v = var[(int64_t)c * F + j] + eps;
    if (!(v > 0.0) || !isfinite(v)) atomicOr(status, ST_BAD_TABLE);
    var[(int64_t)c * F + j] = v;
    g_mu[k] = (float)mu[(int64_t)c * F + j];
    g_ivar[k] = (float)(1.0 / v);
  }
  __syncthreads();
  const double kTwoPi = 6.283185307179586476925;
  __shared__ double red4[8];
  for (int c = 0; c < C; ++c) {
    // sum_j log(2 pi var_cj), and a4_c = sum_j m^2 v over the FP32 tables (a
    // term of the CUDA-core scorer's rounding bound)
    double s = 0.0, s4 = 0.0;
    for (int j = threadIdx.x; j < F; j += blockDim.x) {
      s += log(kTwoPi * var[(int64_t)c * F + j]);
      const double mj = g_mu[(int64_t)j * CP + c];
      s4 += mj * mj * (double)g_ivar[(int64_t)j * CP + c];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      s += __shfl_xor_sync(0xFFFFFFFFu, s, off);
      s4 += __shfl_xor_sync(0xFFFFFFFFu, s4, off);
    }
    if (lane == 0) {
      red[warp] = s;
      red4[warp] = s4;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0, t4 = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        t += red[w];
        t4 += red4[w];
      }
      g_const[C + c] = (float)t4;
      if (!prior_given) {
        if (nc[c] == 0) atomicOr(status, ST_BAD_LABEL);
        log_pi[c] = nc[c] ? log((double)nc[c]) - log((double)n) : 0.0;
      }
      gconst[c] = log_pi[c] - 0.5 * t;
      g_const[c] = (float)gconst[c];
    }
    __syncthreads();
  }
}

nb_status launch_fit_gaussian(nb_model* m, const float* X, int64_t n, int64_t ld,
                              const int32_t* y, const double* log_prior_dev, cudaStream_t st) {
  const int C = m->C, F = m->F, S = C + 1;
  ModelDev& d = m->d;
  NB_TRY_CUDA(cudaMemsetAsync(d.nc, 0, sizeof(uint64_t) * C, st), "memset");
  if (log_prior_dev && log_prior_dev != d.log_pi)
    NB_TRY_CUDA(cudaMemcpyAsync(d.log_pi, log_prior_dev, sizeof(double) * C,
                                cudaMemcpyDeviceToDevice, st),
                "memcpy prior");
  const int sms = num_sms();
  const long long g = (n + 255) / 256;
  count_launch();
  k_label_hist<<<(unsigned)(g < sms * 4 ? g : sms * 4), 256, 0, st>>>(
      y, n, C, reinterpret_cast<unsigned long long*>(d.nc), d.status);
  NB_TRY_CUDA(cudaGetLastError(), "k_label_hist");
  const int64_t chunk_rows = gauss_chunk_rows(n);
  const int nchunk = (int)((n + chunk_rows - 1) / chunk_rows);
  const size_t part_elems = (size_t)nchunk * S * F;
  const size_t extra = (size_t)F * 2;   // mu_all, m2_all
  void* scratch = nullptr;
  NB_TRY_CUDA(cudaMallocAsync(&scratch, sizeof(double) * (part_elems + extra), st),
              "cudaMallocAsync(gauss scratch)");
  double* partial = static_cast<double*>(scratch);
  double* mu_all = partial + part_elems;
  double* m2_all = mu_all + F;
  const int tile = gauss_tile(C);
  const int smem = (int)(sizeof(double) * 8 * S * tile);
  if (smem > kSmemOptIn)
    NB_TRY_CUDA(cudaFuncSetAttribute(k_gauss_partial, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     smem),
                "cudaFuncSetAttribute");
  dim3 grid(nchunk, (F + tile - 1) / tile);
  const int rb = (S * F + 255) / 256;
  for (int pass = 0; pass < 2; ++pass) {
    count_launch();
    k_gauss_partial<<<grid, 256, smem, st>>>(X, ld, n, F, C, y, pass, d.p0, mu_all, partial,
                                             chunk_rows, tile, d.status);
    NB_TRY_CUDA(cudaGetLastError(), "k_gauss_partial");
    count_launch();
    k_gauss_reduce<<<rb < 1024 ? rb : 1024, 256, 0, st>>>(
        partial, nchunk, F, C, reinterpret_cast<unsigned long long*>(d.nc), n, pass, d.p0, mu_all,
        d.p1, m2_all);
    NB_TRY_CUDA(cudaGetLastError(), "k_gauss_reduce");
  }
  count_launch();
  k_gauss_finalize<<<1, 256, 0, st>>>(m2_all, F, m->F_pad, C, m->var_smoothing,
                                       reinterpret_cast<unsigned long long*>(d.nc), n,
                                       log_prior_dev != nullptr, d.p0, d.p1, d.log_pi, d.gconst,
                                       d.g_mu, d.g_ivar, d.g_const, d.status);
  NB_TRY_CUDA(cudaGetLastError(), "k_gauss_finalize");
  NB_TRY_CUDA(cudaFreeAsync(scratch, st), "cudaFreeAsync(gauss scratch)");
  if (d.tcg_kc) return launch_derive_tcg(m, st);
  return NB_OK;
}

}  // namespace nbg
