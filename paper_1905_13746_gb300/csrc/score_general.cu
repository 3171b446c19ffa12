// CUDA-core scorers for any class count (Sec. 4 posterior and decision rule).
//
// Multinomial, C >= 2: s_c = log pi_c + sum_j x_j w_cj with the centred table
// w_cj = log theta_cj - mean_c log theta_cj (the per-feature shift is the same
// for every class, so it cancels in the label, the margin and the log
// posterior, and it keeps |w| small for the error bound).  A block scores 64
// files x 64 classes per pass as a register-tiled FP32 product over 32-feature
// chunks staged in shared memory; the epilogue takes the arg-max (lowest
// index among the maxima), the top-2 margin and the log-sum-exp.
//
// Gaussian: s_c = k_c - 1/2 sum_j (x_j - mu_cj)^2 / var_cj with
// k_c = log pi_c - 1/2 sum_j log(2 pi var_cj) from the FP64 fit.
//
// Both mark rows for the FP64 recheck when a rigorous bound on the FP32
// rounding error cannot guarantee the decision (or the log posteriors).
#include <cuda_fp16.h>
#include <math.h>

#include "device.cuh"
#include "internal.cuh"
#include "seg.cuh"

namespace nbg {

constexpr int GBM = 64;   // rows per tile
constexpr int GBK = 32;   // features per chunk
constexpr int GCB = 64;   // classes per pass

struct GArgs {
  const char* X;
  int64_t ld;        // elements
  int64_t n;
  int F, F_pad, C, dtype, aligned;
  const int64_t* ovf_ptr;
  const uint16_t* ovf_col;
  const uint16_t* ovf_add;
  const int8_t* row_exp;
  const float* w;      // C x F_pad
  const float* bias;   // C
  const float* wmax;
  const double* log_pi;
  uint8_t* label;
  float* margin;
  float* logpost;
  int want_lp, recheck;
  int* status;
};

// element j of a row as float (scalar path, any alignment)
__device__ __forceinline__ float gload1(int dt, const char* rp, int j) {
  switch (dt) {
    case NB_F32: return reinterpret_cast<const float*>(rp)[j];
    case NB_U16: return (float)reinterpret_cast<const uint16_t*>(rp)[j];
    case NB_U8: return (float)reinterpret_cast<const uint8_t*>(rp)[j];
    case NB_BF16: return __uint_as_float((uint32_t)reinterpret_cast<const uint16_t*>(rp)[j] << 16);
    default: return e4m3x2_to_f32((uint16_t)reinterpret_cast<const uint8_t*>(rp)[j]).x;
  }
}

__device__ __forceinline__ void decode16(int dt, const uint4& x, float* v, int& cnt) {
  const uint32_t w[4] = {x.x, x.y, x.z, x.w};
  switch (dt) {
    case NB_F32:
      cnt = 4;
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = __uint_as_float(w[k]);
      break;
    case NB_U16:
      cnt = 8;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        v[2 * k] = u_field_to_f32(w[k], kSelU16Lo);
        v[2 * k + 1] = u_field_to_f32(w[k], kSelU16Hi);
      }
      break;
    case NB_BF16:
      cnt = 8;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        v[2 * k] = __uint_as_float(w[k] << 16);
        v[2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
      }
      break;
    case NB_U8:
      cnt = 16;
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int b = 0; b < 4; ++b) v[4 * k + b] = u_field_to_f32(w[k], sel_u8(b));
      break;
    default:
      cnt = 16;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 lo = e4m3x2_to_f32((uint16_t)(w[k] & 0xFFFFu));
        const float2 hi = e4m3x2_to_f32((uint16_t)(w[k] >> 16));
        v[4 * k] = lo.x;
        v[4 * k + 1] = lo.y;
        v[4 * k + 2] = hi.x;
        v[4 * k + 3] = hi.y;
      }
  }
}

// One tile of GBM rows starting at r0 (all class blocks, epilogue included).
__device__ __forceinline__ void gen_tile(const GArgs& a, int64_t r0, float* gsm) {
  float* Xs = gsm;                         // [GBK][GBM + 4]
  float* Ws = Xs + GBK * (GBM + 4);        // [GBK][GCB + 4]
  float* Ss = Ws + GBK * (GCB + 4);        // [GBM][C_pad]
  const int C_pad = ((a.C + 3) / 4) * 4;
  float* Ts = Ss + GBM * C_pad;            // [GBM]
  float* Tslot = Ts + GBM;                 // [GBM * 8] per-slot |x| sums
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int es = a.dtype == NB_F32 ? 4 : ((a.dtype == NB_U16 || a.dtype == NB_BF16) ? 2 : 1);
  const int epv = 16 / es;
  const int vpr = GBK / epv;               // vectors per row per chunk (2, 4 or 8)
  const float wmax = *a.wmax;
  float bmax = 0.f;
  for (int c = 0; c < a.C; ++c) bmax = fmaxf(bmax, fabsf(a.bias[c]));
  const int nchunk = (a.F + GBK - 1) / GBK;
  float tpart[2] = {0.f, 0.f};   // |x| sums of the (row, vector) slots this thread loads
  for (int cb = 0; cb < a.C; cb += GCB) {
    float run[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) run[i][j] = 0.f;
    for (int ch = 0; ch < nchunk; ++ch) {
      const int k0 = ch * GBK;
      // X tile -> Xs[k][row] (FP32)
      for (int s = 0, slot = tid; slot < GBM * vpr; ++s, slot += 256) {
        const int row = slot / vpr, vv = slot % vpr;
        const int64_t gr = r0 + row;
        float v[16];
        int cnt = epv;
        const int kb = k0 + vv * epv;
        if (gr < a.n) {
          const char* rp = a.X + gr * a.ld * es;
          if (a.aligned && kb + epv <= a.F) {
            decode16(a.dtype, ld_stream16(rp + (int64_t)kb * es), v, cnt);
          } else {
            for (int e = 0; e < epv; ++e) v[e] = kb + e < a.F ? gload1(a.dtype, rp, kb + e) : 0.f;
          }
          if (a.dtype == NB_FP8E4M3 && a.row_exp) {
            const float sc = exp2f((float)a.row_exp[gr]);
            for (int e = 0; e < epv; ++e) v[e] *= sc;
          }
        } else {
          for (int e = 0; e < epv; ++e) v[e] = 0.f;
        }
        float tsum = 0.f;
        for (int e = 0; e < epv; ++e) {
          Xs[(vv * epv + e) * (GBM + 4) + row] = v[e];
          tsum += fabsf(v[e]);
        }
        if (cb == 0) tpart[s] += tsum;
      }
      // W tile -> Ws[k][c]
      for (int slot = tid; slot < GCB * (GBK / 4); slot += 256) {
        const int c = slot / (GBK / 4), kq = slot % (GBK / 4);
        float4 wv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (cb + c < a.C)
          wv = *reinterpret_cast<const float4*>(a.w + (int64_t)(cb + c) * a.F_pad + k0 + kq * 4);
        Ws[(kq * 4 + 0) * (GCB + 4) + c] = wv.x;
        Ws[(kq * 4 + 1) * (GCB + 4) + c] = wv.y;
        Ws[(kq * 4 + 2) * (GCB + 4) + c] = wv.z;
        Ws[(kq * 4 + 3) * (GCB + 4) + c] = wv.w;
      }
      __syncthreads();
      float acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll 8
      for (int k = 0; k < GBK; ++k) {
        const float4 ra = *reinterpret_cast<const float4*>(&Xs[k * (GBM + 4) + ty * 4]);
        const float4 rb = *reinterpret_cast<const float4*>(&Ws[k * (GCB + 4) + tx * 4]);
        const float A[4] = {ra.x, ra.y, ra.z, ra.w};
        const float B[4] = {rb.x, rb.y, rb.z, rb.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(A[i], B[j], acc[i][j]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) run[i][j] += acc[i][j];
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = cb + tx * 4 + j;
        if (c < a.C) Ss[(ty * 4 + i) * C_pad + c] = run[i][j];
      }
  }
  // row |x| totals, summed over the row's slots in a fixed order
  for (int s = 0, slot = tid; slot < GBM * vpr; ++s, slot += 256) Tslot[slot] = tpart[s];
  __syncthreads();
  if (tid < GBM) {
    float t = 0.f;
    for (int vv = 0; vv < vpr; ++vv) t += Tslot[tid * vpr + vv];
    Ts[tid] = t;
  }
  __syncthreads();
  // overflow entries (u8 storage): one thread per (row, class), entries in order
  if (a.dtype == NB_U8 && a.ovf_ptr) {
    for (int q = tid; q < GBM * a.C; q += 256) {
      const int row = q / a.C, c = q % a.C;
      const int64_t gr = r0 + row;
      if (gr >= a.n) continue;
      float s = Ss[row * C_pad + c];
      float t = 0.f;
      for (int64_t k = a.ovf_ptr[gr]; k < a.ovf_ptr[gr + 1]; ++k) {
        const int j = a.ovf_col[k];
        if (j >= a.F) continue;
        const float add = (float)a.ovf_add[k];
        s = fmaf(add, a.w[(int64_t)c * a.F_pad + j], s);
        t += add;
      }
      Ss[row * C_pad + c] = s;
      if (c == 0) Tslot[row] = t;
    }
    __syncthreads();
    if (tid < GBM) Ts[tid] += Tslot[tid];
    __syncthreads();
  }
  // epilogue: a warp per row
  const int warp = tid >> 5, lane = tid & 31;
  for (int row = warp; row < GBM; row += 8) {
    const int64_t gr = r0 + row;
    if (gr >= a.n) continue;
    float best = -INFINITY;
    int bi = 0x7FFFFFFF;
    for (int c = lane; c < a.C; c += 32) {
      const float s = Ss[row * C_pad + c] + a.bias[c];
      if (s > best) { best = s; bi = c; }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float ob = __shfl_xor_sync(0xFFFFFFFFu, best, off);
      const int oi = __shfl_xor_sync(0xFFFFFFFFu, bi, off);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    float second = -INFINITY, se = 0.f;
    for (int c = lane; c < a.C; c += 32) {
      const float s = Ss[row * C_pad + c] + a.bias[c];
      if (c != bi) second = fmaxf(second, s);
      se += expf(s - best);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      second = fmaxf(second, __shfl_xor_sync(0xFFFFFFFFu, second, off));
      se += __shfl_xor_sync(0xFFFFFFFFu, se, off);
    }
    const float lse = best + logf(se);
    const float margin = best - second;
    const int64_t novf = (a.dtype == NB_U8 && a.ovf_ptr) ? a.ovf_ptr[gr + 1] - a.ovf_ptr[gr] : 0;
    const float k = (float)(GBK + nchunk + 3 + novf);
    const float gam = k * 5.9604645e-8f / (1.f - k * 5.9604645e-8f);
    const float tau = 2.f * (gam * (Ts[row] * wmax + bmax) * 1.01f + 1e-12f * (Ts[row] * wmax + bmax)) + 1e-30f;
    bool flag = false;
    if (a.recheck != NB_RECHECK_OFF) {
      flag = !(margin > tau);
      if (a.recheck == NB_RECHECK_LP && tau > 5e-6f * fmaxf(1.f, margin)) flag = true;
    }
    if (lane == 0) {
      a.label[gr] = flag ? kLabelRecheck : (uint8_t)bi;
      a.margin[gr] = margin;
    }
    if (a.want_lp)
      for (int c = lane; c < a.C; c += 32)
        a.logpost[gr * a.C + c] = Ss[row * C_pad + c] + a.bias[c] - lse;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) k_score_gen(const GArgs a) {
  extern __shared__ __align__(16) float gsm[];
  const int64_t ntile = (a.n + GBM - 1) / GBM;
  for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) gen_tile(a, tile * GBM, gsm);
}

// ---------------------------------------------------------------------------
// Gaussian scorer on the CUDA cores (any 2 <= C <= 64, FP32 rows)
// ---------------------------------------------------------------------------
// s_c = k_c - 1/2 sum_j v_cj (x_j - mu_cj)^2 (Sec. 4 with Gaussian class
// conditionals; v = 1/var, k_c = log pi_c - 1/2 sum_j log(2 pi var_cj)).
// A group of LPR lanes scores R rows at once: lane li takes features j = li,
// li + LPR, ..., and for each block of CB classes keeps CB x R partial sums
// q = sum v dx^2.  The block's warps stage mu and v of a chunk of features
// (feature-major tables, CB consecutive classes per feature) in shared
// memory, so that each is read from L2 once per block of rows and from
// shared memory once per R rows.  The group's partial sums are combined by a
// reduce-scatter (each exchange halves the values a lane holds: CB R (LPR -
// 1) / LPR shuffles instead of CB R log2 LPR), which leaves lane li with the
// finished sums of classes-and-rows li CB R / LPR ...; their scores and
// bounds go to shared memory, and the LPR lanes then share each row's
// arg-max, sum of exponentials, recheck tests and log-posterior stores.
struct GGArgs {
  const float* X;
  int64_t ld, n;
  int F, F_pad, C;
  const float* mu;
  const float* ivar;
  const float* kc;
  uint8_t* label;
  float* margin;
  float* logpost;
  int want_lp, recheck;
};

constexpr int kGaussWarps = 8;

// lowest index among equal maxima; NaN never wins
__device__ __forceinline__ void gauss_top2(float& b1, int& i1, float& b2, float ob1, int oi1,
                                           float ob2) {
  const bool other = ob1 > b1 || (ob1 == b1 && oi1 < i1);
  const float lo = other ? b1 : ob1;
  if (other) {
    b1 = ob1;
    i1 = oi1;
  }
  b2 = fmaxf(fmaxf(b2, ob2), lo);
}

template <int LPR, int R, int CB>
__global__ void __launch_bounds__(kGaussWarps * 32, 2) k_score_gauss(const GGArgs a) {
  constexpr int G = 32 / LPR;     // row groups per warp
  constexpr int RPW = G * R;      // rows per warp
  constexpr int RPB = kGaussWarps * RPW;   // rows per block tile
  constexpr int NP = CB * R;      // sums q of a class block
  constexpr int OWN = NP / LPR;   // pairs a lane finishes
  // classes kept per row; 64 + 4 puts the rows of a warp's groups on different
  // banks for the epilogue's reads of class li + LPR m
  constexpr int CM = CB == 4 ? 4 : kTcMaxC + 4;
  constexpr int FPL = LPR == 8 ? 8 : 4;   // features per lane per staged chunk
  constexpr int FC = LPR * FPL;   // features per staged chunk
  // a staged feature holds the class block's mu (CB floats) then v; the row
  // stride keeps eight lanes' 16-byte reads of consecutive features on
  // distinct banks
  constexpr int SR = CB == 4 ? 12 : 2 * CB + 4;
  static_assert(NP % LPR == 0, "the reduce-scatter ends with whole pairs per lane");
  __shared__ __align__(16) float s_tab[FC * SR];
  __shared__ float s_s[kGaussWarps][RPW][CM], s_t[kGaussWarps][RPW][CM];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / LPR, li = lane % LPR;
  const int C = a.C, F = a.F, CP = gauss_cpad(C);
  constexpr float u = 5.9604645e-8f;

  // rounding depth of each sum: F / LPR sequential adds, the log2 LPR
  // combining levels, and 8 for the remaining operations
  int lg = 0;
  while ((1 << lg) < LPR) ++lg;
  const int kdepth = (F + LPR - 1) / LPR + lg + 8;
  const float gam = kdepth * u / (1.f - kdepth * u);

  const int64_t nbt = (a.n + RPB - 1) / RPB;
  for (int64_t bt = blockIdx.x; bt < nbt; bt += gridDim.x) {   // uniform over the block
    const int64_t r0 = bt * RPB + (int64_t)warp * RPW + (int64_t)grp * R;
    const float* xr[R];
    bool ok[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      ok[i] = r0 + i < a.n;
      xr[i] = a.X + (ok[i] ? r0 + i : 0) * a.ld;
    }
    for (int cb = 0; cb < C; cb += CB) {
      // sum p = k R + i: class cb + k, row r0 + i
      float pq[NP];
#pragma unroll
      for (int p = 0; p < NP; ++p) pq[p] = 0.f;
      for (int f0 = 0; f0 < F; f0 += FC) {
        // stage mu and v of features f0 .. f0 + FC - 1, classes cb .. cb + CB - 1
        // (feature-major tables: CB consecutive floats per feature; padding
        // classes and features past F are zero and add nothing)
        __syncthreads();
        for (int e = threadIdx.x; e < FC * (CB / 4) * 2; e += kGaussWarps * 32) {
          const int fl = e / ((CB / 4) * 2), rem = e % ((CB / 4) * 2);
          const int which = rem / (CB / 4), q4 = rem % (CB / 4);
          const int j = f0 + fl;
          float4 v4 = make_float4(0.f, 0.f, 0.f, 0.f);
          if (j < F)
            v4 = __ldg(reinterpret_cast<const float4*>((which ? a.ivar : a.mu) +
                                                       (int64_t)j * CP + cb) + q4);
          *reinterpret_cast<float4*>(s_tab + fl * SR + which * CB + 4 * q4) = v4;
        }
        __syncthreads();
#pragma unroll
        for (int jj = 0; jj < FPL; ++jj) {
          const int fl = li + LPR * jj, j = f0 + fl;
          if (j >= F) break;
          float x[R];
#pragma unroll
          for (int i = 0; i < R; ++i) x[i] = ok[i] ? __ldg(xr[i] + j) : 0.f;
          const float* tb = s_tab + fl * SR;
#pragma unroll
          for (int k4 = 0; k4 < CB / 4; ++k4) {
            const float4 m4 = *reinterpret_cast<const float4*>(tb + 4 * k4);
            const float4 v4 = *reinterpret_cast<const float4*>(tb + CB + 4 * k4);
            const float mm[4] = {m4.x, m4.y, m4.z, m4.w}, vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int k = 4 * k4 + e;
#pragma unroll
              for (int i = 0; i < R; ++i) {
                const float dx = x[i] - mm[e];
                pq[k * R + i] = fmaf(dx * vv[e], dx, pq[k * R + i]);
              }
            }
          }
        }
      }
      // reduce-scatter over the group
#pragma unroll
      for (int off = LPR / 2, n = NP; off > 0; off >>= 1, n >>= 1) {
        const bool up = (li & off) != 0;   // this lane keeps the upper half
#pragma unroll
        for (int p = 0; p < n / 2; ++p) {
          const float sq = up ? pq[p] : pq[p + n / 2], kq = up ? pq[p + n / 2] : pq[p];
          pq[p] = kq + __shfl_xor_sync(0xFFFFFFFFu, sq, off);
        }
      }
      // lane li now holds pairs li OWN .. li OWN + OWN - 1
#pragma unroll
      for (int o = 0; o < OWN; ++o) {
        const int p = li * OWN + o, k = p / R, i = p % R, c = cb + k;
        if (c >= C) continue;
        const float qq = pq[o], kc = a.kc[c];
        // |s - s_FP64| with u = 2^-24: m = fl(mu) and v = fl(1/var) are within
        // u relative, dx = fl(x - m) within u (|dx| + |m|) of x - mu, so each
        // term v dx^2 is within u v (4 dx^2 + 2 |dx| |m|) + 2 u^2 v (dx^2 +
        // m^2); the FP32 sums add gam q; k_c and the final subtraction add
        // u (|k_c| + |s|).  sum v |dx| |m| <= sqrt(sum v dx^2 sum v m^2)
        // (Cauchy-Schwarz on the FP32 values; 1e-3 covers the rounding of the
        // two computed sums); 1% slack covers the FP32 evaluation of the bound.
        const float a4 = a.kc[C + c];   // sum_j m^2 v, from the fit
        const float aa = sqrtf(qq * a4) * 1.001f;
        const float sc = kc - 0.5f * qq;
        s_s[warp][grp * R + i][c] = sc;
        s_t[warp][grp * R + i][c] = (0.5f * (u * (4.f * qq + 2.f * aa) * (1.f + 2.f * u) +
                                             2.f * u * u * (qq + a4) + gam * qq) +
                                     u * (fabsf(kc) + fabsf(sc))) * 1.01f +
                                    1e-12f * (qq + fabsf(kc)) + 1e-30f;
      }
    }
    __syncwarp();
    // epilogue: the group's lanes share each row's classes
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int rl = grp * R + i;
      const float* sr = s_s[warp][rl];
      const float* tr = s_t[warp][rl];
      float b1 = -INFINITY, b2 = -INFINITY, tmax = 0.f;
      int i1 = 0x7FFFFFFF;
      bool nan = false;
      for (int c = li; c < C; c += LPR) {
        const float sv = sr[c];
        nan |= !(sv == sv) || !(tr[c] == tr[c]);
        tmax = fmaxf(tmax, tr[c]);
        gauss_top2(b1, i1, b2, sv, c, -INFINITY);
      }
#pragma unroll
      for (int off = LPR / 2; off > 0; off >>= 1) {
        const float ob1 = __shfl_xor_sync(0xFFFFFFFFu, b1, off);
        const int oi1 = __shfl_xor_sync(0xFFFFFFFFu, i1, off);
        const float ob2 = __shfl_xor_sync(0xFFFFFFFFu, b2, off);
        gauss_top2(b1, i1, b2, ob1, oi1, ob2);
        tmax = fmaxf(tmax, __shfl_xor_sync(0xFFFFFFFFu, tmax, off));
        nan |= __shfl_xor_sync(0xFFFFFFFFu, (int)nan, off) != 0;
      }
      const int bi = i1 < C ? i1 : 0;   // every score NaN: class 0, and the row is marked
      const float sb = sr[bi], tb = tr[bi];
      float P = 0.f;
      for (int c = li; c < C; c += LPR)
        if (c != bi) P += expf(sr[c] - sb);
#pragma unroll
      for (int off = LPR / 2; off > 0; off >>= 1) P += __shfl_xor_sync(0xFFFFFFFFu, P, off);
      const float margin = sb - b2;
      // lp_c = (s_c - s_top) - L: formed from the differences, so that no
      // rounding at the scores' magnitude enters (lp_top = -L exactly)
      const float L = log1pf(P);
      bool flag = false;
      if (a.recheck != NB_RECHECK_OFF) {
        flag = nan;   // a NaN score or bound: FP64 decides
        // label: the top class stays ahead of every other class c by more than
        // the two classes' bounds (a far class's large bound does not matter)
        for (int c = li; c < C; c += LPR)
          if (c != bi && !(sb - sr[c] > (tb + tr[c]) * 1.0001f)) flag = true;
        if (a.recheck == NB_RECHECK_LP) {
          // lp_c = d_c - L with d_c = s_c - s_top and L = log(1 + sum_{k != top}
          // e^{d_k}); each d_k is off by at most D = t_top + t_max, so L is off
          // by at most D e^{2D} P / (1 + P) (mean value; the softmax weights at
          // the intermediate point are within e^{2D} of the computed ones), and
          // lp_c by that plus t_c + t_top (c != top)
          const float D = tb + tmax;
          const float eL = D * expf(2.f * D) * (P / (1.f + P)) * 1.01f + 1e-30f;
          for (int c = li; c < C; c += LPR) {
            const float err = (c == bi ? 0.f : tr[c] + tb) + eL;
            if (err > 5e-6f * fmaxf(1.f, fabsf((sr[c] - sb) - L))) flag = true;
          }
        }
      }
      int fl = flag ? 1 : 0;
#pragma unroll
      for (int off = LPR / 2; off > 0; off >>= 1) fl |= __shfl_xor_sync(0xFFFFFFFFu, fl, off);
      if (ok[i]) {
        const int64_t r = r0 + i;
        if (li == 0) {
          a.label[r] = fl ? kLabelRecheck : (uint8_t)bi;
          a.margin[r] = margin;
        }
        if (a.want_lp)
          for (int c = li; c < C; c += LPR) a.logpost[r * C + c] = (sr[c] - sb) - L;
      }
    }
    __syncwarp();
  }
}

template <int LPR, int R, int CB>
static nb_status run_score_gauss(const GGArgs& a, cudaStream_t st) {
  constexpr int RPW = (32 / LPR) * R;
  const int64_t ntile = (a.n + RPW - 1) / RPW;
  int occ = 0;
  NB_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                  &occ, k_score_gauss<LPR, R, CB>, kGaussWarps * 32, 0),
              "occupancy(k_score_gauss)");
  const int64_t cap = (int64_t)num_sms() * (occ > 0 ? occ : 1);
  int64_t blocks = (ntile + kGaussWarps - 1) / kGaussWarps;
  if (blocks > cap) blocks = cap;
  count_launch();
  k_score_gauss<LPR, R, CB><<<(unsigned)blocks, kGaussWarps * 32, 0, st>>>(a);
  NB_TRY_CUDA(cudaGetLastError(), "k_score_gauss launch");
  return NB_OK;
}

// lanes per row: the features a lane sums in sequence stay at most 32 (the
// rounding depth of the bound); few classes take 4-class blocks of 4 rows
static nb_status launch_score_gauss(const GGArgs& a, cudaStream_t st) {
  if (a.C <= 4) {
    if (a.F > 128) return run_score_gauss<16, 4, 4>(a, st);
    return run_score_gauss<8, 4, 4>(a, st);
  }
  if (a.F > 512) return run_score_gauss<32, 4, 16>(a, st);
  if (a.F > 128) return run_score_gauss<16, 4, 16>(a, st);
  return run_score_gauss<8, 2, 16>(a, st);
}

// ---------------------------------------------------------------------------
// segmented general scorer: 64-row tiles of a group list, each group scored
// with its own model slot (one launch per batch)
// ---------------------------------------------------------------------------
struct GModel {
  int C, F_pad;
  const float* w;
  const float* bias;
  const float* wmax;
};

struct GSegArgs {
  const SegGroup* groups;
  const SegHeader* hdr;
  GModel md[kSegMaxModels];
  int F, dtype, want_lp, recheck;
  int* status;
};

__global__ void __launch_bounds__(256) k_score_gen_seg(const GSegArgs s) {
  extern __shared__ __align__(16) float gsm[];
  const int n_groups = s.hdr->n_groups;
  const long long tiles = s.hdr->tiles;
  const SegGroup* gr = s.groups;
  const int es = s.dtype == NB_F32 ? 4 : ((s.dtype == NB_U16 || s.dtype == NB_BF16) ? 2 : 1);
  for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int g = seg_find(n_groups, t, [gr](int i) { return gr[i].tile0; });
    const SegGroup& G = gr[g];
    const GModel& M = s.md[G.model];
    GArgs a{};
    a.X = G.X;
    a.ld = G.ld_bytes / es;
    a.n = G.n;
    a.F = s.F;
    a.F_pad = M.F_pad;
    a.C = M.C;
    a.dtype = s.dtype;
    a.aligned = ((reinterpret_cast<uintptr_t>(G.X) & 15) == 0) && (G.ld_bytes % 16 == 0);
    a.ovf_ptr = G.ovf_ptr;
    a.ovf_col = G.ovf_col;
    a.ovf_add = G.ovf_add;
    a.row_exp = G.row_exp;
    a.w = M.w;
    a.bias = M.bias;
    a.wmax = M.wmax;
    a.label = G.label;
    a.margin = G.margin;
    a.logpost = G.logpost;
    a.want_lp = s.want_lp;
    a.recheck = s.recheck;
    a.status = s.status;
    gen_tile(a, (t - G.tile0) * GBM, gsm);
  }
}

nb_status launch_score_gen_seg(const SegGroup* groups, const SegHeader* hdr,
                               const nb_model* const* models, int n_models, nb_dtype dt, int F,
                               int want_lp, int recheck, int* status, cudaStream_t st) {
  GSegArgs s{};
  s.groups = groups;
  s.hdr = hdr;
  int C_max = 2;
  for (int i = 0; i < n_models && i < kSegMaxModels; ++i) {
    const nb_model* m = models[i];
    s.md[i] = GModel{m->C, m->F_pad, m->d.w, m->d.bias, m->d.wmax};
    C_max = m->C > C_max ? m->C : C_max;
  }
  s.F = F;
  s.dtype = dt;
  s.want_lp = want_lp;
  s.recheck = recheck;
  s.status = status;
  const int C_pad = ((C_max + 3) / 4) * 4;
  const int smem =
      (int)sizeof(float) * (GBK * (GBM + 4) + GBK * (GCB + 4) + GBM * C_pad + GBM + GBM * 8);
  if (smem > kSmemOptIn)
    NB_TRY_CUDA(cudaFuncSetAttribute(k_score_gen_seg, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     smem),
                "cudaFuncSetAttribute(gen_seg)");
  int occ = 0;
  NB_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_score_gen_seg, 256, smem),
              "occupancy(gen_seg)");
  count_launch();
  k_score_gen_seg<<<num_sms() * (occ > 0 ? occ : 1), 256, smem, st>>>(s);
  NB_TRY_CUDA(cudaGetLastError(), "k_score_gen_seg launch");
  return NB_OK;
}

nb_status launch_score_general(const nb_model* m, const void* X, nb_dtype dt, int64_t n,
                               int64_t ld, const nb_aux* aux, const ScoreOut& o, cudaStream_t st) {
  if (n == 0) return NB_OK;
  if (m->kind == NB_GAUSSIAN) {
    if (dt != NB_F32) {
      set_error("Gaussian models score F32 features");
      return NB_EINVAL;
    }
    GGArgs a{};
    a.X = static_cast<const float*>(X);
    a.ld = ld;
    a.n = n;
    a.F = m->F;
    a.F_pad = m->F_pad;
    a.C = m->C;
    a.mu = m->d.g_mu;
    a.ivar = m->d.g_ivar;
    a.kc = m->d.g_const;
    a.label = o.label;
    a.margin = o.margin;
    a.logpost = o.logpost;
    a.want_lp = o.want_lp;
    a.recheck = o.recheck;
    return launch_score_gauss(a, st);
  }
  const int es = elem_size(dt);
  GArgs a{};
  a.X = static_cast<const char*>(X);
  a.ld = ld;
  a.n = n;
  a.F = m->F;
  a.F_pad = m->F_pad;
  a.C = m->C;
  a.dtype = dt;
  a.aligned = ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && ((ld * es) % 16 == 0);
  a.ovf_ptr = aux ? aux->ovf_ptr : nullptr;
  a.ovf_col = aux ? aux->ovf_col : nullptr;
  a.ovf_add = aux ? aux->ovf_add : nullptr;
  a.row_exp = aux ? aux->row_exp : nullptr;
  a.w = m->d.w;
  a.bias = m->d.bias;
  a.wmax = m->d.wmax;
  a.log_pi = m->d.log_pi;
  a.label = o.label;
  a.margin = o.margin;
  a.logpost = o.logpost;
  a.want_lp = o.want_lp;
  a.recheck = o.recheck;
  a.status = m->d.sstatus;
  const int C_pad = ((m->C + 3) / 4) * 4;
  const int smem =
      (int)sizeof(float) * (GBK * (GBM + 4) + GBK * (GCB + 4) + GBM * C_pad + GBM + GBM * 8);
  if (smem > kSmemOptIn)   // per device and function: set at every launch
    NB_TRY_CUDA(cudaFuncSetAttribute(k_score_gen, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     smem > 96 * 1024 ? smem : 96 * 1024),
                "cudaFuncSetAttribute");
  int occ = 0;
  NB_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_score_gen, 256, smem),
              "occupancy");
  const int64_t tiles = (n + GBM - 1) / GBM;
  const int64_t cap = (int64_t)num_sms() * (occ > 0 ? occ : 1);
  count_launch();
  k_score_gen<<<(unsigned)(tiles < cap ? tiles : cap), 256, smem, st>>>(a);
  NB_TRY_CUDA(cudaGetLastError(), "k_score_gen launch");
  return NB_OK;
}

}  // namespace nbg
