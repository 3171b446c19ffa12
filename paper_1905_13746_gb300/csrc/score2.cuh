// Pieces shared by the two-class scorers (register-streaming and
// TMA-pipelined): launch arguments, the epilogue that turns the log-odds d
// into label / margin / log posteriors and marks rows for the FP64 recheck,
// and the exact decoders of each storage type into FP32.
#pragma once

#include <cuda_fp16.h>

#include "device.cuh"
#include "internal.cuh"

namespace nbg {

struct S2Args {
  const char* X;
  int64_t ld_bytes;
  int64_t n;
  int F;
  int nvec_row;   // 16-byte vectors that hold a row's F features
  int nvec_tab;   // vectors of the padded table (F_pad elements)
  const void* table;
  uint32_t table_bytes;
  const C2Header* hdr;
  const int32_t* delta_q;   // plain fixed-point table (overflow entries)
  const float* delta;       // plain FP32 table (overflow entries)
  const int64_t* ovf_ptr;
  const uint16_t* ovf_col;
  const uint16_t* ovf_add;
  const int8_t* row_exp;
  uint8_t* label;
  float* margin;
  float* logpost;
  int want_lp;
  int recheck;
  unsigned long long* marks;   // counts the rows marked for the recheck, or nullptr
  int k_base;     // FP32 path: rounding depth of a row without overflow entries
  int* status;
};

__device__ __forceinline__ float softplusf(float z) {
  return fmaxf(z, 0.f) + log1pf(expf(-fabsf(z)));
}

// Outputs of one row from its log-odds d and the bound tau on |d - d_exact|:
// label (or the recheck mark), margin |d|, log posteriors -softplus(-+d).
// tau = +inf says that the fast path's sums are not valid for this row at all
// (see c2_tau_u8): the row is marked in every recheck mode, NB_RECHECK_OFF
// included.
__device__ __forceinline__ bool c2_store(uint8_t* label, float* margin, float* logpost,
                                         int want_lp, int recheck, int64_t row, float d,
                                         float tau) {
  bool flag = !(tau < INFINITY);
  const float ad = fabsf(d);
  if (recheck != NB_RECHECK_OFF) {
    flag = flag || !(ad > tau);  // also true for NaN
    if (recheck == NB_RECHECK_LP && tau > 5e-6f * fmaxf(1.f, ad)) flag = true;
  }
  label[row] = flag ? kLabelRecheck : (d > 0.f ? 1 : 0);
  margin[row] = ad;
  if (want_lp) {
    logpost[2 * row] = -softplusf(d);
    logpost[2 * row + 1] = -softplusf(-d);
  }
  return flag;
}

// c2_store for the single-group scorers; the marked rows are also counted into
// a.marks (the call's n_rechecked), one atomic per warp, so that the FP64
// recheck can skip its scan when no row was marked.
__device__ __forceinline__ void c2_epilogue(const S2Args& a, int64_t row, float d, float tau) {
  const bool flag = c2_store(a.label, a.margin, a.logpost, a.want_lp, a.recheck, row, d, tau);
  if (a.marks) {
    const unsigned act = __activemask();
    const unsigned m = __ballot_sync(act, flag);
    if (m && (int)(threadIdx.x & 31) == __ffs(act) - 1)
      atomicAdd(a.marks, (unsigned long long)__popc(m));
  }
}

// The u8 register-streaming scorer stores each row from whichever lane holds
// it, in divergent code; it counts its marked rows per lane and adds them to
// a.marks once per warp here, at the end of the kernel, where every lane of
// the warp arrives.
__device__ __forceinline__ void c2_flush_marks(const S2Args& a, unsigned cnt) {
  if (!a.marks) return;
  cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(a.marks, (unsigned long long)cnt);
}

// Rigorous bound on |d_gpu - d_exact| of the fixed-point u8 path: the Delta
// quantisation (half a step per unit count), the int64 -> FP32 conversion and
// the final add, and slack for the FP64 reference's own rounding.
// Each of the three limb sums is bounded by 128 T (|limb| <= 128) and is held
// in an int32, which is exact only while 128 T < 2^31: a row of T >= 2^24
// stored counts (possible with the overflow list, whose entries add up to
// 65,535 each) gets tau = +inf, i.e. the FP64 recheck in every mode.  T is the
// exact integer total converted to FP32, which keeps the comparison exact.
__device__ __forceinline__ float c2_tau_u8(float T, float Dsum, float b, float inv_scale,
                                           float maxabs) {
  if (T >= 16777216.f) return INFINITY;
  return 0.5f * T * inv_scale * 1.0001f + 2.4e-7f * (fabsf(Dsum) + fabsf(b)) +
         1e-12f * (T * maxabs + fabsf(b)) + 1e-30f;
}

// ---------------------------------------------------------------------------
// FP32 accumulation from any storage type
// ---------------------------------------------------------------------------
template <int DT>
struct Decode;

template <>
struct Decode<NB_F32> {
  static constexpr int EPV = 4;
  __device__ __forceinline__ static void run(const uint4& x, float* v) {
    v[0] = __uint_as_float(x.x);
    v[1] = __uint_as_float(x.y);
    v[2] = __uint_as_float(x.z);
    v[3] = __uint_as_float(x.w);
  }
};
template <>
struct Decode<NB_U16> {
  static constexpr int EPV = 8;
  __device__ __forceinline__ static void run(const uint4& x, float* v) {
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[2 * k] = u_field_to_f32(w[k], kSelU16Lo);
      v[2 * k + 1] = u_field_to_f32(w[k], kSelU16Hi);
    }
  }
};
template <>
struct Decode<NB_BF16> {
  static constexpr int EPV = 8;
  __device__ __forceinline__ static void run(const uint4& x, float* v) {
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[2 * k] = __uint_as_float(w[k] << 16);
      v[2 * k + 1] = __uint_as_float(w[k] & 0xFFFF0000u);
    }
  }
};
template <>
struct Decode<NB_U8> {
  static constexpr int EPV = 16;
  __device__ __forceinline__ static void run(const uint4& x, float* v) {
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
      for (int b = 0; b < 4; ++b) v[4 * k + b] = u_field_to_f32(w[k], sel_u8(b));
    }
  }
};
template <>
struct Decode<NB_FP8E4M3> {
  static constexpr int EPV = 16;
  __device__ __forceinline__ static void run(const uint4& x, float* v) {
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
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
};

// ---------------------------------------------------------------------------
// FP8 E4M3 counts as exact integers
// ---------------------------------------------------------------------------
// Magic pair of a row with row scale 2^e: (M, M) in FP16, M = 2^(10 - e), for
// e = 0 or 1; 0 for any other exponent (the row then fails the check).
__device__ __forceinline__ uint32_t fp8_magic(int e) {
  return e == 0 ? 0x64006400u : (e == 1 ? 0x60006000u : 0u);
}

// Count check state of one row's values.  With u = v + M in FP16 (v the E4M3
// value, converted exactly), v 2^e is an integer in [0, 2^10) exactly when u
// lies in [M, 2M) -- the sign and exponent field of every half equals M's,
// which the OR and the AND of all halves both show -- and u - M == v; the
// count is then the low 10 bits of u.  Fractions, negatives and NaN fail.
struct Fp8Check {
  uint32_t bd = 0u;             // OR of (u - M) ^ v
  uint32_t orv = 0u;            // OR of u
  uint32_t andv = 0xFFFFFFFFu;  // AND of u
};

__device__ __forceinline__ bool fp8_check_ok(const Fp8Check& c, uint32_t m2) {
  return m2 != 0u && c.bd == 0u && (c.orv & 0xFC00FC00u) == m2 && (c.andv & 0xFC00FC00u) == m2;
}

// Four E4M3 codes (features f .. f+3 in the bytes of w) -> u01 = (M + x_f,
// M + x_f+1) and u23 = (M + x_f+2, M + x_f+3) as 16-bit pairs, checked.
__device__ __forceinline__ void fp8_biased_pairs(uint32_t w, uint32_t m2, uint32_t& u01,
                                                 uint32_t& u23, Fp8Check& c) {
  uint32_t h0, h1, b0, b1;
  asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h0) : "h"((unsigned short)(w & 0xFFFFu)));
  asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h1) : "h"((unsigned short)(w >> 16)));
  asm("add.rn.f16x2 %0, %1, %2;" : "=r"(u01) : "r"(h0), "r"(m2));
  asm("add.rn.f16x2 %0, %1, %2;" : "=r"(u23) : "r"(h1), "r"(m2));
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(b0) : "r"(u01), "r"(m2));
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(b1) : "r"(u23), "r"(m2));
  c.bd |= (b0 ^ h0) | (b1 ^ h1);
  c.orv |= u01 | u23;
  c.andv &= u01 & u23;
}

// One 16-byte vector of E4M3 codes against its three limb words, exact:
// the counts x (low 10 bits of each biased half) times the limbs with dp2a,
// and their total.  Any number of vectors per lane (int32 sums stay below
// 128 T).
__device__ __forceinline__ void fp8_vector_limbs(const uint4& x, const uint4& q0, const uint4& q1,
                                                 const uint4& q2, uint32_t m2, int& a0, int& a1,
                                                 int& a2, uint32_t& tt, Fp8Check& c) {
  const uint32_t w[4] = {x.x, x.y, x.z, x.w};
  const uint32_t l0[4] = {q0.x, q0.y, q0.z, q0.w}, l1[4] = {q1.x, q1.y, q1.z, q1.w},
                 l2[4] = {q2.x, q2.y, q2.z, q2.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    uint32_t u01, u23;
    fp8_biased_pairs(w[k], m2, u01, u23, c);
    const uint32_t x01 = u01 & 0x03FF03FFu, x23 = u23 & 0x03FF03FFu;
    a0 = dp2a_hi_us(x23, l0[k], dp2a_lo_us(x01, l0[k], a0));
    a1 = dp2a_hi_us(x23, l1[k], dp2a_lo_us(x01, l1[k], a1));
    a2 = dp2a_hi_us(x23, l2[k], dp2a_lo_us(x01, l2[k], a2));
    tt = (uint32_t)dp2a_hi_us(x23, 0x01010101u, dp2a_lo_us(x01, 0x01010101u, (int)tt));
  }
}

// As fp8_vector_limbs on the biased halves M + x directly: each sum then
// carries M times the sum of the limbs (and M per value in tt), which the
// caller removes once per row (fp8_unbias).  The int32 sums stay exact for up
// to 64 values per lane ((2^15 + 2^10) * 128 * 64 < 2^31).
__device__ __forceinline__ void fp8_vector_limbs_biased(const uint4& x, const uint4& q0,
                                                        const uint4& q1, const uint4& q2,
                                                        uint32_t m2, int& a0, int& a1, int& a2,
                                                        uint32_t& tt, Fp8Check& c) {
  const uint32_t w[4] = {x.x, x.y, x.z, x.w};
  const uint32_t l0[4] = {q0.x, q0.y, q0.z, q0.w}, l1[4] = {q1.x, q1.y, q1.z, q1.w},
                 l2[4] = {q2.x, q2.y, q2.z, q2.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    uint32_t u01, u23;
    fp8_biased_pairs(w[k], m2, u01, u23, c);
    a0 = dp2a_hi_us(u23, l0[k], dp2a_lo_us(u01, l0[k], a0));
    a1 = dp2a_hi_us(u23, l1[k], dp2a_lo_us(u01, l1[k], a1));
    a2 = dp2a_hi_us(u23, l2[k], dp2a_lo_us(u01, l2[k], a2));
    tt = (uint32_t)dp2a_hi_us(u23, 0x01010101u, dp2a_lo_us(u01, 0x01010101u, (int)tt));
  }
}

// Sum of the 16 signed limb bytes of a vector (the bias correction's weight)
__device__ __forceinline__ int limb_byte_sum(const uint4& q) {
  int s = dp4a_us(0x01010101u, q.x, 0);
  s = dp4a_us(0x01010101u, q.y, s);
  s = dp4a_us(0x01010101u, q.z, s);
  return dp4a_us(0x01010101u, q.w, s);
}

// The lane's count total, or 2^24 when one of its values failed the check
// (which sends the row to the FP64 recheck, see c2_tau_u8).
__device__ __forceinline__ uint32_t fp8_lane_total(uint32_t tt, const Fp8Check& c, uint32_t m2) {
  return fp8_check_ok(c, m2) ? tt : 16777216u;
}

// Sums four int32 values over the LPR lanes of a lane group (LPR = 4 .. 32,
// a power of two) with log2(LPR) + 1 shuffles instead of 4 log2(LPR): the
// first two steps halve the set of values each lane carries.  Returns the lane's share: lanes [0, LPR/4) of
// the group hold the sum of a0, then a1, a2 and a3 by quarter.  Integer sums
// are exact, so the order does not matter.
template <int LPR>
__device__ __forceinline__ int sum4_transposed(int a0, int a1, int a2, int a3, int li) {
  const bool h1 = (li & (LPR / 2)) != 0;
  int k0 = h1 ? a2 : a0, k1 = h1 ? a3 : a1;
  const int s0 = h1 ? a0 : a2, s1 = h1 ? a1 : a3;
  k0 += __shfl_xor_sync(0xFFFFFFFFu, s0, LPR / 2);
  k1 += __shfl_xor_sync(0xFFFFFFFFu, s1, LPR / 2);
  const bool h2 = (li & (LPR / 4)) != 0;
  int k = h2 ? k1 : k0;
  const int s = h2 ? k0 : k1;
  k += __shfl_xor_sync(0xFFFFFFFFu, s, LPR / 4);
#pragma unroll
  for (int off = LPR / 8; off > 0; off >>= 1) k += __shfl_xor_sync(0xFFFFFFFFu, k, off);
  return k;
}

}  // namespace nbg
