// Many-class multinomial scorer on the fifth-generation tensor cores.
//
// Sec. 4 scores file x against class c by s_c = log pi_c + sum_j x_j log
// theta_cj and takes the class of largest posterior.  With the centred table
// w_cj = log theta_cj - mean_c log theta_cj (the per-feature shift is common to
// all classes and cancels in the label, the margin and the log posteriors)
// the scores of 128 files against C <= 64 classes are one dense contraction
// S = X W^T, done here with tcgen05.mma (kind::f16, FP32 accumulators in
// tensor memory).
//
// Exactness.  The weights are held in fixed point, Q_cj = round(w_cj 2^S)
// with |Q| <= 2^22, split into three balanced limbs Q = q0 + 2^8 q1 + 2^16 q2
// with |q_l| <= 128, each an exact FP16 integer.  Stored u8 counts (0..255)
// are exact FP16 integers as well, so every product is exact, and a limb's
// sum over a row stays an integer below 2^24 -- exact in the FP32 accumulator
// whatever the order of the tensor core's additions -- when the row holds
// fewer than 2^17 stored counts.  Overflow-list entries (counts above 255) are
// added exactly on the CUDA cores.  FP8 E4M3 rows (row scale 2^e, e in {0, 1})
// and BF16 rows take the same path: E4M3 values convert exactly to FP16 (the
// row scale multiplies the limb sums in the epilogue), and BF16 values below
// 1024 as well; the converters check that every value, scaled, is an integer
// count below 1024 (else the row goes to the FP64 recheck), which keeps the
// argument above with T counted in scaled units.  The only errors are the weight
// quantisation, at most T 2^-(S+1) with T the file's token count, and two FP32
// roundings when the score is formed; the epilogue bounds both and marks the
// row for the FP64 recheck when the bound does not settle the label (or the
// log posteriors).
//
// Data flow.  The operand A (the files' counts as FP16) lives in tensor
// memory: the rows arrive in shared memory by 2-D tensor TMA (128 rows x 128
// bytes per box, 128-byte swizzle, zero fill past the last row and feature),
// converter warps read their rows' bytes, convert them and store them with
// tcgen05.st, so the MMA reads only the weight operand B from shared memory.
// One weight stage (3 C_p limb rows x 64 features, one bulk copy) feeds the
// MMAs of two 128-file tiles, which halves the weight traffic per file.
//
// Two launches of one kernel:
//   pass "pair"    units of 256 files (two 128-file tiles sharing each weight
//                  stage), one FP32 accumulation per row in tensor memory
//                  (2 x 192 columns) plus a ring of two A stages (128
//                  columns); rows of 2^17 or more stored counts could have
//                  rounded and are put on a list of heavy rows;
//   pass "chunked" units of 128 listed heavy rows (read by the converter warps
//                  straight from global memory), accumulated in 512-feature
//                  chunks (255 * 512 * 128 < 2^24: always exact) and joined in
//                  exact int64 sums in tensor memory (2 columns per class).
// Roles of one persistent CTA per SM (608 threads):
//   warps 0-15  convert rows to FP16 A stages, then run the epilogue (drain,
//               arg-max, top-2 margin, log-sum-exp, log posteriors);
//   warp 16     streams the weight-limb stages (one bulk copy each into this
//               CTA's own shared memory);
//   warp 17     allocates tensor memory and issues the MMAs (one thread);
//   warp 18     streams the rows of the pair pass (tensor TMA).
// Every wait is bounded; a wait that runs out raises ST_TIMEOUT, all roles
// stop, issued MMAs are waited for, and tensor memory is freed.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <math.h>

#include "device.cuh"
#include "internal.cuh"
#include "seg.cuh"
#include "tc.cuh"

namespace nbg {

constexpr int TC_M = 128;                  // files per tile (tensor-memory lanes)
constexpr int TC_KS = 64;                  // features per stage (4 MMAs, K = 16)
constexpr int TC_NB = 5;                   // weight stages in shared memory
constexpr int TC_ACC = 192;                // tensor-memory columns per FP32 accumulator
constexpr int TC_ACOL = 384;               // first A column (128 columns of A stages)
constexpr int TC_SUMCOL = 192;             // chunked pass: int64 sums, 2 columns per class
constexpr int TC_CHUNK = 8;                // stages per chunk of the chunked pass
constexpr float TC_T_EXACT = 131072.f;     // 128 T < 2^24: one accumulation is exact
constexpr int TC_WORK = 16;                // converter / epilogue warps
constexpr int TC_THREADS = (TC_WORK + 3) * 32;
constexpr int TC_BOX = 128;                // features per TMA box (128-byte swizzle span)
constexpr int TC_NRAW = 2;                 // row stages in shared memory (pair pass)
constexpr uint32_t TC_RAW_BYTES = 2 * TC_M * TC_BOX;   // both tiles, 128 features
constexpr int TC_PD = 3;                   // row stages loaded ahead into registers
constexpr long long TC_WAIT = 2000000000LL;
constexpr int kTcHeavyCap = 262144;        // heavy rows one call redoes exactly

// Per-pass constants: H tiles per unit (two in the pair pass), P class parts
// per row (the 16 warps cover H x 4 lane quadrants x P parts), BPT bytes of
// its row each converter thread converts per A stage, KA features per A
// stage, NA A stages in the 128 A columns of tensor memory.
template <int MODE>
struct TcPass {
  static constexpr int H = MODE == 0 ? 2 : 1;
  static constexpr int P = 4 / H;
  static constexpr int BPT = MODE == 0 ? 32 : 16;  // bytes per thread per A stage
  static constexpr int NV = BPT / 16;              // 16-byte vectors per thread per A stage
  static constexpr int COLS = BPT / 2;             // A columns per thread per A stage
  static constexpr int KA = BPT * P;               // features per A stage
  static constexpr int SUB = TC_KS / KA;           // A stages per weight stage
  static constexpr int ACOLS = KA / 2;             // A columns per tile per A stage
  static constexpr int NA = 128 / (ACOLS * H);     // A stages in the 128 A columns
  static constexpr int CPP = kTcMaxC / P;          // classes per part
  static constexpr int ROWS = TC_M * H;            // files per unit
};

struct TcModelArg {
  const uint8_t* wlay;
  const int32_t* q;
  const float* bias;
  const TcHeader* hdr;
  int C, Cp, N;
};

struct TcArgs {
  CUtensorMap tmap;         // u8 rows of g0 (single-group launch)
  const CUtensorMap* maps;  // group list: one map per group (device), else nullptr
  const SegGroup* groups;   // group list on the device, or nullptr: g0 alone
  const SegHeader* hdr;     // its header (tiles = 256-row units of the list)
  SegGroup g0;
  long long units0;         // 256-row units of g0
  TcModelArg models[kSegMaxModels];
  int F, nks, want_lp, recheck;
  int pf;                   // stages between the L2 prefetch of a row's bytes and their load
  uint32_t b_bytes;         // bytes of one weight stage slot (largest model)
  long long* heavy;         // pair pass: rows of 2^17+ stored counts (g0 only), or nullptr
  unsigned long long* heavy_n;   // their count (may exceed heavy_cap)
  int heavy_cap;
  int* status;
};

struct TcXch {               // partial epilogue results of each class part and row:
                             // entry part * rows-per-unit + row
  float best[512], second[512], se[512];
  float emax[512], T[512], Tplane[512];
  int idx[512];
};

struct TcShared {
  uint64_t raw_full[TC_NRAW], raw_empty[TC_NRAW];
  uint64_t b_full[TC_NB], b_empty[TC_NB];
  uint64_t a_full[4], a_empty[4];
  uint64_t acc_full, acc_empty, fin;
  uint64_t xfull, xfree;        // exchange written by all parts / read by all parts
  uint32_t tmem;
  int abort;
};

struct TcUnit {
  long long row0;   // first row of the unit within its group (pair pass)
  int g;            // group
  long long n;      // rows of the group
};

__device__ __forceinline__ const SegGroup& tc_group(const TcArgs& a, int g) {
  return a.groups ? a.groups[g] : a.g0;
}

// unit t of the pair pass: group and first row
__device__ __forceinline__ TcUnit tc_unit(const TcArgs& a, int n_groups, long long t) {
  int g = 0;
  if (a.groups && n_groups > 1)
    g = seg_find(n_groups, t, [&](int i) { return a.groups[i].tile0; });
  const SegGroup& G = tc_group(a, g);
  return TcUnit{(t - G.tile0) * 256, g, G.n};
}

__device__ __forceinline__ uint4 lds16(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(addr)
               : "memory");
  return v;
}

// two u8 counts (bytes picked by sel) -> two exact FP16 values: 1024 + b is
// 0x64bb in FP16, and subtracting 1024 is exact
__device__ __forceinline__ uint32_t u8x2_to_f16x2(uint32_t w, uint32_t sel) {
  const uint32_t x = __byte_perm(w, 0x64646464u, sel);
  uint32_t r;
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(0x64006400u));
  return r;
}

// two E4M3 values (the low 16 bits of w) -> two exact FP16 values
__device__ __forceinline__ uint32_t e4m3x2_to_f16x2(uint32_t w) {
  uint32_t r;
  asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(r) : "h"((unsigned short)w));
  return r;
}

// two BF16 values -> two FP16 values (exact for the integers below 1024 that
// the count check accepts)
__device__ __forceinline__ uint32_t bf16x2_to_f16x2(uint32_t w) {
  uint32_t r;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;"
      : "=r"(r)
      : "f"(__uint_as_float(w & 0xFFFF0000u)), "f"(__uint_as_float(w << 16)));
  return r;
}

// non-zero if a BF16 half of w is non-zero with magnitude below 2^-14 (its
// FP16 image would be subnormal or zero, which the count check cannot tell
// from an exact value)
__device__ __forceinline__ uint32_t bf16x2_tiny(uint32_t w) {
  const uint32_t mag = w & 0x7FFF7FFFu;
  const uint32_t nz = mag + 0x7FFF7FFFu;      // bit 15 of a half set: half >= 1
  const uint32_t big = mag + 0x47804780u;     // bit 15 of a half set: half >= 0x3880 (2^-14)
  return nz & ~big & 0x80008000u;
}

// Count check of an FP16 pair h against the magic pair m2 = (M, M), M = 2^(10-e):
// with w = h + M (FP16), a half of h is a non-negative multiple of 2^-e below M
// exactly when that half of w lies in [M, 2M) (its sign and exponent field is
// M's) and w - M == h; its count h 2^e is then the low 10 bits of w.  A failing
// half leaves a bit in bd.  The biased halves M + x are summed into tt (the
// caller removes M per value).
__device__ __forceinline__ void f16x2_count_check(uint32_t h, uint32_t m2, uint32_t& tt,
                                                  uint32_t& bd) {
  uint32_t w, back;
  asm("add.rn.f16x2 %0, %1, %2;" : "=r"(w) : "r"(h), "r"(m2));
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(back) : "r"(w), "r"(m2));
  bd |= (back ^ h) | ((w & 0xFC00FC00u) ^ m2);
  tt = (uint32_t)dp2a_lo_us(w, 0x01010101u, (int)tt);
}

// bounded wait that sleeps in the barrier instead of polling
__device__ __forceinline__ bool tc_wait_sleep(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait_sleep(bar, parity, 100000u)) {
    if (clock64() - t0 > TC_WAIT) return false;
  }
  return true;
}

__device__ __forceinline__ bool tc_aborted(TcShared& sh) {
  return *reinterpret_cast<volatile int*>(&sh.abort) != 0;
}

__device__ __forceinline__ bool tc_wait(TcShared& sh, uint64_t* bar, uint32_t parity, int* status) {
  if (tc_wait_sleep(bar, parity)) return true;
  atomicOr(status, ST_TIMEOUT);
  *reinterpret_cast<volatile int*>(&sh.abort) = 1;
  return false;
}

// every lane waits (each observes the phase, so each may read what it
// guards); the warp follows the outcome together
__device__ __forceinline__ bool tc_wait_warp(TcShared& sh, uint64_t* bar, uint32_t parity,
                                             int* status) {
  const bool mine = tc_wait_sleep(bar, parity);
  const bool all = __all_sync(0xFFFFFFFFu, mine) != 0;
  if (!all && (threadIdx.x & 31) == 0) {
    atomicOr(status, ST_TIMEOUT);
    *reinterpret_cast<volatile int*>(&sh.abort) = 1;
  }
  return all;
}

// D[tmem] (+)= A[tmem] * B[smem]^T, issued by one thread (A: 128 lanes = rows,
// two FP16 values of consecutive features per 32-bit column)
__device__ __forceinline__ void tc_mma_f16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc,
                                              uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}


// ---------------------------------------------------------------------------
// epilogue
// ---------------------------------------------------------------------------
// Exact fixed-point sums of classes cb .. cb+7 of this thread's row from the
// int64 sums of the chunked pass (warp-uniform arguments: the tensor-memory
// loads are warp-wide).
__device__ __forceinline__ void tc_load_sums8(uint32_t lane_base, int cb, long long (&q)[8]) {
  uint32_t sw[16];
  tmem_ld16(lane_base + (uint32_t)(TC_SUMCOL + 2 * cb), sw);
  tmem_ld_wait();
#pragma unroll
  for (int i = 0; i < 8; ++i)
    q[i] = (long long)(((unsigned long long)sw[2 * i + 1] << 32) | sw[2 * i]);
}

// The exact limb sums of classes cb .. cb+7 of tile h (FP32 integers of the
// pair pass), q[i] = a0 + 2^8 a1 + 2^16 a2, one limb at a time.
__device__ __forceinline__ void tc_load_acc8(uint32_t lane_base, int h, int Cp, int cb,
                                             long long (&q)[8]) {
  const uint32_t acc = lane_base + (uint32_t)(TC_ACC * h + cb);
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    uint32_t v[8];
    tmem_ld8(acc + (uint32_t)(l * Cp), v);
    tmem_ld_wait();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const long long x = (long long)__float2int_rn(__uint_as_float(v[i])) << (8 * l);
      q[i] = l == 0 ? x : q[i] + x;
    }
  }
}

// Scores s of classes cb .. cb+7 of this thread's row, and per class e = the
// sum of the magnitudes of the prior and of every rounded FP32 result on the
// way (each rounding is within 2^-24 of its result, the prior's within 2^-24
// of itself).  Pair pass: s = ((a0 sc + b) + a1 2^8 sc) + a2 2^16 sc from the
// exact FP32 limb sums (sc = 2^-S: the products are exact, each FMA rounds
// once), then + (float)(overflow sum) sc.  Chunked pass: the exact int64 sum
// q (overflow entries included) is rounded once to FP32 and enters one FMA
// with the prior.  `added` receives the overflow entries' counts.
template <int MODE>
__device__ __forceinline__ void tc_scores8(const SegGroup& G, const TcModelArg& M, int F,
                                           uint32_t lane_base, int h, int cb, bool any_ovf,
                                           long long k0, long long k1, float rsc, float (&s)[8],
                                           float (&e)[8], float& added) {
  const float sc = M.hdr->scale * rsc;   // rsc: the row's power-of-two scale (FP8 rows)
  added = 0.f;
  if (MODE == 0) {
    // the three limbs' loads in flight together, one wait
    const uint32_t acc = lane_base + (uint32_t)(TC_ACC * h + cb);
    uint32_t v[3][8];
#pragma unroll
    for (int l = 0; l < 3; ++l) tmem_ld8(acc + (uint32_t)(l * M.Cp), v[l]);
    float b[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) b[i] = cb + i < M.C ? M.bias[cb + i] : 0.f;
    tmem_ld_wait();
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      const float w = sc * (float)(1 << (8 * l));
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        s[i] = fmaf(__uint_as_float(v[l][i]), w, l == 0 ? b[i] : s[i]);
        e[i] = (l == 0 ? fabsf(b[i]) : e[i]) + fabsf(s[i]);
      }
    }
  } else {
    long long q[8];
    tc_load_sums8(lane_base, cb, q);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float b = cb + i < M.C ? M.bias[cb + i] : 0.f;
      const float v = fmaf((float)(int)(q[i] >> 24), 16777216.f, (float)(int)(q[i] & 0xFFFFFF));
      s[i] = fmaf(v, sc, b);
      e[i] = fabsf(b) + fabsf(v * sc) + fabsf(s[i]);
    }
  }
  if (any_ovf) {   // overflow entries (counts above 255): exact int64 sums per class
#pragma unroll 1
    for (long long k = k0; k < k1; ++k) {
      const int j = G.ovf_col[k];
      if (j < F) added += (float)G.ovf_add[k];
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (cb + i >= M.C) break;
      long long o = 0;
#pragma unroll 1
      for (long long k = k0; k < k1; ++k) {
        const int j = G.ovf_col[k];
        if (j < F) o += (long long)G.ovf_add[k] * (long long)M.q[(long long)(cb + i) * F + j];
      }
      // the sum joins the score with two roundings (the conversion, the add)
      const float t = (float)o * sc;
      const float si = s[i] + t;
      e[i] += fabsf(t) + fabsf(si);
      s[i] = si;
    }
  }
}

// Epilogue of one row for this thread's class part: pass 1 (arg-max, second
// best, sum of exponentials) over the part's classes, exchange with the other
// parts through shared memory, label / margin / recheck mark by part 0, pass 2
// (log posteriors, the scores formed again).  grow < 0: a row past the end
// (every lane still runs the warp-wide tensor-memory loads).
template <int MODE>
__device__ __forceinline__ bool tc_epilogue(const TcArgs& a, TcShared& sh, TcXch& xe,
                                            const SegGroup& G, const TcModelArg& M,
                                            long long grow, int xr, int h, int part,
                                            uint32_t Tpart, float rsc, uint32_t lane_base,
                                            int& ep) {
  using PS = TcPass<MODE>;
  const int lane = threadIdx.x & 31;
  const bool valid = grow >= 0;
  const int F = a.F;
  const int c0 = PS::CPP * part;
  long long k0 = 0, k1 = 0;
  if (valid && G.ovf_ptr) {
    k0 = G.ovf_ptr[grow];
    k1 = G.ovf_ptr[grow + 1];
  }
  const bool any_ovf = __any_sync(0xFFFFFFFFu, k1 > k0);
  const float tau_unit = M.hdr->tau_unit;
  float T = (float)Tpart;
  // pass 1; the pair pass keeps the part's scores in registers for pass 2
  float best = -INFINITY, second = -INFINITY, emax = 0.f, se = 0.f;
  int bidx = 0x7FFFFFFF;
  float keep[MODE == 0 ? PS::CPP : 1];
#pragma unroll
  for (int ch = 0; ch < PS::CPP / 8; ++ch) {
    const int cb = c0 + 8 * ch;
    if (cb >= M.Cp) break;
    float sc[8], er[8], added;
    tc_scores8<MODE>(G, M, F, lane_base, h, cb, any_ovf, k0, k1, rsc, sc, er, added);
    if (part == 0 && ch == 0) T += added;
    if constexpr (MODE == 0) {
#pragma unroll
      for (int i = 0; i < 8; ++i) keep[8 * ch + i] = sc[i];
    }
    // the chunk's best, second best and sum of exp(s - chunk best), in class
    // order (ties keep the lower index); the exponentials are independent
    float b8 = -INFINITY, s8b = -INFINITY;
    int i8 = 0x7FFFFFFF;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (cb + i >= M.C) break;
      emax = fmaxf(emax, er[i]);
      if (sc[i] > b8) {
        s8b = b8;
        b8 = sc[i];
        i8 = cb + i;
      } else if (sc[i] > s8b) {
        s8b = sc[i];
      }
    }
    float e8 = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (cb + i < M.C) e8 += __expf(sc[i] - b8);   // ~2^-21 relative: lse to ~1e-6
    // merge into the running values (sum of exp(s - best))
    if (b8 > best) {
      se = se * expf(best - b8) + e8;
      second = fmaxf(best, s8b);
      best = b8;
      bidx = i8;
    } else {
      se += e8 * expf(b8 - best);
      second = fmaxf(second, b8);
    }
  }
  const int eph = ep & 1;
  // the exchange of the previous row set must have been read by every part
  if (!tc_wait_warp(sh, &sh.xfree, (uint32_t)eph ^ 1u, a.status)) return false;
  xe.best[part * PS::ROWS + xr] = best;
  xe.second[part * PS::ROWS + xr] = second;
  xe.se[part * PS::ROWS + xr] = se;
  xe.emax[part * PS::ROWS + xr] = emax;
  xe.T[part * PS::ROWS + xr] = T;
  xe.Tplane[part * PS::ROWS + xr] = (float)Tpart;
  xe.idx[part * PS::ROWS + xr] = bidx;
  __syncwarp();
  if (lane == 0) mbar_arrive(&sh.xfull);
  if (!tc_wait_warp(sh, &sh.xfull, (uint32_t)eph, a.status)) return false;
  ++ep;
  // combine the parts in class order (ties go to the lower class index)
  float Bv = -INFINITY, S2 = -INFINITY, em = 0.f, Tt = 0.f, Tp = 0.f;
  int Bi = 0x7FFFFFFF;
#pragma unroll
  for (int k = 0; k < PS::P; ++k) {
    const float xb = xe.best[k * PS::ROWS + xr];
    Tp += xe.Tplane[k * PS::ROWS + xr];
    if (xb > Bv) {
      S2 = fmaxf(Bv, xe.second[k * PS::ROWS + xr]);
      Bv = xb;
      Bi = xe.idx[k * PS::ROWS + xr];
    } else {
      S2 = fmaxf(S2, xb);
    }
    em = fmaxf(em, xe.emax[k * PS::ROWS + xr]);
    Tt += xe.T[k * PS::ROWS + xr];
  }
  float sum = 0.f;
#pragma unroll
  for (int k = 0; k < PS::P; ++k) {
    const float xs = xe.se[k * PS::ROWS + xr];
    if (xs > 0.f) sum += xs * expf(xe.best[k * PS::ROWS + xr] - Bv);
  }
  __syncwarp();
  if (lane == 0) mbar_arrive(&sh.xfree);   // this row set's exchange is read
  const float lse = Bv + logf(sum);
  const float margin = Bv - S2;
  // |s_c - exact| <= T 2^-(S+1) (weight quantisation) + 2^-24 e_c (FP32
  // roundings); two classes form the margin
  const float tau = 2.f * (Tt * tau_unit + 5.9604645e-8f * em) * (1.f + 1.f / 1048576.f) + 1e-30f;
  bool flag = false;
  if (a.recheck != NB_RECHECK_OFF) {
    flag = !(margin > tau);
    if (a.recheck == NB_RECHECK_LP && tau > 5e-6f * fmaxf(1.f, margin)) flag = true;
  }
  // pair pass: a row of 2^17 or more stored counts may have rounded in its
  // single accumulation: marked, and listed for the chunked pass (beyond the
  // list's capacity, or in a batch, the FP64 recheck resolves it)
  const bool heavy = MODE == 0 && !(Tp < TC_T_EXACT);
  if (valid && part == 0) {
    G.label[grow] = (flag || heavy) ? kLabelRecheck : (uint8_t)Bi;
    G.margin[grow] = margin;
    if (heavy && a.heavy) {
      const unsigned long long k = atomicAdd(a.heavy_n, 1ull);
      if (k < (unsigned long long)a.heavy_cap) a.heavy[k] = grow;
    }
  }
  if (a.want_lp && G.logpost) {
    // pass 2; a full chunk of 8 classes goes out as two 16-byte stores when the
    // row's log posteriors are 16-byte aligned
    float* lp = G.logpost + (valid ? grow : 0) * M.C;
    const bool vec = (reinterpret_cast<uintptr_t>(lp) & 15) == 0;
#pragma unroll
    for (int ch = 0; ch < PS::CPP / 8; ++ch) {
      const int cb = c0 + 8 * ch;
      if (cb >= M.Cp) break;
      float sc[8];
      if constexpr (MODE == 0) {
#pragma unroll
        for (int i = 0; i < 8; ++i) sc[i] = keep[8 * ch + i];
      } else {
        float er[8], added;
        tc_scores8<MODE>(G, M, F, lane_base, h, cb, any_ovf, k0, k1, rsc, sc, er, added);
      }
      if (!valid) continue;
      if (vec && cb + 8 <= M.C) {
        float4* d = reinterpret_cast<float4*>(lp + cb);
        d[0] = make_float4(sc[0] - lse, sc[1] - lse, sc[2] - lse, sc[3] - lse);
        d[1] = make_float4(sc[4] - lse, sc[5] - lse, sc[6] - lse, sc[7] - lse);
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (cb + i < M.C) lp[cb + i] = sc[i] - lse;
      }
    }
  }
  return true;
}

// chunked pass: add the chunk's three limb sums (exact integers below 2^24 in
// FP32) into this thread's int64 sums in tensor memory (2 columns per class,
// low word first), 8 classes at a time
__device__ __forceinline__ void tc_drain_chunk(int Cp, int c0, int cpp, bool first,
                                               uint32_t lane_base) {
#pragma unroll 1
  for (int cb = c0; cb < c0 + cpp; cb += 8) {
    if (cb >= Cp) break;
    uint32_t sw[16];
    const uint32_t sum_addr = lane_base + (uint32_t)(TC_SUMCOL + 2 * cb);
    if (first) {
#pragma unroll
      for (int i = 0; i < 16; ++i) sw[i] = 0;
    } else {
      tmem_ld16(sum_addr, sw);
      tmem_ld_wait();
    }
    long long q[8];
    tc_load_acc8(lane_base, 0, Cp, cb, q);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      unsigned long long x = ((unsigned long long)sw[2 * i + 1] << 32) | sw[2 * i];
      x += (unsigned long long)q[i];
      sw[2 * i] = (uint32_t)x;
      sw[2 * i + 1] = (uint32_t)(x >> 32);
    }
    tmem_st16(sum_addr, sw);
    tmem_st_wait();
  }
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------
// This CTA's first weight stage of every unit in the pair pass: CTAs start at
// different stages (in pairs, so that a row stage's two halves stay together;
// only when the stages pair up exactly) and wrap around, so that they do not
// all fetch the same weight stage from L2 at the same time.  The limb sums are
// exact integers, so the order of the stages does not change them.
template <int MODE>
__device__ __forceinline__ int tc_rot(int nks) {
  return (MODE == 0 && nks % 2 == 0) ? 2 * (int)((blockIdx.x * 37u) % (unsigned)(nks / 2)) : 0;
}

// units of this CTA: the pass's unit count, dealt round-robin
template <int MODE>
__device__ __forceinline__ long long tc_units(const TcArgs& a) {
  if (MODE == 0) return a.groups ? a.hdr->tiles : a.units0;
  unsigned long long c = *a.heavy_n;
  if (c > (unsigned long long)a.heavy_cap) c = (unsigned long long)a.heavy_cap;
  return (long long)((c + TC_M - 1) / TC_M);
}

// DT: storage of the rows (NB_U8, NB_FP8E4M3 or NB_BF16; the chunked pass
// takes u8 rows only).  A 128-byte row box holds BOXF features.
template <int MODE, int DT>
__global__ void __launch_bounds__(TC_THREADS, 1) k_score_tc(const __grid_constant__ TcArgs a) {
  using PS = TcPass<MODE>;
  static_assert(MODE == 0 || DT == NB_U8, "the chunked pass reads u8 rows");
  constexpr int ES = DT == NB_BF16 ? 2 : 1;        // bytes per feature
  constexpr int BOXF = TC_BOX / ES;                 // features per row stage
  extern __shared__ __align__(1024) uint8_t tc_smem[];
  TcShared& sh = *reinterpret_cast<TcShared*>(tc_smem);
  TcXch& xe = *reinterpret_cast<TcXch*>(tc_smem + 1024);
  // 1 KB aligned: the swizzled row stages (pair pass only), then the weights
  uint8_t* raw = tc_smem + 1024 + ((sizeof(TcXch) + 1023) / 1024) * 1024;
  uint8_t* B = raw + (MODE == 0 ? (size_t)TC_NRAW * TC_RAW_BYTES : 0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_groups = a.groups ? a.hdr->n_groups : 1;
  const long long n_units = tc_units<MODE>(a);
  const long long my_units =
      n_units > (long long)blockIdx.x ? (n_units - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const int nks = a.nks, F = a.F;
  // chunked pass: the listed rows' count
  long long n_heavy = 0;
  if (MODE == 1) n_heavy = (long long)min(*a.heavy_n, (unsigned long long)a.heavy_cap);

  if (threadIdx.x == 0) {
    for (int i = 0; i < TC_NRAW; ++i) {
      mbar_init(&sh.raw_full[i], 1);
      mbar_init(&sh.raw_empty[i], TC_WORK);
    }
    for (int i = 0; i < TC_NB; ++i) {
      mbar_init(&sh.b_full[i], 1);
      mbar_init(&sh.b_empty[i], 1);
    }
    for (int i = 0; i < PS::NA; ++i) {
      mbar_init(&sh.a_full[i], TC_WORK);
      mbar_init(&sh.a_empty[i], 1);
    }
    mbar_init(&sh.acc_full, 1);
    mbar_init(&sh.acc_empty, TC_WORK);
    mbar_init(&sh.fin, 1);
    mbar_init(&sh.xfull, TC_WORK);
    mbar_init(&sh.xfree, TC_WORK);
    sh.abort = 0;
  }
  if (warp == TC_WORK + 1) tmem_alloc(&sh.tmem, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh.tmem;

  if (warp == TC_WORK) {
    // ---- weight-limb producer -----------------------------------------
    if (lane == 0) {
      long long bi = 0, last[TC_NB];
      for (int s = 0; s < TC_NB; ++s) last[s] = -1;
      bool ok = true;
      for (long long it = 0; it < my_units && ok && !tc_aborted(sh); ++it) {
        const long long t = blockIdx.x + it * gridDim.x;
        const int g = MODE == 0 ? tc_unit(a, n_groups, t).g : 0;
        const TcModelArg& M = a.models[tc_group(a, g).model];
        const uint32_t sb = (uint32_t)M.N * 128u;
        const int rot = tc_rot<MODE>(nks);
        for (int ks = 0; ks < nks; ++ks, ++bi) {
          const int slot = (int)(bi % TC_NB);
          const uint32_t par = (uint32_t)((bi / TC_NB) & 1);
          if (!tc_wait(sh, &sh.b_empty[slot], par ^ 1u, a.status)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&sh.b_full[slot], sb);
          const int kse = ks + rot < nks ? ks + rot : ks + rot - nks;
          bulk_g2s(B + (size_t)slot * a.b_bytes, M.wlay + (size_t)kse * sb, sb, &sh.b_full[slot]);
          last[slot] = bi;
        }
      }
      // copies still in flight land before the CTA exits
      for (int s = 0; s < TC_NB; ++s)
        if (last[s] >= 0)
          tc_wait(sh, &sh.b_full[s], (uint32_t)((last[s] / TC_NB) & 1), a.status);
    }
    __syncwarp();
  } else if (warp == TC_WORK + 2) {
    // ---- row producer (pair pass) ----------------------------------------
    if (MODE == 0 && lane == 0) {
      long long ri = 0, last[TC_NRAW];
      for (int s = 0; s < TC_NRAW; ++s) last[s] = -1;
      bool ok = (smem_addr(raw) & 1023u) == 0;   // the swizzled reads assume 1 KB alignment
      if (!ok) {
        atomicOr(a.status, ST_TIMEOUT);
        *reinterpret_cast<volatile int*>(&sh.abort) = 1;
      }
      const uint64_t map0 = reinterpret_cast<uint64_t>(&a.tmap);
      for (long long it = 0; it < my_units && ok && !tc_aborted(sh); ++it) {
        const long long t = blockIdx.x + it * gridDim.x;
        const TcUnit U = tc_unit(a, n_groups, t);
        // a group's map sits in the work list, rewritten between calls: drop
        // any stale copy the tensor-map proxy may hold
        const uint64_t tmap = a.maps ? reinterpret_cast<uint64_t>(a.maps + U.g) : map0;
        if (a.maps)
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmap)
                       : "memory");
        // row stages of BOXF features; the rotation counts weight stages of TC_KS
        const int nraw = (F + BOXF - 1) / BOXF, rot = tc_rot<MODE>(nks) * TC_KS / BOXF;
        for (int rs = 0; rs < nraw; ++rs, ++ri) {
          const int f0 = BOXF * (rs + rot < nraw ? rs + rot : rs + rot - nraw);
          const int slot = (int)(ri % TC_NRAW);
          const uint32_t par = (uint32_t)((ri / TC_NRAW) & 1);
          if (!tc_wait(sh, &sh.raw_empty[slot], par ^ 1u, a.status)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&sh.raw_full[slot], TC_RAW_BYTES);
          uint8_t* dst = raw + (size_t)slot * TC_RAW_BYTES;
#pragma unroll
          for (int h = 0; h < 2; ++h)
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst + h * (TC_M * TC_BOX))),
                "l"(tmap), "r"(f0), "r"((int)(U.row0 + TC_M * h)),
                "r"(smem_addr(&sh.raw_full[slot]))
                : "memory");
          last[slot] = ri;
        }
      }
      // copies still in flight land before the CTA exits
      for (int s = 0; s < TC_NRAW; ++s)
        if (last[s] >= 0)
          tc_wait(sh, &sh.raw_full[s], (uint32_t)((last[s] / TC_NRAW) & 1), a.status);
    }
    __syncwarp();
  } else if (warp == TC_WORK + 1) {
    // ---- MMA issuer -----------------------------------------------------
    if (lane == 0) {
      long long bi = 0, ai = 0, ci = 0;
      bool ok = true;
      const int chunk = MODE == 0 ? nks : TC_CHUNK;
      for (long long it = 0; it < my_units && ok && !tc_aborted(sh); ++it) {
        const long long t = blockIdx.x + it * gridDim.x;
        const int g = MODE == 0 ? tc_unit(a, n_groups, t).g : 0;
        const TcModelArg& M = a.models[tc_group(a, g).model];
        const uint32_t idesc = tc_idesc_f16(TC_M, M.N);
        int kc = 0;
        for (int ks = 0; ks < nks && ok; ++ks) {
          if (kc == 0 && ci > 0) {   // the accumulators were drained
            if (!tc_wait(sh, &sh.acc_empty, (uint32_t)((ci - 1) & 1), a.status)) {
              ok = false;
              break;
            }
          }
          const int bslot = (int)(bi % TC_NB);
          if (!tc_wait(sh, &sh.b_full[bslot], (uint32_t)((bi / TC_NB) & 1), a.status)) {
            ok = false;
            break;
          }
          const uint32_t bs = smem_addr(B + (size_t)bslot * a.b_bytes);
          // the weight stage's A stages, KA features each
#pragma unroll
          for (int sub = 0; sub < PS::SUB; ++sub) {
            const int aslot = (int)(ai % PS::NA);
            if (!tc_wait(sh, &sh.a_full[aslot], (uint32_t)((ai / PS::NA) & 1), a.status)) {
              ok = false;
              break;
            }
            tc_fence_after();
#pragma unroll
            for (int h = 0; h < PS::H; ++h)
#pragma unroll
              for (int j = 0; j < PS::KA / 16; ++j)
                tc_mma_f16_ts(tmem + (uint32_t)(TC_ACC * h),
                              tmem + (uint32_t)(TC_ACOL + aslot * PS::ACOLS * PS::H +
                                                PS::ACOLS * h + 8 * j),
                              tc_desc(bs + 256u * (uint32_t)(sub * (PS::KA / 16) + j), 128u, 1024u),
                              idesc, (uint32_t)(kc | sub | j));
            tc_commit(&sh.a_empty[aslot]);
            ++ai;
          }
          if (!ok) break;
          tc_commit(&sh.b_empty[bslot]);
          ++bi;
          if (++kc == chunk || ks == nks - 1) {
            tc_commit(&sh.acc_full);
            ++ci;
            kc = 0;
          }
        }
      }
      // every MMA issued so far has completed once this arrives
      tc_commit(&sh.fin);
      tc_wait(sh, &sh.fin, 0, a.status);
    }
    __syncwarp();
  } else {
    // ---- converters / drains / epilogue (warps 0 .. TC_WORK-1) ----------
    const int qd = warp & 3, rest = warp >> 2;
    const int h = rest % PS::H, part = rest / PS::H;
    const int xr = TC_M * h + 32 * qd + lane;     // exchange row of this thread
    const uint32_t lane_base = tmem + ((uint32_t)(32 * qd) << 16);
    const uint32_t a_col = (uint32_t)(TC_ACOL + PS::ACOLS * h + PS::COLS * part);
    const int nka = nks * PS::SUB;                // A stages per row
    const long long total = my_units * nka;
    const int chunk = MODE == 0 ? nka : TC_CHUNK * PS::SUB;   // A stages per accumulation
    int ep = 0;
    long long ai = 0, ci = 0;
    bool ok = true;

    // row of this thread in unit ordinal i (-1: past the end)
    auto row_of = [&](long long i, int& g) -> long long {
      const long long t = blockIdx.x + i * gridDim.x;
      if (MODE == 0) {
        const TcUnit U = tc_unit(a, n_groups, t);
        g = U.g;
        const long long r = U.row0 + TC_M * h + 32 * qd + lane;
        return r < U.n ? r : -1;
      }
      g = 0;
      const long long idx = t * TC_M + 32 * qd + lane;
      return idx < n_heavy ? a.heavy[idx] : -1;
    };

    // chunked pass: the listed rows' bytes come from global memory, TC_PD - 1
    // A stages ahead of the conversion
    long long l_i = 0;
    int l_ka = 0, l_g = 0;
    long long l_row = (MODE == 1 && total > 0) ? row_of(0, l_g) : -1;
    const unsigned char* l_rp =
        l_row >= 0 ? reinterpret_cast<const unsigned char*>(tc_group(a, l_g).X) +
                         l_row * tc_group(a, l_g).ld_bytes
                   : nullptr;
    auto load_next = [&](uint4& dst) {
      const int f = PS::KA * l_ka + PS::BPT * part;
      // the same bytes a.pf stages on are fetched into L2 now
      if (l_rp && f + PS::KA * a.pf < F)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(l_rp + f + PS::KA * a.pf));
      uint4 x = make_uint4(0, 0, 0, 0);
      if (l_rp && f < F) {
        x = ld_stream16(l_rp + f);
        if (f + 16 > F) {   // zero the bytes past F
          const int keep = F - f;
          uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int vb = keep - 4 * k;
            w[k] &= vb >= 4 ? 0xFFFFFFFFu : (vb <= 0 ? 0u : ((1u << (8 * vb)) - 1u));
          }
          x = make_uint4(w[0], w[1], w[2], w[3]);
        }
      }
      dst = x;
      if (++l_ka == nka) {
        l_ka = 0;
        if (++l_i < my_units) {
          l_row = row_of(l_i, l_g);
          const SegGroup& G = tc_group(a, l_g);
          l_rp = l_row >= 0 ? reinterpret_cast<const unsigned char*>(G.X) + l_row * G.ld_bytes
                            : nullptr;
        } else {
          l_rp = nullptr;
        }
      }
    };
    uint4 buf[MODE == 1 ? TC_PD : 1];
    if constexpr (MODE == 1) {
#pragma unroll
      for (int d = 0; d < TC_PD - 1; ++d)
        if (d < total) load_next(buf[d]);
    }
    long long ri = 0;   // pair pass: row stages consumed
    const uint32_t raw_s = smem_addr(raw) + (uint32_t)(h * TC_M * TC_BOX);
    const int rr = 32 * qd + lane;   // row within the tile
    constexpr int RAW_A = BOXF / PS::KA;     // A stages per row stage
    constexpr int NVT = PS::NV * ES;         // 16-byte chunks per thread per A stage
    constexpr int CPA = PS::KA * ES / 16;    // 16-byte chunks of a row per A stage
    // FP8 / BF16 rows: the magic pair of the count check, and the row's flag
    // and scale (set at the start of each unit)
    uint32_t m2 = 0x64006400u, bad = 0u;
    float rsc = 1.f;

    // consumer state
    long long c_i = 0;
    int c_ka = 0, kc = 0;
    uint32_t T = 0;
    for (long long base = 0; base < total && ok; base += TC_PD) {
#pragma unroll
      for (int d = 0; d < TC_PD; ++d) {
        if (base + d >= total || !ok) break;
        if (tc_aborted(sh)) {
          ok = false;
          break;
        }
        uint4 xv[NVT];
        if constexpr (MODE == 1) {
          if (base + d + TC_PD - 1 < total) load_next(buf[(d + TC_PD - 1) % TC_PD]);
          xv[0] = buf[d];
        } else {
          // this thread's bytes of the A stage: 16-byte chunks of its row in
          // the row stage, swizzled by the row (rows and features past the end
          // arrive as zeros)
          const uint32_t slot = (uint32_t)(ri % TC_NRAW);
          if (c_ka % RAW_A == 0 &&
              !tc_wait_warp(sh, &sh.raw_full[slot], (uint32_t)((ri / TC_NRAW) & 1), a.status)) {
            ok = false;
            break;
          }
#pragma unroll
          for (int v = 0; v < NVT; ++v) {
            const int c16 = CPA * (c_ka % RAW_A) + NVT * part + v;
            xv[v] = lds16(raw_s + slot * TC_RAW_BYTES +
                          (uint32_t)(rr * TC_BOX + ((c16 ^ (rr & 7)) << 4)));
          }
        }
        if (DT != NB_U8 && c_ka == 0) {
          // a new unit: this thread's row scale (FP8 rows: 2^e, e in {0, 1};
          // any other exponent sends the row to the FP64 recheck)
          bad = 0u;
          m2 = 0x64006400u;
          rsc = 1.f;
          if (DT == NB_FP8E4M3) {
            int g = 0;
            const long long r = row_of(c_i, g);
            const int8_t* re = tc_group(a, g).row_exp;
            const int e = (re && r >= 0) ? (int)re[r] : 0;
            if (e == 1) {
              m2 = 0x60006000u;
              rsc = 2.f;
            } else if (e != 0) {
              bad = 1u;
            }
          }
        }
        // convert this thread's values to FP16 pairs
        uint32_t o[PS::COLS];
        if constexpr (DT == NB_U8) {
#pragma unroll
          for (int v = 0; v < NVT; ++v) {
            const uint4 x = xv[v];
            T = dp4a_uu(x.x, 0x01010101u, T);
            T = dp4a_uu(x.y, 0x01010101u, T);
            T = dp4a_uu(x.z, 0x01010101u, T);
            T = dp4a_uu(x.w, 0x01010101u, T);
            o[8 * v + 0] = u8x2_to_f16x2(x.x, 0x5140u);
            o[8 * v + 1] = u8x2_to_f16x2(x.x, 0x7362u);
            o[8 * v + 2] = u8x2_to_f16x2(x.y, 0x5140u);
            o[8 * v + 3] = u8x2_to_f16x2(x.y, 0x7362u);
            o[8 * v + 4] = u8x2_to_f16x2(x.z, 0x5140u);
            o[8 * v + 5] = u8x2_to_f16x2(x.z, 0x7362u);
            o[8 * v + 6] = u8x2_to_f16x2(x.w, 0x5140u);
            o[8 * v + 7] = u8x2_to_f16x2(x.w, 0x7362u);
          }
        } else {
#pragma unroll
          for (int v = 0; v < NVT; ++v) {
            const uint32_t w[4] = {xv[v].x, xv[v].y, xv[v].z, xv[v].w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              if constexpr (DT == NB_FP8E4M3) {
                o[8 * v + 2 * k] = e4m3x2_to_f16x2(w[k] & 0xFFFFu);
                o[8 * v + 2 * k + 1] = e4m3x2_to_f16x2(w[k] >> 16);
              } else {
                o[4 * v + k] = bf16x2_to_f16x2(w[k]);
                bad |= bf16x2_tiny(w[k]);
              }
            }
          }
          // every value an integer count x = v 2^e below 1024: x sits in the
          // low 10 bits of v + M; T sums M + x (at most 2^15 + 2^10 for each of
          // 32 values per A stage: no wrap below 2^32 for F <= 8192)
#pragma unroll
          for (int k = 0; k < PS::COLS; ++k) f16x2_count_check(o[k], m2, T, bad);
        }
        if constexpr (MODE == 0) {
          if (c_ka % RAW_A == RAW_A - 1 || c_ka == nka - 1) {   // done with the row stage
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh.raw_empty[ri % TC_NRAW]);
            ++ri;
          }
        }
        const int aslot = (int)(ai % PS::NA);
        if (!tc_wait_warp(sh, &sh.a_empty[aslot], (uint32_t)((ai / PS::NA) & 1) ^ 1u,
                          a.status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        if constexpr (PS::COLS == 16) tmem_st16(lane_base + a_col + (uint32_t)(aslot * PS::ACOLS * PS::H), o);
        else tmem_st8(lane_base + a_col + (uint32_t)(aslot * PS::ACOLS * PS::H), o);
        tmem_st_wait();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.a_full[aslot]);
        ++ai;
        const bool unit_end = c_ka == nka - 1;
        if (++kc == chunk || unit_end) {
          // the accumulation cycle is complete: drain (chunked) and / or run
          // the epilogue of the unit
          kc = 0;
          if (!tc_wait_warp(sh, &sh.acc_full, (uint32_t)(ci & 1), a.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          if (MODE == 1) {
            tc_drain_chunk(a.models[0].Cp, PS::CPP * part, PS::CPP, c_ka < chunk, lane_base);
            // the chunk's sums are in the int64 columns: the MMAs may go on
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh.acc_empty);
          }
          if (unit_end) {
            int g = 0;
            const long long r = row_of(c_i, g);
            const SegGroup& G = tc_group(a, g);
            uint32_t Tu = T;
            if (DT != NB_U8) {
              // the unit's check; then the counts' total without the bias M of
              // each of the 2 COLS values of every A stage
              Tu = bad != 0u ? 0xFFFFFFFFu
                        : T - (m2 & 0xFFFFu) * (uint32_t)(2 * PS::COLS) * (uint32_t)nka;
            }
            if (!tc_epilogue<MODE>(a, sh, xe, G, a.models[G.model], r, xr, h, part, Tu, rsc,
                                   lane_base, ep)) {
              ok = false;
              break;
            }
            T = 0;
          }
          if (MODE == 0) {   // the accumulators are read: the next unit's MMAs may start
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh.acc_empty);
          }
          ++ci;
        }
        if (++c_ka == nka) {
          c_ka = 0;
          ++c_i;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == TC_WORK + 1) tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------------------
// tables: fixed-point weights and their FP16 limbs in the MMA operand layout
// ---------------------------------------------------------------------------
__global__ void k_derive_tc(const double* log_theta, int C, int F, int Cp, int nks,
                            const float* wmax, uint8_t* wlay, int32_t* q, TcHeader* hdr) {
  const int N = 3 * Cp;
  // |w| <= wmax (1 + 2^-24) < 2^e; then |Q| = |round(w 2^S)| <= 2^22
  const float wm = *wmax;
  int e = 0;
  if (wm > 0.f && isfinite(wm)) frexpf(wm * (1.f + 1.f / 1048576.f), &e);
  int S = 22 - e;
  if (S > 120) S = 120;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    hdr->S = S;
    hdr->scale = ldexpf(1.f, -S);
    hdr->tau_unit = ldexpf(1.f, -S - 1);
    hdr->pad = 0;
  }
  const double sc = ldexp(1.0, S);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nks * TC_KS;
       j += gridDim.x * blockDim.x) {
    double m = 0.0;
    if (j < F) {
      for (int c = 0; c < C; ++c) m += log_theta[(size_t)c * F + j];
      m /= (double)C;
    }
    const int ks = j / TC_KS, kk = j % TC_KS;
    uint8_t* stage = wlay + (size_t)ks * N * 128;
    for (int c = 0; c < Cp; ++c) {
      int Q = 0;
      if (c < C && j < F) {
        const double w = log_theta[(size_t)c * F + j] - m;
        Q = isfinite(w) ? (int)rint(w * sc) : 0;
        q[(size_t)c * F + j] = Q;
      }
      const int q0 = ((Q + 128) & 255) - 128;
      const int Q1 = (Q - q0) >> 8;
      const int q1 = ((Q1 + 128) & 255) - 128;
      const int q2 = (Q1 - q1) >> 8;
      const int limb[3] = {q0, q1, q2};
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        const int n = l * Cp + c;
        __half* p = reinterpret_cast<__half*>(stage + (n >> 3) * 1024 + (kk >> 3) * 128 +
                                              (n & 7) * 16 + (kk & 7) * 2);
        *p = __int2half_rn(limb[l]);
      }
    }
  }
}

nb_status launch_derive_tc(nb_model* m, cudaStream_t st) {
  const int nks = (m->F + TC_KS - 1) / TC_KS;
  const int threads = 256;
  const int blocks = (nks * TC_KS + threads - 1) / threads;
  count_launch();
  k_derive_tc<<<blocks, threads, 0, st>>>(m->d.p0, m->C, m->F, tc_classes_padded(m->C), nks,
                                          m->d.wmax, m->d.tc_w, m->d.tc_q, m->d.tc_hdr);
  NB_TRY_CUDA(cudaGetLastError(), "k_derive_tc");
  return NB_OK;
}


// ---------------------------------------------------------------------------
// launch
// ---------------------------------------------------------------------------
bool tc_eligible(const nb_model* m, nb_dtype dt, const void* X, int64_t ld) {
  return m->kind == NB_MULTINOMIAL && m->d.tc_w != nullptr &&
         (dt == NB_U8 || dt == NB_FP8E4M3 || dt == NB_BF16) &&
         (ld * elem_size(dt)) % 16 == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
         m->tile.variant != NB_VARIANT_REGISTER;
}

static TcModelArg tc_model_arg(const nb_model* m) {
  TcModelArg r;
  r.wlay = m->d.tc_w;
  r.q = m->d.tc_q;
  r.bias = m->d.bias;
  r.hdr = m->d.tc_hdr;
  r.C = m->C;
  r.Cp = tc_classes_padded(m->C);
  r.N = 3 * r.Cp;
  return r;
}

// shared memory of a launch whose largest model has N limb rows
static size_t tc_smem_bytes(int mode, int N) {
  return 1024 + ((sizeof(TcXch) + 1023) / 1024) * 1024 +
         (mode == 0 ? (size_t)TC_NRAW * TC_RAW_BYTES : 0) + (size_t)TC_NB * (uint32_t)N * 128u;
}

template <int MODE, int DT>
static nb_status run_tc(TcArgs& a, int maxN, long long units_hint, cudaStream_t st) {
  constexpr size_t kMax = 227 * 1024;
  const size_t smem = tc_smem_bytes(MODE, maxN);
  if (smem > kMax) {
    set_error("tensor-core scorer: shared memory %zu bytes exceeds the limit", smem);
    return NB_EUNSUPPORTED;
  }
  a.b_bytes = (uint32_t)maxN * 128u;
  a.pf = 8;
  // more than half the shared memory of an SM keeps one CTA (and one
  // tensor-memory allocation) per SM
  const size_t launch_smem = smem < 120 * 1024 ? 120 * 1024 : smem;
  NB_TRY_CUDA(cudaFuncSetAttribute(k_score_tc<MODE, DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)launch_smem),
              "cudaFuncSetAttribute(k_score_tc)");
  long long grid = num_sms();
  if (units_hint > 0 && units_hint < grid) grid = units_hint;
  count_launch();
  k_score_tc<MODE, DT><<<(unsigned)grid, TC_THREADS, launch_smem, st>>>(a);
  NB_TRY_CUDA(cudaGetLastError(), "k_score_tc launch");
  return NB_OK;
}

// cuTensorMapEncodeTiled from the driver, fetched once through the runtime
static PFN_cuTensorMapEncodeTiled_v12000 tc_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  }
  return fn;
}

// 2-D map of n rows x F features of es bytes (1: u8 or FP8, 2: BF16; row pitch
// ld bytes): boxes of 128 rows x 128 bytes, 128-byte swizzle, zero fill out of
// bounds
static nb_status tc_row_map(CUtensorMap* map, const void* X, int64_t n, int F, int64_t ld,
                            int es = 1) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tc_encode_fn();
  if (!enc) {
    set_error("tensor-core scorer: cuTensorMapEncodeTiled is not available");
    return NB_ECUDA;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)F, (cuuint64_t)(n > 0 ? n : 1)};
  const cuuint64_t strides[1] = {(cuuint64_t)ld};
  const cuuint32_t box[2] = {(cuuint32_t)(TC_BOX / es), (cuuint32_t)TC_M};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, es == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8,
                         2, const_cast<void*>(X), dims, strides,
                         box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("tensor-core scorer: cuTensorMapEncodeTiled failed (%d)", (int)r);
    return NB_ECUDA;
  }
  return NB_OK;
}

nb_status launch_score_tc(const nb_model* m, const void* X, nb_dtype dt, int64_t n, int64_t ld,
                          const nb_aux* aux, const ScoreOut& o, cudaStream_t st) {
  TcArgs a{};
  const int es = elem_size(dt);
  nb_status ms = tc_row_map(&a.tmap, X, n, m->F, ld * es, es);
  if (ms != NB_OK) return ms;
  a.maps = nullptr;
  a.groups = nullptr;
  a.hdr = nullptr;
  SegGroup& g = a.g0;
  const bool u8 = dt == NB_U8;
  g.X = static_cast<const char*>(X);
  g.ld_bytes = ld * es;
  g.n = n;
  g.ovf_ptr = (u8 && aux) ? aux->ovf_ptr : nullptr;
  g.ovf_col = (u8 && aux) ? aux->ovf_col : nullptr;
  g.ovf_add = (u8 && aux) ? aux->ovf_add : nullptr;
  g.row_exp = (dt == NB_FP8E4M3 && aux) ? aux->row_exp : nullptr;
  g.label = o.label;
  g.margin = o.margin;
  g.logpost = o.want_lp ? o.logpost : nullptr;
  g.tile0 = 0;
  g.chunk0 = 0;
  g.model = 0;
  g.family = 2;
  a.units0 = (n + 2 * TC_M - 1) / (2 * TC_M);
  a.models[0] = tc_model_arg(m);
  a.F = m->F;
  a.nks = (m->F + TC_KS - 1) / TC_KS;
  a.want_lp = o.want_lp;
  a.recheck = o.recheck;
  a.status = m->d.sstatus;
  if (!u8) {
    // FP8 / BF16 rows: heavy or unchecked rows stay marked for the FP64 recheck
    a.heavy = nullptr;
    a.heavy_n = nullptr;
    a.heavy_cap = 0;
    return dt == NB_FP8E4M3 ? run_tc<0, NB_FP8E4M3>(a, a.models[0].N, a.units0, st)
                            : run_tc<0, NB_BF16>(a, a.models[0].N, a.units0, st);
  }
  // the list of heavy rows (and its count) for the chunked pass: stream-ordered
  // scratch of this call
  const int cap = n < kTcHeavyCap ? (int)n : kTcHeavyCap;
  void* scratch = nullptr;
  NB_TRY_CUDA(cudaMallocAsync(&scratch, 16 + sizeof(long long) * (size_t)cap, st),
              "cudaMallocAsync(heavy rows)");
  a.heavy_n = static_cast<unsigned long long*>(scratch);
  a.heavy = reinterpret_cast<long long*>(static_cast<char*>(scratch) + 16);
  a.heavy_cap = cap;
  const cudaError_t me = cudaMemsetAsync(scratch, 0, 16, st);
  nb_status s = me == cudaSuccess ? NB_OK : cuda_status(me, "memset(heavy count)");
  if (s == NB_OK) s = run_tc<0, NB_U8>(a, a.models[0].N, a.units0, st);
  if (s == NB_OK) s = run_tc<1, NB_U8>(a, a.models[0].N, 0, st);
  const cudaError_t fe = cudaFreeAsync(scratch, st);
  if (s != NB_OK) return s;
  NB_TRY_CUDA(fe, "cudaFreeAsync(heavy rows)");
  return NB_OK;
}

// tensor map of a group's rows (es bytes per feature) for a batch work list
// (128 bytes at map)
nb_status tc_encode_rows(void* map, const void* X, int64_t n, int F, int64_t ld_bytes, int es) {
  return tc_row_map(static_cast<CUtensorMap*>(map), X, n, F, ld_bytes, es);
}

bool tc_group_eligible(const nb_model* m, nb_dtype dt, const void* X, int64_t ld) {
  return tc_eligible(m, dt, X, ld);
}

nb_status launch_score_tc_seg(const SegGroup* groups, const SegHeader* hdr, const void* maps,
                              const nb_model* const* models, int n_models, nb_dtype dt, int F,
                              int want_lp, int recheck, int* status, cudaStream_t st) {
  TcArgs a{};
  a.maps = static_cast<const CUtensorMap*>(maps);
  a.groups = groups;
  a.hdr = hdr;
  int maxN = 48;
  for (int i = 0; i < n_models && i < kSegMaxModels; ++i) {
    a.models[i] = tc_model_arg(models[i]);
    if (a.models[i].N > maxN) maxN = a.models[i].N;
  }
  a.F = F;
  a.nks = (F + TC_KS - 1) / TC_KS;
  a.want_lp = want_lp;
  a.recheck = recheck;
  a.status = status;
  // heavy rows of a batch stay marked for the segmented FP64 recheck
  a.heavy = nullptr;
  a.heavy_n = nullptr;
  a.heavy_cap = 0;
  if (dt == NB_FP8E4M3) return run_tc<0, NB_FP8E4M3>(a, maxN, 0, st);
  if (dt == NB_BF16) return run_tc<0, NB_BF16>(a, maxN, 0, st);
  return run_tc<0, NB_U8>(a, maxN, 0, st);
}

}  // namespace nbg
