// Many-class Gaussian scorer on the fifth-generation tensor cores.
//
// Sec. 4 scores file x against class c by its joint log probability; for
// real-valued features with class-conditional Gaussians,
//   s_c = log pi_c - 1/2 sum_j [log(2 pi var_cj) + (x_j - mu_cj)^2 / var_cj].
// With per-feature centres m_j (the mean of the class means) and
// x~_j = x_j - m_j, d_cj = mu_cj - m_j, the square expands exactly into
//   s_c = K_c + sum_j x~_j B_cj + sum_j x~_j^2 A_cj,
//   B_cj = d_cj / var_cj,  A_cj = -1 / (2 var_cj),
//   K_c = log pi_c - 1/2 sum_j [log(2 pi var_cj) + d_cj^2 / var_cj],
// a dense contraction of the rows [x~, x~^2] with the class table [B; A]:
// tcgen05.mma kind::f16 with FP32 accumulators in tensor memory.
//
// Precision.  x~ and q = x~^2 (FP32) and the FP64 weights are each split into
// two FP16 limbs, hi = fp16(v), lo = fp16(v - hi) (|v - hi - lo| <= 2^-22 |v|);
// every feature contributes the eight limb products (x_hi + x_lo)(B_hi + B_lo)
// + (q_hi + q_lo)(A_hi + A_lo), each exact in FP32.  The tensor core's FP32
// sums are not exact: each of the K = 8F additions is taken to err by at most
// one FP32 ulp of a partial sum, i.e. 2^-23 of P = sum_j (|x~_j| max_c |B_cj| +
// q_j max_c |A_cj|), which bounds every partial sum.  The rigorous per-row bound
// tau = 2 [((8F + 16) 2^-23 + 2^-20) P (1 + 2^-9) + 2^-24 (Q + W + e_max)]
// (Q, W: the subnormal slack of the low limbs; e_max: the final roundings)
// settles the label when the margin exceeds it; rows it does not settle, and
// every row in the log-posterior mode whose bound is above 5e-6 of its margin,
// go to the FP64 recheck.  Because P is the sum of the terms' magnitudes, not
// of the result, the bound is loose against the cancelling expansion: the
// label mode marks few rows, the log-posterior mode most (which is why the
// library routes that mode to the CUDA-core scorer, whose direct form keeps
// the bound relative to the result).
//
// One persistent CTA per SM (736 threads): a row producer (2-D tensor TMA of
// 128 rows x 32 FP32 features, 128-byte swizzle, zero fill), a weight producer
// (one bulk copy of C_p x 64 FP16 limbs per 8-feature stage, up to 96 KB in
// flight; a table that fits is loaded once and stays), one MMA issuer (M = 128,
// N = C_p, K = 16, A from tensor memory), sixteen converter warps (one row and
// two features per thread and stage: FP32 -> centred FP16 limbs, tcgen05.st
// into eight A stages) and four epilogue warps (one thread per row, every
// class), the accumulators double buffered so that a tile's epilogue overlaps
// the next tile's MMAs.  Every wait
// is bounded; a wait that runs out raises ST_TIMEOUT and all roles stop.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <math.h>

#include "device.cuh"
#include "internal.cuh"
#include "tc.cuh"

namespace nbg {

constexpr int TG_M = 128;                  // files per tile (tensor-memory lanes)
constexpr int TG_FS = kTcgFS;              // features per stage
constexpr int TG_KS = 8 * TG_FS;           // K elements per stage (eight per feature)
constexpr int TG_BOXF = 32;                // FP32 features per TMA box (128 bytes)
constexpr int TG_SPB = TG_BOXF / TG_FS;    // stages per row box
constexpr int TG_NRAW = 4;                 // row boxes in shared memory
constexpr int TG_NB = 32;                  // most weight stages in shared memory
constexpr uint32_t TG_B_BYTES = 128 * 1024;  // shared memory for weight stages
constexpr int TG_CONV = 16;                // converter warps: 4 lane quadrants x 4 parts
constexpr int TG_PARTS = TG_CONV / 4;      // parts of a stage's features
constexpr int TG_FPW = TG_FS / TG_PARTS;   // features per converter thread per stage
constexpr int TG_EPI = 4;                  // epilogue warps: one per lane quadrant
constexpr int TG_THREADS = (TG_CONV + TG_EPI + 3) * 32;
constexpr uint32_t TG_RAW_BYTES = TG_M * TG_BOXF * 4;   // 16 KB
// a row slot: the box, then the box's features' centres, B bounds and A
// bounds (TG_BOXF floats each), padded to keep the next box 1 KB aligned
constexpr uint32_t TG_TAB_BYTES = 3 * TG_BOXF * 4;
constexpr uint32_t TG_SLOT_BYTES = TG_RAW_BYTES + 1024;
static_assert(TG_TAB_BYTES <= 1024 && TG_BOXF == TG_FS, "a row slot holds one stage's tables");
constexpr int TG_ACC = 64;                 // accumulator buffer b at columns 64 b
constexpr int TG_ACOL = 2 * TG_ACC;        // A stage s at columns 128 + TG_ACOLS s
constexpr int TG_ACOLS = TG_KS / 2;        // tensor-memory columns of an A stage
constexpr int TG_NA = (512 - TG_ACOL) / TG_ACOLS;   // A stages in tensor memory
constexpr long long TG_WAIT = 2000000000LL;
static_assert(TG_BOXF % TG_FS == 0 && TG_FS % TG_PARTS == 0, "stage shape");
static_assert(TG_FPW == 2 || TG_FPW == 4 || TG_FPW == 8, "features per converter thread");

struct TgArgs {
  CUtensorMap tmap;          // n rows x F FP32 features
  int64_t n;
  int F, nks, C, Cp;
  int nb;                    // weight stages in flight (nks of them: the table stays resident)
  const uint8_t* wlay;       // nks stages x Cp rows x TG_KS FP16 limbs (K-major core matrices)
  const TcgHeader* hdr;
  const float* kc;           // C
  const float* ctr;          // nks * TG_FS centres
  const float* bmax;         // nks * TG_FS: max_c |B_cj| (rounded up)
  const float* amax;         // nks * TG_FS: max_c |A_cj| (rounded up)
  uint8_t* label;
  float* margin;
  float* logpost;
  int want_lp, recheck;
  int* status;
};

struct TgShared {
  uint64_t raw_full[TG_NRAW], raw_empty[TG_NRAW];
  uint64_t b_full[TG_NB], b_empty[TG_NB];
  uint64_t a_full[TG_NA], a_empty[TG_NA];
  uint64_t acc_full[2], acc_empty[2], pr_full[2], pr_empty[2];
  uint64_t fin;
  uint32_t tmem;
  int abort;
  float rowP[2][TG_PARTS][TG_M];   // per tile buffer, converter part, row: the bound's sum P
  float rowQ[2][TG_PARTS][TG_M];   // ... and sum (|x~| + q)
};

__device__ __forceinline__ bool tg_aborted(TgShared& sh) {
  return *reinterpret_cast<volatile int*>(&sh.abort) != 0;
}

__device__ __forceinline__ bool tg_wait_sleep(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait_sleep(bar, parity, 100000u)) {
    if (clock64() - t0 > TG_WAIT) return false;
  }
  return true;
}

__device__ __forceinline__ bool tg_wait(TgShared& sh, uint64_t* bar, uint32_t parity,
                                        int* status) {
  if (tg_wait_sleep(bar, parity)) return true;
  atomicOr(status, ST_TIMEOUT);
  *reinterpret_cast<volatile int*>(&sh.abort) = 1;
  return false;
}

__device__ __forceinline__ bool tg_wait_warp(TgShared& sh, uint64_t* bar, uint32_t parity,
                                             int* status) {
  const bool mine = tg_wait_sleep(bar, parity);
  const bool all = __all_sync(0xFFFFFFFFu, mine) != 0;
  if (!all && (threadIdx.x & 31) == 0) {
    atomicOr(status, ST_TIMEOUT);
    *reinterpret_cast<volatile int*>(&sh.abort) = 1;
  }
  return all;
}

template <int N>
__device__ __forceinline__ void tg_lds(uint32_t addr, float (&x)[N]) {
  static_assert(N == 2 || N == 4 || N == 8, "two, four or eight features per load");
  if constexpr (N == 8) {
    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(x[0]), "=f"(x[1]), "=f"(x[2]), "=f"(x[3])
                 : "r"(addr)
                 : "memory");
    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(x[4]), "=f"(x[5]), "=f"(x[6]), "=f"(x[7])
                 : "r"(addr + 16u)
                 : "memory");
  } else if constexpr (N == 4) {
    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(x[0]), "=f"(x[1]), "=f"(x[2]), "=f"(x[3])
                 : "r"(addr)
                 : "memory");
  } else {
    asm volatile("ld.shared.v2.f32 {%0,%1}, [%2];" : "=f"(x[0]), "=f"(x[1]) : "r"(addr) : "memory");
  }
}

// N consecutive floats of a per-feature table (4 N-byte aligned)
template <int N>
__device__ __forceinline__ void tg_ldg(const float* p, float (&v)[N]) {
  if constexpr (N == 8) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    const float4 u = __ldg(reinterpret_cast<const float4*>(p) + 1);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    v[4] = u.x; v[5] = u.y; v[6] = u.z; v[7] = u.w;
  } else if constexpr (N == 4) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else {
    const float2 t = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = t.x; v[1] = t.y;
  }
}

// one thread's 4 N limb words of a stage into tensor memory
template <int N>
__device__ __forceinline__ void tg_st(uint32_t col, const uint32_t (&o)[4 * N]) {
  if constexpr (N == 8) tmem_st32(col, o);
  else if constexpr (N == 4) tmem_st16(col, o);
  else tmem_st8(col, o);
}

// D[tmem] (+)= A[tmem] * B[smem]^T, issued by one thread
__device__ __forceinline__ void tg_mma(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// one lane of a converged warp (the MMA issuer's)
__device__ __forceinline__ bool tg_elect() {
  uint32_t p;
  asm volatile("{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n selp.u32 %0, 1, 0, e;\n}\n"
               : "=r"(p));
  return p != 0;
}

// the bits of an FP16 pair (two consecutive K elements)
__device__ __forceinline__ uint32_t tg_h2u(__half2 h) {
  return *reinterpret_cast<const uint32_t*>(&h);
}

__global__ void __launch_bounds__(TG_THREADS, 1) k_score_tcg(const __grid_constant__ TgArgs a) {
  extern __shared__ __align__(1024) uint8_t tg_smem[];
  TgShared& sh = *reinterpret_cast<TgShared*>(tg_smem);
  uint8_t* raw = tg_smem + ((sizeof(TgShared) + 1023) / 1024) * 1024;   // 1 KB aligned
  uint8_t* B = raw + (size_t)TG_NRAW * TG_SLOT_BYTES;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long n_units = (a.n + TG_M - 1) / TG_M;
  const long long my_units =
      n_units > (long long)blockIdx.x ? (n_units - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const int nks = a.nks, F = a.F, nb = a.nb;
  const uint32_t b_bytes = (uint32_t)a.Cp * (uint32_t)(2 * TG_KS);
  // a table of at most nb stages is loaded once and stays in shared memory
  const bool resident = nks <= nb;
  // Every role walks a tile's stages in the same order, rotated per CTA by
  // whole 32-feature row boxes (TG_SPB stages): stage i of a tile is (i + s0)
  // mod nks, so that the CTAs spread their weight reads over the table.
  const int nbox = (nks + TG_SPB - 1) / TG_SPB;
  const int rbox = (int)((blockIdx.x * 37u) % (unsigned)nbox), s0 = TG_SPB * rbox;

  if (threadIdx.x == 0) {
    for (int i = 0; i < TG_NRAW; ++i) {
      mbar_init(&sh.raw_full[i], 1);
      mbar_init(&sh.raw_empty[i], TG_CONV);
    }
    for (int i = 0; i < nb; ++i) {
      mbar_init(&sh.b_full[i], 1);
      mbar_init(&sh.b_empty[i], 1);
    }
    for (int i = 0; i < TG_NA; ++i) {
      mbar_init(&sh.a_full[i], TG_CONV);
      mbar_init(&sh.a_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&sh.acc_full[i], 1);
      mbar_init(&sh.acc_empty[i], TG_EPI);
      mbar_init(&sh.pr_full[i], TG_CONV);
      mbar_init(&sh.pr_empty[i], TG_EPI);
    }
    mbar_init(&sh.fin, 1);
    sh.abort = 0;
  }
  if (warp == TG_CONV + TG_EPI + 1) tmem_alloc(&sh.tmem, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh.tmem;

  if (warp == TG_CONV + TG_EPI) {
    // ---- row producer -------------------------------------------------
    if (lane == 0) {
      long long ri = 0, last[TG_NRAW] = {-1, -1, -1, -1};
      bool ok = (smem_addr(raw) & 1023u) == 0;   // the swizzled reads assume 1 KB alignment
      if (!ok) {
        atomicOr(a.status, ST_TIMEOUT);
        *reinterpret_cast<volatile int*>(&sh.abort) = 1;
      }
      const uint64_t map = reinterpret_cast<uint64_t>(&a.tmap);
      for (long long it = 0; it < my_units && ok && !tg_aborted(sh); ++it) {
        const long long t = blockIdx.x + it * gridDim.x;
        for (int b = 0; b < nbox; ++b, ++ri) {
          const int f0 = TG_BOXF * (rbox + b < nbox ? rbox + b : rbox + b - nbox);
          const int slot = (int)(ri % TG_NRAW);
          if (!tg_wait(sh, &sh.raw_empty[slot], (uint32_t)((ri / TG_NRAW) & 1) ^ 1u, a.status)) {
            ok = false;
            break;
          }
          uint8_t* dst = raw + (size_t)slot * TG_SLOT_BYTES;
          mbar_expect_tx(&sh.raw_full[slot], TG_RAW_BYTES + TG_TAB_BYTES);
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
              " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
              "l"(map), "r"(f0), "r"((int)(t * TG_M)), "r"(smem_addr(&sh.raw_full[slot]))
              : "memory");
          // the box's per-feature tables (the tables are padded to a multiple
          // of TG_FS features, so f0 + TG_BOXF stays inside them)
          bulk_g2s(dst + TG_RAW_BYTES, a.ctr + f0, 4 * TG_BOXF, &sh.raw_full[slot]);
          bulk_g2s(dst + TG_RAW_BYTES + 4 * TG_BOXF, a.bmax + f0, 4 * TG_BOXF, &sh.raw_full[slot]);
          bulk_g2s(dst + TG_RAW_BYTES + 8 * TG_BOXF, a.amax + f0, 4 * TG_BOXF, &sh.raw_full[slot]);
          last[slot] = ri;
        }
      }
      for (int s = 0; s < TG_NRAW; ++s)
        if (last[s] >= 0)
          tg_wait(sh, &sh.raw_full[s], (uint32_t)((last[s] / TG_NRAW) & 1), a.status);
    }
    __syncwarp();
  } else if (warp == TG_CONV + TG_EPI + 2) {
    // ---- weight producer ------------------------------------------------
    if (lane == 0) {
      // ring position (slot, phase) of the next stage; lastph[s]: phase of the
      // last copy into slot s, or -1
      int slot = 0, ph = 0, lastph[TG_NB];
      for (int s = 0; s < TG_NB; ++s) lastph[s] = -1;
      bool ok = true;
      const long long loads = resident ? (my_units > 0 ? 1 : 0) : my_units;
      for (long long it = 0; it < loads && ok && !tg_aborted(sh); ++it) {
        for (int i = 0; i < nks; ++i) {
          const int ks = i + s0 < nks ? i + s0 : i + s0 - nks;
          const int sl = resident ? ks : slot;   // resident: stage ks in slot ks
          if (!resident && !tg_wait(sh, &sh.b_empty[sl], (uint32_t)ph ^ 1u, a.status)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&sh.b_full[sl], b_bytes);
          bulk_g2s(B + (size_t)sl * b_bytes, a.wlay + (size_t)ks * b_bytes, b_bytes,
                   &sh.b_full[sl]);
          lastph[sl] = resident ? 0 : ph;
          if (++slot == nb) {
            slot = 0;
            ph ^= 1;
          }
        }
      }
      for (int s = 0; s < nb; ++s)
        if (lastph[s] >= 0) tg_wait(sh, &sh.b_full[s], (uint32_t)lastph[s], a.status);
    }
    __syncwarp();
  } else if (warp == TG_CONV + TG_EPI + 1) {
    // ---- MMA issuer: the whole warp waits, one elected lane issues ----------
    {
      int bslot_r = 0, bph = 0, aslot = 0, aph = 0;   // ring positions of B and A stages
      bool ok = true;
      const uint32_t idesc = tc_idesc_f16(TG_M, a.Cp);
      // descriptor of weight slot 0 (core matrices 128 bytes apart along K,
      // 8-class groups one stage row apart); slot s and K16 step j add
      // (s b_bytes + 256 j) / 16 to its start-address field (14 bits: no
      // carry below 256 KB)
      const uint64_t bdesc0 = tc_desc(smem_addr(B), 128u, (uint32_t)(16 * TG_KS));
      for (long long it = 0; it < my_units && ok && !__any_sync(0xFFFFFFFFu, tg_aborted(sh));
           ++it) {
        const int buf = (int)(it & 1);
        const long long use = it >> 1;   // earlier uses of this accumulator buffer
        if (use > 0 &&
            !tg_wait_warp(sh, &sh.acc_empty[buf], (uint32_t)((use - 1) & 1), a.status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d0 = tmem + (uint32_t)(TG_ACC * buf);
        for (int i = 0; i < nks; ++i) {
          const int ks = i + s0 < nks ? i + s0 : i + s0 - nks;
          // resident table: stage ks in slot ks, its one phase completed
          const int bslot = resident ? ks : bslot_r;
          if (!tg_wait_warp(sh, &sh.b_full[bslot], resident ? 0u : (uint32_t)bph, a.status) ||
              !tg_wait_warp(sh, &sh.a_full[aslot], (uint32_t)aph, a.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t bd = bdesc0 + (uint64_t)(((uint32_t)bslot * b_bytes) >> 4);
          const uint32_t at = tmem + (uint32_t)(TG_ACOL + TG_ACOLS * aslot);
          if (tg_elect()) {
#pragma unroll
            for (int j = 0; j < TG_KS / 16; ++j)
              tg_mma(d0, at + 8u * j, bd + 16u * j, idesc, (i > 0 || j > 0) ? 1u : 0u);
            if (!resident) tc_commit(&sh.b_empty[bslot]);
            tc_commit(&sh.a_empty[aslot]);
          }
          __syncwarp();
          if (++bslot_r == nb) {
            bslot_r = 0;
            bph ^= 1;
          }
          if (++aslot == TG_NA) {
            aslot = 0;
            aph ^= 1;
          }
        }
        if (!ok) break;
        if (tg_elect()) tc_commit(&sh.acc_full[buf]);
        __syncwarp();
      }
      if (tg_elect()) tc_commit(&sh.fin);
      __syncwarp();
      tg_wait_warp(sh, &sh.fin, 0, a.status);
    }
  } else if (warp < TG_CONV) {
    // ---- converters -------------------------------------------------------
    const int qd = warp & 3, part = warp >> 2;
    const int r = 32 * qd + lane;                       // row within the tile
    const uint32_t lane_base = tmem + ((uint32_t)(32 * qd) << 16);
    const uint32_t raw_s = smem_addr(raw) + (uint32_t)(r * 128);
    long long ri = 0;
    int aslot = 0, aph = 0;   // ring position of the next A stage
    bool ok = true;
    // A stage whose tensor-memory store is still in flight: its completion is
    // awaited (and the stage handed to the MMA) after the next stage's
    // arithmetic, so that the store latency overlaps it
    int pend = -1;
    for (long long it = 0; it < my_units && ok; ++it) {
      float P = 0.f, Q = 0.f, qmax = 0.f;
      for (int i = 0; i < nks; ++i) {
        const int ks = i + s0 < nks ? i + s0 : i + s0 - nks;
        if (__any_sync(0xFFFFFFFFu, tg_aborted(sh))) {   // warp-uniform exit
          ok = false;
          break;
        }
        const uint32_t slot = (uint32_t)(ri % TG_NRAW);
        if (ks % TG_SPB == 0 &&
            !tg_wait_warp(sh, &sh.raw_full[slot], (uint32_t)((ri / TG_NRAW) & 1), a.status)) {
          ok = false;
          break;
        }
        // features TG_FS ks + TG_FPW part .. of the row: byte 4 TG_FS (ks % TG_SPB) +
        // 4 TG_FPW part of the row's 128-byte segment, whose 16-byte chunks are
        // swizzled by the row
        const int byte = 4 * TG_FS * (ks % TG_SPB) + 4 * TG_FPW * part;
        const uint32_t rs = raw_s + slot * TG_SLOT_BYTES;
        float xs[TG_FPW];
        if constexpr (TG_FPW == 8) {
          float lo[4], hi[4];
          tg_lds(rs + (uint32_t)((((byte >> 4) ^ (r & 7)) << 4)), lo);
          tg_lds(rs + (uint32_t)(((((byte >> 4) + 1) ^ (r & 7)) << 4)), hi);
#pragma unroll
          for (int f = 0; f < 4; ++f) {
            xs[f] = lo[f];
            xs[4 + f] = hi[f];
          }
        } else {
          tg_lds(rs + (uint32_t)((((byte >> 4) ^ (r & 7)) << 4) | (byte & 15)), xs);
        }
        // this thread's features' centres and bounds, staged with the box
        float ctr[TG_FPW], bm[TG_FPW], am[TG_FPW];
        const uint32_t tab = smem_addr(raw) + slot * TG_SLOT_BYTES + TG_RAW_BYTES +
                             (uint32_t)(4 * TG_FPW * part);   // the same for every row
        tg_lds(tab, ctr);
        tg_lds(tab + 4 * TG_BOXF, bm);
        tg_lds(tab + 8 * TG_BOXF, am);
        if (ks % TG_SPB == TG_SPB - 1 || ks == nks - 1) {   // done with the row box
          __syncwarp();
          if (lane == 0) mbar_arrive(&sh.raw_empty[slot]);
          ++ri;
        }
        uint32_t o[4 * TG_FPW];
#pragma unroll
        for (int f = 0; f < TG_FPW; ++f) {
          const float xt = xs[f] - ctr[f];
          const float q = xt * xt;
          // each limb twice, as one FP16 pair (one packed conversion)
          const __half2 xh = __floats2half2_rn(xt, xt);
          const float xr = xt - __low2float(xh);
          const __half2 qh = __floats2half2_rn(q, q);
          const float qr = q - __low2float(qh);
          o[4 * f + 0] = tg_h2u(xh);
          o[4 * f + 1] = tg_h2u(__floats2half2_rn(xr, xr));
          o[4 * f + 2] = tg_h2u(qh);
          o[4 * f + 3] = tg_h2u(__floats2half2_rn(qr, qr));
          P = fmaf(fabsf(xt), bm[f], fmaf(q, am[f], P));   // NaN and inf carry into P
          Q += fabsf(xt) + q;
          qmax = fmaxf(qmax, q);
        }
        if (pend >= 0) {
          tmem_st_wait();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&sh.a_full[pend]);
          pend = -1;
        }
        if (!tg_wait_warp(sh, &sh.a_empty[aslot], (uint32_t)aph ^ 1u, a.status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t col =
            lane_base + (uint32_t)(TG_ACOL + TG_ACOLS * aslot + 4 * TG_FPW * part);
        tg_st<TG_FPW>(col, o);
        pend = aslot;
        if (++aslot == TG_NA) {
          aslot = 0;
          aph ^= 1;
        }
      }
      if (!ok) break;
      // the tile's bound sums for the epilogue
      const int buf = (int)(it & 1);
      const long long use = it >> 1;
      if (use > 0 &&
          !tg_wait_warp(sh, &sh.pr_empty[buf], (uint32_t)((use - 1) & 1), a.status)) {
        ok = false;
        break;
      }
      // x~ and q inside the FP16 range (q < 2^15 bounds |x~| < 182 too)
      sh.rowP[buf][part][r] = qmax < 32768.f ? P : INFINITY;
      sh.rowQ[buf][part][r] = Q;
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.pr_full[buf]);
    }
    if (pend >= 0) {
      tmem_st_wait();
      tc_fence_before();
      __syncwarp();
      if (ok && lane == 0) mbar_arrive(&sh.a_full[pend]);
    }
  } else {
    // ---- epilogue: one thread per row, every class ------------------------
    const int qd = warp - TG_CONV;
    const int r = 32 * qd + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * qd) << 16);
    const float W = a.hdr->wsum, fsl = (float)(8 * F + 16) * 1.1920929e-7f + 9.5367432e-7f;
    const bool tab_ok = a.hdr->bad == 0;
    const bool want_lp = a.want_lp && a.logpost;   // the exponential sums only for lp
    for (long long it = 0; it < my_units; ++it) {
      const long long t = blockIdx.x + it * gridDim.x;
      const int buf = (int)(it & 1);
      const uint32_t par = (uint32_t)((it >> 1) & 1);
      if (!tg_wait_warp(sh, &sh.acc_full[buf], par, a.status) ||
          !tg_wait_warp(sh, &sh.pr_full[buf], par, a.status))
        break;
      tc_fence_after();
      float P = 0.f, Q = 0.f;
#pragma unroll
      for (int p = 0; p < TG_PARTS; ++p) {
        P += sh.rowP[buf][p][r];
        Q += sh.rowQ[buf][p][r];
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.pr_empty[buf]);
      const long long grow = t * TG_M + r;
      const bool valid = grow < a.n;
      const uint32_t acc = lane_base + (uint32_t)(TG_ACC * buf);
      // pass 1: best, second best, sum of exp(s - best), largest rounding term
      float best = -INFINITY, second = -INFINITY, se = 0.f, emax = 0.f;
      int bidx = 0;
      for (int cb = 0; cb < a.Cp; cb += 16) {
        uint32_t v[16];
        tmem_ld16(acc + (uint32_t)cb, v);
        tmem_ld_wait();
        float b16 = -INFINITY, s16 = -INFINITY, e16 = 0.f;
        int i16 = 0;
        float sc[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int c = cb + i;
          sc[i] = -INFINITY;
          if (c >= a.C) continue;
          const float k = __ldg(a.kc + c);
          sc[i] = __uint_as_float(v[i]) + k;
          emax = fmaxf(emax, fabsf(k) + fabsf(sc[i]));
          if (sc[i] > b16) {
            s16 = b16;
            b16 = sc[i];
            i16 = c;
          } else if (sc[i] > s16) {
            s16 = sc[i];
          }
        }
        if (want_lp) {
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (cb + i < a.C) e16 += __expf(sc[i] - b16);
        }
        if (cb == 0 || b16 > best) {
          if (want_lp) se = (cb == 0 ? 0.f : se * __expf(best - b16)) + e16;
          second = cb == 0 ? s16 : fmaxf(best, s16);
          best = b16;
          bidx = i16;
        } else {
          if (want_lp) se += e16 * __expf(b16 - best);
          second = fmaxf(second, b16);
        }
      }
      const float lse = want_lp ? best + logf(se) : 0.f;
      const float margin = best - second;
      const float tau = 2.f * (fsl * P * (1.f + 1.f / 512.f) +
                               5.9604645e-8f * (Q + W + emax)) + 1e-30f;
      bool flag = !tab_ok || !(tau < INFINITY);
      if (a.recheck != NB_RECHECK_OFF) {
        flag = flag || !(margin > tau);
        if (a.recheck == NB_RECHECK_LP && tau > 5e-6f * fmaxf(1.f, margin)) flag = true;
      }
      if (valid) {
        a.label[grow] = flag ? kLabelRecheck : (uint8_t)bidx;
        a.margin[grow] = margin;
      }
      if (want_lp) {
        float* lp = a.logpost + (valid ? grow : 0) * a.C;
        for (int cb = 0; cb < a.Cp; cb += 16) {
          uint32_t v[16];
          tmem_ld16(acc + (uint32_t)cb, v);
          tmem_ld_wait();
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (valid && cb + i < a.C) lp[cb + i] = __uint_as_float(v[i]) + __ldg(a.kc + cb + i) - lse;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.acc_empty[buf]);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == TG_CONV + TG_EPI + 1) tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------------------
// tables: centres, FP16 limbs of B and A in the MMA operand layout, K_c
// ---------------------------------------------------------------------------
// One thread per feature j (nks * TG_FS of them): m_j = the mean of the class
// means, rounded to FP32 (the expansion uses that FP32 value), the eight limb
// values of every class in one 16-byte record, the per-feature maxima.
__global__ void k_derive_tcg(const double* mu, const double* var, int C, int F, int Cp, int nks,
                             uint8_t* wlay, float* ctr, float* bmax, float* amax, TcgHeader* hdr) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nks * TG_FS) return;
  double m = 0.0;
  if (j < F) {
    for (int c = 0; c < C; ++c) m += mu[(int64_t)c * F + j];
    m /= (double)C;
  }
  const float mf = (float)m;
  const double md = (double)mf;
  const int ks = j / TG_FS, jj = j % TG_FS;
  uint8_t* stage = wlay + (size_t)ks * Cp * (2 * TG_KS);
  double bm = 0.0, am = 0.0;
  bool ok = true;
  for (int c = 0; c < Cp; ++c) {
    __half h[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) h[t] = __float2half_rn(0.f);
    if (c < C && j < F) {
      const double iv = 1.0 / var[(int64_t)c * F + j];
      const double Bv = (mu[(int64_t)c * F + j] - md) * iv, Av = -0.5 * iv;
      ok = ok && fabs(Bv) < 32768.0 && fabs(Av) < 32768.0;
      bm = fmax(bm, fabs(Bv));
      am = fmax(am, fabs(Av));
      const __half bh = __double2half(Bv), ah = __double2half(Av);
      const __half bl = __double2half(Bv - (double)__half2float(bh));
      const __half al = __double2half(Av - (double)__half2float(ah));
      // K elements 8 jj + t: (x_hi, x_hi, x_lo, x_lo) x (B_hi, B_lo, B_hi, B_lo),
      // then (q_hi, q_hi, q_lo, q_lo) x (A_hi, A_lo, A_hi, A_lo)
      h[0] = bh; h[1] = bl; h[2] = bh; h[3] = bl;
      h[4] = ah; h[5] = al; h[6] = ah; h[7] = al;
    }
    // core matrix (c / 8, jj): 8 rows of 16 bytes; row c % 8 holds this record
    *reinterpret_cast<uint4*>(stage + (c >> 3) * (16 * TG_KS) + jj * 128 + (c & 7) * 16) =
        *reinterpret_cast<const uint4*>(h);
  }
  if (!ok) hdr->bad = 1;   // a weight outside the FP16 range: every row to FP64
  ctr[j] = j < F ? mf : 0.f;
  bmax[j] = (float)(bm * (1.0 + 1.0 / 1048576.0));
  amax[j] = (float)(am * (1.0 + 1.0 / 1048576.0));
}

// K_c (one block per class) and W = sum_j (max|B| + max|A|) (block 0)
__global__ void __launch_bounds__(256) k_derive_tcg_k(const double* mu, const double* var,
                                                      const double* gconst, const float* ctr,
                                                      const float* bmax, const float* amax,
                                                      int F, float* kc, TcgHeader* hdr) {
  __shared__ double red[8];
  const int c = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double s = 0.0, w = 0.0;
  for (int j = threadIdx.x; j < F; j += blockDim.x) {
    const double d = mu[(int64_t)c * F + j] - (double)ctr[j];
    s += d * d / var[(int64_t)c * F + j];
    w += (double)bmax[j] + (double)amax[j];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    s += __shfl_xor_sync(0xFFFFFFFFu, s, off);
    w += __shfl_xor_sync(0xFFFFFFFFu, w, off);
  }
  if (lane == 0) red[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    kc[c] = (float)(gconst[c] - 0.5 * t);
  }
  __syncthreads();
  if (c == 0) {
    if (lane == 0) red[warp] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
      hdr->wsum = (float)(t * (1.0 + 1.0 / 1048576.0));
    }
  }
}

nb_status launch_derive_tcg(nb_model* m, cudaStream_t st) {
  const int nks = (m->F + TG_FS - 1) / TG_FS;
  const int Cp = tc_classes_padded(m->C);
  NB_TRY_CUDA(cudaMemsetAsync(m->d.tcg_hdr, 0, sizeof(TcgHeader), st), "memset(tcg header)");
  count_launch();
  k_derive_tcg<<<(nks * TG_FS + 255) / 256, 256, 0, st>>>(m->d.p0, m->d.p1, m->C, m->F, Cp, nks,
                                                           m->d.tc_w, m->d.tcg_ctr,
                                                           m->d.tcg_bmax, m->d.tcg_amax,
                                                           m->d.tcg_hdr);
  NB_TRY_CUDA(cudaGetLastError(), "k_derive_tcg");
  count_launch();
  k_derive_tcg_k<<<m->C, 256, 0, st>>>(m->d.p0, m->d.p1, m->d.gconst, m->d.tcg_ctr,
                                       m->d.tcg_bmax, m->d.tcg_amax, m->F, m->d.tcg_kc,
                                       m->d.tcg_hdr);
  NB_TRY_CUDA(cudaGetLastError(), "k_derive_tcg_k");
  return NB_OK;
}

// ---------------------------------------------------------------------------
// launch
// ---------------------------------------------------------------------------
bool tcg_eligible(const nb_model* m, const void* X, int64_t ld, int recheck) {
  if (m->kind != NB_GAUSSIAN || m->d.tcg_kc == nullptr || ld % 4 != 0 ||
      (reinterpret_cast<uintptr_t>(X) & 15) != 0 || m->tile.variant == NB_VARIANT_REGISTER)
    return false;
  // the log-posterior mode goes to the CUDA-core scorer (see the bound above)
  // unless the tensor-core path is asked for
  return recheck != NB_RECHECK_LP || m->tile.variant == NB_VARIANT_PIPELINED;
}

static PFN_cuTensorMapEncodeTiled_v12000 tg_encode_fn() {
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

nb_status launch_score_tcg(const nb_model* m, const float* X, int64_t n, int64_t ld,
                           const ScoreOut& o, cudaStream_t st) {
  TgArgs a{};
  PFN_cuTensorMapEncodeTiled_v12000 enc = tg_encode_fn();
  if (!enc) {
    set_error("Gaussian tensor-core scorer: cuTensorMapEncodeTiled is not available");
    return NB_ECUDA;
  }
  // n rows x F FP32 features, 32 x 128 boxes, 128-byte swizzle, zero fill
  const cuuint64_t dims[2] = {(cuuint64_t)m->F, (cuuint64_t)(n > 0 ? n : 1)};
  const cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
  const cuuint32_t box[2] = {(cuuint32_t)TG_BOXF, (cuuint32_t)TG_M};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(&a.tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(X), dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("Gaussian tensor-core scorer: cuTensorMapEncodeTiled failed (%d)", (int)r);
    return NB_ECUDA;
  }
  a.n = n;
  a.F = m->F;
  a.nks = (m->F + TG_FS - 1) / TG_FS;
  a.C = m->C;
  a.Cp = tc_classes_padded(m->C);
  a.nb = (int)(TG_B_BYTES / ((uint32_t)a.Cp * (uint32_t)(2 * TG_KS)));
  if (a.nb > TG_NB) a.nb = TG_NB;
  a.wlay = m->d.tc_w;
  a.hdr = m->d.tcg_hdr;
  a.kc = m->d.tcg_kc;
  a.ctr = m->d.tcg_ctr;
  a.bmax = m->d.tcg_bmax;
  a.amax = m->d.tcg_amax;
  a.label = o.label;
  a.margin = o.margin;
  a.logpost = o.want_lp ? o.logpost : nullptr;
  a.want_lp = o.want_lp;
  a.recheck = o.recheck;
  a.status = m->d.sstatus;
  const size_t smem = ((sizeof(TgShared) + 1023) / 1024) * 1024 + (size_t)TG_NRAW * TG_SLOT_BYTES +
                      (size_t)a.nb * a.Cp * (2 * TG_KS);
  // more than half the shared memory of an SM keeps one CTA (and one
  // tensor-memory allocation) per SM
  const size_t launch_smem = smem < 120 * 1024 ? 120 * 1024 : smem;
  NB_TRY_CUDA(cudaFuncSetAttribute(k_score_tcg, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)launch_smem),
              "cudaFuncSetAttribute(k_score_tcg)");
  const long long units = (n + TG_M - 1) / TG_M;
  long long grid = num_sms();
  if (units < grid) grid = units;
  count_launch();
  k_score_tcg<<<(unsigned)grid, TG_THREADS, launch_smem, st>>>(a);
  NB_TRY_CUDA(cudaGetLastError(), "k_score_tcg launch");
  return NB_OK;
}

}  // namespace nbg
