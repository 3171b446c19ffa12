// Many-class multinomial scorer on the fifth-generation tensor cores.
//
// Sec. 4 scores file x against class c by s_c = log pi_c + sum_j x_j log
// theta_cj and takes the class of largest posterior.  With the centred table
// w_cj = log theta_cj - mean_c log theta_cj (the per-feature shift is common to
// all classes and cancels in the label, the margin and the log posteriors)
// the scores of a tile of 128 files against C <= 64 classes are one dense
// contraction S = X W^T, done here with tcgen05.mma (kind::f16, FP32
// accumulators in tensor memory).
//
// Exactness.  The weights are held in fixed point, Q_cj = round(w_cj 2^S)
// with |Q| <= 2^22, split into three balanced limbs Q = q0 + 2^8 q1 + 2^16 q2
// with |q_l| <= 128, each an exact FP16 integer.  Stored u8 counts (0..255)
// are exact FP16 integers as well, so every product is exact and every
// partial sum of one limb over 512 features is an integer of magnitude below
// 255 * 512 * 128 < 2^24: the FP32 accumulator holds it exactly, whatever the
// order of the tensor core's additions.  Every 512 features the accumulators
// are drained into int32 registers (exact: |sum_j x_j q_j| <= 255 F 128 <
// 2^31 for F <= 32768) and the limbs are combined exactly in int64 at the end,
// overflow-list entries (counts above 255) added exactly on the CUDA cores.
// The only errors are the weight quantisation, at most T 2^-(S+1) with T the
// file's token count, and two FP32 roundings when the score is formed; the
// epilogue bounds both and marks the row for the FP64 recheck when the bound
// does not settle the label (or the log posteriors).
//
// Roles of one persistent CTA per SM (352 threads):
//   warps 0-7  convert u8 rows to FP16 operand tiles, drain the accumulators,
//              run the epilogue (arg-max, top-2 margin, log-sum-exp);
//   warp 8     streams the rows of each tile into shared memory (bulk copies);
//   warp 9     allocates tensor memory and issues the MMAs (one thread);
//   warp 10    streams the weight-limb stages (bulk copies).
// Every wait is bounded; a wait that runs out raises ST_TIMEOUT, all roles
// stop, outstanding copies and MMAs are waited for, and tensor memory is freed.
#include <cuda_fp16.h>
#include <math.h>

#include "device.cuh"
#include "internal.cuh"
#include "seg.cuh"
#include "tc.cuh"

namespace nbg {

constexpr int TC_M = 128;                  // files per tile (tensor-memory lanes)
constexpr int TC_KS = 64;                  // features per MMA stage (4 MMAs, K = 16)
constexpr int TC_KR = 256;                 // features per row copy
constexpr int TC_RAW_PITCH = TC_KR + 16;   // padded row pitch of a row stage
constexpr int TC_CHUNK = 8;                // MMA stages per exact accumulation chunk
constexpr int TC_NAB = 3;                  // operand stages
constexpr int TC_MAX_RAW = 4;              // row stages
constexpr int TC_ACC_COLS = 256;           // tensor-memory columns per accumulator
constexpr int TC_WORK = 16;                // converter / epilogue warps (4 per lane quadrant)
constexpr int TC_PARTS = TC_WORK / 4;      // class parts per row
constexpr int TC_CLS = 16;                 // classes per part (kTcMaxC = TC_PARTS * TC_CLS)
constexpr int TC_THREADS = (TC_WORK + 3) * 32;
constexpr int TC_LAG = 2;                  // stages converted before a drain
constexpr long long TC_WAIT = 2000000000LL;
constexpr uint32_t TC_A_BYTES = TC_M * TC_KS * 2;   // 16 KB

struct TcModelArg {
  const uint8_t* wlay;
  const int32_t* q;
  const float* bias;
  const TcHeader* hdr;
  int C, Cp, N;
};

struct TcArgs {
  const SegGroup* groups;   // group list on the device, or nullptr: g0 alone
  const SegHeader* hdr;     // its header (tiles = 128-row tiles of the list)
  SegGroup g0;
  long long tiles0;
  TcModelArg models[kSegMaxModels];
  int F, nks, nraw, want_lp, recheck;
  uint32_t b_bytes;         // bytes of one weight stage (largest model)
  int* status;
};

struct TcXch {               // per row and half: partial epilogue results
  float best, second, se, smax, bmax, T;
  int idx, pad;
};

struct TcShared {
  uint64_t raw_full[TC_MAX_RAW], raw_empty[TC_MAX_RAW];
  uint64_t b_full[TC_NAB], a_full[TC_NAB], ab_empty[TC_NAB];
  uint64_t acc_full[2], acc_empty[2], xb[2], fin;
  uint32_t tmem;
  int abort;
};

struct TcTile {
  long long row0;
  int nr, g;
};

__device__ __forceinline__ const SegGroup& tc_group(const TcArgs& a, int g) {
  return a.groups ? a.groups[g] : a.g0;
}

__device__ __forceinline__ TcTile tc_tile(const TcArgs& a, int n_groups, long long t) {
  int g = 0;
  if (a.groups && n_groups > 1)
    g = seg_find(n_groups, t, [&](int i) { return a.groups[i].tile0; });
  const SegGroup& G = tc_group(a, g);
  TcTile r;
  r.g = g;
  r.row0 = (t - G.tile0) * TC_M;
  const long long left = G.n - r.row0;
  r.nr = (int)(left < TC_M ? left : TC_M);
  return r;
}

__device__ __forceinline__ uint4 lds16(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(addr)
               : "memory");
  return v;
}

__device__ __forceinline__ void sts16(uint32_t addr, const uint4& v) {
  asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w)
               : "memory");
}

// two u8 counts (bytes picked by sel) -> two exact FP16 values: 1024 + b is
// 0x64bb in FP16, and subtracting 1024 is exact
__device__ __forceinline__ uint32_t u8x2_to_f16x2(uint32_t w, uint32_t sel) {
  const uint32_t x = __byte_perm(w, 0x64646464u, sel);
  uint32_t r;
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(0x64006400u));
  return r;
}

__device__ __forceinline__ bool tc_wait(TcShared& sh, uint64_t* bar, uint32_t parity, int* status) {
  if (mbar_wait_bounded(bar, parity, TC_WAIT)) return true;
  atomicOr(status, ST_TIMEOUT);
  *reinterpret_cast<volatile int*>(&sh.abort) = 1;
  return false;
}

__device__ __forceinline__ bool tc_aborted(TcShared& sh) {
  return *reinterpret_cast<volatile int*>(&sh.abort) != 0;
}

// every lane waits (each observes the phase, so each may read what it
// guards); the warp follows the outcome together
__device__ __forceinline__ bool tc_wait_warp(TcShared& sh, uint64_t* bar, uint32_t parity,
                                             int* status) {
  const bool mine = mbar_wait_bounded(bar, parity, TC_WAIT);
  const bool all = __all_sync(0xFFFFFFFFu, mine) != 0;
  if (!all && (threadIdx.x & 31) == 0) {
    atomicOr(status, ST_TIMEOUT);
    *reinterpret_cast<volatile int*>(&sh.abort) = 1;
  }
  return all;
}

struct TcDrain {
  long long row0;
  uint32_t T;
  int trigger;
  int nr, g;
  int bits;        // accumulator buffer | phase << 1 | last chunk of the tile << 2
};

// Drain one accumulation chunk into the int32 limb sums of this thread's row
// and 16 classes; after the last chunk of a tile, form the scores and write
// label, margin and log posteriors.
__device__ __forceinline__ bool tc_drain(const TcArgs& a, TcShared& sh, TcXch* xch,
                                         const TcDrain& p, int qd, int part, int lane,
                                         uint32_t tmem, int& ep, int (&a0)[TC_CLS],
                                         int (&a1)[TC_CLS], int (&a2)[TC_CLS]) {
  const int r = 32 * qd + lane;
  const int F = a.F;
  const int c0 = TC_CLS * part;
  const int buf = p.bits & 1;
  if (!tc_wait_warp(sh, &sh.acc_full[buf], (uint32_t)(p.bits >> 1) & 1u, a.status)) return false;
  tc_fence_after();
  const SegGroup& G = tc_group(a, p.g);
  const TcModelArg& M = a.models[G.model];
  if (c0 < M.Cp) {
    const uint32_t base =
        tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(buf * TC_ACC_COLS + c0);
    uint32_t v[TC_CLS];
    tmem_ld16(base, v);
    tmem_ld_wait();
#pragma unroll
    for (int i = 0; i < TC_CLS; ++i) a0[i] += __float2int_rn(__uint_as_float(v[i]));
    tmem_ld16(base + (uint32_t)M.Cp, v);
    tmem_ld_wait();
#pragma unroll
    for (int i = 0; i < TC_CLS; ++i) a1[i] += __float2int_rn(__uint_as_float(v[i]));
    tmem_ld16(base + (uint32_t)(2 * M.Cp), v);
    tmem_ld_wait();
#pragma unroll
    for (int i = 0; i < TC_CLS; ++i) a2[i] += __float2int_rn(__uint_as_float(v[i]));
  }
  tc_fence_before();
  __syncwarp();
  if (lane == 0) mbar_arrive(&sh.acc_empty[buf]);
  if (!(p.bits & 4)) return true;

  // ---- epilogue of the tile: scores, arg-max, margin, log-sum-exp ----------
  const long long gr = p.row0 + r;
  const bool valid = r < p.nr;
  const float scale = M.hdr->scale, tau_unit = M.hdr->tau_unit;
  long long k0 = 0, k1 = 0;
  if (valid && G.ovf_ptr) {
    k0 = G.ovf_ptr[gr];
    k1 = G.ovf_ptr[gr + 1];
  }
  // overflow entries (counts above 255) join the limb sums exactly: add * q_l
  // is below 2^23, and the sums stay below 2^31 while the row has fewer than
  // 2^24 tokens (rows with more are sent to the recheck below)
  float T = (float)p.T;
#pragma unroll 1
  for (long long k = k0; k < k1; ++k) {
    const int j = G.ovf_col[k];
    if (j >= F) continue;
    const int add = G.ovf_add[k];
    if (part == 0) T += (float)add;
#pragma unroll
    for (int i = 0; i < TC_CLS; ++i) {
      if (c0 + i >= M.C) break;
      const int Q = M.q[(long long)(c0 + i) * F + j];
      const int q0 = ((Q + 128) & 255) - 128;
      const int Q1 = (Q - q0) >> 8;
      const int q1 = ((Q1 + 128) & 255) - 128;
      a0[i] += add * q0;
      a1[i] += add * q1;
      a2[i] += add * ((Q1 - q1) >> 8);
    }
  }
  // the scores replace the limb sums in a0 (as float bits)
  float best = -INFINITY, second = -INFINITY, smax = 0.f, bmax = 0.f;
  int bidx = 0x7FFFFFFF;
#pragma unroll
  for (int i = 0; i < TC_CLS; ++i) {
    const int c = c0 + i;
    float sc = -INFINITY;
    if (c < M.C) {
      const long long q =
          ((long long)a2[i] << 16) + ((long long)a1[i] << 8) + (long long)a0[i];
      // q = hi 2^24 + lo exactly; one rounding to FP32, one in the FMA
      const float v = fmaf((float)(int)(q >> 24), 16777216.f, (float)(int)(q & 0xFFFFFF));
      const float b = M.bias[c];
      sc = fmaf(v, scale, b);
      smax = fmaxf(smax, fabsf(sc));
      bmax = fmaxf(bmax, fabsf(b));
      if (sc > best) {
        second = best;
        best = sc;
        bidx = c;
      } else if (sc > second) {
        second = sc;
      }
    }
    a0[i] = __float_as_int(sc);
    a1[i] = 0;
    a2[i] = 0;
  }
  float se = 0.f;
#pragma unroll
  for (int i = 0; i < TC_CLS; ++i)
    if (c0 + i < M.C) se += expf(__int_as_float(a0[i]) - best);
  TcXch* xe = xch + (size_t)(ep & 1) * TC_M * TC_PARTS;
  xe[r * TC_PARTS + part] = TcXch{best, second, se, smax, bmax, T, bidx, 0};
  __syncwarp();
  if (lane == 0) mbar_arrive(&sh.xb[ep & 1]);
  if (!tc_wait_warp(sh, &sh.xb[ep & 1], (uint32_t)((ep >> 1) & 1), a.status)) return false;
  ++ep;
  if (!valid) {
#pragma unroll
    for (int i = 0; i < TC_CLS; ++i) a0[i] = 0;
    return true;
  }
  // combine the parts in class order (ties go to the lower class index)
  float Bv = -INFINITY, S2 = -INFINITY, sm = 0.f, bm = 0.f, Tt = 0.f;
  int Bi = 0x7FFFFFFF;
#pragma unroll 1
  for (int k = 0; k < TC_PARTS; ++k) {
    const TcXch x = xe[r * TC_PARTS + k];
    if (x.best > Bv) {
      S2 = fmaxf(Bv, x.second);
      Bv = x.best;
      Bi = x.idx;
    } else {
      S2 = fmaxf(S2, x.best);
    }
    sm = fmaxf(sm, x.smax);
    bm = fmaxf(bm, x.bmax);
    Tt += x.T;
  }
  float sum = 0.f;
#pragma unroll 1
  for (int k = 0; k < TC_PARTS; ++k) {
    const TcXch x = xe[r * TC_PARTS + k];
    if (x.se > 0.f) sum += x.se * expf(x.best - Bv);
  }
  const float lse = Bv + logf(sum);
  const float margin = Bv - S2;
  // |s_c - exact| <= T 2^-(S+1) (weight quantisation) + 2^-23 (|s| + |b|) (the
  // FP32 roundings of the score and of the prior); two classes form the margin
  const float tau =
      2.f * Tt * tau_unit * (1.f + 1.f / 1048576.f) + 2.3841858e-7f * (sm + bm) + 1e-30f;
  bool flag = false;
  if (a.recheck != NB_RECHECK_OFF) {
    flag = !(margin > tau) || !(Tt < 16777216.f);
    if (a.recheck == NB_RECHECK_LP && tau > 5e-6f * fmaxf(1.f, margin)) flag = true;
  }
  if (part == 0) {
    G.label[gr] = flag ? kLabelRecheck : (uint8_t)Bi;
    G.margin[gr] = margin;
  }
  if (a.want_lp && G.logpost) {
    float* lp = G.logpost + gr * M.C;
#pragma unroll
    for (int i = 0; i < TC_CLS; ++i)
      if (c0 + i < M.C) lp[c0 + i] = __int_as_float(a0[i]) - lse;
  }
#pragma unroll
  for (int i = 0; i < TC_CLS; ++i) a0[i] = 0;
  return true;
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_score_tc(const __grid_constant__ TcArgs a) {
  extern __shared__ __align__(1024) uint8_t tc_smem[];
  TcShared& sh = *reinterpret_cast<TcShared*>(tc_smem);
  TcXch* xch = reinterpret_cast<TcXch*>(tc_smem + 1024);   // [2][128][TC_PARTS]
  uint8_t* raw = tc_smem + 1024 + 2 * TC_M * TC_PARTS * sizeof(TcXch);
  uint8_t* A = raw + (size_t)a.nraw * TC_M * TC_RAW_PITCH;
  uint8_t* B = A + (size_t)TC_NAB * TC_A_BYTES;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_groups = a.groups ? a.hdr->n_groups : 1;
  const long long n_tiles = a.groups ? a.hdr->tiles : a.tiles0;
  const int nks = a.nks, F = a.F;

  if (threadIdx.x == 0) {
    for (int i = 0; i < a.nraw; ++i) {
      mbar_init(&sh.raw_full[i], 1);
      mbar_init(&sh.raw_empty[i], TC_WORK);
    }
    for (int i = 0; i < TC_NAB; ++i) {
      mbar_init(&sh.b_full[i], 1);
      mbar_init(&sh.a_full[i], TC_WORK);
      mbar_init(&sh.ab_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&sh.acc_full[i], 1);
      mbar_init(&sh.acc_empty[i], TC_WORK);
      mbar_init(&sh.xb[i], TC_WORK);
    }
    mbar_init(&sh.fin, 1);
    sh.abort = 0;
  }
  if (warp == TC_WORK + 1) tmem_alloc(&sh.tmem, 2 * TC_ACC_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh.tmem;

  if (warp == TC_WORK) {
    // ---- row producer -------------------------------------------------
    long long ri = 0, last[TC_MAX_RAW] = {-1, -1, -1, -1};
    for (long long t = blockIdx.x; t < n_tiles && !tc_aborted(sh); t += gridDim.x) {
      const TcTile tl = tc_tile(a, n_groups, t);
      const SegGroup& G = tc_group(a, tl.g);
      const char* X = G.X + tl.row0 * G.ld_bytes;
      bool ok = true;
      for (int f0 = 0; f0 < F; f0 += TC_KR, ++ri) {
        const int slot = (int)(ri % a.nraw);
        if (!tc_wait_warp(sh, &sh.raw_empty[slot], (uint32_t)((ri / a.nraw) & 1) ^ 1u,
                          a.status)) {
          ok = false;
          break;
        }
        const uint32_t bytes = (uint32_t)(F - f0 < TC_KR ? F - f0 : TC_KR);
        if (lane == 0) mbar_expect_tx(&sh.raw_full[slot], bytes * (uint32_t)tl.nr);
        __syncwarp();
        uint8_t* dst = raw + (size_t)slot * TC_M * TC_RAW_PITCH;
        for (int r = lane; r < tl.nr; r += 32)
          bulk_g2s(dst + r * TC_RAW_PITCH, X + r * G.ld_bytes + f0, bytes, &sh.raw_full[slot]);
        last[slot] = ri;
      }
      if (!ok) break;
    }
    // the phases of a slot complete in order: wait for its last copies
    if (lane == 0)
      for (int s = 0; s < a.nraw; ++s)
        if (last[s] >= 0) tc_wait(sh, &sh.raw_full[s], (uint32_t)((last[s] / a.nraw) & 1), a.status);
  } else if (warp == TC_WORK + 2) {
    // ---- weight-limb producer -----------------------------------------
    long long bi = 0, last[TC_NAB] = {-1, -1, -1};
    for (long long t = blockIdx.x; t < n_tiles && !tc_aborted(sh); t += gridDim.x) {
      const TcTile tl = tc_tile(a, n_groups, t);
      const TcModelArg& M = a.models[tc_group(a, tl.g).model];
      const uint32_t sb = (uint32_t)M.N * 128u;
      bool ok = true;
      for (int ks = 0; ks < nks; ++ks, ++bi) {
        const int slot = (int)(bi % TC_NAB);
        if (!tc_wait_warp(sh, &sh.ab_empty[slot], (uint32_t)((bi / TC_NAB) & 1) ^ 1u,
                          a.status)) {
          ok = false;
          break;
        }
        if (lane == 0) {
          mbar_expect_tx(&sh.b_full[slot], sb);
          bulk_g2s(B + (size_t)slot * a.b_bytes, M.wlay + (size_t)ks * sb, sb, &sh.b_full[slot]);
        }
        last[slot] = bi;
        __syncwarp();
      }
      if (!ok) break;
    }
    if (lane == 0)
      for (int s = 0; s < TC_NAB; ++s)
        if (last[s] >= 0) tc_wait(sh, &sh.b_full[s], (uint32_t)((last[s] / TC_NAB) & 1), a.status);
  } else if (warp == TC_WORK + 1) {
    // ---- MMA issuer ---------------------------------------------------
    if (lane == 0) {
      long long bi = 0, di = 0;
      bool ok = true;
      for (long long t = blockIdx.x; t < n_tiles && ok && !tc_aborted(sh); t += gridDim.x) {
        const TcTile tl = tc_tile(a, n_groups, t);
        const TcModelArg& M = a.models[tc_group(a, tl.g).model];
        const uint32_t idesc = tc_idesc_f16(TC_M, M.N);
        uint32_t d = tmem;
        int buf = 0;
        for (int ks = 0; ks < nks; ++ks, ++bi) {
          if (ks % TC_CHUNK == 0) {
            buf = (int)(di & 1);
            if (!tc_wait(sh, &sh.acc_empty[buf], (uint32_t)((di >> 1) & 1) ^ 1u, a.status)) {
              ok = false;
              break;
            }
            tc_fence_after();
            d = tmem + (uint32_t)(buf * TC_ACC_COLS);
          }
          const int slot = (int)(bi % TC_NAB);
          const uint32_t par = (uint32_t)((bi / TC_NAB) & 1);
          if (!tc_wait(sh, &sh.b_full[slot], par, a.status) ||
              !tc_wait(sh, &sh.a_full[slot], par, a.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t as = smem_addr(A + (size_t)slot * TC_A_BYTES);
          const uint32_t bs = smem_addr(B + (size_t)slot * a.b_bytes);
#pragma unroll
          for (int j = 0; j < TC_KS / 16; ++j)
            tc_mma_f16(d, tc_desc(as + 256u * j, 128u, 1024u), tc_desc(bs + 256u * j, 128u, 1024u),
                       idesc, (uint32_t)((ks % TC_CHUNK) | j));
          tc_commit(&sh.ab_empty[slot]);
          if (ks % TC_CHUNK == TC_CHUNK - 1 || ks == nks - 1) {
            tc_commit(&sh.acc_full[buf]);
            ++di;
          }
        }
      }
      // every MMA issued so far has completed once this arrives
      tc_commit(&sh.fin);
      tc_wait(sh, &sh.fin, 0, a.status);
    }
    __syncwarp();
  } else {
    // ---- converters / drain / epilogue (warps 0 .. TC_WORK-1) ----------
    const int qd = warp & 3, part = warp >> 2;
    const int r = 32 * qd + lane;          // tile row = tensor-memory lane
    int a0[TC_CLS], a1[TC_CLS], a2[TC_CLS];
#pragma unroll
    for (int i = 0; i < TC_CLS; ++i) a0[i] = a1[i] = a2[i] = 0;
    TcDrain p0{}, p1{};      // pending drains, oldest first
    int np = 0;
    int ri = 0, bi = 0, di = 0, gs = 0, ep = 0;   // ring counters of this CTA
    const uint32_t raw_s = smem_addr(raw), a_s = smem_addr(A);
    bool ok = true;


    for (long long t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
      const TcTile tl = tc_tile(a, n_groups, t);
      uint32_t T = 0;
      int rslot = 0;
      for (int ks = 0; ks < nks; ++ks) {
        if (tc_aborted(sh)) {
          ok = false;
          break;
        }
        const int sub = ks & 3;
        if (sub == 0) {
          rslot = (int)(ri % a.nraw);
          if (!tc_wait_warp(sh, &sh.raw_full[rslot], (uint32_t)((ri / a.nraw) & 1), a.status)) {
            ok = false;
            break;
          }
        }
        const int slot = (int)(bi % TC_NAB);
        if (!tc_wait_warp(sh, &sh.ab_empty[slot], (uint32_t)((bi / TC_NAB) & 1) ^ 1u,
                          a.status)) {
          ok = false;
          break;
        }
        // row r, features ks*64 + 16 part .. +15 -> core matrices 2 part, 2 part + 1
        const int f0 = ks * TC_KS + 16 * part;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (r < tl.nr && f0 < F)
          v = lds16(raw_s + (uint32_t)(rslot * TC_M * TC_RAW_PITCH + r * TC_RAW_PITCH +
                                       sub * TC_KS + 16 * part));
        T = dp4a_uu(v.x, 0x01010101u, T);
        T = dp4a_uu(v.y, 0x01010101u, T);
        T = dp4a_uu(v.z, 0x01010101u, T);
        T = dp4a_uu(v.w, 0x01010101u, T);
        const uint32_t at = a_s + (uint32_t)slot * TC_A_BYTES +
                            (uint32_t)((r >> 3) * 1024 + (r & 7) * 16 + 2 * part * 128);
        uint4 o;
        o.x = u8x2_to_f16x2(v.x, 0x5140u);
        o.y = u8x2_to_f16x2(v.x, 0x7362u);
        o.z = u8x2_to_f16x2(v.y, 0x5140u);
        o.w = u8x2_to_f16x2(v.y, 0x7362u);
        sts16(at, o);
        o.x = u8x2_to_f16x2(v.z, 0x5140u);
        o.y = u8x2_to_f16x2(v.z, 0x7362u);
        o.z = u8x2_to_f16x2(v.w, 0x5140u);
        o.w = u8x2_to_f16x2(v.w, 0x7362u);
        sts16(at + 128, o);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.a_full[slot]);
        ++bi;
        if (sub == 3 || ks == nks - 1) {
          if (lane == 0) mbar_arrive(&sh.raw_empty[rslot]);
          ++ri;
        }
        ++gs;
        while (np > 0 && p0.trigger <= gs) {
          if (!tc_drain(a, sh, xch, p0, qd, part, lane, tmem, ep, a0, a1, a2)) {
            ok = false;
            break;
          }
          p0 = p1;
          --np;
        }
        if (!ok) break;
        if (ks % TC_CHUNK == TC_CHUNK - 1 || ks == nks - 1) {
          if (np == 2) {   // very short rows: drain the oldest before queueing
            if (!tc_drain(a, sh, xch, p0, qd, part, lane, tmem, ep, a0, a1, a2)) {
              ok = false;
              break;
            }
            p0 = p1;
            --np;
          }
          TcDrain p;
          p.row0 = tl.row0;
          p.nr = tl.nr;
          p.g = tl.g;
          p.bits = (di & 1) | (((di >> 1) & 1) << 1) | ((ks == nks - 1) ? 4 : 0);
          p.T = T;
          p.trigger = gs + TC_LAG;
          if (np == 0) p0 = p; else p1 = p;
          ++np;
          ++di;
        }
      }
    }
    while (ok && np > 0) {
      if (!tc_drain(a, sh, xch, p0, qd, part, lane, tmem, ep, a0, a1, a2)) break;
      p0 = p1;
      --np;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == TC_WORK + 1) tmem_dealloc(tmem, 2 * TC_ACC_COLS);
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
  return m->kind == NB_MULTINOMIAL && m->d.tc_w != nullptr && dt == NB_U8 && m->F % 16 == 0 &&
         ld % 16 == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
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
static size_t tc_smem_bytes(int nraw, int N) {
  return 1024 + 2 * TC_M * TC_PARTS * sizeof(TcXch) + (size_t)nraw * TC_M * TC_RAW_PITCH +
         (size_t)TC_NAB * (TC_A_BYTES + (uint32_t)N * 128u);
}

static nb_status run_tc(TcArgs& a, int maxN, long long tiles_hint, cudaStream_t st) {
  constexpr size_t kMax = 227 * 1024;
  int nraw = TC_MAX_RAW;
  while (nraw > 2 && tc_smem_bytes(nraw, maxN) > kMax) --nraw;
  const size_t smem = tc_smem_bytes(nraw, maxN);
  if (smem > kMax) {
    set_error("tensor-core scorer: shared memory %zu bytes exceeds the limit", smem);
    return NB_EUNSUPPORTED;
  }
  a.nraw = nraw;
  a.b_bytes = (uint32_t)maxN * 128u;
  // more than half the shared memory of an SM keeps one CTA (and one
  // tensor-memory allocation) per SM
  const size_t launch_smem = smem < 120 * 1024 ? 120 * 1024 : smem;
  NB_TRY_CUDA(cudaFuncSetAttribute(k_score_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)launch_smem),
              "cudaFuncSetAttribute(k_score_tc)");
  long long grid = num_sms();
  if (tiles_hint > 0 && tiles_hint < grid) grid = tiles_hint;
  count_launch();
  k_score_tc<<<(unsigned)grid, TC_THREADS, launch_smem, st>>>(a);
  NB_TRY_CUDA(cudaGetLastError(), "k_score_tc launch");
  return NB_OK;
}

nb_status launch_score_tc(const nb_model* m, const void* X, int64_t n, int64_t ld,
                          const nb_aux* aux, const ScoreOut& o, cudaStream_t st) {
  TcArgs a{};
  a.groups = nullptr;
  a.hdr = nullptr;
  SegGroup& g = a.g0;
  g.X = static_cast<const char*>(X);
  g.ld_bytes = ld;
  g.n = n;
  g.ovf_ptr = aux ? aux->ovf_ptr : nullptr;
  g.ovf_col = aux ? aux->ovf_col : nullptr;
  g.ovf_add = aux ? aux->ovf_add : nullptr;
  g.row_exp = nullptr;
  g.label = o.label;
  g.margin = o.margin;
  g.logpost = o.want_lp ? o.logpost : nullptr;
  g.tile0 = 0;
  g.chunk0 = 0;
  g.model = 0;
  g.family = 2;
  a.tiles0 = (n + TC_M - 1) / TC_M;
  a.models[0] = tc_model_arg(m);
  a.F = m->F;
  a.nks = (m->F + TC_KS - 1) / TC_KS;
  a.want_lp = o.want_lp;
  a.recheck = o.recheck;
  a.status = m->d.status;
  return run_tc(a, a.models[0].N, a.tiles0, st);
}

}  // namespace nbg
