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
// are drained and the limbs joined into one exact int64 sum per class, kept in
// tensor memory next to the two accumulator buffers (2 x 192 + 128 columns);
// overflow-list entries (counts above 255) are added exactly on the CUDA cores.
// The only errors are the weight quantisation, at most T 2^-(S+1) with T the
// file's token count, and two FP32 roundings when the score is formed; the
// epilogue bounds both and marks the row for the FP64 recheck when the bound
// does not settle the label (or the log posteriors).
//
// Roles of one persistent CTA per SM (608 threads):
//   warps 0-15  convert u8 rows to FP16 operand tiles (four warps per tensor-
//               memory lane quadrant), drain the accumulators, run the
//               epilogue (arg-max, top-2 margin, log-sum-exp), 16 classes each;
//   warp 16     streams each tile's rows into shared memory (2-D tensor TMA,
//               128 rows x 128 features per box, 128-byte swizzle, zero fill
//               past the last row and feature);
//   warp 17     allocates tensor memory and issues the MMAs (one thread);
//   warp 18     streams the weight-limb stages (one bulk copy per stage into
//               this CTA's own shared memory).
// Every wait is bounded; a wait that runs out raises ST_TIMEOUT, all roles
// stop, outstanding copies and MMAs are waited for, and tensor memory is freed.
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
constexpr int TC_KS = 64;                  // features per MMA stage (4 MMAs, K = 16)
constexpr int TC_KR = 128;                 // features per row stage (one TMA box)
constexpr int TC_BOX = 128;                // features per TMA box (128-byte swizzle span)
constexpr uint32_t TC_RAW_BYTES = TC_M * TC_KR;   // 16 KB
constexpr int TC_CHUNK = 8;                // MMA stages per chunk of the exact mode
constexpr float TC_T_EXACT = 131072.f;     // 128 T < 2^24: one accumulator is exact
constexpr int TC_REDO_CAP = 64;            // tiles a CTA can queue for the exact pass
constexpr int TC_PF = 6;                   // row stages prefetched into L2 ahead of the loads
constexpr int TC_NAB = 4;                  // operand stages
constexpr int TC_MAX_RAW = 4;              // row stages
constexpr int TC_ACC_COLS = 192;           // tensor-memory columns per FP32 accumulator
constexpr int TC_SUM_COL = 2 * TC_ACC_COLS; // exact int64 sums: 2 columns per class
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
  CUtensorMap tmap;         // u8 rows of the group (single-group launch)
  const CUtensorMap* maps;  // group list: one map per group (device), else nullptr
  const SegGroup* groups;   // group list on the device, or nullptr: g0 alone
  const SegHeader* hdr;     // its header (tiles = 128-row tiles of the list)
  SegGroup g0;
  long long tiles0;
  TcModelArg models[kSegMaxModels];
  int F, nks, nraw, want_lp, recheck;
  int single;               // 1: one accumulation per row, heavy rows redone exactly
  uint32_t b_bytes;         // bytes of one weight stage (largest model)
  int* status;
};

struct TcXch {               // partial epilogue results of each class part and row
  float best[TC_PARTS][TC_M], second[TC_PARTS][TC_M], se[TC_PARTS][TC_M];
  float smax[TC_PARTS][TC_M], bmax[TC_PARTS][TC_M], T[TC_PARTS][TC_M], Tplane[TC_PARTS][TC_M];
  int idx[TC_PARTS][TC_M];
};

struct TcShared {
  uint64_t raw_full[TC_MAX_RAW], raw_empty[TC_MAX_RAW];
  uint64_t b_full[TC_NAB], a_full[TC_NAB], ab_empty[TC_NAB];
  uint64_t acc_full[2], acc_empty[2], fin, redo_ready;
  uint64_t xfull, xfree;        // exchange written by all parts / read by all parts
  uint32_t tmem;
  int abort;
  int redo_flag[2];
  int redo_n;                   // tiles queued for the exact pass (phase 1)
  int redo_list[TC_REDO_CAP];
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
  r.nr = (int)(left <= 0 ? 0 : (left < TC_M ? left : TC_M));
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

// bounded wait that sleeps in the barrier instead of polling
__device__ __forceinline__ bool tc_wait_sleep(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait_sleep(bar, parity, 100000u)) {
    if (clock64() - t0 > TC_WAIT) return false;
  }
  return true;
}

__device__ __forceinline__ bool tc_wait(TcShared& sh, uint64_t* bar, uint32_t parity, int* status) {
  if (tc_wait_sleep(bar, parity)) return true;
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
  const bool mine = tc_wait_sleep(bar, parity);
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
  int nr, g, tile;
  int bits;        // accumulator buffer | phase << 1 | last chunk of the tile << 2
};

// score of class c from its exact sum q: q = hi 2^24 + lo exactly, one
// rounding to FP32, one in the FMA with the prior
__device__ __forceinline__ float tc_score(uint32_t lo, uint32_t hi, float scale, float b) {
  const long long q = (long long)(((unsigned long long)hi << 32) | lo);
  const float v = fmaf((float)(int)(q >> 24), 16777216.f, (float)(int)(q & 0xFFFFFF));
  return fmaf(v, scale, b);
}

// Epilogue of a tile: the thread's exact sums stay in its tensor-memory lane
// until it starts its next tile, so they are read twice, 8 classes at a time
// (pass 1: arg-max, second best and sum of exponentials; pass 2: log
// posteriors), which keeps the epilogue's registers small.
__device__ __forceinline__ bool tc_epilogue(const TcArgs& a, TcShared& sh, TcXch* xch,
                                            long long row0, int nr, int g, int tile,
                                            bool check_heavy, uint32_t Tpart,
                                            int qd, int part, int lane, uint32_t tmem,
                                            int& ep) {
  const int r = 32 * qd + lane;
  const int F = a.F;
  const int c0 = TC_CLS * part;
  const SegGroup& G = tc_group(a, g);
  const TcModelArg& M = a.models[G.model];
  const uint32_t lane_base = tmem + ((uint32_t)(32 * qd) << 16);
  const long long gr = row0 + r;
  const bool valid = r < nr;
  long long k0 = 0, k1 = 0;
  if (valid && G.ovf_ptr) {
    k0 = G.ovf_ptr[gr];
    k1 = G.ovf_ptr[gr + 1];
  }
  const float scale = M.hdr->scale, tau_unit = M.hdr->tau_unit;
  float T = (float)Tpart;
  // overflow entries (counts above 255) join the sums exactly (rare path)
  if (__any_sync(0xFFFFFFFFu, k1 > k0)) {
#pragma unroll 1
    for (int hh = 0; hh < 2; ++hh) {
      const int cb = c0 + 8 * hh;
      if (cb >= M.Cp) break;
      uint32_t sw[16];
      const uint32_t addr = lane_base + (uint32_t)(TC_SUM_COL + 2 * cb);
      tmem_ld16(addr, sw);
      tmem_ld_wait();
#pragma unroll 1
      for (long long k = k0; k < k1; ++k) {
        const int j = G.ovf_col[k];
        if (j >= F) continue;
        const long long add = G.ovf_add[k];
        if (part == 0 && hh == 0) T += (float)add;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          if (cb + i >= M.C) break;
          unsigned long long x = ((unsigned long long)sw[2 * i + 1] << 32) | sw[2 * i];
          x += (unsigned long long)(add * M.q[(long long)(cb + i) * F + j]);
          sw[2 * i] = (uint32_t)x;
          sw[2 * i + 1] = (uint32_t)(x >> 32);
        }
      }
      __syncwarp();   // the lanes' overflow loops differ in length
      tmem_st16(addr, sw);
      tmem_st_wait();
    }
  }
  // pass 1
  float best = -INFINITY, second = -INFINITY, smax = 0.f, bmax = 0.f, se = 0.f;
  int bidx = 0x7FFFFFFF;
#pragma unroll 1
  for (int hh = 0; hh < 2; ++hh) {
    const int cb = c0 + 8 * hh;
    if (cb >= M.Cp) break;
    uint32_t sw[16];
    tmem_ld16(lane_base + (uint32_t)(TC_SUM_COL + 2 * cb), sw);
    tmem_ld_wait();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int c = cb + i;
      if (c >= M.C) break;
      const float b = M.bias[c];
      const float sc = tc_score(sw[2 * i], sw[2 * i + 1], scale, b);
      smax = fmaxf(smax, fabsf(sc));
      bmax = fmaxf(bmax, fabsf(b));
      if (sc > best) {            // running sum of exp(s - best)
        se = se * expf(best - sc) + 1.f;
        second = best;
        best = sc;
        bidx = c;
      } else {
        se += expf(sc - best);
        if (sc > second) second = sc;
      }
    }
  }
  TcXch& xe = *xch;
  const int eph = ep & 1;
  // the exchange of the previous tile must have been read by every part
  if (!tc_wait_warp(sh, &sh.xfree, (uint32_t)eph ^ 1u, a.status)) return false;
  // the flag of the next tile of the other parity is free once xfull passes
  if (r == 0 && part == 0) sh.redo_flag[eph ^ 1] = 0;
  xe.best[part][r] = best;
  xe.second[part][r] = second;
  xe.se[part][r] = se;
  xe.smax[part][r] = smax;
  xe.bmax[part][r] = bmax;
  xe.T[part][r] = T;
  xe.Tplane[part][r] = (float)Tpart;
  xe.idx[part][r] = bidx;
  __syncwarp();
  if (lane == 0) mbar_arrive(&sh.xfull);
  if (!tc_wait_warp(sh, &sh.xfull, (uint32_t)eph, a.status)) return false;
  ++ep;
  // combine the parts in class order (ties go to the lower class index); every
  // lane stays to the end, since the tensor-memory loads below need the warp
  // converged, and only rows of the tile store results
  float Bv = -INFINITY, S2 = -INFINITY, sm = 0.f, bm = 0.f, Tt = 0.f, Tp = 0.f;
  int Bi = 0x7FFFFFFF;
#pragma unroll 1
  for (int k = 0; k < TC_PARTS; ++k) {
    const float xb = xe.best[k][r];
    Tp += xe.Tplane[k][r];
    if (xb > Bv) {
      S2 = fmaxf(Bv, xe.second[k][r]);
      Bv = xb;
      Bi = xe.idx[k][r];
    } else {
      S2 = fmaxf(S2, xb);
    }
    sm = fmaxf(sm, xe.smax[k][r]);
    bm = fmaxf(bm, xe.bmax[k][r]);
    Tt += xe.T[k][r];
  }
  float sum = 0.f;
#pragma unroll 1
  for (int k = 0; k < TC_PARTS; ++k) {
    const float xs = xe.se[k][r];
    if (xs > 0.f) sum += xs * expf(xe.best[k][r] - Bv);
  }
  __syncwarp();
  if (lane == 0) mbar_arrive(&sh.xfree);   // this tile's exchange is read
  const float lse = Bv + logf(sum);
  const float margin = Bv - S2;
  // |s_c - exact| <= T 2^-(S+1) (weight quantisation) + 2^-23 (|s| + |b|) (the
  // FP32 roundings of the score and of the prior); two classes form the margin
  const float tau =
      2.f * Tt * tau_unit * (1.f + 1.f / 1048576.f) + 2.3841858e-7f * (sm + bm) + 1e-30f;
  bool flag = false;
  if (a.recheck != NB_RECHECK_OFF) {
    flag = !(margin > tau);
    if (a.recheck == NB_RECHECK_LP && tau > 5e-6f * fmaxf(1.f, margin)) flag = true;
  }
  // A row of 2^17 or more stored counts may have rounded in the single
  // accumulation: it is marked for the FP64 recheck and its tile queued for the
  // exact (chunked) pass, which overwrites the tile's results.
  const bool heavy = check_heavy && !(Tp < TC_T_EXACT);
  if (valid && part == 0) {
    G.label[gr] = (flag || heavy) ? kLabelRecheck : (uint8_t)Bi;
    G.margin[gr] = margin;
    if (heavy && atomicExch(&sh.redo_flag[eph], 1) == 0) {
      const int k = atomicAdd(&sh.redo_n, 1);
      if (k < TC_REDO_CAP) sh.redo_list[k] = tile;   // beyond: the FP64 recheck
    }
  }
  if (a.want_lp && G.logpost) {
    // pass 2
    float* lp = G.logpost + (valid ? gr : 0) * M.C;
#pragma unroll 1
    for (int hh = 0; hh < 2; ++hh) {
      const int cb = c0 + 8 * hh;
      if (cb >= M.Cp) break;
      uint32_t sw[16];
      tmem_ld16(lane_base + (uint32_t)(TC_SUM_COL + 2 * cb), sw);
      tmem_ld_wait();
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int c = cb + i;
        if (c >= M.C) break;
        if (valid) lp[c] = tc_score(sw[2 * i], sw[2 * i + 1], scale, M.bias[c]) - lse;
      }
    }
  }
  return true;
}

// Drain one accumulation chunk: add its three limb sums (exact integers
// below 2^24 in FP32) into this thread's 16 exact int64 sums, which live in
// tensor memory (2 columns per class, low word first), 8 classes at a time.
// After the last chunk of a tile, run the epilogue.
__device__ __forceinline__ bool tc_drain(const TcArgs& a, TcShared& sh, TcXch* xch,
                                         const TcDrain& p, int qd, int part, int lane,
                                         uint32_t tmem, int& ep) {
  const int c0 = TC_CLS * part;
  const int buf = p.bits & 1;
  if (!tc_wait_warp(sh, &sh.acc_full[buf], (uint32_t)(p.bits >> 1) & 1u, a.status)) return false;
  tc_fence_after();
  const int Cp = a.models[tc_group(a, p.g).model].Cp;
  const uint32_t lane_base = tmem + ((uint32_t)(32 * qd) << 16);
#pragma unroll
  for (int hh = 0; hh < 2; ++hh) {
    const int cb = c0 + 8 * hh;
    if (cb < Cp) {
      uint32_t sw[16];
      const uint32_t sum_addr = lane_base + (uint32_t)(TC_SUM_COL + 2 * cb);
      if (p.bits & 8) {        // first chunk of the tile
#pragma unroll
        for (int i = 0; i < 16; ++i) sw[i] = 0;
      } else {
        tmem_ld16(sum_addr, sw);
        tmem_ld_wait();
      }
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        uint32_t v[8];
        tmem_ld8(lane_base + (uint32_t)(buf * TC_ACC_COLS + l * Cp + cb), v);
        tmem_ld_wait();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          unsigned long long x = ((unsigned long long)sw[2 * i + 1] << 32) | sw[2 * i];
          x += (unsigned long long)((long long)__float2int_rn(__uint_as_float(v[i])) << (8 * l));
          sw[2 * i] = (uint32_t)x;
          sw[2 * i + 1] = (uint32_t)(x >> 32);
        }
      }
      tmem_st16(sum_addr, sw);
      tmem_st_wait();
    }
  }
  tc_fence_before();
  __syncwarp();
  if (lane == 0) mbar_arrive(&sh.acc_empty[buf]);
  if (!(p.bits & 4)) return true;
  return tc_epilogue(a, sh, xch, p.row0, p.nr, p.g, p.tile, (p.bits & 16) != 0, p.T, qd,
                     part, lane, tmem, ep);
}

// Tiles of this CTA: phase 0 its share of all tiles (blockIdx.x + i gridDim.x),
// phase 1 the tiles it queued for the exact pass.
__device__ __forceinline__ long long tc_ntiles(const TcArgs& a, TcShared& sh, long long n_tiles,
                                               int phase) {
  if (phase) {
    const int c = *reinterpret_cast<volatile int*>(&sh.redo_n);
    return c < TC_REDO_CAP ? c : TC_REDO_CAP;
  }
  const long long k = blockIdx.x;
  return k < n_tiles ? (n_tiles - k + gridDim.x - 1) / gridDim.x : 0;
}
__device__ __forceinline__ long long tc_tile_at(const TcArgs& a, TcShared& sh, int phase,
                                                long long i) {
  if (phase) return (long long)sh.redo_list[i];
  return (long long)blockIdx.x + i * (long long)gridDim.x;
}
// MMA stages per accumulation chunk: the whole row in the single-accumulation
// phase, 512 features (always exact) otherwise
__device__ __forceinline__ int tc_chunk(const TcArgs& a, int phase) {
  return (a.single && phase == 0) ? a.nks : TC_CHUNK;
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_score_tc(const __grid_constant__ TcArgs a) {
  extern __shared__ __align__(1024) uint8_t tc_smem[];
  TcShared& sh = *reinterpret_cast<TcShared*>(tc_smem);
  TcXch* xch = reinterpret_cast<TcXch*>(tc_smem + 1024);
  uint8_t* raw = tc_smem + 1024 + sizeof(TcXch);            // 1 KB aligned
  uint8_t* A = raw + (size_t)a.nraw * TC_RAW_BYTES;
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

    }
    mbar_init(&sh.fin, 1);
    mbar_init(&sh.xfull, TC_WORK);
    mbar_init(&sh.xfree, TC_WORK);
    mbar_init(&sh.redo_ready, TC_WORK);
    sh.abort = 0;
    sh.redo_flag[0] = sh.redo_flag[1] = 0;
    sh.redo_n = 0;
  }
  if (warp == TC_WORK + 1) tmem_alloc(&sh.tmem, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh.tmem;

  if (warp == TC_WORK) {
    // ---- row producer -------------------------------------------------
    long long ri = 0, last[TC_MAX_RAW] = {-1, -1, -1, -1};
    uint32_t lastp[TC_MAX_RAW] = {0, 0, 0, 0};
    int rs = 0;          // slot of the next row stage
    uint32_t rp = 0;     // its phase parity
    if ((smem_addr(raw) & 1023u) != 0) {   // the swizzled reads assume 1 KB alignment
      if (lane == 0) {
        atomicOr(a.status, ST_TIMEOUT);
        *reinterpret_cast<volatile int*>(&sh.abort) = 1;
      }
    }
    bool ok = true;
    const uint64_t map = reinterpret_cast<uint64_t>(&a.tmap);
    // L2 prefetch cursor of phase 0, TC_PF row stages ahead of the loads: the
    // shared-memory stages then fill from L2, so few of them keep HBM busy
    long long pit = 0, npf = 0;
    int pf0 = 0;
    const long long nt0 = tc_ntiles(a, sh, n_tiles, 0);
    for (int phase = 0; phase < 2 && ok; ++phase) {
     if (phase == 1 && !tc_wait_warp(sh, &sh.redo_ready, 0, a.status)) break;
     const long long nt = tc_ntiles(a, sh, n_tiles, phase);
     for (long long it = 0; it < nt && ok && !tc_aborted(sh); ++it) {
      const long long t = tc_tile_at(a, sh, phase, it);
      const TcTile tl = tc_tile(a, n_groups, t);
      // a group's map sits in the work list, rewritten between calls: drop any
      // stale copy the tensor-map proxy may hold
      const uint64_t tmap = a.maps ? reinterpret_cast<uint64_t>(a.maps + tl.g) : map;
      if (a.maps && lane == 0)
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmap)
                     : "memory");
      for (int f0 = 0; f0 < F; f0 += TC_KR, ++ri) {
        if (phase == 0 && lane == 0)
          for (; npf < ri + TC_PF && pit < nt0; ++npf) {
            const TcTile pt = tc_tile(a, n_groups, tc_tile_at(a, sh, 0, pit));
#pragma unroll
            for (int b = 0; b < TC_KR / TC_BOX; ++b)
              asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                               a.maps ? reinterpret_cast<uint64_t>(a.maps + pt.g) : map),
                           "r"(pf0 + b * TC_BOX), "r"((int)pt.row0)
                           : "memory");
            pf0 += TC_KR;
            if (pf0 >= F) {
              pf0 = 0;
              ++pit;
            }
          }
        const int slot = rs;
        const uint32_t rpar = rp;
        if (++rs == a.nraw) {
          rs = 0;
          rp ^= 1u;
        }
        if (!tc_wait_warp(sh, &sh.raw_empty[slot], rpar ^ 1u, a.status)) {
          ok = false;
          break;
        }
        if (lane == 0) {
          mbar_expect_tx(&sh.raw_full[slot], TC_RAW_BYTES);
          uint8_t* dst = raw + (size_t)slot * TC_RAW_BYTES;
          const int y = (int)tl.row0;
#pragma unroll
          for (int b = 0; b < TC_KR / TC_BOX; ++b)
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst + b * (TC_M * TC_BOX))),
                "l"(tmap), "r"(f0 + b * TC_BOX), "r"(y), "r"(smem_addr(&sh.raw_full[slot]))
                : "memory");
        }
        last[slot] = ri;
        lastp[slot] = rpar;
        __syncwarp();
      }
     }
    }
    // the phases of a slot complete in order: wait for its last copies
    if (lane == 0)
      for (int s = 0; s < a.nraw; ++s)
        if (last[s] >= 0) tc_wait(sh, &sh.raw_full[s], lastp[s], a.status);
  } else if (warp == TC_WORK + 2) {
    // ---- weight-limb producer -----------------------------------------
    long long bi = 0, last[TC_NAB] = {-1, -1, -1, -1};
    bool ok = true;
    for (int phase = 0; phase < 2 && ok; ++phase) {
     if (phase == 1 && !tc_wait_warp(sh, &sh.redo_ready, 0, a.status)) break;
     const long long nt = tc_ntiles(a, sh, n_tiles, phase);
     for (long long it = 0; it < nt && ok && !tc_aborted(sh); ++it) {
      const TcTile tl = tc_tile(a, n_groups, tc_tile_at(a, sh, phase, it));
      const TcModelArg& M = a.models[tc_group(a, tl.g).model];
      const uint32_t sb = (uint32_t)M.N * 128u;
      for (int ks = 0; ks < nks; ++ks, ++bi) {
        const int slot = (int)((unsigned long long)bi & (TC_NAB - 1));
        const uint32_t bpar = (uint32_t)(((unsigned long long)bi / TC_NAB) & 1);
        if (!tc_wait_warp(sh, &sh.ab_empty[slot], bpar ^ 1u, a.status)) {
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
     }
    }
    if (lane == 0)
      for (int s = 0; s < TC_NAB; ++s)
        if (last[s] >= 0)
          tc_wait(sh, &sh.b_full[s], (uint32_t)(((unsigned long long)last[s] / TC_NAB) & 1),
                  a.status);
  } else if (warp == TC_WORK + 1) {
    // ---- MMA issuer ---------------------------------------------------
    if (lane == 0) {
      long long bi = 0, di = 0;
      bool ok = true;
      for (int phase = 0; phase < 2 && ok; ++phase) {
       if (phase == 1 && !tc_wait(sh, &sh.redo_ready, 0, a.status)) break;
       const long long nt = tc_ntiles(a, sh, n_tiles, phase);
       const int chunk = tc_chunk(a, phase);
       for (long long it = 0; it < nt && ok && !tc_aborted(sh); ++it) {
        const TcTile tl = tc_tile(a, n_groups, tc_tile_at(a, sh, phase, it));
        const TcModelArg& M = a.models[tc_group(a, tl.g).model];
        const uint32_t idesc = tc_idesc_f16(TC_M, M.N);
        uint32_t d = tmem;
        int buf = 0, kc = 0;   // kc: MMA stage within the accumulation chunk
        for (int ks = 0; ks < nks; ++ks, ++bi) {
          if (kc == 0) {
            buf = (int)(di & 1);
            if (!tc_wait(sh, &sh.acc_empty[buf], (uint32_t)((di >> 1) & 1) ^ 1u, a.status)) {
              ok = false;
              break;
            }
            tc_fence_after();
            d = tmem + (uint32_t)(buf * TC_ACC_COLS);
          }
          const int slot = (int)((unsigned long long)bi & (TC_NAB - 1));
          const uint32_t par = (uint32_t)(((unsigned long long)bi / TC_NAB) & 1);
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
                       idesc, (uint32_t)(kc | j));
          tc_commit(&sh.ab_empty[slot]);
          if (++kc == chunk || ks == nks - 1) {
            tc_commit(&sh.acc_full[buf]);
            ++di;
            kc = 0;
          }
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
    TcDrain p0{}, p1{};      // pending drains, oldest first
    int np = 0;
    int ri = 0, bi = 0, di = 0, gs = 0, ep = 0;   // ring counters of this CTA
    int rs = 0;          // slot of the next row stage
    uint32_t rp = 0;     // its phase parity
    const uint32_t raw_s = smem_addr(raw), a_s = smem_addr(A);
    bool ok = true;


    for (int phase = 0; phase < 2 && ok; ++phase) {
     if (phase == 1) {
      // every epilogue of phase 0 is done once all converter warps arrive
      while (ok && np > 0) {
        if (!tc_drain(a, sh, xch, p0, qd, part, lane, tmem, ep)) ok = false;
        p0 = p1;
        --np;
      }
      if (!ok) break;
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.redo_ready);
      if (!tc_wait_warp(sh, &sh.redo_ready, 0, a.status)) break;
     }
     const long long nt = tc_ntiles(a, sh, n_tiles, phase);
     const int chunk = tc_chunk(a, phase);
     const int heavy_bit = (a.single && phase == 0) ? 16 : 0;
     for (long long it = 0; it < nt && ok; ++it) {
      const long long t = tc_tile_at(a, sh, phase, it);
      const TcTile tl = tc_tile(a, n_groups, t);
      uint32_t T = 0, rpar = 0;
      int rslot = 0, kc = 0;
      for (int ks = 0; ks < nks; ++ks) {
        if (tc_aborted(sh)) {
          ok = false;
          break;
        }
        const int sub = ks & 1;   // MMA stage within the row stage
        if (sub == 0) {
          rslot = rs;
          rpar = rp;
          if (++rs == a.nraw) {
            rs = 0;
            rp ^= 1u;
          }
          if (!tc_wait_warp(sh, &sh.raw_full[rslot], rpar, a.status)) {
            ok = false;
            break;
          }
        }
        const int slot = bi & (TC_NAB - 1);
        if (!tc_wait_warp(sh, &sh.ab_empty[slot], ((uint32_t)bi / TC_NAB & 1u) ^ 1u, a.status)) {
          ok = false;
          break;
        }
        // row r, features ks*64 + 16 part .. +15 -> core matrices 2 part, 2 part + 1
        // 16-byte chunk sub*4 + part of row r, swizzled by r & 7; rows and
        // features past the end arrive as zeros
        const int c16 = (sub << 2) + part;
        const uint4 v = lds16(raw_s + (uint32_t)rslot * TC_RAW_BYTES +
                              (uint32_t)(r * TC_BOX + ((c16 ^ (r & 7)) << 4)));
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
        if (sub == 1 || ks == nks - 1) {
          if (lane == 0) mbar_arrive(&sh.raw_empty[rslot]);
          ++ri;
        }
        ++gs;
        while (np > 0 && p0.trigger <= gs) {
          if (!tc_drain(a, sh, xch, p0, qd, part, lane, tmem, ep)) {
            ok = false;
            break;
          }
          p0 = p1;
          --np;
        }
        if (!ok) break;
        const bool chunk_end = ++kc == chunk || ks == nks - 1;
        if (chunk_end) {
          if (np == 2) {   // very short rows: drain the oldest before queueing
            if (!tc_drain(a, sh, xch, p0, qd, part, lane, tmem, ep)) {
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
          p.tile = (int)t;
          p.bits = (di & 1) | (((di >> 1) & 1) << 1) | ((ks == nks - 1) ? 4 : 0) |
                   (ks < chunk ? 8 : 0) | heavy_bit;
          kc = 0;
          p.T = T;
          p.trigger = gs + TC_LAG;
          if (np == 0) p0 = p; else p1 = p;
          ++np;
          ++di;
        }
      }
     }
    }
    while (ok && np > 0) {
      if (!tc_drain(a, sh, xch, p0, qd, part, lane, tmem, ep)) break;
      p0 = p1;
      --np;
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
  return m->kind == NB_MULTINOMIAL && m->d.tc_w != nullptr && dt == NB_U8 &&
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
  return 1024 + sizeof(TcXch) + (size_t)nraw * TC_RAW_BYTES +
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
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(TC_THREADS);
  cfg.dynamicSmemBytes = launch_smem;
  cfg.stream = st;
  long long grid = num_sms();
  if (tiles_hint > 0 && tiles_hint < grid) grid = tiles_hint;
  cfg.gridDim = dim3((unsigned)grid);
  count_launch();
  NB_TRY_CUDA(cudaLaunchKernelEx(&cfg, k_score_tc, a), "k_score_tc launch");
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

// 2-D map of n rows x F u8 features (row pitch ld bytes): 128 x 128 boxes,
// 128-byte swizzle, zero fill out of bounds
static nb_status tc_row_map(CUtensorMap* map, const void* X, int64_t n, int F, int64_t ld) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tc_encode_fn();
  if (!enc) {
    set_error("tensor-core scorer: cuTensorMapEncodeTiled is not available");
    return NB_ECUDA;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)F, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)ld};
  const cuuint32_t box[2] = {(cuuint32_t)TC_BOX, (cuuint32_t)TC_M};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(X), dims, strides,
                         box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("tensor-core scorer: cuTensorMapEncodeTiled failed (%d)", (int)r);
    return NB_ECUDA;
  }
  return NB_OK;
}

nb_status launch_score_tc(const nb_model* m, const void* X, int64_t n, int64_t ld,
                          const nb_aux* aux, const ScoreOut& o, cudaStream_t st) {
  TcArgs a{};
  nb_status ms = tc_row_map(&a.tmap, X, n, m->F, ld);
  if (ms != NB_OK) return ms;
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
  a.status = m->d.sstatus;
  a.single = 1;
  return run_tc(a, a.models[0].N, a.tiles0, st);
}

// tensor map of a group's u8 rows for a batch work list (128 bytes at map)
nb_status tc_encode_rows(void* map, const void* X, int64_t n, int F, int64_t ld_bytes) {
  return tc_row_map(static_cast<CUtensorMap*>(map), X, n, F, ld_bytes);
}

bool tc_group_eligible(const nb_model* m, const void* X, int64_t ld_bytes) {
  return tc_eligible(m, NB_U8, X, ld_bytes);
}

nb_status launch_score_tc_seg(const SegGroup* groups, const SegHeader* hdr, const void* maps,
                              const nb_model* const* models, int n_models, int F, int want_lp,
                              int recheck, int* status, cudaStream_t st) {
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
  a.single = 1;
  return run_tc(a, maxN, 0, st);
}

}  // namespace nbg
