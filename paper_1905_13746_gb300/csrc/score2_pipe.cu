// TMA-pipelined two-class scorer (Sec. 4 posterior and decision rule, in the
// log-odds form d = b + sum_j x_j Delta_j).
//
// Each block owns a contiguous range of files.  The producer warp
// (pipe.cuh) streams blocks of RS consecutive rows and their overflow-list
// slices into shared-memory stages.  NCW consumer warps work on RPW rows at a
// time each, LPR = 32 / RPW lanes per row: lane i of a row's lane group owns
// the row's 16-byte vectors v = i, i + LPR, ..., and holds the Delta table
// slice of those vectors in registers (staged once per block by a bulk copy).
//
// u8 storage: the three int8 limbs of the fixed-point Delta and the count
// total T are accumulated with dp4a in four int32 sums per row (FP8 E4M3
// storage: the values as exact integer counts in 16-bit pairs, with dp2a),
// reduced by a
// butterfly inside the lane group (exact), and combined into an int64 only
// when the row is finished.  Overflow entries (count - 255 at a column) are
// split over the row's lanes and added limb by limb, the column's three limbs
// read as one packed word (staged after the limb planes).  FP32 paths decode
// each vector and FMA into four accumulators, then the same butterfly.
//
// Finished rows wait in registers (lane j holds the j-th) and are finalised
// 32 at a time, one lane per row: label, margin, log posteriors, FP64-recheck
// mark.  Integer sums make the u8 results independent of the tile shape.
#include "pipe.cuh"
#include "score2.cuh"

namespace nbg {


template <int LPR, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int off = LPR / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
  return v;
}

struct RowSum {   // one finished row waiting for its epilogue
  int a0, a1, a2;  // limb sums (u8) ...
  uint32_t t;      // ... and count total
  float s, tf;     // FP32 sum and |x| total (other storage)
};

template <int DT>
__device__ __forceinline__ void finish_row(const S2Args& a, float hb, float inv_scale, float maxabs,
                                           long long row, const RowSum& r) {
  if (DT == NB_U8 || DT == NB_FP8E4M3) {
    const long long D = ((long long)r.a2 << 16) + ((long long)r.a1 << 8) + (long long)r.a0;
    const float Dsum = (float)D * inv_scale;
    const float d = Dsum + hb;
    c2_epilogue(a, row, d, c2_tau_u8((float)r.t, Dsum, hb, inv_scale, maxabs));
  } else {
    float scale = 1.f;
    if (DT == NB_FP8E4M3 && a.row_exp) scale = exp2f((float)a.row_exp[row]);
    const float sum = r.s * scale;
    const float d = sum + hb;
    const float kk = (float)a.k_base;
    const float gam = kk * 5.9604645e-8f / (1.f - kk * 5.9604645e-8f);
    const float A = r.tf * scale * maxabs * 1.001f;
    const float tau = gam * (A + fabsf(hb)) * 1.01f + 1e-12f * (A + fabsf(hb)) + 1e-30f;
    c2_epilogue(a, row, d, tau);
  }
}

// mask of the first vb (clamped to 0..4) bytes of a 32-bit word
__device__ __forceinline__ uint32_t u8_keep_mask(int vb) {
  vb = vb < 0 ? 0 : (vb > 4 ? 4 : vb);
  return vb >= 4 ? 0xFFFFFFFFu : ((1u << (8 * vb)) - 1u);
}

// FULL: every lane's KV vectors lie inside the row (no bound or tail checks);
// the kernel then carries no per-vector branches.  OVF (u8 only): the rows
// carry an overflow list, and the packed limb words (one 32-bit word per
// feature, limb l in byte l) follow the three limb planes in shared memory.
template <int DT, int KV, int RPW, int NCW, bool FULL, bool OVF>
__global__ void __launch_bounds__((NCW + 1) * 32, NCW == 8 ? 2 : 1)
    k_score2_pipe(const S2Args a, const PipeArgs p) {
  constexpr int LPR = 32 / RPW;
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint64_t full[kMaxStages], empty[kMaxStages], tabbar;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / LPR, li = lane % LPR;
  const long long t0 = p.tiles * blockIdx.x / gridDim.x;
  const long long t1 = p.tiles * (blockIdx.x + 1) / gridDim.x;
  const long long ntl = t1 - t0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NCW);
    }
    mbar_init(&tabbar, 1);
  }
  __syncthreads();

  if (warp == NCW) {
    const PipeSrc src{a.X, a.ld_bytes, a.n, a.ovf_ptr, a.ovf_col, a.ovf_add, nullptr, a.table,
                      a.status};
    pipe_produce(src, p, sm, full, empty, &tabbar, t0, ntl);
    return;
  }

  // ------------------------------------------------------------- consumers
  using Dec = Decode<DT>;
  constexpr int EPV = Dec::EPV, QPV = EPV / 4;
  constexpr bool LIMBS = DT == NB_U8 || DT == NB_FP8E4M3;   // fixed-point limbs, exact
  const float hb = a.hdr->b, inv_scale = a.hdr->inv_scale, maxabs = a.hdr->maxabs;
  if (!mbar_wait_bounded(&tabbar, 0)) {
    if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
    return;
  }
  const int nv = a.nvec_row, nt = a.nvec_tab;
  uint4 q0[KV], q1[KV], q2[KV];
  float4 wq[KV][QPV];
#pragma unroll
  for (int kv = 0; kv < KV; ++kv) {
    const int v = li + LPR * kv;
    if (LIMBS) {
      const uint4* tab = reinterpret_cast<const uint4*>(sm);
      const uint4 z = make_uint4(0, 0, 0, 0);
      q0[kv] = (FULL || v < nv) ? tab[v] : z;
      q1[kv] = (FULL || v < nv) ? tab[nt + v] : z;
      q2[kv] = (FULL || v < nv) ? tab[2 * nt + v] : z;
    } else {
      const float4* tab = reinterpret_cast<const float4*>(sm);
#pragma unroll
      for (int q = 0; q < QPV; ++q)
        wq[kv][q] = (FULL || v < nv) ? tab[q * nt + v] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  // FP8 rows: each lane's limb byte sums and value count remove the bias of
  // the biased dp2a sums once per row
  int fs0 = 0, fs1 = 0, fs2 = 0, fnv = 0;
  if (DT == NB_FP8E4M3) {
#pragma unroll
    for (int kv = 0; kv < KV; ++kv) {
      if (!(FULL || li + LPR * kv < nv)) continue;
      fs0 += limb_byte_sum(q0[kv]);
      fs1 += limb_byte_sum(q1[kv]);
      fs2 += limb_byte_sum(q2[kv]);
      fnv += 16;
    }
  }
  // u8 overflow entries: the packed limb words after the three planes
  const uint32_t* limbw = reinterpret_cast<const uint32_t*>(sm + (size_t)3 * nt * 16);
  const int tail_v = (!FULL && a.F < nv * EPV) ? nv - 1 : -1;

  RowSum res{0, 0, 0, 0u, 0.f, 0.f};
  long long rrow = -1;
  int nres = 0;

  for (long long k = 0; k < ntl; ++k) {
    const int s = (int)(k % p.S);
    const uint32_t ph = (uint32_t)((k / p.S) & 1);
    if (!mbar_wait_bounded(&full[s], ph)) {
      if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
      return;
    }
    const unsigned char* st = sm + p.stages_off + (size_t)s * p.stage_bytes;
    const StageMeta* mp = reinterpret_cast<const StageMeta*>(st + p.meta_off);
    const int nr = mp->nr;
    const long long row0 = mp->row0;
    const int in_smem = mp->in_smem;
    const long long ebase = mp->ebase;
    const long long* sp = reinterpret_cast<const long long*>(st + p.ptr_off);
    const uint16_t* scol = reinterpret_cast<const uint16_t*>(st + p.col_off);
    const uint16_t* sadd = reinterpret_cast<const uint16_t*>(st + p.add_off);
    for (int r0 = warp * RPW; r0 < nr; r0 += NCW * RPW) {
      if (nres + RPW > 32) {
        if (lane < nres) finish_row<DT>(a, hb, inv_scale, maxabs, rrow, res);
        nres = 0;
      }
      const int r = r0 + grp;             // this lane group's row
      const bool valid = r < nr;
      const unsigned char* rp = st + (size_t)(valid ? r : 0) * a.ld_bytes;
      RowSum mine{0, 0, 0, 0u, 0.f, 0.f};
      if (DT == NB_U8) {
        // the row's staged overflow range (stage-relative), read before the
        // dense part so that its latency hides behind the dp4a chains
        int e0 = 0, e1 = 0;
        if (OVF && valid && in_smem) {
          e0 = (int)(sp[r] - ebase);
          e1 = (int)(sp[r + 1] - ebase);
        }
        // two independent sets of the four dp4a chains (even / odd vectors)
        int c0[2] = {0, 0}, c1[2] = {0, 0}, c2[2] = {0, 0};
        uint32_t ct[2] = {0u, 0u};
#pragma unroll
        for (int kv = 0; kv < KV; ++kv) {
          const int v = li + LPR * kv, e = kv & 1;
          if (FULL || v < nv) {
            uint4 x = *reinterpret_cast<const uint4*>(rp + (size_t)v * 16);
            if (!FULL && v == tail_v) {   // zero the bytes past F (masks made here: rare)
              const int keep = a.F - 16 * (nv - 1);   // valid bytes of the last vector
              x.x &= u8_keep_mask(keep);
              x.y &= u8_keep_mask(keep - 4);
              x.z &= u8_keep_mask(keep - 8);
              x.w &= u8_keep_mask(keep - 12);
            }
            c0[e] = dp4a_us(x.x, q0[kv].x, c0[e]);
            c1[e] = dp4a_us(x.x, q1[kv].x, c1[e]);
            c2[e] = dp4a_us(x.x, q2[kv].x, c2[e]);
            ct[e] = dp4a_uu(x.x, 0x01010101u, ct[e]);
            c0[e] = dp4a_us(x.y, q0[kv].y, c0[e]);
            c1[e] = dp4a_us(x.y, q1[kv].y, c1[e]);
            c2[e] = dp4a_us(x.y, q2[kv].y, c2[e]);
            ct[e] = dp4a_uu(x.y, 0x01010101u, ct[e]);
            c0[e] = dp4a_us(x.z, q0[kv].z, c0[e]);
            c1[e] = dp4a_us(x.z, q1[kv].z, c1[e]);
            c2[e] = dp4a_us(x.z, q2[kv].z, c2[e]);
            ct[e] = dp4a_uu(x.z, 0x01010101u, ct[e]);
            c0[e] = dp4a_us(x.w, q0[kv].w, c0[e]);
            c1[e] = dp4a_us(x.w, q1[kv].w, c1[e]);
            c2[e] = dp4a_us(x.w, q2[kv].w, c2[e]);
            ct[e] = dp4a_uu(x.w, 0x01010101u, ct[e]);
          }
        }
        int a0 = c0[0] + c0[1], a1 = c1[0] + c1[1], a2 = c2[0] + c2[1];
        uint32_t tt = ct[0] + ct[1];
        if (OVF && valid) {
          if (in_smem) {
            for (int e = e0 + li; e < e1; e += LPR) {
              const uint32_t col = scol[e];
              const int add = sadd[e];
              if (col < (uint32_t)a.F) {
                const uint32_t w = limbw[col];
                a0 += add * (int)(int8_t)(w & 255u);
                a1 += add * (int)(int8_t)((w >> 8) & 255u);
                a2 += add * (int)(int8_t)((w >> 16) & 255u);
                tt += (uint32_t)add;
              } else {
                atomicOr(a.status, ST_OVF_RANGE);
              }
            }
          } else {
            const long long k0 = sp[r], k1 = sp[r + 1];
            for (long long e = k0 + li; e < k1; e += LPR) {
              const uint32_t col = a.ovf_col[e];
              const int add = a.ovf_add[e];
              if (col < (uint32_t)a.F) {
                const uint32_t w = limbw[col];
                a0 += add * (int)(int8_t)(w & 255u);
                a1 += add * (int)(int8_t)((w >> 8) & 255u);
                a2 += add * (int)(int8_t)((w >> 16) & 255u);
                tt += (uint32_t)add;
              } else {
                atomicOr(a.status, ST_OVF_RANGE);
              }
            }
          }
        }
        // the group's sums end up in its four lane quarters (see sum4_transposed)
        mine.a0 = sum4_transposed<LPR>(a0, a1, a2, (int)tt, li);
      } else if (DT == NB_FP8E4M3) {
        // the row's scale selects the magic pair of the count check
        const uint32_t m2 =
            fp8_magic((a.row_exp && valid) ? (int)a.row_exp[row0 + r] : 0);
        int a0 = 0, a1 = 0, a2 = 0;
        uint32_t tt = 0u;
        Fp8Check chk;
#pragma unroll
        for (int kv = 0; kv < KV; ++kv) {
          const int v = li + LPR * kv;
          if (FULL || v < nv) {
            uint4 x = *reinterpret_cast<const uint4*>(rp + (size_t)v * 16);
            if (!FULL && v == tail_v) {   // E4M3 zero past F
              const int keep = a.F - 16 * (nv - 1);
              x.x &= u8_keep_mask(keep);
              x.y &= u8_keep_mask(keep - 4);
              x.z &= u8_keep_mask(keep - 8);
              x.w &= u8_keep_mask(keep - 12);
            }
            fp8_vector_limbs_biased(x, q0[kv], q1[kv], q2[kv], m2, a0, a1, a2, tt, chk);
          }
        }
        // remove the bias M of every value (exact integer arithmetic)
        const int mh = (int)(m2 & 0xFFFFu);
        a0 -= mh * fs0;
        a1 -= mh * fs1;
        a2 -= mh * fs2;
        tt -= (uint32_t)(mh * fnv);
        mine.a0 = sum4_transposed<LPR>(a0, a1, a2, (int)fp8_lane_total(tt, chk, m2), li);
      } else {
        float acc[4] = {0.f, 0.f, 0.f, 0.f}, tf = 0.f;
#pragma unroll
        for (int kv = 0; kv < KV; ++kv) {
          const int v = li + LPR * kv;
          if (FULL || v < nv) {
            const uint4 x = *reinterpret_cast<const uint4*>(rp + (size_t)v * 16);
            float val[EPV];
            Dec::run(x, val);
            if (!FULL && v == tail_v) {
#pragma unroll
              for (int e = 0; e < EPV; ++e)
                if (v * EPV + e >= a.F) val[e] = 0.f;
            }
#pragma unroll
            for (int q = 0; q < QPV; ++q) {
              acc[0] = fmaf(val[4 * q + 0], wq[kv][q].x, acc[0]);
              acc[1] = fmaf(val[4 * q + 1], wq[kv][q].y, acc[1]);
              acc[2] = fmaf(val[4 * q + 2], wq[kv][q].z, acc[2]);
              acc[3] = fmaf(val[4 * q + 3], wq[kv][q].w, acc[3]);
              tf += fabsf(val[4 * q + 0]) + fabsf(val[4 * q + 1]) + fabsf(val[4 * q + 2]) +
                    fabsf(val[4 * q + 3]);
            }
          }
        }
        mine.s = group_sum<LPR>((acc[0] + acc[1]) + (acc[2] + acc[3]));
        mine.tf = group_sum<LPR>(tf);
      }
      // lane nres + g takes row r0 + g of this pass from lane g * LPR
      const int src = (lane - nres) * LPR;
      const bool take = lane >= nres && lane < nres + RPW && r0 + (lane - nres) < nr;
      const int sl = take ? src : 0;
      RowSum got;
      if (LIMBS) {
        got.a0 = __shfl_sync(0xFFFFFFFFu, mine.a0, sl);
        got.a1 = __shfl_sync(0xFFFFFFFFu, mine.a0, sl + LPR / 4);
        got.a2 = __shfl_sync(0xFFFFFFFFu, mine.a0, sl + LPR / 2);
        got.t = (uint32_t)__shfl_sync(0xFFFFFFFFu, mine.a0, sl + 3 * LPR / 4);
        got.s = 0.f;
        got.tf = 0.f;
      } else {
        got = RowSum{0, 0, 0, 0u, __shfl_sync(0xFFFFFFFFu, mine.s, sl),
                     __shfl_sync(0xFFFFFFFFu, mine.tf, sl)};
      }
      if (take) {
        res = got;
        rrow = row0 + r0 + (lane - nres);
      }
      nres += (nr - r0) < RPW ? (nr - r0) : RPW;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
    if (nres + RPW > 32) {
      if (lane < nres) finish_row<DT>(a, hb, inv_scale, maxabs, rrow, res);
      nres = 0;
    }
  }
  if (lane < nres) finish_row<DT>(a, hb, inv_scale, maxabs, rrow, res);
}

// ---------------------------------------------------------------------------
// launcher: NB_EUNSUPPORTED when the row does not fit (the caller then uses
// the register-streaming kernel)
// ---------------------------------------------------------------------------
template <int DT, int KV, int RPW, int NCW, bool FULL, bool OVF>
static nb_status run_pipe(const S2Args& a, const PipeArgs& p, int smem, cudaStream_t st) {
  auto kern = k_score2_pipe<DT, KV, RPW, NCW, FULL, OVF>;
  if (smem > kSmemOptIn)   // per device and function: set at every launch
    NB_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                "cudaFuncSetAttribute(pipe)");
  int occ = 0;
  NB_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, (NCW + 1) * 32, smem),
              "occupancy(pipe)");
  if (occ < 1) {
    set_error("pipelined scorer does not fit on an SM");
    return NB_EUNSUPPORTED;
  }
  long long blocks = (long long)num_sms() * occ;
  if (blocks > p.tiles) blocks = p.tiles;
  count_launch();
  kern<<<(unsigned)blocks, (NCW + 1) * 32, smem, st>>>(a, p);
  NB_TRY_CUDA(cudaGetLastError(), "k_score2_pipe launch");
  return NB_OK;
}

// Shapes: rows per warp pass (RPW = 1 or 2, lanes per row 32 / RPW), vectors
// per lane (KV) and consumer warps (NCW).  Eight consumer warps and two blocks
// per SM when the Delta slice fits the 96-register budget, or for u8 rows of
// 64 vectors at two rows per pass when the stages leave room for two blocks;
// else twelve consumers and one block.
nb_status launch_score2_pipe(const S2Args& a, nb_dtype dt, int stages, int rows_per_stage,
                             int rows_per_warp, int stage_entries, cudaStream_t st) {
  const int rpw = rows_per_warp == 2 ? 2 : 1;
  const int lpr = 32 / rpw;
  const int kv = (a.nvec_row + lpr - 1) / lpr;
  const int kv_max = dt == NB_F32 ? 8 : 4;
  if (kv < 1 || kv > kv_max || a.ld_bytes > 8192) return NB_EUNSUPPORTED;
  // u8 rows with an overflow list also stage the packed limb words (4 bytes a
  // feature) after the three limb planes
  const bool ovf = dt == NB_U8 && a.ovf_ptr != nullptr;
  const uint32_t tab_all = ovf ? 7u * (uint32_t)(a.nvec_tab * 16) : a.table_bytes;
  // Stage plan for `ncw` consumer warps: rows per stage in whole passes of
  // ncw * rpw rows, 16-48 KB; stages filling ~100 KB (eight consumers, two
  // blocks per SM) or ~180 KB (twelve, one block) unless given.
  auto plan = [&](int ncw, PipeArgs& p) {
    const int pass_rows = ncw * rpw;
    long long per = 32768 / ((long long)pass_rows * a.ld_bytes);
    int rs = rows_per_stage > 0 ? rows_per_stage : pass_rows * (int)(per > 0 ? per : 1);
    if (rs > kMaxStageRows) rs = kMaxStageRows;
    if (rs < 1) rs = 1;
    const unsigned budget = ncw == 8 ? 100u * 1024u : 180u * 1024u;   // per block
    int S = stages;
    if (S <= 0) {
      PipeArgs q{};
      pipe_layout(q, rs, 1, a.ld_bytes, stage_entries != 0, false, tab_all, a.n);
      S = q.stages_off + q.stage_bytes > budget ? 2 : (int)((budget - q.stages_off) / q.stage_bytes);
    }
    S = S < 2 ? 2 : (S > kMaxStages ? kMaxStages : S);
    pipe_layout(p, rs, S, a.ld_bytes, stage_entries != 0, false, tab_all, a.n);
    return (int)(p.stages_off + (uint32_t)p.S * p.stage_bytes);
  };
  int ncw = (rpw == 1 && (dt == NB_F32 ? kv <= 8 : kv <= 2)) ? 8 : 12;
  PipeArgs p{};
  int smem = 0;
  // two u8 rows per pass: eight consumer warps whenever the stages leave room
  // for two blocks (18 warps) per SM
  if (dt == NB_U8 && rpw == 2 && kv == 4) {
    smem = plan(8, p);
    if (smem <= 112 * 1024) ncw = 8;
  }
  if (ncw == 12 || smem == 0) smem = plan(ncw, p);
  if (smem > 220 * 1024) return NB_EUNSUPPORTED;
  // rounding depth of the FP32 paths: serial FMAs per accumulator, the four
  // accumulators, the lane-group butterfly, the weight and final roundings
  S2Args ak = a;
  ak.k_base = kv * ((16 / elem_size(dt)) / 4) + 2 + (rpw == 2 ? 4 : 5) + 2;
  // rows that fill every lane's vectors exactly take the branch-free kernel
  const bool full = a.nvec_row == kv * lpr && (a.F * elem_size(dt)) % 16 == 0;
#define NB_PIPE_CASE(D, K, R, N)                                                            \
  if (dt == D && kv == K && rpw == R && ncw == N) {                                         \
    if (D == NB_U8 && ovf)                                                                  \
      return full ? run_pipe<D, K, R, N, true, D == NB_U8>(ak, p, smem, st)                 \
                  : run_pipe<D, K, R, N, false, D == NB_U8>(ak, p, smem, st);               \
    return full ? run_pipe<D, K, R, N, true, false>(ak, p, smem, st)                        \
                : run_pipe<D, K, R, N, false, false>(ak, p, smem, st);                      \
  }
#define NB_PIPE_DT(D)                                                                        \
  NB_PIPE_CASE(D, 1, 1, 8) NB_PIPE_CASE(D, 2, 1, 8) NB_PIPE_CASE(D, 3, 1, 12)                 \
  NB_PIPE_CASE(D, 4, 1, 12) NB_PIPE_CASE(D, 1, 2, 12) NB_PIPE_CASE(D, 2, 2, 12)               \
  NB_PIPE_CASE(D, 3, 2, 12) NB_PIPE_CASE(D, 4, 2, 12)
  NB_PIPE_DT(NB_U8)
  NB_PIPE_CASE(NB_U8, 4, 2, 8)
  NB_PIPE_DT(NB_FP8E4M3)
  NB_PIPE_DT(NB_U16)
  NB_PIPE_DT(NB_BF16)
  NB_PIPE_CASE(NB_F32, 1, 1, 8) NB_PIPE_CASE(NB_F32, 2, 1, 8) NB_PIPE_CASE(NB_F32, 3, 1, 8)
  NB_PIPE_CASE(NB_F32, 4, 1, 8) NB_PIPE_CASE(NB_F32, 5, 1, 8) NB_PIPE_CASE(NB_F32, 6, 1, 8)
  NB_PIPE_CASE(NB_F32, 7, 1, 8) NB_PIPE_CASE(NB_F32, 8, 1, 8)
  NB_PIPE_CASE(NB_F32, 1, 2, 12) NB_PIPE_CASE(NB_F32, 2, 2, 12) NB_PIPE_CASE(NB_F32, 3, 2, 12)
  NB_PIPE_CASE(NB_F32, 4, 2, 12)
#undef NB_PIPE_DT
#undef NB_PIPE_CASE
  return NB_EUNSUPPORTED;
}

}  // namespace nbg
