// Two-class multinomial scoring (Sec. 4 posterior and decision rule).
//
// For C = 2 the decision needs only the log-odds
//     d = s_1 - s_0 = b + sum_j x_j Delta_j,
//     b = log pi_1 - log pi_0,  Delta_j = log theta_1j - log theta_0j,
// and the outputs follow from d alone: label = [d > 0] (a tie, d = 0, goes to
// benign), margin = |d|, log P(1|x) = -softplus(-d), log P(0|x) = -softplus(d).
// Each file is read once from HBM with 16-byte streaming loads; the Delta
// table is staged into shared memory by bulk copies (TMA) behind an mbarrier.
//
// Two inner products:
//   * u8 storage: Delta is held as a 22-bit fixed-point integer split into
//     three signed 8-bit limbs; dp4a accumulates x * limb exactly in int32, so
//     the only error is the quantisation of Delta (<= 2^-S / 2 per count).
//     FP8 E4M3 storage takes the same limbs: its values become exact integer
//     counts (row scale 2^0 or 2^1, checked per value, see fp8_count_pairs)
//     in 16-bit pairs, accumulated with dp2a.
//   * f32 / u16 / bf16 storage: decode to FP32 and FMA against the FP32 Delta
//     table, four accumulators per row per lane.
// Every row also gets a rigorous bound tau on |d_gpu - d_exact|; rows whose
// sign (or whose log posteriors to 1e-5) the bound cannot guarantee are marked
// for the FP64 recheck.
#include <cuda_fp16.h>

#include "score2.cuh"

namespace nbg {

// ---------------------------------------------------------------------------
// u8 storage, fixed-point Delta, exact integer accumulation
// ---------------------------------------------------------------------------
template <int DT, int LPR, int R>
__global__ void __launch_bounds__(256) k_score2_u8(const S2Args a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t bar;
  if (!stage_table(smem_raw, a.table, a.table_bytes, &bar, a.status, ST_TIMEOUT)) return;
  const uint4* tab = reinterpret_cast<const uint4*>(smem_raw);
  const C2Header h = *a.hdr;

  constexpr int SUBS = 32 / LPR;
  constexpr int RPW = SUBS * R;
  const int lane = threadIdx.x & 31;
  const int sub = lane / LPR, li = lane % LPR;
  const int nv = a.nvec_row, nt = a.nvec_tab;
  const int64_t ntiles = (a.n + RPW - 1) / RPW;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);

  // byte masks of the last (partial) vector
  const int keep = a.F - 16 * (nv - 1);
  uint32_t tm[4];
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    int vb = keep - 4 * w;
    vb = vb < 0 ? 0 : (vb > 4 ? 4 : vb);
    tm[w] = vb >= 4 ? 0xFFFFFFFFu : ((1u << (8 * vb)) - 1u);
  }
  const bool has_tail = keep < 16;

  // rows this lane marked for the FP64 recheck, added up once per warp at the
  // end (faster here than an atomic per marked row; the FP kernel below keeps
  // the atomic, which holds no register through its loop)
  unsigned marks = 0;
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < ntiles;
       t += nwarps) {
    const int64_t row0 = t * RPW + (int64_t)sub * R;
    int acc0[R], acc1[R], acc2[R];
    uint32_t tot[R], m2[R];
    Fp8Check chk[R];
    const char* rp[R];
    bool ok[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      acc0[r] = acc1[r] = acc2[r] = 0;
      tot[r] = 0;
      ok[r] = row0 + r < a.n;
      rp[r] = a.X + (ok[r] ? row0 + r : 0) * a.ld_bytes;
      m2[r] = DT == NB_FP8E4M3 ? fp8_magic((a.row_exp && ok[r]) ? (int)a.row_exp[row0 + r] : 0)
                               : 0u;
    }
#pragma unroll 2
    for (int v = li; v < nv; v += LPR) {
      const uint4 q0 = tab[v], q1 = tab[nt + v], q2 = tab[2 * nt + v];
      uint4 x[R];
#pragma unroll
      for (int r = 0; r < R; ++r)
        x[r] = ok[r] ? ld_stream16(rp[r] + (int64_t)v * 16) : make_uint4(0, 0, 0, 0);
      if (has_tail && v == nv - 1) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          x[r].x &= tm[0];
          x[r].y &= tm[1];
          x[r].z &= tm[2];
          x[r].w &= tm[3];
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (DT == NB_FP8E4M3) {
          fp8_vector_limbs(x[r], q0, q1, q2, m2[r], acc0[r], acc1[r], acc2[r], tot[r], chk[r]);
          continue;
        }
        acc0[r] = dp4a_us(x[r].x, q0.x, acc0[r]);
        acc0[r] = dp4a_us(x[r].y, q0.y, acc0[r]);
        acc0[r] = dp4a_us(x[r].z, q0.z, acc0[r]);
        acc0[r] = dp4a_us(x[r].w, q0.w, acc0[r]);
        acc1[r] = dp4a_us(x[r].x, q1.x, acc1[r]);
        acc1[r] = dp4a_us(x[r].y, q1.y, acc1[r]);
        acc1[r] = dp4a_us(x[r].z, q1.z, acc1[r]);
        acc1[r] = dp4a_us(x[r].w, q1.w, acc1[r]);
        acc2[r] = dp4a_us(x[r].x, q2.x, acc2[r]);
        acc2[r] = dp4a_us(x[r].y, q2.y, acc2[r]);
        acc2[r] = dp4a_us(x[r].z, q2.z, acc2[r]);
        acc2[r] = dp4a_us(x[r].w, q2.w, acc2[r]);
        tot[r] = dp4a_uu(x[r].x, 0x01010101u, tot[r]);
        tot[r] = dp4a_uu(x[r].y, 0x01010101u, tot[r]);
        tot[r] = dp4a_uu(x[r].z, 0x01010101u, tot[r]);
        tot[r] = dp4a_uu(x[r].w, 0x01010101u, tot[r]);
      }
    }
    long long D[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      D[r] = ((long long)acc2[r] << 16) + ((long long)acc1[r] << 8) + (long long)acc0[r];
      if (DT == NB_FP8E4M3) tot[r] = fp8_lane_total(tot[r], chk[r], m2[r]);
    }
    if (DT == NB_U8 && a.ovf_ptr) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!ok[r]) continue;
        const int64_t k0 = a.ovf_ptr[row0 + r], k1 = a.ovf_ptr[row0 + r + 1];
        for (int64_t k = k0 + li; k < k1; k += LPR) {
          const uint32_t col = a.ovf_col[k], add = a.ovf_add[k];
          if (col < (uint32_t)a.F) {
            D[r] += (long long)add * (long long)a.delta_q[col];
            tot[r] += add;
          } else {
            atomicOr(a.status, ST_OVF_RANGE);
          }
        }
      }
    }
#pragma unroll
    for (int off = LPR / 2; off > 0; off >>= 1) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        D[r] += __shfl_xor_sync(0xFFFFFFFFu, D[r], off);
        tot[r] += __shfl_xor_sync(0xFFFFFFFFu, tot[r], off);
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!ok[r] || (r % LPR) != li) continue;
      const float Dsum = (float)D[r] * h.inv_scale;
      const float d = Dsum + h.b;
      // quantisation of Delta + int64->f32 and final-add roundings + FP64 slack;
      // +inf past the int32 range of the limb sums
      const float tau = c2_tau_u8((float)tot[r], Dsum, h.b, h.inv_scale, h.maxabs);
      marks += c2_store(a.label, a.margin, a.logpost, a.want_lp, a.recheck, row0 + r, d, tau);
    }
  }
  c2_flush_marks(a, marks);
}

template <int DT, int LPR, int R>
__global__ void __launch_bounds__(256) k_score2_fp(const S2Args a) {
  using Dec = Decode<DT>;
  constexpr int EPV = Dec::EPV, QPV = EPV / 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t bar;
  if (!stage_table(smem_raw, a.table, a.table_bytes, &bar, a.status, ST_TIMEOUT)) return;
  const float4* tab = reinterpret_cast<const float4*>(smem_raw);
  const C2Header h = *a.hdr;

  constexpr int SUBS = 32 / LPR;
  constexpr int RPW = SUBS * R;
  const int lane = threadIdx.x & 31;
  const int sub = lane / LPR, li = lane % LPR;
  const int nv = a.nvec_row, nt = a.nvec_tab;
  const int64_t ntiles = (a.n + RPW - 1) / RPW;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const bool has_tail = a.F < nv * EPV;

  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < ntiles;
       t += nwarps) {
    const int64_t row0 = t * RPW + (int64_t)sub * R;
    float acc[R][4], tot[R];
    const char* rp[R];
    bool ok[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      acc[r][0] = acc[r][1] = acc[r][2] = acc[r][3] = 0.f;
      tot[r] = 0.f;
      ok[r] = row0 + r < a.n;
      rp[r] = a.X + (ok[r] ? row0 + r : 0) * a.ld_bytes;
    }
#pragma unroll 2
    for (int v = li; v < nv; v += LPR) {
      float4 wq[QPV];
#pragma unroll
      for (int q = 0; q < QPV; ++q) wq[q] = tab[q * nt + v];
      uint4 x[R];
#pragma unroll
      for (int r = 0; r < R; ++r)
        x[r] = ok[r] ? ld_stream16(rp[r] + (int64_t)v * 16) : make_uint4(0, 0, 0, 0);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float val[EPV];
        Dec::run(x[r], val);
        if (has_tail && v == nv - 1) {
#pragma unroll
          for (int e = 0; e < EPV; ++e)
            if (v * EPV + e >= a.F) val[e] = 0.f;
        }
#pragma unroll
        for (int q = 0; q < QPV; ++q) {
          acc[r][0] = fmaf(val[4 * q + 0], wq[q].x, acc[r][0]);
          acc[r][1] = fmaf(val[4 * q + 1], wq[q].y, acc[r][1]);
          acc[r][2] = fmaf(val[4 * q + 2], wq[q].z, acc[r][2]);
          acc[r][3] = fmaf(val[4 * q + 3], wq[q].w, acc[r][3]);
          tot[r] += fabsf(val[4 * q + 0]) + fabsf(val[4 * q + 1]) + fabsf(val[4 * q + 2]) +
                    fabsf(val[4 * q + 3]);
        }
      }
    }
    float s[R];
    int nov[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      s[r] = (acc[r][0] + acc[r][1]) + (acc[r][2] + acc[r][3]);
      nov[r] = 0;
    }
    if (DT == NB_U8 && a.ovf_ptr) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!ok[r]) continue;
        const int64_t k0 = a.ovf_ptr[row0 + r], k1 = a.ovf_ptr[row0 + r + 1];
        for (int64_t k = k0 + li; k < k1; k += LPR) {
          const uint32_t col = a.ovf_col[k];
          const float add = (float)a.ovf_add[k];
          if (col < (uint32_t)a.F) {
            s[r] = fmaf(add, a.delta[col], s[r]);
            tot[r] += add;
            ++nov[r];
          } else {
            atomicOr(a.status, ST_OVF_RANGE);
          }
        }
      }
    }
#pragma unroll
    for (int off = LPR / 2; off > 0; off >>= 1) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        s[r] += __shfl_xor_sync(0xFFFFFFFFu, s[r], off);
        tot[r] += __shfl_xor_sync(0xFFFFFFFFu, tot[r], off);
        nov[r] = max(nov[r], __shfl_xor_sync(0xFFFFFFFFu, nov[r], off));
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!ok[r] || (r % LPR) != li) continue;
      float scale = 1.f;
      if (DT == NB_FP8E4M3 && a.row_exp) scale = exp2f((float)a.row_exp[row0 + r]);
      const float sum = s[r] * scale;
      const float d = sum + h.b;
      const float k = (float)(a.k_base + nov[r]);
      const float gam = k * 5.9604645e-8f / (1.f - k * 5.9604645e-8f);
      const float A = tot[r] * scale * h.maxabs * 1.001f;
      const float tau = gam * (A + fabsf(h.b)) * 1.01f + 1e-12f * (A + fabsf(h.b)) + 1e-30f;
      // marked rows are rare: one atomic each, no state carried through the loop
      if (c2_store(a.label, a.margin, a.logpost, a.want_lp, a.recheck, row0 + r, d, tau) && a.marks)
        atomicAdd(a.marks, 1ull);
    }
  }
}

// ---------------------------------------------------------------------------
// launcher
// ---------------------------------------------------------------------------
template <typename K>
static nb_status launch_persistent(K kernel, int smem, int64_t ntiles_warp, const S2Args& a,
                                   cudaStream_t st) {
  static thread_local const void* last_k = nullptr;
  static thread_local int last_smem = -1, last_occ = 0;
  if (smem > kSmemOptIn) {
    NB_TRY_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                "cudaFuncSetAttribute");
  }
  int occ;
  if (last_k == (const void*)kernel && last_smem == smem) {
    occ = last_occ;
  } else {
    NB_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 256, smem),
                "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    last_k = (const void*)kernel;
    last_smem = smem;
    last_occ = occ;
  }
  if (occ < 1) occ = 1;
  int64_t blocks = (ntiles_warp + 7) / 8;
  const int64_t cap = (int64_t)num_sms() * occ;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  count_launch();
  kernel<<<(unsigned)blocks, 256, smem, st>>>(a);
  NB_TRY_CUDA(cudaGetLastError(), "score2 launch");
  return NB_OK;
}

static int pick_lpr(int nvec_row) {
  int lpr = 1;
  while (lpr < 32 && lpr * 2 < nvec_row) lpr *= 2;
  return lpr;
}

// u8 and FP8 rows: about eight 16-byte vectors per lane and at least two lanes
// per row (measured, 4M files: u8 F = 256 at 89% of HBM against 61% with two
// vectors per lane, F = 64 at 65% against 61%, F = 4096 unchanged at 98%; FP8
// F = 256 at 54% against 36%, F = 1024 at 48% against 37%)
static int pick_lpr_u8(int nvec_row) {
  int lpr = 2;
  while (lpr < 32 && lpr * 8 < nvec_row) lpr *= 2;
  return lpr;
}

static int ilog2(int v) {
  int k = 0;
  while ((1 << k) < v) ++k;
  return k;
}

template <int LPR>
static nb_status dispatch_dt(nb_dtype dt, S2Args& a, int smem, cudaStream_t st) {
  constexpr int R = 4;
  const int64_t rpw = (32 / LPR) * R;
  const int64_t ntiles = (a.n + rpw - 1) / rpw;
  switch (dt) {
    case NB_U8:
      if (a.nvec_row < 16) {   // short rows: two rows per lane group, twice the warps per SM
        const int64_t rpw2 = (32 / LPR) * 2;
        return launch_persistent(k_score2_u8<NB_U8, LPR, 2>, smem, (a.n + rpw2 - 1) / rpw2, a,
                                 st);
      }
      return launch_persistent(k_score2_u8<NB_U8, LPR, R>, smem, ntiles, a, st);
    case NB_F32:
      return launch_persistent(k_score2_fp<NB_F32, LPR, R>, smem, ntiles, a, st);
    case NB_U16:
      return launch_persistent(k_score2_fp<NB_U16, LPR, R>, smem, ntiles, a, st);
    case NB_BF16:
      return launch_persistent(k_score2_fp<NB_BF16, LPR, R>, smem, ntiles, a, st);
    case NB_FP8E4M3:
      if (a.nvec_row < 16) {
        const int64_t rpw2 = (32 / LPR) * 2;
        return launch_persistent(k_score2_u8<NB_FP8E4M3, LPR, 2>, smem, (a.n + rpw2 - 1) / rpw2,
                                 a, st);
      }
      return launch_persistent(k_score2_u8<NB_FP8E4M3, LPR, R>, smem, ntiles, a, st);
  }
  set_error("unknown dtype");
  return NB_EINVAL;
}

nb_status launch_score2(const nb_model* m, const void* X, nb_dtype dt, int64_t n, int64_t ld,
                        const nb_aux* aux, const ScoreOut& o, cudaStream_t st) {
  const int es = elem_size(dt);
  S2Args a{};
  a.X = static_cast<const char*>(X);
  a.ld_bytes = ld * es;
  a.n = n;
  a.F = m->F;
  a.nvec_row = (m->F * es + 15) / 16;
  a.hdr = m->d.c2;
  a.delta_q = m->d.delta_q;
  a.delta = m->d.delta;
  a.ovf_ptr = aux ? aux->ovf_ptr : nullptr;
  a.ovf_col = aux ? aux->ovf_col : nullptr;
  a.ovf_add = aux ? aux->ovf_add : nullptr;
  a.row_exp = aux ? aux->row_exp : nullptr;
  a.label = o.label;
  a.margin = o.margin;
  a.logpost = o.logpost;
  a.want_lp = o.want_lp;
  a.recheck = o.recheck;
  a.marks = o.counted ? reinterpret_cast<unsigned long long*>(o.n_rechecked) : nullptr;
  a.status = m->d.sstatus;
  int smem;
  if (dt == NB_U8 || dt == NB_FP8E4M3) {   // fixed-point limbs, exact sums
    a.nvec_tab = m->nvec8;
    a.table = m->d.limbs;
    smem = 3 * m->nvec8 * 16;
  } else {
    const int epv = 16 / es;
    a.nvec_tab = m->F_pad / epv;
    a.table = m->d.il[es == 4 ? 0 : (es == 2 ? 1 : 2)];
    smem = m->F_pad * 4;
  }
  a.table_bytes = (uint32_t)smem;
  if (n == 0) return NB_OK;
  const nb_tile_config& cfg = m->tile;
  if (cfg.variant != NB_VARIANT_REGISTER) {
    // overflow slices are staged by bulk copies only from 16-byte aligned arrays
    S2Args ap = a;
    const int epv = 16 / es;
    ap.k_base = ((a.nvec_row + 31) / 32) * (epv / 4) + 2 + 5 + 2;
    const bool side_ok = !a.ovf_ptr || ((reinterpret_cast<uintptr_t>(a.ovf_col) & 15) == 0 &&
                                        (reinterpret_cast<uintptr_t>(a.ovf_add) & 15) == 0);
    const nb_status s =
        launch_score2_pipe(ap, dt, cfg.stages, cfg.rows_per_stage, cfg.rows_per_warp,
                           side_ok ? 1 : 0, st);
    if (s != NB_EUNSUPPORTED || cfg.variant == NB_VARIANT_PIPELINED) return s;
  }
  const int lpr = (dt == NB_U8 || dt == NB_FP8E4M3) ? pick_lpr_u8(a.nvec_row)
                                                    : pick_lpr(a.nvec_row);
  {
    const int epv = 16 / es;
    const int per_lane = (a.nvec_row + lpr - 1) / lpr;
    a.k_base = per_lane * (epv / 4) + 2 + ilog2(lpr) + 2;
  }
  switch (lpr) {
    case 1: return dispatch_dt<1>(dt, a, smem, st);
    case 2: return dispatch_dt<2>(dt, a, smem, st);
    case 4: return dispatch_dt<4>(dt, a, smem, st);
    case 8: return dispatch_dt<8>(dt, a, smem, st);
    case 16: return dispatch_dt<16>(dt, a, smem, st);
    default: return dispatch_dt<32>(dt, a, smem, st);
  }
}

}  // namespace nbg
