// Segmented persistent two-class scorer: one launch scores a whole batch of
// file groups of uneven size (1 .. 50,000 files and more), several resident
// models, under a captured CUDA graph (the paper's groups, Sec. 3 / Sec. 4,
// classified with their group's model).
//
// The launch reads its work list from device memory (header + one descriptor
// per group, see seg.cuh), so a graph captured once serves every batch.  The
// persistent grid splits the list's tiles (RS rows of one group) into
// contiguous ranges per block; the producer warp walks the groups of its range
// and streams each tile's rows and overflow slice into shared-memory stages
// (pipe.cuh).  Every model's Delta table is staged once per block; a consumer
// warp reloads its register slice when the stage's group uses another model.
// Finished rows keep their group and are finalised 32 at a time.  The
// per-row arithmetic is the single-group kernel's (32 lanes per row), so a
// group gives the same bits alone and inside any batch.
#include "pipe.cuh"
#include "score2.cuh"
#include "seg.cuh"

namespace nbg {


// tiles of a block's range, walking the group list
struct SegSrc {
  const SegGroup* groups;
  int n_groups;
  long long t0;
  int RS;
  int g;
  TileInfo gi;      // fields of group g
  long long gt0;    // its first tile
  __device__ __forceinline__ void load(int gg) {
    const SegGroup& G = groups[gg];
    g = gg;
    gt0 = G.tile0;
    gi.X = G.X;
    gi.ld_bytes = G.ld_bytes;
    gi.group = gg;
    gi.ovf_ptr = G.ovf_ptr;
    gi.ovf_col = G.ovf_col;
    gi.ovf_add = G.ovf_add;
    gi.E = G.ovf_ptr ? G.ovf_ptr[G.n] : 0;
    gi.y = nullptr;
    gi.sizes = nullptr;
    gi.row0 = G.n;   // holds n until a tile is cut
  }
  __device__ __forceinline__ void init() {
    const SegGroup* gr = groups;
    load(seg_find(n_groups, t0, [gr](int i) { return gr[i].tile0; }));
  }
  __device__ __forceinline__ TileInfo tile(long long k) {
    const long long t = t0 + k;
    while (g + 1 < n_groups && groups[g + 1].tile0 <= t) load(g + 1);
    TileInfo r = gi;
    const long long n = gi.row0;
    r.row0 = (t - gt0) * RS;
    r.nr = (int)min((long long)RS, n - r.row0);
    return r;
  }
};

template <int DT, int KV, int RPW, int NCW>
__global__ void __launch_bounds__((NCW + 1) * 32, NCW == 8 ? 2 : 1)
    k_score2_seg(const SegArgs a, PipeArgs p) {
  constexpr int LPR = 32 / RPW;   // lanes per row: RPW rows per warp pass
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint64_t full[kMaxStages], empty[kMaxStages], tabbar;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / LPR, li = lane % LPR;
  const int n_groups = a.hdr->n_groups;
  const long long tiles = a.hdr->tiles;
  const long long t0 = tiles * blockIdx.x / gridDim.x;
  const long long t1 = tiles * (blockIdx.x + 1) / gridDim.x;
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
    pipe_stage_tables(sm, a.tables, a.n_models, a.table_bytes, a.table_stride, &tabbar);
    if (ntl > 0) {
      SegSrc src{a.groups, n_groups, t0, p.RS, 0, TileInfo{}, 0};
      src.init();
      pipe_produce_tiles(src, p, sm, full, empty, ntl, a.status);
    }
    return;
  }

  // ------------------------------------------------------------- consumers
  using Dec = Decode<DT>;
  constexpr int EPV = Dec::EPV, QPV = EPV / 4;
  if (!mbar_wait_bounded(&tabbar, 0)) {
    if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
    return;
  }
  const int nv = a.nvec_row, nt = a.nvec_tab;
  uint4 q0[KV], q1[KV], q2[KV];
  float4 wq[KV][QPV];
  int cur_g = -1, cur_m = -1;
  long long ld_bytes = 0;
  const signed char* limb = nullptr;
  const int keep = a.F * (16 / EPV) - 16 * (nv - 1);
  uint32_t tm[4];
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    int vb = keep - 4 * w;
    vb = vb < 0 ? 0 : (vb > 4 ? 4 : vb);
    tm[w] = vb >= 4 ? 0xFFFFFFFFu : ((1u << (8 * vb)) - 1u);
  }
  const int tail_v = a.F < nv * EPV ? nv - 1 : -1;

  int ra0 = 0, ra1 = 0, ra2 = 0;
  uint32_t rt = 0;
  float rs = 0.f, rtf = 0.f;
  long long rrow = -1;
  int rgrp = 0, nres = 0;

  auto finish = [&]() {
    if (lane < nres) {
      const SegGroup& G = a.groups[rgrp];
      const C2Header& H = *a.chdr[G.model];
      if (DT == NB_U8) {
        const long long D = ((long long)ra2 << 16) + ((long long)ra1 << 8) + (long long)ra0;
        const float Dsum = (float)D * H.inv_scale;
        const float d = Dsum + H.b;
        const float tau = c2_tau_u8((float)rt, Dsum, H.b, H.inv_scale, H.maxabs);
        c2_store(G.label, G.margin, G.logpost, a.want_lp, a.recheck, rrow, d, tau);
      } else {
        float scale = 1.f;
        if (DT == NB_FP8E4M3 && G.row_exp) scale = exp2f((float)G.row_exp[rrow]);
        const float d = rs * scale + H.b;
        const float kk = (float)a.k_base;
        const float gam = kk * 5.9604645e-8f / (1.f - kk * 5.9604645e-8f);
        const float A = rtf * scale * H.maxabs * 1.001f;
        const float tau = gam * (A + fabsf(H.b)) * 1.01f + 1e-12f * (A + fabsf(H.b)) + 1e-30f;
        c2_store(G.label, G.margin, G.logpost, a.want_lp, a.recheck, rrow, d, tau);
      }
    }
    nres = 0;
  };

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
    const int g = mp->group;
    const int in_smem = mp->in_smem;
    const long long ebase = mp->ebase;
    if (g != cur_g) {
      cur_g = g;
      const SegGroup& G = a.groups[g];
      ld_bytes = G.ld_bytes;
      const int m = G.model;
      if (m != cur_m) {
        cur_m = m;
        const unsigned char* tb = sm + (size_t)m * a.table_stride;
        limb = reinterpret_cast<const signed char*>(tb);
#pragma unroll
        for (int kv = 0; kv < KV; ++kv) {
          const int v = li + LPR * kv;
          if (DT == NB_U8) {
            const uint4* tab = reinterpret_cast<const uint4*>(tb);
            const uint4 z = make_uint4(0, 0, 0, 0);
            q0[kv] = v < nv ? tab[v] : z;
            q1[kv] = v < nv ? tab[nt + v] : z;
            q2[kv] = v < nv ? tab[2 * nt + v] : z;
          } else {
            const float4* tab = reinterpret_cast<const float4*>(tb);
#pragma unroll
            for (int q = 0; q < QPV; ++q)
              wq[kv][q] = v < nv ? tab[q * nt + v] : make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
      }
    }
    const SegGroup& G = a.groups[g];
    const long long* sp = reinterpret_cast<const long long*>(st + p.ptr_off);
    const uint16_t* scol = reinterpret_cast<const uint16_t*>(st + p.col_off);
    const uint16_t* sadd = reinterpret_cast<const uint16_t*>(st + p.add_off);
    for (int r0 = warp * RPW; r0 < nr; r0 += NCW * RPW) {
      if (nres + RPW > 32) finish();
      const int r = r0 + grp;             // this lane group's row
      const bool valid = r < nr;
      const unsigned char* rp = st + (size_t)(valid ? r : 0) * ld_bytes;
      int c0[2] = {0, 0}, c1[2] = {0, 0}, c2[2] = {0, 0};   // even / odd vector chains
      uint32_t ct[2] = {0u, 0u};
      float acc[4] = {0.f, 0.f, 0.f, 0.f}, tf = 0.f;
#pragma unroll
      for (int kv = 0; kv < KV; ++kv) {
        const int v = li + LPR * kv, e = kv & 1;
        if (v < nv) {
          uint4 x = *reinterpret_cast<const uint4*>(rp + (size_t)v * 16);
          if (DT == NB_U8) {
            if (v == tail_v) {
              x.x &= tm[0]; x.y &= tm[1]; x.z &= tm[2]; x.w &= tm[3];
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
          } else {
            float val[EPV];
            Dec::run(x, val);
            if (v == tail_v) {
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
      }
      int a0 = c0[0] + c0[1], a1 = c1[0] + c1[1], a2 = c2[0] + c2[1];
      uint32_t tt = ct[0] + ct[1];
      if (DT == NB_U8 && G.ovf_ptr && valid) {
        const long long k0 = sp[r], k1 = sp[r + 1];
        for (long long e = k0 + li; e < k1; e += LPR) {
          const uint32_t col = in_smem ? scol[e - ebase] : G.ovf_col[e];
          const int add = in_smem ? sadd[e - ebase] : G.ovf_add[e];
          if (col < (uint32_t)a.F) {
            const int vv = col >> 4, b = col & 15;
            a0 += add * (int)limb[(size_t)vv * 16 + b];
            a1 += add * (int)limb[((size_t)nt + vv) * 16 + b];
            a2 += add * (int)limb[((size_t)2 * nt + vv) * 16 + b];
            tt += (uint32_t)add;
          } else {
            atomicOr(a.status, ST_OVF_RANGE);
          }
        }
      }
      // lane nres + j takes row r0 + j of this pass from its group's first lane
      const int src = (lane - nres) * LPR;
      const bool take = lane >= nres && lane < nres + RPW && r0 + (lane - nres) < nr;
      const int sl = take ? src : 0;
      if (DT == NB_U8) {
        // the group's four sums end up in its four lane quarters
        const int k4 = sum4_transposed<LPR>(a0, a1, a2, (int)tt, li);
        const int s0 = __shfl_sync(0xFFFFFFFFu, k4, sl);
        const int s1 = __shfl_sync(0xFFFFFFFFu, k4, sl + LPR / 4);
        const int s2 = __shfl_sync(0xFFFFFFFFu, k4, sl + LPR / 2);
        const uint32_t st_ = (uint32_t)__shfl_sync(0xFFFFFFFFu, k4, sl + 3 * LPR / 4);
        if (take) {
          ra0 = s0, ra1 = s1, ra2 = s2, rt = st_;
        }
      } else {
        float sum = (acc[0] + acc[1]) + (acc[2] + acc[3]);
#pragma unroll
        for (int off = LPR / 2; off > 0; off >>= 1) {
          sum += __shfl_xor_sync(0xFFFFFFFFu, sum, off);
          tf += __shfl_xor_sync(0xFFFFFFFFu, tf, off);
        }
        const float ss = __shfl_sync(0xFFFFFFFFu, sum, sl);
        const float stf = __shfl_sync(0xFFFFFFFFu, tf, sl);
        if (take) {
          rs = ss, rtf = stf;
        }
      }
      if (take) {
        rrow = row0 + r0 + (lane - nres);
        rgrp = g;
      }
      nres += (nr - r0) < RPW ? (nr - r0) : RPW;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
    if (nres + RPW > 32) finish();
  }
  finish();
}

// ---------------------------------------------------------------------------
template <int DT, int KV, int RPW, int NCW>
static nb_status run_seg(const SegArgs& a, const PipeArgs& p, int smem, int* grid,
                         cudaStream_t st) {
  auto kern = k_score2_seg<DT, KV, RPW, NCW>;
  if (smem > kSmemOptIn)
    NB_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                "cudaFuncSetAttribute(seg)");
  int occ = 0;
  NB_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, (NCW + 1) * 32, smem),
              "occupancy(seg)");
  if (occ < 1) {
    set_error("segmented scorer does not fit on an SM");
    return NB_EUNSUPPORTED;
  }
  *grid = num_sms() * occ;
  count_launch();
  kern<<<*grid, (NCW + 1) * 32, smem, st>>>(a, p);
  NB_TRY_CUDA(cudaGetLastError(), "k_score2_seg launch");
  return NB_OK;
}

// Plan of a segmented two-class launch for rows of at most max_ld_bytes.
// u8 rows of up to 16 (32) vectors take 8 (16) lanes per row, four (two) rows
// per warp pass, so that short rows (a few hundred selected opcodes) keep all
// lanes busy; exact integer sums make the result independent of the shape.
// FP32 rows keep 32 lanes per row (their reduction order is that of the
// single-group scorer).
//
// Rows per stage: at most 48 when groups may carry side arrays (the producer's
// lanes hold the overflow pointers of a tile), up to 240 for plain rows, so
// that stages of short rows still move tens of KB.
nb_status seg2_plan(nb_dtype dt, int F, int F_pad, long long max_ld_bytes, int n_models,
                    bool plain_rows, PipeArgs* p, int* kv_out, int* rpw_out, int* ncw_out,
                    int* smem_out) {
  const int es = elem_size(dt);
  const int nvec_row = (F * es + 15) / 16;
  const int rpw = dt == NB_U8 ? (nvec_row <= 16 ? 4 : (nvec_row <= 32 ? 2 : 1)) : 1;
  const int lpr = 32 / rpw;
  const int kv = (nvec_row + lpr - 1) / lpr;
  const int kv_max = dt == NB_F32 ? 8 : 4;
  if (kv < 1 || kv > kv_max || max_ld_bytes > 8192) {
    set_error("batched two-class scoring supports rows of at most %d vectors and 8 KB",
              32 * kv_max);
    return NB_EUNSUPPORTED;
  }
  const int ncw = rpw > 1 ? 12 : ((dt == NB_F32 ? kv <= 8 : kv <= 2) ? 8 : 12);
  const uint32_t tab = dt == NB_U8 ? (uint32_t)(3 * F_pad) : (uint32_t)(4 * F_pad);
  const uint32_t stride = (tab + 127) / 128 * 128;
  long long per = 32768 / ((long long)ncw * rpw * max_ld_bytes);
  int rs = ncw * rpw * (int)(per > 0 ? per : 1);
  const int max_rows = plain_rows ? 240 : kMaxStageRows;
  if (rs > max_rows) {
    rs = max_rows - max_rows % (ncw * rpw);   // whole warp passes
    if (rs < 1) rs = max_rows;
  }
  const unsigned budget = ncw == 8 ? 100u * 1024u : 180u * 1024u;
  PipeArgs q{};
  pipe_layout(q, rs, 1, max_ld_bytes, !plain_rows, false, stride * (uint32_t)n_models, 0);
  int S = q.stages_off + q.stage_bytes > budget ? 2 : (int)((budget - q.stages_off) / q.stage_bytes);
  S = S < 2 ? 2 : (S > kMaxStages ? kMaxStages : S);
  pipe_layout(*p, rs, S, max_ld_bytes, !plain_rows, false, stride * (uint32_t)n_models, 0);
  *kv_out = kv;
  *rpw_out = rpw;
  *ncw_out = ncw;
  *smem_out = (int)(p->stages_off + (uint32_t)p->S * p->stage_bytes);
  if (*smem_out > 220 * 1024) {
    set_error("batched two-class scoring: %d models do not fit in shared memory", n_models);
    return NB_EUNSUPPORTED;
  }
  return NB_OK;
}

nb_status launch_score2_seg(const SegArgs& a, const PipeArgs& p, nb_dtype dt, int kv, int rpw,
                            int ncw, int smem, int* grid, cudaStream_t st) {
#define NB_SEG_CASE(D, K, R, N) \
  if (dt == D && kv == K && rpw == R && ncw == N) return run_seg<D, K, R, N>(a, p, smem, grid, st);
  NB_SEG_CASE(NB_U8, 1, 1, 8) NB_SEG_CASE(NB_U8, 2, 1, 8) NB_SEG_CASE(NB_U8, 3, 1, 12)
  NB_SEG_CASE(NB_U8, 4, 1, 12)
  NB_SEG_CASE(NB_U8, 1, 4, 12) NB_SEG_CASE(NB_U8, 2, 4, 12)
  NB_SEG_CASE(NB_U8, 1, 2, 12) NB_SEG_CASE(NB_U8, 2, 2, 12)
  NB_SEG_CASE(NB_F32, 1, 1, 8) NB_SEG_CASE(NB_F32, 2, 1, 8) NB_SEG_CASE(NB_F32, 3, 1, 8)
  NB_SEG_CASE(NB_F32, 4, 1, 8) NB_SEG_CASE(NB_F32, 5, 1, 8) NB_SEG_CASE(NB_F32, 6, 1, 8)
  NB_SEG_CASE(NB_F32, 7, 1, 8) NB_SEG_CASE(NB_F32, 8, 1, 8)
#undef NB_SEG_CASE
  set_error("batched two-class scoring supports u8 and f32 storage");
  return NB_EUNSUPPORTED;
}

}  // namespace nbg
