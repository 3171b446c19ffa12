// Shared-memory stage pipeline used by the two-class scorer and the
// two-class fit: a producer warp streams blocks of RS consecutive file rows
// (one contiguous range of HBM), the rows' slice of the overflow list and
// (for the fit) their labels into a ring of S stages with cp.async.bulk, each
// stage completing on a "full" mbarrier; consumer warps release a stage on
// its "empty" mbarrier.  All waits are bounded (ST_TIMEOUT, early return).
#pragma once

#include "device.cuh"
#include "internal.cuh"

namespace nbg {

constexpr int kMaxStages = 6;
constexpr int kMaxStageRows = 48;   // producer lanes hold ptr[row0 .. row0 + 63]

struct PipeArgs {
  int RS;               // rows per stage (<= 32)
  int S;                // stages
  int ent_cap;          // overflow entries per stage kept in shared memory
  uint32_t xs_bytes;    // RS * ld_bytes
  uint32_t ptr_off, col_off, add_off, y_off, meta_off, stage_bytes;
  uint32_t tab_bytes;   // parameter table bytes staged at offset 0 (multiple of 16)
  uint32_t stages_off;  // offset of stage 0 in dynamic shared memory
  long long tiles;      // ceil(n / RS)
};

struct StageMeta {
  long long row0;       // first row of the stage within its group
  long long ebase;      // first overflow entry staged (aligned down to 8)
  int nr;
  int in_smem;
  int group;            // group of a segmented launch (0 otherwise)
  int pad;
};

// One tile (up to RS rows of one group) as the producer streams it.
struct TileInfo {
  const char* X;             // the group's matrix
  long long ld_bytes;
  long long row0;            // first row of the tile within the group
  int nr;                    // rows in the tile
  int group;
  const int64_t* ovf_ptr;    // the group's overflow list, or nullptr
  const uint16_t* ovf_col;
  const uint16_t* ovf_add;
  long long E;               // entries in the group's list (ovf_ptr[n])
  const int32_t* y;          // the group's labels (fit), or nullptr
  const int64_t* sizes;      // file sizes (group-wise scorer), or nullptr
};

// what the producer streams
struct PipeSrc {
  const char* X;
  long long ld_bytes;
  long long n;
  const int64_t* ovf_ptr;
  const uint16_t* ovf_col;
  const uint16_t* ovf_add;
  const int32_t* y;        // labels (fit), or nullptr
  const void* table;       // parameter table for offset 0, or nullptr
  int* status;
  const int64_t* sizes;    // file sizes whose model slots go to the y area, or nullptr
};

// Size group -> model slot map of the group-wise scorer (in the staged table):
// a row's slot is map[min(max(size, 0) / bin_bytes, n_bins - 1)].
struct SizeMap {
  int64_t bin_bytes;
  int n_bins;
  uint32_t map_off;         // offset of the map (one byte per size group) in shared memory
};

// Layout of the per-stage side areas after RS rows of ld_bytes each.
inline void pipe_layout(PipeArgs& p, int rs, int stages, long long ld_bytes, bool stage_entries,
                        bool want_y, uint32_t tab_bytes, long long n) {
  p.RS = rs;
  p.S = stages;
  p.ent_cap = stage_entries ? 16 * rs + 16 : 0;
  p.xs_bytes = (uint32_t)(rs * ld_bytes);
  const uint32_t ptr_bytes = (uint32_t)((8 * (rs + 2) + 15) / 16 * 16);
  const uint32_t ent_bytes = (uint32_t)((2 * (p.ent_cap + 8) + 15) / 16 * 16);
  const uint32_t y_bytes = want_y ? (uint32_t)((4 * rs + 15) / 16 * 16) : 0u;
  p.ptr_off = (p.xs_bytes + 127) / 128 * 128;
  p.col_off = p.ptr_off + ptr_bytes;
  p.add_off = p.col_off + ent_bytes;
  p.y_off = p.add_off + ent_bytes;
  p.meta_off = p.y_off + y_bytes;
  p.stage_bytes = (p.meta_off + (uint32_t)sizeof(StageMeta) + 127) / 128 * 128;
  p.tab_bytes = tab_bytes;
  p.stages_off = (tab_bytes + 127) / 128 * 128;
  p.tiles = (n + rs - 1) / rs;
}

// Tiles of one matrix (the single-group case).
struct SingleSrc {
  const PipeSrc* src;
  const PipeArgs* p;
  long long t0;
  long long E;
  __device__ __forceinline__ void init() {
    E = src->ovf_ptr ? src->ovf_ptr[src->n] : 0;
  }
  __device__ __forceinline__ TileInfo tile(long long k) const {
    TileInfo t;
    t.X = src->X;
    t.ld_bytes = src->ld_bytes;
    t.row0 = (t0 + k) * p->RS;
    t.nr = (int)min((long long)p->RS, src->n - t.row0);
    t.group = 0;
    t.ovf_ptr = src->ovf_ptr;
    t.ovf_col = src->ovf_col;
    t.ovf_add = src->ovf_add;
    t.E = E;
    t.y = src->y;
    t.sizes = src->sizes;
    return t;
  }
};

// Stage the parameter tables: table i (bytes each) goes to sm + i * stride.
__device__ __forceinline__ void pipe_stage_tables(unsigned char* sm, const void* const* tables,
                                                  int n_tables, uint32_t bytes, uint32_t stride,
                                                  uint64_t* tabbar) {
  if ((threadIdx.x & 31) != 0 || n_tables == 0) return;
  mbar_expect_tx(tabbar, bytes * (uint32_t)n_tables);
  for (int i = 0; i < n_tables; ++i)
    for (uint32_t off = 0; off < bytes; off += 32768) {
      const uint32_t len = bytes - off < 32768 ? bytes - off : 32768;
      bulk_g2s(sm + (size_t)i * stride + off, static_cast<const char*>(tables[i]) + off, len,
               tabbar);
    }
}

// Per-tile values the producer reads from global memory (the overflow
// pointers ptr[row0 + i], i <= nr, and the labels), loaded two tiles ahead so
// that their latency hides behind the copies of the tiles before.
struct TilePre {
  long long pa, pb;   // ptr[row0 + lane], ptr[row0 + 32 + lane]
  int32_t ya, yb;     // y[row0 + lane], y[row0 + 32 + lane]
  long long za, zb;   // sizes[row0 + lane], sizes[row0 + 32 + lane]
};

__device__ __forceinline__ TilePre pipe_preload(const TileInfo& t, int lane) {
  TilePre r{0, 0, 0, 0, 0, 0};
  if (t.ovf_ptr) {
    r.pa = lane <= t.nr ? t.ovf_ptr[t.row0 + lane] : 0;
    r.pb = lane + 32 <= t.nr ? t.ovf_ptr[t.row0 + 32 + lane] : 0;
  }
  if (t.y) {
    r.ya = lane < t.nr ? t.y[t.row0 + lane] : 0;
    r.yb = lane + 32 < t.nr ? t.y[t.row0 + 32 + lane] : 0;
  }
  if (t.sizes) {
    r.za = lane < t.nr ? t.sizes[t.row0 + lane] : 0;
    r.zb = lane + 32 < t.nr ? t.sizes[t.row0 + 32 + lane] : 0;
  }
  return r;
}

__device__ __forceinline__ int32_t size_slot(long long z, const SizeMap& sm,
                                             const unsigned char* smem, int* status) {
  if (z < 0) {   // flagged, counted as size 0
    atomicOr(status, ST_BAD_ROUTE);
    z = 0;
  }
  long long b = z / sm.bin_bytes;
  if (b > sm.n_bins - 1) b = sm.n_bins - 1;
  return (int32_t)smem[sm.map_off + b];
}

// Producer warp: the whole warp calls it; lane 0 issues the copies.  `src`
// describes tiles k = 0 .. ntl-1 of this block.
template <class Src>
__device__ __forceinline__ void pipe_produce_tiles(Src& src, const PipeArgs& p,
                                                   unsigned char* sm, uint64_t* full,
                                                   uint64_t* empty, long long ntl, int* status,
                                                   const SizeMap* zmap = nullptr,
                                                   uint64_t* tabbar = nullptr) {
  const int lane = threadIdx.x & 31;
  TileInfo cur, nxt;
  TilePre pc{0, 0, 0, 0, 0, 0}, pn{0, 0, 0, 0, 0, 0};
  if (zmap && ntl > 0) {   // the size map arrives with the table
    bool ok = true;
    if (lane == 0) ok = mbar_wait_bounded(tabbar, 0);
    ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
    if (!ok) {
      if (lane == 0) atomicOr(status, ST_TIMEOUT);
      return;
    }
  }
  if (ntl > 0) {
    cur = src.tile(0);
    pc = pipe_preload(cur, lane);
  }
  if (ntl > 1) {
    nxt = src.tile(1);
    pn = pipe_preload(nxt, lane);
  }
  for (long long k = 0; k < ntl; ++k) {
    // tile k + 2: its global values are in flight while tile k is staged
    TileInfo nn = nxt;
    TilePre p2{0, 0, 0, 0, 0, 0};
    if (k + 2 < ntl) {
      nn = src.tile(k + 2);
      p2 = pipe_preload(nn, lane);
    }
    const int s = (int)(k % p.S);
    const uint32_t ph = (uint32_t)((k / p.S) & 1);
    if (k >= p.S) {
      bool ok = true;
      if (lane == 0) ok = mbar_wait_bounded(&empty[s], ph ^ 1u);
      ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
      if (!ok) {
        if (lane == 0) atomicOr(status, ST_TIMEOUT);
        return;
      }
    }
    unsigned char* st = sm + p.stages_off + (size_t)s * p.stage_bytes;
    const int nr = cur.nr;
    const bool ovf = cur.ovf_ptr != nullptr;
    long long e0 = 0, e1 = 0;
    if (ovf) {
      long long* sp = reinterpret_cast<long long*>(st + p.ptr_off);
      if (lane <= nr) sp[lane] = pc.pa;
      if (lane + 32 <= nr) sp[lane + 32] = pc.pb;
      e0 = __shfl_sync(0xFFFFFFFFu, pc.pa, 0);
      const long long tail_a = __shfl_sync(0xFFFFFFFFu, pc.pa, nr & 31);
      const long long tail_b = __shfl_sync(0xFFFFFFFFu, pc.pb, nr & 31);
      e1 = nr < 32 ? tail_a : tail_b;
    }
    if (cur.y) {
      // labels through registers (rows of a stage need not start 16-byte aligned)
      int32_t* sy = reinterpret_cast<int32_t*>(st + p.y_off);
      if (lane < nr) sy[lane] = pc.ya;
      if (lane + 32 < nr) sy[lane + 32] = pc.yb;
    } else if (cur.sizes && zmap) {
      // the rows' model slots from their sizes
      int32_t* sy = reinterpret_cast<int32_t*>(st + p.y_off);
      if (lane < nr) sy[lane] = size_slot(pc.za, *zmap, sm, status);
      if (lane + 32 < nr) sy[lane + 32] = size_slot(pc.zb, *zmap, sm, status);
    }
    // the lanes' shared-memory writes are ordered before lane 0's arrive
    // (a release) by the warp barrier
    __syncwarp();
    if (lane == 0) {
      StageMeta* m = reinterpret_cast<StageMeta*>(st + p.meta_off);
      m->row0 = cur.row0;
      m->nr = nr;
      m->group = cur.group;
      const uint32_t xb = (uint32_t)nr * (uint32_t)cur.ld_bytes;
      uint32_t total = xb;
      const long long eb = e0 & ~7LL, ee = (e1 + 7) & ~7LL;
      int in_smem = 0;
      if (ovf && e1 > e0 && ee - eb <= p.ent_cap && ee <= cur.E) in_smem = 1;
      m->in_smem = in_smem;
      m->ebase = eb;
      const uint32_t eb_bytes = in_smem ? (uint32_t)(ee - eb) * 2u : 0u;
      total += 2u * eb_bytes;
      mbar_expect_tx(&full[s], total);
      const char* x = cur.X + cur.row0 * cur.ld_bytes;
      for (uint32_t off = 0; off < xb; off += 32768) {
        const uint32_t len = xb - off < 32768 ? xb - off : 32768;
        bulk_g2s(st + off, x + off, len, &full[s]);
      }
      if (eb_bytes) {
        bulk_g2s(st + p.col_off, cur.ovf_col + eb, eb_bytes, &full[s]);
        bulk_g2s(st + p.add_off, cur.ovf_add + eb, eb_bytes, &full[s]);
      }
    }
    cur = nxt;
    pc = pn;
    nxt = nn;
    pn = p2;
  }
}

// Single-matrix producer (the table, if any, is staged at offset 0).
__device__ __forceinline__ void pipe_produce(const PipeSrc& src, const PipeArgs& p,
                                             unsigned char* sm, uint64_t* full, uint64_t* empty,
                                             uint64_t* tabbar, long long t0, long long ntl,
                                             const SizeMap* zmap = nullptr) {
  if (src.table) pipe_stage_tables(sm, &src.table, 1, p.tab_bytes, 0, tabbar);
  SingleSrc ss{&src, &p, t0, 0};
  ss.init();
  pipe_produce_tiles(ss, p, sm, full, empty, ntl, src.status, zmap, tabbar);
}

}  // namespace nbg
