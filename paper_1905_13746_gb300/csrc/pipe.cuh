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
  long long row0;
  long long ebase;      // first overflow entry staged (aligned down to 8)
  int nr;
  int in_smem;
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
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

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

// Producer warp: the whole warp calls it; lane 0 issues the copies.
// Tiles [t0, t0 + ntl) of this block; the table (if any) goes on `tabbar`.
__device__ __forceinline__ void pipe_produce(const PipeSrc& src, const PipeArgs& p,
                                             unsigned char* sm, uint64_t* full, uint64_t* empty,
                                             uint64_t* tabbar, long long t0, long long ntl) {
  const int lane = threadIdx.x & 31;
  const bool ovf = src.ovf_ptr != nullptr;
  if (lane == 0 && src.table) {
    mbar_expect_tx(tabbar, p.tab_bytes);
    for (uint32_t off = 0; off < p.tab_bytes; off += 32768) {
      const uint32_t len = p.tab_bytes - off < 32768 ? p.tab_bytes - off : 32768;
      bulk_g2s(sm + off, static_cast<const char*>(src.table) + off, len, tabbar);
    }
  }
  const long long E = ovf ? src.ovf_ptr[src.n] : 0;   // entries in the list
  // overflow pointers of the next tile, one tile ahead: lane i holds
  // ptr[row0 + i] and ptr[row0 + 32 + i]
  long long pa = 0, pb = 0;
  if (ovf && ntl > 0) {
    const long long r0 = t0 * p.RS;
    const long long nr = min((long long)p.RS, src.n - r0);
    pa = lane <= nr ? src.ovf_ptr[r0 + lane] : 0;
    pb = lane + 32 <= nr ? src.ovf_ptr[r0 + 32 + lane] : 0;
  }
  for (long long k = 0; k < ntl; ++k) {
    long long na = 0, nb = 0;
    if (ovf && k + 1 < ntl) {
      const long long r0 = (t0 + k + 1) * p.RS;
      const long long nr = min((long long)p.RS, src.n - r0);
      na = lane <= nr ? src.ovf_ptr[r0 + lane] : 0;
      nb = lane + 32 <= nr ? src.ovf_ptr[r0 + 32 + lane] : 0;
    }
    const int s = (int)(k % p.S);
    const uint32_t ph = (uint32_t)((k / p.S) & 1);
    if (k >= p.S) {
      bool ok = true;
      if (lane == 0) ok = mbar_wait_bounded(&empty[s], ph ^ 1u);
      ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
      if (!ok) {
        if (lane == 0) atomicOr(src.status, ST_TIMEOUT);
        return;
      }
    }
    unsigned char* st = sm + p.stages_off + (size_t)s * p.stage_bytes;
    const long long row0 = (t0 + k) * p.RS;
    const int nr = (int)min((long long)p.RS, src.n - row0);
    long long e0 = 0, e1 = 0;
    if (ovf) {
      long long* sp = reinterpret_cast<long long*>(st + p.ptr_off);
      if (lane <= nr) sp[lane] = pa;
      if (lane + 32 <= nr) sp[lane + 32] = pb;
      e0 = __shfl_sync(0xFFFFFFFFu, pa, 0);
      const long long tail_a = __shfl_sync(0xFFFFFFFFu, pa, nr & 31);
      const long long tail_b = __shfl_sync(0xFFFFFFFFu, pb, nr & 31);
      e1 = nr < 32 ? tail_a : tail_b;
    }
    if (src.y) {
      // labels through registers (rows of a stage need not start 16-byte aligned)
      int32_t* sy = reinterpret_cast<int32_t*>(st + p.y_off);
      if (lane < nr) sy[lane] = src.y[row0 + lane];
      if (lane + 32 < nr) sy[lane + 32] = src.y[row0 + 32 + lane];
    }
    __threadfence_block();
    __syncwarp();
    if (lane == 0) {
      StageMeta* m = reinterpret_cast<StageMeta*>(st + p.meta_off);
      m->row0 = row0;
      m->nr = nr;
      const uint32_t xb = (uint32_t)nr * (uint32_t)src.ld_bytes;
      uint32_t total = xb;
      const long long eb = e0 & ~7LL, ee = (e1 + 7) & ~7LL;
      int in_smem = 0;
      if (ovf && e1 > e0 && ee - eb <= p.ent_cap && ee <= E) in_smem = 1;
      m->in_smem = in_smem;
      m->ebase = eb;
      const uint32_t eb_bytes = in_smem ? (uint32_t)(ee - eb) * 2u : 0u;
      total += 2u * eb_bytes;
      mbar_expect_tx(&full[s], total);
      const char* x = src.X + row0 * src.ld_bytes;
      for (uint32_t off = 0; off < xb; off += 32768) {
        const uint32_t len = xb - off < 32768 ? xb - off : 32768;
        bulk_g2s(st + off, x + off, len, &full[s]);
      }
      if (eb_bytes) {
        bulk_g2s(st + p.col_off, src.ovf_col + eb, eb_bytes, &full[s]);
        bulk_g2s(st + p.add_off, src.ovf_add + eb, eb_bytes, &full[s]);
      }
    }
    pa = na;
    pb = nb;
  }
}

}  // namespace nbg
