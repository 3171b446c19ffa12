// The group-wise method around the scorer (Sec. 3 size groups and top-k
// opcode selection, Sec. 4 per-group models and the small-group rule):
//
//   nb_group_fallback   host: model group of every size group;
//   nb_route            size -> group (-> model) per file, and a stable
//                       counting sort of the files by group (three kernels:
//                       per-tile warp-ranked counts, one scan, scatter);
//   nb_select_features  exact top-k opcode ranking of two-class models;
//   nb_gather           rows by a permutation, columns by each row's group's
//                       selection, into a dense padded matrix;
//   nb_groupwise_*      all of it for scoring: route, gather, one batched
//                       two-class launch over every group with a work list
//                       built on the device, FP64 recheck, and the results
//                       put back in the files' order.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "pipe.cuh"
#include "score2.cuh"
#include "seg.cuh"

namespace nbg {

constexpr int kRouteWarps = 8;
constexpr int kRouteSub = 512;                          // files per warp and tile
constexpr int kRouteTile = kRouteWarps * kRouteSub;     // files per block
constexpr int kRouteMaxGroups = 512;
constexpr int kRouteMaxClassCells = 4096;               // n_bins * C with labels

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Group of file i and its size group in *bin.  A negative size or a model_of
// entry outside [0, n_out) raises ST_BAD_ROUTE and counts as 0, so that every
// file still gets a group and the order stays a permutation.
__device__ __forceinline__ int route_of(const int64_t* sizes, int64_t i, int64_t bin_bytes,
                                        int n_bins, const int32_t* model_of, int n_out,
                                        int* bin, int* status) {
  long long s = sizes[i];
  if (s < 0) {
    atomicOr(status, ST_BAD_ROUTE);
    s = 0;
  }
  long long g = s / bin_bytes;
  if (g > n_bins - 1) g = n_bins - 1;
  *bin = (int)g;
  int m = model_of ? model_of[g] : (int)g;
  if (m < 0 || m >= n_out) {
    atomicOr(status, ST_BAD_ROUTE);
    m = 0;
  }
  return m;
}

// Pass 1: group of every file, per-block counts per group (hist[b * n_out + g])
// and, with labels, files per (size group, class).
__global__ void __launch_bounds__(kRouteWarps * 32)
    k_route_count(const int64_t* sizes, int64_t n, int64_t bin_bytes, int n_bins,
                  const int32_t* model_of, int n_out, const int32_t* y, int C,
                  int32_t* group, int64_t* hist, int64_t* class_counts, int* status) {
  __shared__ int cnt[kRouteWarps][kRouteMaxGroups];
  __shared__ int ccnt[kRouteMaxClassCells];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int t = threadIdx.x; t < kRouteWarps * kRouteMaxGroups; t += blockDim.x)
    (&cnt[0][0])[t] = 0;
  if (y)
    for (int t = threadIdx.x; t < n_bins * C; t += blockDim.x) ccnt[t] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRouteTile + (int64_t)warp * kRouteSub;
  for (int step = 0; step < kRouteSub / 32; ++step) {
    const int64_t i = base + step * 32 + lane;
    int bin = -1, g = -1;
    if (i < n) {
      g = route_of(sizes, i, bin_bytes, n_bins, model_of, n_out, &bin, status);
      group[i] = g;
      if (y) {
        const int c = y[i];
        if (c >= 0 && c < C) atomicAdd(&ccnt[bin * C + c], 1);
        else atomicOr(status, ST_BAD_ROUTE);
      }
    }
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, g);
    if (g >= 0 && lane == __ffs(peers) - 1) cnt[warp][g] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  for (int g = threadIdx.x; g < n_out; g += blockDim.x) {
    int s = 0;
#pragma unroll
    for (int w = 0; w < kRouteWarps; ++w) s += cnt[w][g];
    hist[(int64_t)blockIdx.x * n_out + g] = s;
  }
  if (y)
    for (int t = threadIdx.x; t < n_bins * C; t += blockDim.x)
      if (ccnt[t]) atomicAdd(reinterpret_cast<unsigned long long*>(&class_counts[t]),
                             (unsigned long long)ccnt[t]);
}

// Pass 2 (one block of 1024 threads): thread (p, g), g < n_out, p < P =
// 1024 / n_out, owns a slice of the blocks of column g of hist; it sums the
// slice (coalesced across g), the slices' sums are scanned per group and the
// group totals across groups (offsets[g], offsets[n_out] = n), then each
// thread rewrites its slice as exclusive prefixes within the group: block b's
// first position of group g is offsets[g] + hist[b * n_out + g].
__global__ void __launch_bounds__(1024)
    k_route_scan(int64_t* hist, int nblk, int n_out, int64_t* offsets) {
  __shared__ int64_t part[1024];
  __shared__ int64_t tot[kRouteMaxGroups];
  const int t = threadIdx.x;
  const int P = 1024 / n_out;
  const int g = t % n_out, p = t / n_out;
  const bool on = p < P;
  const int b0 = on ? (int)((int64_t)nblk * p / P) : 0;
  const int b1 = on ? (int)((int64_t)nblk * (p + 1) / P) : 0;
  int64_t s = 0;
#pragma unroll 4
  for (int b = b0; b < b1; ++b) s += hist[(int64_t)b * n_out + g];
  part[t] = on ? s : 0;
  __syncthreads();
  int64_t start = 0, total = 0;
  if (on) {
    for (int q = 0; q < P; ++q) {
      const int64_t v = part[q * n_out + g];
      if (q < p) start += v;
      total += v;
    }
    if (p == 0) tot[g] = total;
  }
  __syncthreads();
  if (t < 32) {   // exclusive scan of the group totals by one warp
    const int per = (n_out + 31) / 32;
    const int a = t * per, e = min(n_out, a + per);
    int64_t sum = 0;
    for (int i = a; i < e; ++i) sum += tot[i];
    int64_t v = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int64_t u = __shfl_up_sync(0xFFFFFFFFu, v, off);
      if (t >= off) v += u;
    }
    int64_t run = v - sum;
    for (int i = a; i < e; ++i) {
      const int64_t x = tot[i];
      tot[i] = run;
      offsets[i] = run;
      run += x;
    }
    if (t == 31) offsets[n_out] = v;
  }
  if (on) {
    int64_t run = start;
    for (int b = b0; b < b1; ++b) {
      const int64_t h = hist[(int64_t)b * n_out + g];
      hist[(int64_t)b * n_out + g] = run;
      run += h;
    }
  }
}

// Pass 3: each file's position; ranks inside a warp step from the peers of
// the same group, so the order within a group is the files' order (stable).
__global__ void __launch_bounds__(kRouteWarps * 32)
    k_route_scatter(const int32_t* group, int64_t n, int n_out, const int64_t* first,
                    const int64_t* offsets, int64_t* order) {
  __shared__ int cnt[kRouteWarps][kRouteMaxGroups];
  __shared__ int64_t run[kRouteWarps][kRouteMaxGroups / 2];   // two passes of 256 groups
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int t = threadIdx.x; t < kRouteWarps * kRouteMaxGroups; t += blockDim.x)
    (&cnt[0][0])[t] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRouteTile + (int64_t)warp * kRouteSub;
  for (int step = 0; step < kRouteSub / 32; ++step) {
    const int64_t i = base + step * 32 + lane;
    const int g = i < n ? group[i] : -1;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, g);
    if (g >= 0 && lane == __ffs(peers) - 1) cnt[warp][g] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // groups [h * 256, h * 256 + 256) per pass keep their running positions in `run`
  for (int h = 0; h * (kRouteMaxGroups / 2) < n_out; ++h) {
    const int g0 = h * (kRouteMaxGroups / 2);
    for (int t = threadIdx.x; t < kRouteMaxGroups / 2; t += blockDim.x) {
      const int g = g0 + t;
      if (g >= n_out) continue;
      int64_t p = offsets[g] + first[(int64_t)blockIdx.x * n_out + g];
      for (int w = 0; w < kRouteWarps; ++w) {
        run[w][t] = p;
        p += cnt[w][g];
      }
    }
    __syncthreads();
    for (int step = 0; step < kRouteSub / 32; ++step) {
      const int64_t i = base + step * 32 + lane;
      const int g = i < n ? group[i] : -1;
      const bool mine = g >= g0 && g < g0 + kRouteMaxGroups / 2;
      const unsigned peers = __match_any_sync(0xFFFFFFFFu, mine ? g : -1);
      if (mine) order[run[warp][g - g0] + __popc(peers & lanemask_lt())] = i;
      __syncwarp();
      if (mine && lane == __ffs(peers) - 1) run[warp][g - g0] += __popc(peers);
      __syncwarp();
    }
    __syncthreads();
  }
}

size_t route_workspace(int64_t n, int n_out) {
  const int64_t nblk = n > 0 ? (n + kRouteTile - 1) / kRouteTile : 1;
  return (size_t)(nblk * n_out) * sizeof(int64_t);
}

nb_status launch_route(const int64_t* sizes, int64_t n, int64_t bin_bytes, int n_bins,
                       const int32_t* model_of, int n_out, const int32_t* y, int C,
                       int32_t* group, int64_t* order, int64_t* offsets,
                       int64_t* class_counts, int64_t* hist, int* status, cudaStream_t st) {
  const int64_t nblk = n > 0 ? (n + kRouteTile - 1) / kRouteTile : 0;
  if (class_counts)
    NB_TRY_CUDA(cudaMemsetAsync(class_counts, 0, sizeof(int64_t) * n_bins * C, st),
                "memset(class_counts)");
  if (nblk == 0) {
    NB_TRY_CUDA(cudaMemsetAsync(offsets, 0, sizeof(int64_t) * (n_out + 1), st),
                "memset(offsets)");
    return NB_OK;
  }
  count_launch();
  k_route_count<<<(unsigned)nblk, kRouteWarps * 32, 0, st>>>(
      sizes, n, bin_bytes, n_bins, model_of, n_out, class_counts ? y : nullptr, C, group, hist,
      class_counts, status);
  NB_TRY_CUDA(cudaGetLastError(), "k_route_count launch");
  count_launch();
  k_route_scan<<<1, 1024, 0, st>>>(hist, (int)nblk, n_out, offsets);
  NB_TRY_CUDA(cudaGetLastError(), "k_route_scan launch");
  if (order) {
    count_launch();
    k_route_scatter<<<(unsigned)nblk, kRouteWarps * 32, 0, st>>>(group, n, n_out, hist,
                                                                  offsets, order);
    NB_TRY_CUDA(cudaGetLastError(), "k_route_scatter launch");
  }
  return NB_OK;
}

// ---------------------------------------------------------------------------
// top-k opcode selection (two-class models): key_j = |N_1j D_0 - N_0j D_1|
// over the common denominator D_0 D_1 (a class with D_c = 0 counts as D_c = 1,
// its N_cj being 0), compared exactly in 128-bit integers; rank_j = number
// of opcodes with a larger key or an equal key and a lower index.
// ---------------------------------------------------------------------------
constexpr int kSelMaxModels = 128;
constexpr int kSelThreads = 256;
constexpr int kSelPer = 4;                        // candidates per thread
constexpr int kSelBlock = kSelThreads * kSelPer;  // candidates per block
constexpr int kSelTile = 1024;                    // keys staged per round

struct SelModel {
  const uint64_t* counts;   // 2 x F
  const uint64_t* nc;       // 2
  int F;
};

struct SelArgs {
  SelModel m[kSelMaxModels];
  int k, norm;
  int32_t* cols;
};

typedef unsigned __int128 u128;

__device__ __forceinline__ u128 sel_key(const uint64_t* N, int F, int j, uint64_t D0,
                                        uint64_t D1) {
  const u128 a = (u128)N[F + j] * D0, b = (u128)N[j] * D1;
  return a > b ? a - b : b - a;
}

__global__ void __launch_bounds__(kSelThreads) k_select_topk(const SelArgs a) {
  __shared__ uint64_t khi[kSelTile], klo[kSelTile];
  __shared__ unsigned long long red[2][kSelThreads / 32];
  const SelModel M = a.m[blockIdx.y];
  const int F = M.F, t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if ((int64_t)blockIdx.x * kSelBlock >= F) return;   // uniform per block
  uint64_t D0, D1;
  if (a.norm == NB_SELECT_FILES) {
    D0 = M.nc[0];
    D1 = M.nc[1];
  } else {
    unsigned long long s0 = 0, s1 = 0;
    for (int j = t; j < F; j += blockDim.x) {
      s0 += M.counts[j];
      s1 += M.counts[F + j];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      s0 += __shfl_xor_sync(0xFFFFFFFFu, s0, off);
      s1 += __shfl_xor_sync(0xFFFFFFFFu, s1, off);
    }
    if (lane == 0) {
      red[0][warp] = s0;
      red[1][warp] = s1;
    }
    __syncthreads();
    s0 = s1 = 0;
    for (int w = 0; w < kSelThreads / 32; ++w) {
      s0 += red[0][w];
      s1 += red[1][w];
    }
    D0 = s0;
    D1 = s1;
  }
  if (D0 == 0) D0 = 1;
  if (D1 == 0) D1 = 1;
  u128 key[kSelPer];
  int jj[kSelPer], rank[kSelPer];
#pragma unroll
  for (int q = 0; q < kSelPer; ++q) {
    jj[q] = blockIdx.x * kSelBlock + q * kSelThreads + t;
    key[q] = jj[q] < F ? sel_key(M.counts, F, jj[q], D0, D1) : (u128)0;
    rank[q] = 0;
  }
  for (int i0 = 0; i0 < F; i0 += kSelTile) {
    __syncthreads();
    for (int u = t; u < kSelTile; u += blockDim.x) {
      const int i = i0 + u;
      const u128 v = i < F ? sel_key(M.counts, F, i, D0, D1) : (u128)0;
      khi[u] = (uint64_t)(v >> 64);
      klo[u] = (uint64_t)v;
    }
    __syncthreads();
    const int m = F - i0 < kSelTile ? F - i0 : kSelTile;
    for (int u = 0; u < m; ++u) {
      const u128 v = ((u128)khi[u] << 64) | klo[u];
      const int i = i0 + u;
#pragma unroll
      for (int q = 0; q < kSelPer; ++q) rank[q] += (v > key[q] || (v == key[q] && i < jj[q]));
    }
  }
#pragma unroll
  for (int q = 0; q < kSelPer; ++q)
    if (jj[q] < F && rank[q] < a.k) a.cols[(int64_t)blockIdx.y * a.k + rank[q]] = jj[q];
}

// ---------------------------------------------------------------------------
// gather: out[r][t] = X[src(r)][cols[grp * k + t]], t < k, zero up to ld_out
// (src(r) = order[r] or r; grp = group[src(r)] or 0; cols == nullptr: t).
// One warp per output row; the u8 kernel packs four bytes per lane.
// ---------------------------------------------------------------------------
template <int ES>
__global__ void __launch_bounds__(256)
    k_gather(const char* X, int64_t ld, int F, int64_t n_src, int64_t n, const int64_t* order,
             const int32_t* group, int n_groups, const int32_t* cols, int k, char* out,
             int64_t ld_out, int* status) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n;
       r += warps) {
    int64_t i = order ? order[r] : r;
    int g = 0;
    if (i < 0 || i >= n_src) {       // no source row: zero row
      if (lane == 0) atomicOr(status, ST_BAD_ROUTE);
      i = 0;
      g = -1;
    } else if (group) {
      g = group[i];
    }
    if (g >= n_groups) g = -1;
    if (g < 0) {                     // no selection to take: zero row
      if (lane == 0) atomicOr(status, ST_BAD_ROUTE);
      g = -1;
    }
    const int32_t* cg = cols && g >= 0 ? cols + (int64_t)g * k : nullptr;
    const int kk = g >= 0 ? k : 0;
    if (ES == 1) {
      const unsigned char* src = reinterpret_cast<const unsigned char*>(X) + i * ld;
      uint32_t* dst = reinterpret_cast<uint32_t*>(out + r * ld_out);
      for (int64_t t0 = 4 * lane; t0 < ld_out; t0 += 128) {
        uint32_t w = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int t = (int)t0 + b;
          if (t < kk) {
            const int c = cg ? cg[t] : t;
            if ((unsigned)c < (unsigned)F) w |= (uint32_t)src[c] << (8 * b);
            else atomicOr(status, ST_BAD_ROUTE);
          }
        }
        dst[t0 >> 2] = w;
      }
    } else {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(X + i * ld * 4);
      uint32_t* dst = reinterpret_cast<uint32_t*>(out + r * ld_out * 4);
      for (int64_t t = lane; t < ld_out; t += 32) {
        uint32_t v = 0;
        if (t < kk) {
          const int c = cg ? cg[t] : (int)t;
          if ((unsigned)c < (unsigned)F) v = src[c];
          else atomicOr(status, ST_BAD_ROUTE);
        }
        dst[t] = v;
      }
    }
  }
}

// u8 rows through shared memory.  A warp takes chunks of 32 consecutive
// output rows; lane j loads row j's source index and group once per chunk (the
// next chunk's while the current one is gathered), so no row waits on a
// dependent index load.  Each row is copied with 16-byte cp.async copies
// (coalesced, one HBM pass) while the previous one is gathered (two buffers
// per warp); the group's selection stays in shared memory while consecutive
// rows share the group (rows come sorted by group); bytes are gathered from
// shared memory, four per lane per output word.
constexpr int kGatherWarps = 8;

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait1() {
  asm volatile("cp.async.wait_group 1;" ::: "memory");
}

// source row (-1: none) and group (-1: none) of output row r
__device__ __forceinline__ void gather_index(int64_t r, int64_t n, const int64_t* order,
                                             const int32_t* group, int n_groups, int64_t n_src,
                                             int64_t* i, int* g) {
  *i = -1;
  *g = -1;
  if (r >= n) return;
  int64_t s = order ? order[r] : r;
  if (s < 0 || s >= n_src) return;
  *i = s;
  int gg = group ? group[s] : 0;
  *g = gg < 0 || gg >= n_groups ? -1 : gg;
}

__global__ void __launch_bounds__(kGatherWarps * 32)
    k_gather_u8s(const unsigned char* X, int64_t ld, int F, int64_t n_src, int64_t n,
                 const int64_t* order, const int32_t* group, int n_groups, const int32_t* cols,
                 int k, unsigned char* out, int64_t ld_out, int row_bytes, int* status) {
  extern __shared__ __align__(16) unsigned char gsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* buf = gsm + (size_t)warp * 2 * row_bytes;
  const int kq = (k + 3) & ~3;   // selection stride: 16-byte aligned rows of sel
  int32_t* sel = reinterpret_cast<int32_t*>(gsm + (size_t)kGatherWarps * 2 * row_bytes) +
                 (size_t)warp * kq;
  const int nv = (F + 15) >> 4;
  const int64_t nchunks = (n + 31) / 32;
  const int64_t wstride = (int64_t)gridDim.x * kGatherWarps;
  int64_t c = (int64_t)blockIdx.x * kGatherWarps + warp;
  if (c >= nchunks) return;
  // lane j: source row and group of row j of the current and the next chunk
  int64_t ci, ni;
  int cg, ng;
  gather_index(c * 32 + lane, n, order, group, n_groups, n_src, &ci, &cg);
  gather_index((c + wstride) * 32 + lane, n, order, group, n_groups, n_src, &ni, &ng);
  auto fetch = [&](int64_t i, unsigned char* dst) {
    if (i >= 0) {
      const unsigned char* src = X + i * ld;
      for (int v = lane; v < nv; v += 32) cp_async16(dst + 16 * v, src + 16 * v);
    }
    cp_async_commit();
  };
  fetch(__shfl_sync(0xFFFFFFFFu, ci, 0), buf);
  int held = -2;   // group whose selection sel holds (-1: identity)
  int b = 0;
  for (; c < nchunks; c += wstride) {
    const int rows = (int)min((int64_t)32, n - c * 32);
    for (int j = 0; j < rows; ++j, b ^= 1) {
      const int64_t i = __shfl_sync(0xFFFFFFFFu, ci, j);
      const int g = __shfl_sync(0xFFFFFFFFu, cg, j);
      // the next row (this chunk's j + 1, else the next chunk's first) lands meanwhile
      const int64_t inext = j + 1 < rows ? __shfl_sync(0xFFFFFFFFu, ci, (j + 1) & 31)
                                         : __shfl_sync(0xFFFFFFFFu, ni, 0);
      fetch(inext, buf + (size_t)(b ^ 1) * row_bytes);
      cp_async_wait1();   // this thread's copies of the current row
      const bool bad = i < 0 || g < 0;
      if (bad && lane == 0) atomicOr(status, ST_BAD_ROUTE);
      const int want = cols ? g : -1;
      if (!bad && want != held) {
        for (int t = lane; t < k; t += 32) sel[t] = cols ? cols[(int64_t)g * k + t] : t;
        held = want;
      }
      __syncwarp();       // every lane's copies and sel visible
      const unsigned char* row = buf + (size_t)b * row_bytes;
      uint32_t* dst = reinterpret_cast<uint32_t*>(out + (c * 32 + j) * ld_out);
      for (int64_t t0 = 4 * lane; t0 < ld_out; t0 += 128) {
        uint32_t w = 0;
        if (!bad && t0 + 3 < k) {
          const int4 c4 = *reinterpret_cast<const int4*>(sel + t0);
          const unsigned cmax = max(max((unsigned)c4.x, (unsigned)c4.y),
                                    max((unsigned)c4.z, (unsigned)c4.w));
          if (cmax < (unsigned)F) {
            w = (uint32_t)row[c4.x] | ((uint32_t)row[c4.y] << 8) | ((uint32_t)row[c4.z] << 16) |
                ((uint32_t)row[c4.w] << 24);
          } else {
            atomicOr(status, ST_BAD_ROUTE);
          }
        } else if (!bad) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int t = (int)t0 + q;
            if (t < k) {
              const int cc = sel[t];
              if ((unsigned)cc < (unsigned)F) w |= (uint32_t)row[cc] << (8 * q);
              else atomicOr(status, ST_BAD_ROUTE);
            }
          }
        }
        dst[t0 >> 2] = w;
      }
      __syncwarp();       // buffer b is free for the row after next
    }
    ci = ni;
    cg = ng;
    gather_index((c + 2 * wstride) * 32 + lane, n, order, group, n_groups, n_src, &ni, &ng);
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

nb_status launch_gather(const void* X, nb_dtype dt, int64_t ld, int F, int64_t n_src,
                        int64_t n, const int64_t* order, const int32_t* group, int n_groups,
                        const int32_t* cols, int k, void* out, int64_t ld_out, int* status,
                        cudaStream_t st) {
  if (n == 0) return NB_OK;
  int64_t blocks = (n + 7) / 8;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  int64_t cblocks = ((n + 31) / 32 + kGatherWarps - 1) / kGatherWarps;   // 32-row chunks
  if (cblocks > cap) cblocks = cap;
  // staged u8 path: 16-byte aligned rows whose copies and selections fit
  const int row_bytes = (F + 15) / 16 * 16;
  const size_t smem =
      (size_t)kGatherWarps * 2 * row_bytes + (size_t)kGatherWarps * ((k + 3) & ~3) * 4;
  if (elem_size(dt) == 1 && (ld % 16) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
      smem <= 96 * 1024) {
    if ((int)smem > kSmemOptIn)   // per device and function: set at every launch
      NB_TRY_CUDA(cudaFuncSetAttribute(k_gather_u8s, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem),
                  "cudaFuncSetAttribute(gather)");
    count_launch();
    k_gather_u8s<<<(unsigned)cblocks, kGatherWarps * 32, smem, st>>>(
        static_cast<const unsigned char*>(X), ld, F, n_src, n, order, group, n_groups, cols, k,
        static_cast<unsigned char*>(out), ld_out, row_bytes, status);
    NB_TRY_CUDA(cudaGetLastError(), "k_gather_u8s launch");
    return NB_OK;
  }
  count_launch();
  if (elem_size(dt) == 1)
    k_gather<1><<<(unsigned)blocks, 256, 0, st>>>(static_cast<const char*>(X), ld, F, n_src, n,
                                                   order, group, n_groups, cols, k,
                                                   static_cast<char*>(out), ld_out, status);
  else
    k_gather<4><<<(unsigned)blocks, 256, 0, st>>>(static_cast<const char*>(X), ld, F, n_src, n,
                                                   order, group, n_groups, cols, k,
                                                   static_cast<char*>(out), ld_out, status);
  NB_TRY_CUDA(cudaGetLastError(), "k_gather launch");
  return NB_OK;
}

// ---------------------------------------------------------------------------
// device-built work list of the batched two-class launch: group m = the rows
// offsets[m] .. offsets[m+1]-1 of the gathered matrix, scored by model slot m
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128)
    k_gw_worklist(SegHeader* hdr, SegGroup* list, int n_models, const int64_t* offsets,
                  const char* xs, int64_t ld_bytes, uint8_t* label, float* margin,
                  float* logpost, int64_t rs) {
  // one thread per model slot (n_models <= 128); first tiles and chunks by a
  // block-wide exclusive scan
  __shared__ long long wt[4], wc[4];
  const int m = threadIdx.x, lane = m & 31, warp = m >> 5;
  int64_t o = 0, nm = 0;
  if (m < n_models) {
    o = offsets[m];
    nm = offsets[m + 1] - o;
  }
  const long long t = (nm + rs - 1) / rs, c = (nm + 31) / 32;
  long long it = t, ic = c;   // inclusive scans within the warp
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const long long ut = __shfl_up_sync(0xFFFFFFFFu, it, off);
    const long long uc = __shfl_up_sync(0xFFFFFFFFu, ic, off);
    if (lane >= off) {
      it += ut;
      ic += uc;
    }
  }
  if (lane == 31) {
    wt[warp] = it;
    wc[warp] = ic;
  }
  __syncthreads();
  long long bt = 0, bc = 0, tt = 0, tc = 0;
  for (int w = 0; w < 4; ++w) {
    if (w < warp) {
      bt += wt[w];
      bc += wc[w];
    }
    tt += wt[w];
    tc += wc[w];
  }
  if (m < n_models) {
    SegGroup& d = list[m];
    d.X = xs + o * ld_bytes;
    d.ld_bytes = ld_bytes;
    d.n = nm;
    d.ovf_ptr = nullptr;
    d.ovf_col = nullptr;
    d.ovf_add = nullptr;
    d.row_exp = nullptr;
    d.label = label + o;
    d.margin = margin + o;
    d.logpost = logpost ? logpost + 2 * o : nullptr;
    d.tile0 = bt + it - t;
    d.chunk0 = bc + ic - c;
    d.model = m;
    d.family = 0;
  }
  if (m < 3) {
    hdr[m].n_groups = m == 0 ? n_models : 0;
    hdr[m].pad = 0;
    hdr[m].tiles = m == 0 ? tt : 0;
    hdr[m].chunks = m == 0 ? tc : 0;
    hdr[m].pad2 = 0;
  }
}

// results back in the files' order
__global__ void k_gw_unpermute(const int64_t* order, int64_t n, const uint8_t* label_s,
                               const float* margin_s, const float* lp_s, uint8_t* label,
                               float* margin, float* logpost) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = order[r];
    label[i] = label_s[r];
    margin[i] = margin_s[r];
    if (logpost) {
      const float2 v = reinterpret_cast<const float2*>(lp_s)[r];
      logpost[2 * i] = v.x;
      logpost[2 * i + 1] = v.y;
    }
  }
}

// ---------------------------------------------------------------------------
// Fused group-wise scorer (u8 histograms, two-class models on k opcodes): one
// streaming pass over the full histograms in the files' order.  A pack staged
// once per block in shared memory holds, per model, W four-feature records
// {4 opcode columns (uint16), limb-0 bytes, limb-1 bytes} plus a plane of
// limb-2 words, its two-class header, and the model slot of each size group.
// The model's (opcode, weight) pairs are sorted by opcode and dealt so that
// the 8 lanes of a row, at each of their four byte gathers, read 8 neighbouring
// selected columns (few shared-memory bank conflicts); the k pairs are padded
// to a multiple of 32 with column 0 and zero weights.  The producer warp
// streams RS-row tiles of the histograms and each row's model slot
// (pipe.cuh); a row's lanes gather four counts per record and accumulate them
// against the limbs with dp4a.  Integer sums do not depend on the order, so
// the results are the bits of scoring the gathered row.
// ---------------------------------------------------------------------------
constexpr int kGwLPR = 8;                  // lanes per row
constexpr int kGwRPW = 32 / kGwLPR;        // rows per warp pass
constexpr int kGwNCW = 12;                 // consumer warps

struct GwArgs {
  const char* X;
  int64_t ld_bytes;
  int64_t n;
  const int64_t* sizes;
  int64_t bin_bytes;
  int n_bins, W, npad;     // records per model (a multiple of 8); padded pairs
  const void* pack;
  uint32_t pack_bytes, l2_off, hdr_off, map_off;
  uint8_t* label;
  float* margin;
  float* logpost;
  int want_lp, recheck;
  int* status;
  unsigned long long* marks;   // the call's n_rechecked: marked rows are counted here, or null
};

__global__ void __launch_bounds__((kGwNCW + 1) * 32, 1)
    k_score_gw(const GwArgs a, const PipeArgs p) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint64_t full[kMaxStages], empty[kMaxStages], tabbar;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / kGwLPR, li = lane % kGwLPR;
  const long long t0 = p.tiles * blockIdx.x / gridDim.x;
  const long long t1 = p.tiles * (blockIdx.x + 1) / gridDim.x;
  const long long ntl = t1 - t0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < p.S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kGwNCW);
    }
    mbar_init(&tabbar, 1);
  }
  __syncthreads();
  if (warp == kGwNCW) {
    const PipeSrc src{a.X, a.ld_bytes, a.n, nullptr, nullptr, nullptr, nullptr, a.pack,
                      a.status, a.sizes};
    const SizeMap zm{a.bin_bytes, a.n_bins, a.map_off};
    pipe_produce(src, p, sm, full, empty, &tabbar, t0, ntl, &zm);
    return;
  }
  if (!mbar_wait_bounded(&tabbar, 0)) {
    if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
    return;
  }
  const uint4* recs = reinterpret_cast<const uint4*>(sm);                       // m * W
  const uint32_t* l2s = reinterpret_cast<const uint32_t*>(sm + a.l2_off);       // m * W
  const C2Header* hdrs = reinterpret_cast<const C2Header*>(sm + a.hdr_off);

  int ra0 = 0, ra1 = 0, ra2 = 0, rmod = 0;
  uint32_t rt = 0;
  long long rrow = -1;
  int nres = 0;
  auto finish = [&]() {
    if (lane < nres) {
      const C2Header& H = hdrs[rmod];
      const long long D = ((long long)ra2 << 16) + ((long long)ra1 << 8) + (long long)ra0;
      const float Dsum = (float)D * H.inv_scale;
      const float d = Dsum + H.b;
      const float tau = c2_tau_u8((float)rt, Dsum, H.b, H.inv_scale, H.maxabs);
      const bool flag = c2_store(a.label, a.margin, a.logpost, a.want_lp, a.recheck, rrow, d, tau);
      if (a.marks) {
        // one atomic per warp, so that the recheck can skip its scan when no row is marked
        const unsigned act = __activemask();
        const unsigned mk = __ballot_sync(act, flag);
        if (mk && lane == __ffs(act) - 1) atomicAdd(a.marks, (unsigned long long)__popc(mk));
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
    const int32_t* slot = reinterpret_cast<const int32_t*>(st + p.y_off);   // model per row
    for (int r0 = warp * kGwRPW; r0 < nr; r0 += kGwNCW * kGwRPW) {
      if (nres + kGwRPW > 32) finish();
      const int r = r0 + grp;
      const bool valid = r < nr;
      const int m = valid ? slot[r] : 0;
      int c0 = 0, c1 = 0, c2 = 0;
      uint32_t ct = 0;
      if (valid) {
        const unsigned char* rp = st + (size_t)r * a.ld_bytes;
        const uint4* rg = recs + (size_t)m * a.W;
        const uint32_t* l2g = l2s + (size_t)m * a.W;
        // the four rows of a pass sit 1,024-byte multiples apart (the same
        // banks for the same column): each row group starts at another block
        // of records, so their gathers fall in different parts of the rows
        const int J = a.W / kGwLPR;
        int jj = grp % J;
        for (int it = 0; it < J; ++it, jj = jj + 1 == J ? 0 : jj + 1) {
          const int w = jj * kGwLPR + li;
          const uint4 rc = rg[w];
          const uint32_t x = (uint32_t)rp[rc.x & 0xFFFFu] | ((uint32_t)rp[rc.x >> 16] << 8) |
                             ((uint32_t)rp[rc.y & 0xFFFFu] << 16) |
                             ((uint32_t)rp[rc.y >> 16] << 24);
          c0 = dp4a_us(x, rc.z, c0);
          c1 = dp4a_us(x, rc.w, c1);
          c2 = dp4a_us(x, l2g[w], c2);
          ct = dp4a_uu(x, 0x01010101u, ct);
        }
        // the padding pairs read column 0 with zero weights: take them out of T
        if (li == 0) ct -= (uint32_t)a.npad * (uint32_t)rp[0];
      }
      const int k4 = sum4_transposed<kGwLPR>(c0, c1, c2, (int)ct, li);
      // lane nres + j takes row r0 + j of this pass from its group's first lane
      const int src = (lane - nres) * kGwLPR;
      const bool take = lane >= nres && lane < nres + kGwRPW && r0 + (lane - nres) < nr;
      const int sl = take ? src : 0;
      const int s0 = __shfl_sync(0xFFFFFFFFu, k4, sl);
      const int s1 = __shfl_sync(0xFFFFFFFFu, k4, sl + kGwLPR / 4);
      const int s2 = __shfl_sync(0xFFFFFFFFu, k4, sl + kGwLPR / 2);
      const uint32_t sT = (uint32_t)__shfl_sync(0xFFFFFFFFu, k4, sl + 3 * kGwLPR / 4);
      const int sm_ = __shfl_sync(0xFFFFFFFFu, m, sl);
      if (take) {
        ra0 = s0, ra1 = s1, ra2 = s2, rt = sT, rmod = sm_;
        rrow = row0 + r0 + (lane - nres);
      }
      nres += (nr - r0) < kGwRPW ? (nr - r0) : kGwRPW;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
    if (nres + kGwRPW > 32) finish();
  }
  finish();
}

}  // namespace nbg

using namespace nbg;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" nb_status nb_group_fallback(const int64_t* class_counts, int32_t n_bins, int32_t C,
                                       int64_t min_files, int32_t* model_of) {
  if (!class_counts || !model_of || n_bins < 1 || C < 1) {
    set_error("nb_group_fallback: bad arguments");
    return NB_EINVAL;
  }
  std::vector<char> trained((size_t)n_bins, 0);
  bool any = false;
  for (int g = 0; g < n_bins; ++g) {
    int64_t lo = class_counts[(size_t)g * C];
    for (int c = 1; c < C; ++c) {
      const int64_t v = class_counts[(size_t)g * C + c];
      lo = v < lo ? v : lo;
    }
    trained[g] = lo >= min_files;
    any = any || trained[g];
  }
  if (!any) {
    set_error("nb_group_fallback: no group has %lld files of every class", (long long)min_files);
    return NB_EINVAL;
  }
  for (int g = 0; g < n_bins; ++g) {
    int m = -1;
    for (int h = g; h < n_bins && m < 0; ++h)
      if (trained[h]) m = h;
    for (int h = g - 1; h >= 0 && m < 0; --h)
      if (trained[h]) m = h;
    model_of[g] = m;
  }
  return NB_OK;
}

extern "C" size_t nb_route_workspace(int64_t n, int32_t n_groups) {
  return route_workspace(n < 0 ? 0 : n, n_groups < 1 ? 1 : n_groups);
}

extern "C" nb_status nb_route(const int64_t* sizes, int64_t n, int64_t bin_bytes, int32_t n_bins,
                              const int32_t* model_of, int32_t n_groups, const int32_t* y,
                              int32_t C, int32_t* group, int64_t* order, int64_t* offsets,
                              int64_t* class_counts, void* workspace, size_t workspace_bytes,
                              int* status, void* cuda_stream) {
  if (n < 0 || bin_bytes < 1 || n_bins < 1 || n_groups < 1 || n_groups > kRouteMaxGroups ||
      (!model_of && n_groups != n_bins) || (n > 0 && (!sizes || !group)) || !offsets ||
      (class_counts && (!y || C < 1 || (int64_t)n_bins * C > kRouteMaxClassCells)) ||
      !status || workspace_bytes < route_workspace(n, n_groups) || !workspace) {
    set_error("nb_route: bad arguments (n_groups <= %d, n_bins * C <= %d with labels, "
              "workspace >= nb_route_workspace)", kRouteMaxGroups, kRouteMaxClassCells);
    return NB_EINVAL;
  }
  return launch_route(sizes, n, bin_bytes, n_bins, model_of, n_groups, y, C, group, order,
                      offsets, class_counts, static_cast<int64_t*>(workspace), status,
                      static_cast<cudaStream_t>(cuda_stream));
}

extern "C" nb_status nb_select_features(const nb_model* const* models, int32_t n_models,
                                        int32_t k, int32_t norm, int32_t* cols,
                                        void* cuda_stream) {
  if (!models || n_models < 1 || n_models > kSelMaxModels || !cols ||
      (norm != NB_SELECT_TOTAL && norm != NB_SELECT_FILES)) {
    set_error("nb_select_features: need 1 <= n_models <= %d, a norm, cols", kSelMaxModels);
    return NB_EINVAL;
  }
  SelArgs a{};
  int maxF = 0;
  for (int i = 0; i < n_models; ++i) {
    const nb_model* m = models[i];
    if (!m || m->kind != NB_MULTINOMIAL || m->C != 2 || k < 1 || k > m->F) {
      set_error("nb_select_features: model %d: needs a two-class multinomial model with "
                "F >= k >= 1", i);
      return NB_EINVAL;
    }
    a.m[i] = SelModel{m->d.counts, m->d.nc, m->F};
    if (m->F > maxF) maxF = m->F;
  }
  a.k = k;
  a.norm = norm;
  a.cols = cols;
  dim3 grid((unsigned)((maxF + kSelBlock - 1) / kSelBlock), (unsigned)n_models);
  count_launch();
  k_select_topk<<<grid, kSelThreads, 0, static_cast<cudaStream_t>(cuda_stream)>>>(a);
  NB_TRY_CUDA(cudaGetLastError(), "k_select_topk launch");
  return NB_OK;
}

extern "C" nb_status nb_gather(const void* X, nb_dtype dtype, int64_t ld, int32_t F,
                               int64_t n_src, int64_t n, const int64_t* order, const int32_t* group, int32_t n_groups,
                               const int32_t* cols, int32_t k, void* out, int64_t ld_out,
                               int* status, void* cuda_stream) {
  const int es = elem_size(dtype);
  if ((es != 1 && es != 4) || n < 0 || F < 1 || ld < F || k < 1 || ld_out < k ||
      (!order && n_src < n) || (n > 0 && n_src < 1) ||
      (!cols && k > F) || (n > 0 && (!X || !out)) || !status || (group && n_groups < 1) ||
      (es == 1 && (ld_out % 4) != 0) || (es == 1 && (reinterpret_cast<uintptr_t>(out) & 3)) ||
      (es == 4 && ((reinterpret_cast<uintptr_t>(out) | reinterpret_cast<uintptr_t>(X)) & 3))) {
    set_error("nb_gather: bad arguments (1- or 4-byte elements, ld >= F, ld_out >= k, "
              "u8 ld_out a multiple of 4, aligned buffers)");
    return NB_EINVAL;
  }
  return launch_gather(X, dtype, ld, F, n_src, n, order, group, group ? n_groups : 1, cols, k, out,
                       ld_out, status, static_cast<cudaStream_t>(cuda_stream));
}

// ---------------------------------------------------------------------------
// the group-wise scorer object
// ---------------------------------------------------------------------------
struct nb_groupwise {
  nb_batch* batch = nullptr;
  int n_models = 0, k = 0, F_full = 0, n_bins = 0, want_lp = 0, recheck = NB_RECHECK_LP;
  int64_t bin_bytes = 0, max_files = 0, ld_out = 0;
  nb_dtype dtype = NB_U8;
  void* mem = nullptr;        // one device allocation for everything below
  int32_t* model_of = nullptr;
  int32_t* cols = nullptr;
  int32_t* group = nullptr;
  int64_t* order = nullptr;
  int64_t* offsets = nullptr;
  int64_t* hist = nullptr;
  char* xs = nullptr;
  uint8_t* label_s = nullptr;
  float* margin_s = nullptr;
  float* lp_s = nullptr;
  int* status = nullptr;
  // fused scorer (u8): the shared-memory pack and its layout
  std::vector<const nb_model*> models;
  unsigned char* pack = nullptr;
  uint32_t pack_bytes = 0, l2_off = 0, hdr_off = 0, map_off = 0;
  int kp = 0, W = 0, npad = 0;
};

namespace nbg {
// batch.cu
nb_status batch_device_list(nb_batch* b, SegHeader** hdr, SegGroup** list0, int64_t* rs);
nb_status batch_create(const nb_model* const* models, int n_models, nb_dtype dtype,
                       int64_t max_ld, int max_groups, const nb_score_opts* opts, bool plain,
                       nb_batch** out);
nb_status batch_launch_device(nb_batch* b, cudaStream_t st, int64_t* n_rechecked);
nb_status launch_recheck_gw(const unsigned char* X, int64_t ld, int64_t n, const int64_t* sizes,
                            int64_t bin_bytes, int n_bins, int k, const int32_t* model_of,
                            const int32_t* cols, const nb_model* const* models, int n_models,
                            uint8_t* label, float* margin, float* logpost, int want_lp,
                            int64_t* n_rechecked, bool counted, cudaStream_t st);
}  // namespace nbg

extern "C" void nb_groupwise_destroy(nb_groupwise* g) {
  if (!g) return;
  if (g->batch) nb_batch_destroy(g->batch);
  if (g->mem) {
    cudaDeviceSynchronize();
    cudaFree(g->mem);
  }
  delete g;
}

extern "C" nb_status nb_groupwise_create(const nb_model* const* models, int32_t n_models,
                                         const int32_t* cols, int32_t k,
                                         const int32_t* model_of, int32_t n_bins,
                                         int64_t bin_bytes, int32_t F_full, nb_dtype dtype,
                                         int64_t max_files, const nb_score_opts* opts,
                                         nb_groupwise** out) {
  if (!out || !models || n_models < 1 || n_models > kSegMaxModels || !cols || !model_of ||
      n_bins < 1 || bin_bytes < 1 || F_full < 1 || k < 1 || k > F_full || max_files < 0 ||
      (dtype != NB_U8 && dtype != NB_F32)) {
    set_error("nb_groupwise_create: bad arguments (1 <= n_models <= %d, U8 or F32)",
              kSegMaxModels);
    return NB_EINVAL;
  }
  *out = nullptr;
  for (int i = 0; i < n_models; ++i)
    if (!models[i] || models[i]->kind != NB_MULTINOMIAL || models[i]->C != 2 ||
        models[i]->F != k) {
      set_error("nb_groupwise_create: model %d must be two-class multinomial with F = k", i);
      return NB_EINVAL;
    }
  for (int b = 0; b < n_bins; ++b)
    if (model_of[b] < 0 || model_of[b] >= n_models) {
      set_error("nb_groupwise_create: model_of[%d] = %d is not a model slot", b, model_of[b]);
      return NB_EINVAL;
    }
  nb_groupwise* g = new (std::nothrow) nb_groupwise();
  if (!g) {
    set_error("nb_groupwise_create: out of host memory");
    return NB_ENOMEM;
  }
  g->n_models = n_models;
  g->k = k;
  g->F_full = F_full;
  g->n_bins = n_bins;
  g->bin_bytes = bin_bytes;
  g->max_files = max_files;
  g->dtype = dtype;
  g->want_lp = opts ? opts->want_logpost : 0;
  g->recheck = opts ? (int)opts->recheck : (int)NB_RECHECK_LP;
  const int es = elem_size(dtype);
  g->ld_out = ((int64_t)k * es + 15) / 16 * 16 / es;   // rows 16-byte aligned
  auto fail = [&](nb_status s) {
    nb_groupwise_destroy(g);
    return s;
  };
  nb_status s = batch_create(models, n_models, dtype, g->ld_out, n_models, opts, true, &g->batch);
  if (s != NB_OK) return fail(s);
  // one allocation, 256-byte aligned pieces
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  };
  const int64_t nf = max_files > 0 ? max_files : 1;
  const size_t o_model = take(sizeof(int32_t) * n_bins);
  const size_t o_cols = take(sizeof(int32_t) * (size_t)n_models * k);
  const size_t o_group = take(sizeof(int32_t) * nf);
  const size_t o_order = take(sizeof(int64_t) * nf);
  const size_t o_offs = take(sizeof(int64_t) * (n_models + 1));
  const size_t o_hist = take(route_workspace(nf, n_models));
  const size_t o_xs = take((size_t)nf * g->ld_out * es);
  const size_t o_lab = take(nf);
  const size_t o_mar = take(sizeof(float) * nf);
  const size_t o_lp = take(g->want_lp ? sizeof(float) * 2 * nf : 0);
  const size_t o_st = take(sizeof(int));
  // fused-scorer pack: records (16 B per four features), limb-2 words, headers,
  // size group -> slot bytes; 16-byte aligned sections
  g->kp = models[0]->F_pad;
  g->models.assign(models, models + n_models);
  g->W = (k + 31) / 32 * 8;
  g->npad = 4 * g->W - k;
  g->l2_off = (uint32_t)(16 * g->W * n_models);
  g->hdr_off = g->l2_off + (uint32_t)(4 * g->W * n_models + 15) / 16 * 16;
  g->map_off = g->hdr_off + (uint32_t)(sizeof(C2Header) * n_models);
  g->pack_bytes = g->map_off + (uint32_t)(n_bins + 15) / 16 * 16;
  const size_t o_pack = dtype == NB_U8 ? take(g->pack_bytes) : 0;
  std::vector<int32_t> hcols((size_t)n_models * k);
  cudaError_t e = cudaMemcpy(hcols.data(), cols, sizeof(int32_t) * hcols.size(), cudaMemcpyDefault);
  if (e != cudaSuccess) return fail(cuda_status(e, "memcpy(cols)"));
  for (size_t i = 0; i < hcols.size(); ++i)
    if (hcols[i] < 0 || hcols[i] >= F_full) {
      set_error("nb_groupwise_create: cols[%zu] = %d is not an opcode column", i, hcols[i]);
      return fail(NB_EINVAL);
    }
  e = cudaMalloc(&g->mem, off);
  if (e != cudaSuccess) return fail(cuda_status(e, "cudaMalloc(groupwise)"));
  char* base = static_cast<char*>(g->mem);
  g->model_of = reinterpret_cast<int32_t*>(base + o_model);
  g->cols = reinterpret_cast<int32_t*>(base + o_cols);
  g->group = reinterpret_cast<int32_t*>(base + o_group);
  g->order = reinterpret_cast<int64_t*>(base + o_order);
  g->offsets = reinterpret_cast<int64_t*>(base + o_offs);
  g->hist = reinterpret_cast<int64_t*>(base + o_hist);
  g->xs = base + o_xs;
  g->label_s = reinterpret_cast<uint8_t*>(base + o_lab);
  g->margin_s = reinterpret_cast<float*>(base + o_mar);
  g->lp_s = g->want_lp ? reinterpret_cast<float*>(base + o_lp) : nullptr;
  g->status = reinterpret_cast<int*>(base + o_st);
  NB_TRY_CUDA(cudaMemset(g->mem, 0, off), "memset(groupwise)");
  e = cudaMemcpy(g->model_of, model_of, sizeof(int32_t) * n_bins, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(g->cols, hcols.data(), sizeof(int32_t) * hcols.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(cuda_status(e, "memcpy(groupwise tables)"));
  if (dtype == NB_U8) {
    g->pack = reinterpret_cast<unsigned char*>(base + o_pack);
    const int W = g->W, kp = g->kp;
    std::vector<uint32_t> hrec((size_t)n_models * W * 4, 0u), hl2((size_t)n_models * W, 0u);
    std::vector<unsigned char> hl(3 * (size_t)kp);
    std::vector<int> ord(k);
    for (int m = 0; m < n_models && e == cudaSuccess; ++m) {
      // the model's three limb planes (feature t at byte t of each)
      e = cudaMemcpy(hl.data(), models[m]->d.limbs, hl.size(), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) break;
      const int32_t* cm = hcols.data() + (size_t)m * k;
      for (int t = 0; t < k; ++t) ord[t] = t;
      std::stable_sort(ord.begin(), ord.end(), [cm](int u, int v) { return cm[u] < cm[v]; });
      for (int pos = 0; pos < 4 * W; ++pos) {
        // sorted pair pos goes to record j * 8 + lane, byte q, where
        // pos = 32 j + 8 q + lane
        const int j = pos / 32, q = (pos % 32) / 8, ln = pos % 8;
        const size_t r = (size_t)m * W + (size_t)j * 8 + ln;
        uint32_t col = 0, l0 = 0, l1 = 0, l2 = 0;
        if (pos < k) {
          const int t = ord[pos];
          col = (uint32_t)cm[t];
          l0 = hl[t];
          l1 = hl[(size_t)kp + t];
          l2 = hl[2 * (size_t)kp + t];
        }
        hrec[4 * r + (q >> 1)] |= col << (16 * (q & 1));
        hrec[4 * r + 2] |= l0 << (8 * q);
        hrec[4 * r + 3] |= l1 << (8 * q);
        hl2[r] |= l2 << (8 * q);
      }
      e = cudaMemcpy(g->pack + g->hdr_off + sizeof(C2Header) * m, models[m]->d.c2,
                     sizeof(C2Header), cudaMemcpyDeviceToDevice);
    }
    std::vector<unsigned char> hmap((size_t)n_bins);
    for (int b = 0; b < n_bins; ++b) hmap[b] = (unsigned char)model_of[b];
    if (e == cudaSuccess)
      e = cudaMemcpy(g->pack, hrec.data(), 4 * hrec.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(g->pack + g->l2_off, hl2.data(), 4 * hl2.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(g->pack + g->map_off, hmap.data(), hmap.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(cuda_status(e, "memcpy(groupwise pack)"));
  }
  *out = g;
  return NB_OK;
}

// The fused path (k_score_gw + k_recheck_gw): u8 histograms, 16-byte aligned
// rows, and a pack plus two row stages that fit in shared memory; else
// NB_EUNSUPPORTED and the caller routes, gathers and batches.
static nb_status groupwise_fused(nb_groupwise* g, const void* X, int64_t ld, const int64_t* sizes,
                                 int64_t n, uint8_t* label, float* margin, float* logpost,
                                 cudaStream_t st, int64_t* n_rechecked) {
  if (!g->pack || (reinterpret_cast<uintptr_t>(X) & 15) != 0 || (ld % 16) != 0 || ld > 8192)
    return NB_EUNSUPPORTED;
  // the largest stage of 48, 32, 24 or 16 rows of which two fit beside the pack
  PipeArgs p{};
  const uint32_t budget = 220u * 1024u;
  int rs = 0;
  for (int cand : {48, 32, 24, 16}) {
    pipe_layout(p, cand, 1, ld, false, true, g->pack_bytes, n);
    if (p.stages_off + 2 * p.stage_bytes <= budget) {
      rs = cand;
      break;
    }
  }
  if (rs == 0) return NB_EUNSUPPORTED;
  int S = (int)((budget - p.stages_off) / p.stage_bytes);
  S = S > kMaxStages ? kMaxStages : S;
  pipe_layout(p, rs, S, ld, false, true, g->pack_bytes, n);
  const int smem = (int)(p.stages_off + (uint32_t)S * p.stage_bytes);
  if (n_rechecked) NB_TRY_CUDA(cudaMemsetAsync(n_rechecked, 0, sizeof(int64_t), st), "memset");
  if (n == 0) return NB_OK;
  GwArgs a{};
  a.X = static_cast<const char*>(X);
  a.ld_bytes = ld;
  a.n = n;
  a.sizes = sizes;
  a.bin_bytes = g->bin_bytes;
  a.n_bins = g->n_bins;
  a.W = g->W;
  a.npad = g->npad;
  a.pack = g->pack;
  a.pack_bytes = g->pack_bytes;
  a.l2_off = g->l2_off;
  a.hdr_off = g->hdr_off;
  a.map_off = g->map_off;
  a.label = label;
  a.margin = margin;
  a.logpost = g->want_lp ? logpost : nullptr;
  a.want_lp = g->want_lp;
  a.recheck = g->recheck;
  a.status = g->status;
  const bool counted = n_rechecked != nullptr;
  a.marks = counted ? reinterpret_cast<unsigned long long*>(n_rechecked) : nullptr;
  if (smem > kSmemOptIn)   // per device and function: set at every launch
    NB_TRY_CUDA(cudaFuncSetAttribute(k_score_gw, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                "cudaFuncSetAttribute(k_score_gw)");
  int occ = 0;
  NB_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_score_gw, (kGwNCW + 1) * 32,
                                                            smem),
              "occupancy(k_score_gw)");
  if (occ < 1) return NB_EUNSUPPORTED;
  long long blocks = (long long)num_sms() * occ;
  if (blocks > p.tiles) blocks = p.tiles;
  count_launch();
  k_score_gw<<<(unsigned)blocks, (kGwNCW + 1) * 32, smem, st>>>(a, p);
  NB_TRY_CUDA(cudaGetLastError(), "k_score_gw launch");
  return launch_recheck_gw(static_cast<const unsigned char*>(X), ld, n, sizes, g->bin_bytes,
                           g->n_bins, g->k, g->model_of, g->cols, g->models.data(), g->n_models,
                           label, margin, g->want_lp ? logpost : nullptr, g->want_lp, n_rechecked,
                           counted, st);
}

extern "C" nb_status nb_groupwise_classify(nb_groupwise* g, const void* X, int64_t ld,
                                           const int64_t* sizes, int64_t n, uint8_t* label,
                                           float* margin, float* logpost, void* cuda_stream,
                                           int64_t* n_rechecked) {
  if (!g || n < 0 || n > g->max_files || ld < g->F_full ||
      (n > 0 && (!X || !sizes || !label || !margin || (g->want_lp && !logpost)))) {
    set_error("nb_groupwise_classify: bad arguments (n <= max_files, ld >= F)");
    return NB_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  {
    nb_status fs = groupwise_fused(g, X, ld, sizes, n, label, margin, logpost, st, n_rechecked);
    if (fs != NB_EUNSUPPORTED) return fs;
  }
  nb_status s = launch_route(sizes, n, g->bin_bytes, g->n_bins, g->model_of, g->n_models,
                             nullptr, 0, g->group, g->order, g->offsets, nullptr, g->hist,
                             g->status, st);
  if (s != NB_OK) return s;
  s = launch_gather(X, g->dtype, ld, g->F_full, n, n, g->order, g->group, g->n_models, g->cols,
                    g->k, g->xs, g->ld_out, g->status, st);
  if (s != NB_OK) return s;
  SegHeader* hdr = nullptr;
  SegGroup* list0 = nullptr;
  int64_t rs = 1;
  s = batch_device_list(g->batch, &hdr, &list0, &rs);
  if (s != NB_OK) return s;
  count_launch();
  k_gw_worklist<<<1, 128, 0, st>>>(hdr, list0, g->n_models, g->offsets, g->xs,
                                  g->ld_out * elem_size(g->dtype), g->label_s, g->margin_s,
                                  g->want_lp ? g->lp_s : nullptr, rs);
  NB_TRY_CUDA(cudaGetLastError(), "k_gw_worklist launch");
  s = batch_launch_device(g->batch, st, n_rechecked);
  if (s != NB_OK) return s;
  if (n > 0) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)num_sms() * 8) blocks = (int64_t)num_sms() * 8;
    count_launch();
    k_gw_unpermute<<<(unsigned)blocks, 256, 0, st>>>(g->order, n, g->label_s, g->margin_s,
                                                    g->want_lp ? g->lp_s : nullptr, label,
                                                    margin, g->want_lp ? logpost : nullptr);
    NB_TRY_CUDA(cudaGetLastError(), "k_gw_unpermute launch");
  }
  return NB_OK;
}

extern "C" nb_status nb_groupwise_status(nb_groupwise* g, int* host_status) {
  if (!g || !host_status) {
    set_error("nb_groupwise_status: bad arguments");
    return NB_EINVAL;
  }
  NB_TRY_CUDA(cudaMemcpy(host_status, g->status, sizeof(int), cudaMemcpyDeviceToHost),
              "memcpy(status)");
  return NB_OK;
}
