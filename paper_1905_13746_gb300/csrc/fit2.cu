// Two-class multinomial fit reduction (Sec. 4, "trained the model"):
//   n_c = #{i : y_i = c},  N_cj = sum_{i : y_i = c} x_ij   (exact, uint64)
// streamed through the shared-memory stage pipeline of pipe.cuh.
//
// Rows are read in their natural order (no bucketing by class): a consumer
// warp works on one row at a time with its lanes over the row's 16-byte
// vectors, so the row's class is the same for the whole warp and selects
// which of two per-lane accumulator sets receives the row.  u8 rows are
// summed as packed 16-bit lanes (even and odd bytes of each word), which
// cannot overflow before 257 rows; every 256 rows of a warp the sums move into
// a per-block histogram in shared memory, which is added to the global uint64
// counts once per block.  Overflow bounds: u8 (at most 255 + 65,535 per
// element) and u16 rows keep 32-bit block sums, with at most 32,768 rows per
// block; FP32 / BF16 / FP8 counts (below 2^24) flush their 32-bit lane sums
// every 255 rows into a 64-bit block histogram.  Integer sums are exact in
// any order.
//
// The overflow list of u8 storage (counts above 255) is not staged with the
// rows: a second, short kernel (k_fit2_ovf) adds its entries to the counts,
// so that the row pipeline streams plain u8 rows.
#include <type_traits>

#include "pipe.cuh"
#include "score2.cuh"

namespace nbg {

struct Fit2Args {
  const char* X;
  long long ld_bytes;
  long long n;
  int F;
  int F_pad;
  int nvec_row;
  const int32_t* y;
  const int8_t* row_exp;
  unsigned long long* counts;   // 2 x F
  unsigned long long* nc;       // 2
  int* status;
};

__device__ __forceinline__ uint32_t even_bytes(uint32_t w) { return w & 0x00FF00FFu; }
__device__ __forceinline__ uint32_t odd_bytes(uint32_t w) { return __byte_perm(w, 0u, 0x4341u); }

__device__ __forceinline__ uint32_t count_of(float v, int* status) {
  if (!(v >= 0.f) || v != floorf(v) || v >= 16777216.f) {
    atomicOr(status, ST_BAD_VALUE);
    return 0u;
  }
  return (uint32_t)v;
}

// block histogram word: 32 bits where the bounds above allow it, else 64
template <int DT>
using Fit2Hist = typename std::conditional<DT == NB_U8 || DT == NB_U16, unsigned int,
                                           unsigned long long>::type;
// rows between flushes of a warp's 32-bit lane sums
template <int DT>
constexpr int fit2_flush_rows() {
  return DT == NB_U8 ? 256 : (DT == NB_U16 ? 32768 : 255);
}
constexpr long long kFit2BlockRows = 32768;   // most rows of one block (32-bit sums)

// move a warp's per-lane sums into the block histogram and clear them
template <int DT, int KV, int NA, int EPV>
__device__ __forceinline__ void fit2_flush(uint32_t (&acc)[2][KV][NA], Fit2Hist<DT>* hist,
                                           int F, int F_pad, int lane, int nv) {
#pragma unroll
  for (int kv = 0; kv < KV; ++kv) {
    const int v = lane + 32 * kv;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
#pragma unroll
      for (int e = 0; e < EPV; ++e) {
        uint32_t val;
        if (DT == NB_U8) {
          const int w = e >> 2, b = e & 3;
          const uint32_t pk = acc[c][kv][2 * w + (b & 1)];
          val = (b >> 1) ? (pk >> 16) : (pk & 0xFFFFu);
        } else {
          val = acc[c][kv][e];
        }
        const int j = v * EPV + e;
        if (v < nv && val && j < F) atomicAdd(&hist[c * F_pad + j], (Fit2Hist<DT>)val);
      }
#pragma unroll
      for (int e = 0; e < NA; ++e) acc[c][kv][e] = 0u;
    }
  }
}

// FULL: every lane's KV vectors lie inside the row (no bound or tail checks).
template <int DT, int KV, int NCW, bool FULL>
__global__ void __launch_bounds__((NCW + 1) * 32, NCW == 8 ? 2 : 1) k_fit2_pipe(const Fit2Args f, const PipeArgs p) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint64_t full[kMaxStages], empty[kMaxStages], tabbar;
  __shared__ unsigned int ncount[2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long t0 = p.tiles * blockIdx.x / gridDim.x;
  const long long t1 = p.tiles * (blockIdx.x + 1) / gridDim.x;
  const long long ntl = t1 - t0;
  Fit2Hist<DT>* hist = reinterpret_cast<Fit2Hist<DT>*>(sm);   // [2][F_pad]

  for (int k = threadIdx.x; k < 2 * f.F_pad; k += blockDim.x) hist[k] = 0;
  if (threadIdx.x == 0) {
    ncount[0] = ncount[1] = 0u;
    for (int s = 0; s < p.S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NCW);
    }
    mbar_init(&tabbar, 1);
  }
  __syncthreads();

  if (warp == NCW) {
    const PipeSrc src{f.X, f.ld_bytes, f.n, nullptr, nullptr, nullptr, f.y, nullptr, f.status};
    pipe_produce(src, p, sm, full, empty, &tabbar, t0, ntl);
    return;
  }

  // per-lane sums for vectors v = lane + 32 kv, one set per class
  constexpr int NA = DT == NB_U8 ? 8 : (DT == NB_F32 ? 4 : (DT == NB_FP8E4M3 ? 16 : 8));
  uint32_t acc[2][KV][NA];
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int kv = 0; kv < KV; ++kv)
#pragma unroll
      for (int e = 0; e < NA; ++e) acc[c][kv][e] = 0u;
  const int nv = f.nvec_row;
  constexpr int EPV = DT == NB_F32 ? 4 : ((DT == NB_U16 || DT == NB_BF16) ? 8 : 16);
  const int esz = 16 / EPV;
  // byte masks of a partial last vector, computed once
  const int keep = f.F * esz - 16 * (nv - 1);
  uint32_t tm[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int vb = keep - 4 * q;
    vb = vb < 0 ? 0 : (vb > 4 ? 4 : vb);
    tm[q] = vb >= 4 ? 0xFFFFFFFFu : ((1u << (8 * vb)) - 1u);
  }
  const int tail_v = (!FULL && f.F < nv * EPV) ? nv - 1 : -1;
  uint32_t cnt0 = 0u, cnt1 = 0u;   // rows per class (lane 0); scalars, not an array indexed by c
  int since_flush = 0;
  bool dead = false;   // a wait ran out: skip to the common exit (the named barrier)


  for (long long k = 0; k < ntl; ++k) {
    const int s = (int)(k % p.S);
    const uint32_t ph = (uint32_t)((k / p.S) & 1);
    if (dead || !mbar_wait_bounded(&full[s], ph)) {
      if (lane == 0) atomicOr(f.status, ST_TIMEOUT);
      dead = true;
      break;
    }
    const unsigned char* st = sm + p.stages_off + (size_t)s * p.stage_bytes;
    const StageMeta m = *reinterpret_cast<const StageMeta*>(st + p.meta_off);
    const int32_t* sy = reinterpret_cast<const int32_t*>(st + p.y_off);
    for (int rr = warp; rr < m.nr; rr += NCW) {
      const int c = sy[rr];
      if (c < 0 || c > 1) {
        if (lane == 0) atomicOr(f.status, ST_BAD_LABEL);
        continue;
      }
      ++since_flush;
      if (lane == 0) {
        cnt0 += c == 0;
        cnt1 += c == 1;
      }
      const unsigned char* rp = st + (size_t)rr * f.ld_bytes;
      const int8_t ex = (DT == NB_FP8E4M3 && f.row_exp) ? f.row_exp[m.row0 + rr] : (int8_t)0;
#pragma unroll
      for (int kv = 0; kv < KV; ++kv) {
        const int v = lane + 32 * kv;
        if (!FULL && v >= nv) continue;
        const uint4 xv = *reinterpret_cast<const uint4*>(rp + (size_t)v * 16);
        uint32_t w[4] = {xv.x, xv.y, xv.z, xv.w};
        if (!FULL && v == tail_v) {
#pragma unroll
          for (int q = 0; q < 4; ++q) w[q] &= tm[q];
        }
        const uint4 x = make_uint4(w[0], w[1], w[2], w[3]);
        // class-uniform branch: c is the same for the whole warp
        if (DT == NB_U8) {
          if (c == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              acc[0][kv][2 * q] += even_bytes(w[q]);
              acc[0][kv][2 * q + 1] += odd_bytes(w[q]);
            }
          } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              acc[1][kv][2 * q] += even_bytes(w[q]);
              acc[1][kv][2 * q + 1] += odd_bytes(w[q]);
            }
          }
        } else if (DT == NB_U16) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (c == 0) {
              acc[0][kv][2 * q] += w[q] & 0xFFFFu;
              acc[0][kv][2 * q + 1] += w[q] >> 16;
            } else {
              acc[1][kv][2 * q] += w[q] & 0xFFFFu;
              acc[1][kv][2 * q + 1] += w[q] >> 16;
            }
          }
        } else {
          float val[EPV];
          Decode<DT>::run(x, val);
          const float sc = DT == NB_FP8E4M3 ? exp2f((float)ex) : 1.f;
#pragma unroll
          for (int e = 0; e < EPV; ++e) {
            const uint32_t u = count_of(val[e] * sc, f.status);
            if (c == 0) acc[0][kv][e] += u; else acc[1][kv][e] += u;
          }
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
    // a warp takes at most ceil(RS / NCW) rows per stage, so flushing here
    // keeps the packed 16-bit lanes below 257 rows
    if (since_flush + (p.RS + NCW - 1) / NCW > fit2_flush_rows<DT>()) {
      fit2_flush<DT, KV, NA, EPV>(acc, hist, f.F, f.F_pad, lane, nv);
      since_flush = 0;
    }
  }
  fit2_flush<DT, KV, NA, EPV>(acc, hist, f.F, f.F_pad, lane, nv);
  if (lane == 0) {
    if (cnt0) atomicAdd(&ncount[0], cnt0);
    if (cnt1) atomicAdd(&ncount[1], cnt1);
  }
  // consumer warps only (the producer has left): named barrier 1
  asm volatile("bar.sync 1, %0;" ::"r"(NCW * 32) : "memory");
  for (int j = threadIdx.x; j < 2 * f.F_pad; j += NCW * 32) {
    const int c = j / f.F_pad, jj = j % f.F_pad;
    const Fit2Hist<DT> v = hist[j];
    if (v && jj < f.F) atomicAdd(&f.counts[(long long)c * f.F + jj], (unsigned long long)v);
  }
  if (threadIdx.x < 2 && ncount[threadIdx.x])
    atomicAdd(&f.nc[threadIdx.x], (unsigned long long)ncount[threadIdx.x]);
}

// Overflow entries of u8 rows (Sec. 4 counts; the part of each count above
// 255), after the row pipeline.  A warp takes 32 rows and walks their entries
// as one contiguous range (coalesced loads, 32 entries per pass); the row of
// an entry is the last of the 32 row pointers at or below it, found by a
// five-step search over the pointers held one per lane.  Entries go to 32-bit
// (class, column) bins in shared memory, and the bins to the uint64 counts
// once per block.  Rows labelled outside {0, 1} were flagged by the row kernel
// and are skipped.  A bin takes at most 65,535 per row and a block at most
// kFit2BlockRows rows, so 32 bits do not overflow.
constexpr int kOvfThreads = 512;

__global__ void __launch_bounds__(kOvfThreads) k_fit2_ovf(const int64_t* ptr, const uint16_t* col,
                                                          const uint16_t* add, const int32_t* y,
                                                          int64_t n, int F,
                                                          unsigned long long* counts, int* status) {
  extern __shared__ unsigned int bins[];   // [2][F]
  for (int k = threadIdx.x; k < 2 * F; k += blockDim.x) bins[k] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t nchunk = (n + 31) / 32;
  const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t ch = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); ch < nchunk;
       ch += wstride) {
    const int64_t r0 = ch * 32;
    const int nr = (int)min((int64_t)32, n - r0);
    // lane l holds the first entry of row r0 + l (lanes past the last row: the end)
    const int64_t pl = ptr[r0 + (lane < nr ? lane : nr)];
    const int64_t pend = ptr[r0 + nr];
    const int yl = lane < nr ? y[r0 + lane] : -1;
    const int64_t e0 = __shfl_sync(0xFFFFFFFFu, pl, 0);
    for (int64_t base = e0; base < pend; base += 32) {
      const int64_t e = base + lane;
      const bool valid = e < pend;
      uint32_t j = 0u, a = 0u;
      if (valid) {
        j = col[e];
        a = add[e];
      }
      int lo = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int64_t v = __shfl_sync(0xFFFFFFFFu, pl, lo + step);
        if (v <= e) lo += step;
      }
      const int c = __shfl_sync(0xFFFFFFFFu, yl, lo);
      if (valid && (c == 0 || c == 1)) {
        if (j < (uint32_t)F)
          atomicAdd(&bins[c * F + j], a);
        else
          atomicOr(status, ST_OVF_RANGE);
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 2 * F; k += blockDim.x)
    if (bins[k]) atomicAdd(&counts[k], (unsigned long long)bins[k]);
  // launched programmatically after the row kernel, whose output this kernel
  // does not read: it starts on SMs as row blocks leave, and waits for the row
  // kernel only here, so that its own completion (which the finish kernel
  // waits for) implies the row kernel's
  pdl_wait();
}

static nb_status launch_fit2_ovf(nb_model* m, const nb_aux* aux, const int32_t* y, int64_t n,
                                 cudaStream_t st) {
  const int F = m->F;
  const int smem = (int)(2 * sizeof(unsigned int) * (size_t)F);   // F <= 8,192 here
  if (smem > kSmemOptIn)   // per device and function: set at every launch
    NB_TRY_CUDA(cudaFuncSetAttribute(k_fit2_ovf, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                "cudaFuncSetAttribute(k_fit2_ovf)");
  // 32 rows per warp pass, four blocks per SM; at most kFit2BlockRows rows per block
  const long long rows_per_block = 32LL * (kOvfThreads / 32);
  long long blocks = (n + rows_per_block - 1) / rows_per_block;
  const long long cap = (long long)num_sms() * 4;
  if (blocks > cap) blocks = cap;
  if (blocks < (n + kFit2BlockRows - 1) / kFit2BlockRows) blocks = (n + kFit2BlockRows - 1) / kFit2BlockRows;
  count_launch();
  NB_TRY_CUDA(launch_pdl(k_fit2_ovf, dim3((unsigned)blocks), dim3(kOvfThreads), (size_t)smem, st,
                         aux->ovf_ptr, aux->ovf_col, aux->ovf_add, y, (int64_t)n, F,
                         reinterpret_cast<unsigned long long*>(m->d.counts), m->d.status),
              "k_fit2_ovf launch");
  return NB_OK;
}

template <int DT, int KV, int kFitNCW, bool FULL>
static nb_status run_fit2(const Fit2Args& f, const PipeArgs& p, int smem, cudaStream_t st) {
  auto kern = k_fit2_pipe<DT, KV, kFitNCW, FULL>;
  if (smem > kSmemOptIn)   // per device and function: set at every launch
    NB_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                "cudaFuncSetAttribute(fit2)");
  int occ = 0;
  NB_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, (kFitNCW + 1) * 32, smem),
              "occupancy(fit2)");
  if (occ < 1) return NB_EUNSUPPORTED;
  long long blocks = (long long)num_sms() * occ;
  const long long need = (f.n + kFit2BlockRows - 1) / kFit2BlockRows;   // 32-bit block sums
  if (blocks < need) blocks = need;
  if (blocks > p.tiles) blocks = p.tiles;
  count_launch();
  kern<<<(unsigned)blocks, (kFitNCW + 1) * 32, smem, st>>>(f, p);
  NB_TRY_CUDA(cudaGetLastError(), "k_fit2_pipe launch");
  return NB_OK;
}

// Two-class count reduction through the pipeline; NB_EUNSUPPORTED when the
// shape does not fit (the caller then uses the class-bucketed kernels).
nb_status launch_fit2_pipe(nb_model* m, const void* X, nb_dtype dt, int64_t n, int64_t ld,
                           const int32_t* y, const nb_aux* aux, cudaStream_t st) {
  if (m->C != 2 || n <= 0) return NB_EUNSUPPORTED;
  const int es = elem_size(dt);
  Fit2Args f{};
  f.X = static_cast<const char*>(X);
  f.ld_bytes = ld * es;
  f.n = n;
  f.F = m->F;
  f.F_pad = m->F_pad;
  f.nvec_row = (m->F * es + 15) / 16;
  f.y = y;
  f.row_exp = aux ? aux->row_exp : nullptr;
  f.counts = reinterpret_cast<unsigned long long*>(m->d.counts);
  f.nc = reinterpret_cast<unsigned long long*>(m->d.nc);
  f.status = m->d.status;
  const bool aligned = ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && (f.ld_bytes % 16 == 0);
  const int kv = (f.nvec_row + 31) / 32;
  const int kv_max = dt == NB_F32 ? 8 : (dt == NB_FP8E4M3 ? 2 : 4);
  if (!aligned || kv > kv_max || f.ld_bytes > 8192) return NB_EUNSUPPORTED;
  // eight consumer warps and two blocks per SM for u8 rows of <= 64 vectors
  const int ncw = (dt == NB_U8 && kv <= 2) ? 8 : 12;
  // eight consumers (two blocks per SM): two stages of up to 48 rows (~48 KB);
  // twelve: stages of ~24 KB, rows of 2 KB or more one row per consumer warp per
  // stage (as many stages as fit, at least two), so that no warp idles
  int rs = (int)((ncw == 8 ? 49152 : 24576) / f.ld_bytes);
  rs = rs > (ncw == 8 ? 48 : 32) ? (ncw == 8 ? 48 : 32) : (rs < 1 ? 1 : rs);
  if (f.ld_bytes >= 2048 && rs < ncw) rs = ncw;
  PipeArgs p{};
  const uint32_t hist_bytes = (uint32_t)((dt == NB_U8 || dt == NB_U16 ? 8 : 16) * m->F_pad);
  pipe_layout(p, rs, 4, f.ld_bytes, false, true, hist_bytes, n);
  int S = ncw == 8 ? 2 : 4;
  while (S > 2 && p.stages_off + (uint32_t)S * p.stage_bytes > 220u * 1024u) --S;
  pipe_layout(p, rs, S, f.ld_bytes, false, true, hist_bytes, n);
  const int smem = (int)(p.stages_off + (uint32_t)p.S * p.stage_bytes);
  if (smem > 220 * 1024) return NB_EUNSUPPORTED;
  nb_status s = NB_EUNSUPPORTED;
  // rows that fill every lane's vectors exactly take the branch-free kernel
  const bool full = f.nvec_row == 32 * kv && (m->F * es) % 16 == 0;
#define NB_FIT2_CASE(D, K)                                                              \
  if (dt == D && kv == K)                                                               \
    s = ncw == 8 ? (full ? run_fit2<D, K, 8, true>(f, p, smem, st)                      \
                         : run_fit2<D, K, 8, false>(f, p, smem, st))                    \
                 : (full ? run_fit2<D, K, 12, true>(f, p, smem, st)                     \
                         : run_fit2<D, K, 12, false>(f, p, smem, st));                  \
  else
  NB_FIT2_CASE(NB_U8, 1) NB_FIT2_CASE(NB_U8, 2) NB_FIT2_CASE(NB_U8, 3) NB_FIT2_CASE(NB_U8, 4)
  NB_FIT2_CASE(NB_U16, 1) NB_FIT2_CASE(NB_U16, 2) NB_FIT2_CASE(NB_U16, 3)
  NB_FIT2_CASE(NB_U16, 4)
  NB_FIT2_CASE(NB_BF16, 1) NB_FIT2_CASE(NB_BF16, 2) NB_FIT2_CASE(NB_BF16, 3)
  NB_FIT2_CASE(NB_BF16, 4)
  NB_FIT2_CASE(NB_F32, 1) NB_FIT2_CASE(NB_F32, 2) NB_FIT2_CASE(NB_F32, 3) NB_FIT2_CASE(NB_F32, 4)
  NB_FIT2_CASE(NB_F32, 5) NB_FIT2_CASE(NB_F32, 6) NB_FIT2_CASE(NB_F32, 7) NB_FIT2_CASE(NB_F32, 8)
  NB_FIT2_CASE(NB_FP8E4M3, 1) NB_FIT2_CASE(NB_FP8E4M3, 2)
  {}
#undef NB_FIT2_CASE
  if (s != NB_OK) return s;
  if (dt == NB_U8 && aux && aux->ovf_ptr) return launch_fit2_ovf(m, aux, y, n, st);
  return NB_OK;
}

}  // namespace nbg
