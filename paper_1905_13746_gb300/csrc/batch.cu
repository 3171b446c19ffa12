// Batches of file groups: the host side of the segmented launches.
//
// A batch holds the resident models (two-class ones go to the pipelined
// two-class kernel; the others to the tensor-core kernel when the group
// allows it -- u8 rows, 16-byte aligned, a model with tensor tables -- else to
// the general kernel), a device work list (three headers, three descriptor
// lists and the tensor maps of the tensor-core groups) and two pinned host
// copies of it.
// nb_batch_score writes the groups into the next host copy, copies it to the
// device and launches (or replays the captured graphs of) the scoring kernels
// and the FP64 recheck: a fixed number of launches whatever the number of
// groups.
#include <string.h>

#include <new>
#include <vector>

#include "pipe.cuh"
#include "seg.cuh"

namespace nbg {

constexpr int kFamilies = 3;

struct WorkList {   // device and host layout of one work list buffer
  SegHeader hdr[kFamilies];
  // followed by SegGroup lists[kFamilies][max_groups], then 128-byte tensor
  // maps [max_groups] (128-byte aligned)
};

}  // namespace nbg

using namespace nbg;

struct nb_batch {
  nb_dtype dtype;
  int F, F_pad;
  int max_groups;
  int want_lp, recheck;
  bool plain = false;   // groups carry no side arrays (longer stages)
  // family 0 (two-class pipelined), 1 (general) and 2 (tensor-core) models;
  // a many-class slot sits in family 1 and, with tensor tables, in family 2
  std::vector<const nb_model*> fam[kFamilies];
  std::vector<int> slot_family, slot_index, slot_index2;   // slot -> family, indices
  size_t maps_off = 0;
  // two-class launch plan
  PipeArgs plan{};
  int kv = 0, rpw = 1, ncw = 0, smem = 0;
  SegArgs seg{};
  // work lists
  size_t bytes = 0;
  void* dev = nullptr;
  void* host[2] = {nullptr, nullptr};
  cudaEvent_t done[2] = {nullptr, nullptr};
  int cur = 0;
  int64_t* counter = nullptr;   // device: rows rechecked by the last call
  int* status = nullptr;        // device: ST_* bits
  // graphs
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  bool captured = false;
};

static SegHeader* hdr_of(void* base) { return static_cast<SegHeader*>(base); }
static SegGroup* list_of(void* base, int fam, int max_groups) {
  return reinterpret_cast<SegGroup*>(static_cast<char*>(base) + kFamilies * sizeof(SegHeader)) +
         (size_t)fam * max_groups;
}

// The launches of one call (work list already on the device).
static nb_status batch_launch(nb_batch* b, cudaStream_t st) {
  SegHeader* dh = hdr_of(b->dev);
  NB_TRY_CUDA(cudaMemsetAsync(b->counter, 0, sizeof(int64_t), st), "memset(counter)");
  if (!b->fam[0].empty()) {
    SegArgs a = b->seg;
    a.groups = list_of(b->dev, 0, b->max_groups);
    a.hdr = dh;
    int grid = 0;
    nb_status s =
        launch_score2_seg(a, b->plan, b->dtype, b->kv, b->rpw, b->ncw, b->smem, &grid, st);
    if (s != NB_OK) return s;
  }
  if (!b->fam[1].empty()) {
    nb_status s = launch_score_gen_seg(list_of(b->dev, 1, b->max_groups), dh + 1,
                                       b->fam[1].data(), (int)b->fam[1].size(), b->dtype, b->F,
                                       b->want_lp, b->recheck, b->status, st);
    if (s != NB_OK) return s;
  }
  if (!b->fam[2].empty()) {
    nb_status s = launch_score_tc_seg(list_of(b->dev, 2, b->max_groups), dh + 2,
                                      static_cast<char*>(b->dev) + b->maps_off,
                                      b->fam[2].data(), (int)b->fam[2].size(), b->dtype, b->F,
                                      b->want_lp, b->recheck, b->status, st);
    if (s != NB_OK) return s;
  }
  // also under NB_RECHECK_OFF: rows a scorer could not compute at all are marked
  for (int f = 0; f < kFamilies; ++f) {
    if (b->fam[f].empty()) continue;
    nb_status s = launch_recheck_seg(list_of(b->dev, f, b->max_groups), dh + f,
                                     b->fam[f].data(), (int)b->fam[f].size(), b->dtype, b->F,
                                     b->want_lp, b->counter, st);
    if (s != NB_OK) return s;
  }
  return NB_OK;
}

namespace nbg {

// The family-0 (two-class) work list on the device, for callers that build it
// with a kernel (the group-wise scorer), and its rows per tile.
nb_status batch_device_list(nb_batch* b, SegHeader** hdr, SegGroup** list0, int64_t* rs) {
  if (!b || !b->fam[1].empty() || !b->fam[2].empty()) {
    set_error("device-built work lists hold two-class groups only");
    return NB_EINVAL;
  }
  *hdr = hdr_of(b->dev);
  *list0 = list_of(b->dev, 0, b->max_groups);
  *rs = b->fam[0].empty() ? 1 : b->plan.RS;
  return NB_OK;
}

// The batch's launches on a work list already written on the device.
nb_status batch_launch_device(nb_batch* b, cudaStream_t st, int64_t* n_rechecked) {
  nb_status s = batch_launch(b, st);
  if (s != NB_OK) return s;
  if (n_rechecked)
    NB_TRY_CUDA(cudaMemcpyAsync(n_rechecked, b->counter, sizeof(int64_t),
                                cudaMemcpyDeviceToDevice, st),
                "memcpy(n_rechecked)");
  return NB_OK;
}

}  // namespace nbg

namespace nbg {
nb_status batch_create(const nb_model* const* models, int n_models, nb_dtype dtype,
                       int64_t max_ld, int max_groups, const nb_score_opts* opts, bool plain,
                       nb_batch** out);
}

extern "C" nb_status nb_batch_create(const nb_model* const* models, int n_models, nb_dtype dtype,
                                     int64_t max_ld, int max_groups, const nb_score_opts* opts,
                                     nb_batch** out) {
  return batch_create(models, n_models, dtype, max_ld, max_groups, opts, false, out);
}

// plain: every group is dense rows without side arrays (nb_batch_score rejects
// others), which allows longer pipeline stages.
nb_status nbg::batch_create(const nb_model* const* models, int n_models, nb_dtype dtype,
                            int64_t max_ld, int max_groups, const nb_score_opts* opts, bool plain,
                            nb_batch** out) {
  if (!out || !models || n_models < 1 || n_models > kSegMaxModels || max_groups < 1 ||
      elem_size(dtype) == 0) {
    set_error("nb_batch_create: need 1 <= n_models <= %d, max_groups >= 1, a valid dtype",
              kSegMaxModels);
    return NB_EINVAL;
  }
  *out = nullptr;
  const int F = models[0]->F;
  for (int i = 0; i < n_models; ++i) {
    if (!models[i] || models[i]->kind != NB_MULTINOMIAL || models[i]->F != F) {
      set_error("nb_batch_create: models must be multinomial with the same F");
      return NB_EINVAL;
    }
  }
  if (max_ld < F) {
    set_error("nb_batch_create: max_ld must be >= F");
    return NB_EINVAL;
  }
  nb_batch* b = new (std::nothrow) nb_batch();
  if (!b) {
    set_error("nb_batch_create: out of host memory");
    return NB_ENOMEM;
  }
  b->dtype = dtype;
  b->F = F;
  b->F_pad = models[0]->F_pad;
  b->max_groups = max_groups;
  b->want_lp = opts ? opts->want_logpost : 0;
  b->plain = plain;
  b->recheck = opts ? (int)opts->recheck : (int)NB_RECHECK_LP;
  for (int i = 0; i < n_models; ++i) {
    const int f = models[i]->C == 2 ? 0 : 1;
    b->slot_family.push_back(f);
    b->slot_index.push_back((int)b->fam[f].size());
    b->fam[f].push_back(models[i]);
    int i2 = -1;
    if (f == 1 && (dtype == NB_U8 || dtype == NB_FP8E4M3 || dtype == NB_BF16) &&
        models[i]->d.tc_w) {
      i2 = (int)b->fam[2].size();
      b->fam[2].push_back(models[i]);
    }
    b->slot_index2.push_back(i2);
  }
  auto fail = [&](nb_status s) {
    nb_batch_destroy(b);
    return s;
  };
  const int es = elem_size(dtype);
  if (!b->fam[0].empty() && dtype != NB_U8 && dtype != NB_F32) {
    set_error("nb_batch_create: two-class models batch U8 or F32 rows");
    return fail(NB_EINVAL);
  }
  if (!b->fam[0].empty()) {
    nb_status s = seg2_plan(dtype, F, b->F_pad, max_ld * es, (int)b->fam[0].size(), plain,
                            &b->plan, &b->kv, &b->rpw, &b->ncw, &b->smem);
    if (s != NB_OK) return fail(s);
  }
  b->maps_off = (kFamilies * sizeof(SegHeader) + kFamilies * (size_t)max_groups * sizeof(SegGroup) +
                 127) / 128 * 128;
  b->bytes = b->maps_off + (b->fam[2].empty() ? 0 : (size_t)max_groups * kTcMapBytes);
  cudaError_t e = cudaMalloc(&b->dev, b->bytes + 64);
  if (e != cudaSuccess) return fail(cuda_status(e, "cudaMalloc(batch)"));
  b->counter = reinterpret_cast<int64_t*>(static_cast<char*>(b->dev) + b->bytes);
  b->status = reinterpret_cast<int*>(static_cast<char*>(b->dev) + b->bytes + 16);
  for (int i = 0; i < 2; ++i) {
    e = cudaMallocHost(&b->host[i], b->bytes);
    if (e != cudaSuccess) return fail(cuda_status(e, "cudaMallocHost(batch)"));
    memset(b->host[i], 0, b->bytes);
    e = cudaEventCreateWithFlags(&b->done[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return fail(cuda_status(e, "cudaEventCreate"));
  }
  e = cudaMemset(b->dev, 0, b->bytes + 64);
  if (e != cudaSuccess) return fail(cuda_status(e, "cudaMemset(batch)"));
  if (!b->fam[0].empty()) {
    SegArgs& a = b->seg;
    a.n_models = (int)b->fam[0].size();
    const uint32_t tab = dtype == NB_U8 ? (uint32_t)(3 * b->F_pad) : (uint32_t)(4 * b->F_pad);
    a.table_bytes = tab;
    a.table_stride = (tab + 127) / 128 * 128;
    for (int i = 0; i < a.n_models; ++i) {
      const nb_model* m = b->fam[0][i];
      a.tables[i] = dtype == NB_U8 ? static_cast<const void*>(m->d.limbs)
                                   : static_cast<const void*>(m->d.il[0]);
      a.chdr[i] = m->d.c2;
    }
    a.F = F;
    a.nvec_row = (F * es + 15) / 16;
    a.nvec_tab = dtype == NB_U8 ? b->F_pad / 16 : b->F_pad / 4;
    a.want_lp = b->want_lp;
    a.recheck = b->recheck;
    a.k_base = b->kv * ((16 / es) / 4) + 2 + 5 + 2;
    a.status = b->status;
  }
  *out = b;
  return NB_OK;
}

extern "C" nb_status nb_batch_score(nb_batch* b, const nb_group* groups, int n_groups,
                                    void* cuda_stream, int64_t* n_rechecked) {
  if (!b || n_groups < 0 || n_groups > b->max_groups || (n_groups > 0 && !groups)) {
    set_error("nb_batch_score: bad batch or group count (max %d)", b ? b->max_groups : 0);
    return NB_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int es = elem_size(b->dtype);
  // the host copy of this call was last used two calls ago
  NB_TRY_CUDA(cudaEventSynchronize(b->done[b->cur]), "cudaEventSynchronize");
  void* h = b->host[b->cur];
  SegHeader* hh = hdr_of(h);
  memset(hh, 0, kFamilies * sizeof(SegHeader));
  long long tiles[kFamilies] = {0, 0, 0}, chunks[kFamilies] = {0, 0, 0};
  const long long rs = b->fam[0].empty() ? 1 : b->plan.RS;
  for (int i = 0; i < n_groups; ++i) {
    const nb_group& g = groups[i];
    if (g.model < 0 || g.model >= (int)b->slot_family.size() || g.n < 0 ||
        (g.n > 0 && (!g.X || !g.label || !g.margin || (b->want_lp && !g.logpost) ||
                     g.ld < b->F))) {
      set_error("nb_batch_score: group %d: bad model slot, sizes or pointers", i);
      return NB_EINVAL;
    }
    int f = b->slot_family[g.model];
    // a many-class group takes the tensor-core kernel exactly when scoring it
    // alone would, so both give the same bits
    if (f == 1 && g.n > 0 && b->slot_index2[g.model] >= 0 &&
        tc_group_eligible(b->fam[1][b->slot_index[g.model]], b->dtype, g.X, g.ld))
      f = 2;
    if (f == 0 && g.n > 0 &&
        (((reinterpret_cast<uintptr_t>(g.X) & 15) != 0) || ((g.ld * es) % 16) != 0 ||
         g.ld * es > b->plan.xs_bytes / (rs > 0 ? rs : 1))) {
      set_error("nb_batch_score: group %d: X must be 16-byte aligned, ld * element size a "
                "multiple of 16 and ld <= the batch's max_ld",
                i);
      return NB_EINVAL;
    }
    if (b->plain && (g.aux.ovf_ptr || g.aux.row_exp)) {
      set_error("nb_batch_score: group %d: this batch takes dense rows only", i);
      return NB_EINVAL;
    }
    if (g.aux.ovf_ptr && (!g.aux.ovf_col || !g.aux.ovf_add)) {
      set_error("nb_batch_score: group %d: overflow list needs ovf_col and ovf_add", i);
      return NB_EINVAL;
    }
    SegGroup* L = list_of(h, f, b->max_groups);
    SegGroup& d = L[hh[f].n_groups++];
    d.X = static_cast<const char*>(g.X);
    d.ld_bytes = g.ld * es;
    d.n = g.n;
    // the overflow list belongs to u8 rows, the row scale to FP8 rows
    const bool u8 = b->dtype == NB_U8;
    d.ovf_ptr = u8 ? g.aux.ovf_ptr : nullptr;
    d.ovf_col = u8 ? g.aux.ovf_col : nullptr;
    d.ovf_add = u8 ? g.aux.ovf_add : nullptr;
    d.row_exp = b->dtype == NB_FP8E4M3 ? g.aux.row_exp : nullptr;
    d.label = g.label;
    d.margin = g.margin;
    d.logpost = b->want_lp ? g.logpost : nullptr;
    d.tile0 = tiles[f];
    d.chunk0 = chunks[f];
    d.model = f == 2 ? b->slot_index2[g.model] : b->slot_index[g.model];
    d.family = f;
    if (f == 2) {
      nb_status ms = tc_encode_rows(static_cast<char*>(h) + b->maps_off +
                                        (size_t)(hh[2].n_groups - 1) * kTcMapBytes,
                                    g.X, g.n, b->F, g.ld * es, es);
      if (ms != NB_OK) return ms;
    }
    tiles[f] += f == 0 ? (g.n + rs - 1) / rs : (f == 1 ? (g.n + 63) / 64 : (g.n + 255) / 256);
    chunks[f] += (g.n + 31) / 32;
  }
  for (int f = 0; f < kFamilies; ++f) {
    hh[f].tiles = tiles[f];
    hh[f].chunks = chunks[f];
  }
  if (b->captured) {
    NB_TRY_CUDA(cudaGraphLaunch(b->exec[b->cur], st), "cudaGraphLaunch");
  } else {
    NB_TRY_CUDA(cudaMemcpyAsync(b->dev, h, b->bytes, cudaMemcpyHostToDevice, st),
                "memcpy(work list)");
    nb_status s = batch_launch(b, st);
    if (s != NB_OK) return s;
  }
  NB_TRY_CUDA(cudaEventRecord(b->done[b->cur], st), "cudaEventRecord");
  b->cur ^= 1;
  if (n_rechecked)
    NB_TRY_CUDA(cudaMemcpyAsync(n_rechecked, b->counter, sizeof(int64_t),
                                cudaMemcpyDeviceToDevice, st),
                "memcpy(n_rechecked)");
  return NB_OK;
}

extern "C" nb_status nb_batch_capture(nb_batch* b, void* cuda_stream) {
  if (!b) {
    set_error("nb_batch_capture: NULL batch");
    return NB_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (!st) {
    set_error("nb_batch_capture: needs a non-default stream");
    return NB_EINVAL;
  }
  NB_TRY_CUDA(cudaStreamSynchronize(st), "sync");
  for (int i = 0; i < 2; ++i) {
    if (b->exec[i]) {
      cudaGraphExecDestroy(b->exec[i]);
      b->exec[i] = nullptr;
    }
    cudaGraph_t graph = nullptr;
    NB_TRY_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal),
                "cudaStreamBeginCapture");
    cudaError_t e = cudaMemcpyAsync(b->dev, b->host[i], b->bytes, cudaMemcpyHostToDevice, st);
    nb_status s = e == cudaSuccess ? batch_launch(b, st) : cuda_status(e, "memcpy(capture)");
    cudaError_t e2 = cudaStreamEndCapture(st, &graph);
    if (s != NB_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    NB_TRY_CUDA(e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->exec[i], graph, 0);
    cudaGraphDestroy(graph);
    NB_TRY_CUDA(e, "cudaGraphInstantiate");
  }
  b->captured = true;
  return NB_OK;
}

extern "C" void nb_batch_destroy(nb_batch* b) {
  if (!b) return;
  for (int i = 0; i < 2; ++i) {
    if (b->done[i]) {
      cudaEventSynchronize(b->done[i]);
      cudaEventDestroy(b->done[i]);
    }
    if (b->exec[i]) cudaGraphExecDestroy(b->exec[i]);
    if (b->host[i]) cudaFreeHost(b->host[i]);
  }
  if (b->dev) {
    cudaDeviceSynchronize();
    cudaFree(b->dev);
  }
  delete b;
}
