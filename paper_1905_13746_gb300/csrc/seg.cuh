// Device work list of a segmented (batched) launch: groups of files of uneven
// size, each with its own matrix, overflow list, outputs and model slot, all
// scored by one persistent launch per kernel family.
#pragma once

#include <stdint.h>

#include "internal.cuh"

namespace nbg {

constexpr int kSegMaxModels = 128;   // kernel arguments hold one entry per model

struct SegGroup {
  const char* X;
  long long ld_bytes;
  long long n;
  const int64_t* ovf_ptr;
  const uint16_t* ovf_col;
  const uint16_t* ovf_add;
  const int8_t* row_exp;
  uint8_t* label;
  float* margin;
  float* logpost;
  long long tile0;    // first tile of the group in its family's launch
  long long chunk0;   // first 32-row chunk of the group (recheck scan)
  int model;          // model index within its family's model list
  int family;         // 0: two-class pipelined, 1: general CUDA-core, 2: tensor-core
};

struct SegHeader {
  int n_groups;       // groups of this list
  int pad;
  long long tiles;    // tiles of the list: stage rows (two-class), 64 rows (general),
                      // 256 rows (tensor-core)
  long long chunks;   // 32-row chunks of the list (recheck)
  long long pad2;
};

// First group g of a list with key(g) <= t (keys non-decreasing, key(0) = 0).
template <class Key>
__device__ __forceinline__ int seg_find(int n_groups, long long t, Key key) {
  int lo = 0, hi = n_groups;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (key(mid) <= t) lo = mid; else hi = mid;
  }
  return lo;
}

// kernel arguments of the segmented two-class scorer
struct SegArgs {
  const SegGroup* groups;
  const SegHeader* hdr;
  int n_models;
  const void* tables[kSegMaxModels];
  const C2Header* chdr[kSegMaxModels];
  uint32_t table_bytes, table_stride;
  int F, nvec_row, nvec_tab, want_lp, recheck, k_base;
  int* status;
};

struct PipeArgs;

// launchers (score2_seg.cu, score_general.cu, recheck.cu)
nb_status seg2_plan(nb_dtype dt, int F, int F_pad, long long max_ld_bytes, int n_models,
                    bool plain_rows, PipeArgs* p, int* kv_out, int* rpw_out, int* ncw_out,
                    int* smem_out);
nb_status launch_score2_seg(const SegArgs& a, const PipeArgs& p, nb_dtype dt, int kv, int rpw,
                            int ncw, int smem, int* grid, cudaStream_t st);
nb_status launch_score_gen_seg(const SegGroup* groups, const SegHeader* hdr,
                               const nb_model* const* models, int n_models, nb_dtype dt, int F,
                               int want_lp, int recheck, int* status, cudaStream_t st);
nb_status launch_score_tc_seg(const SegGroup* groups, const SegHeader* hdr, const void* maps,
                              const nb_model* const* models, int n_models, nb_dtype dt, int F,
                              int want_lp, int recheck, int* status, cudaStream_t st);
nb_status tc_encode_rows(void* map, const void* X, int64_t n, int F, int64_t ld_bytes, int es);
bool tc_group_eligible(const nb_model* m, nb_dtype dt, const void* X, int64_t ld);
constexpr size_t kTcMapBytes = 128;
nb_status launch_recheck_seg(const SegGroup* groups, const SegHeader* hdr,
                             const nb_model* const* models, int n_models, nb_dtype dt, int F,
                             int want_lp, int64_t* n_rechecked, cudaStream_t st);

}  // namespace nbg
