// Tile configuration of the two-class scorer and its autotuner.
//
// The autotuner times each candidate configuration (pipeline depth, rows per
// shared-memory stage, register-streaming variant) on the caller's data with
// CUDA events and keeps the fastest.  For u8 storage all candidates give
// bit-identical results; for the FP32 paths the variant is only varied where
// both kernels share the per-row reduction order.
#include <vector>

#include "internal.cuh"

using namespace nbg;

extern "C" nb_status nb_set_tile_config(nb_model* m, const nb_tile_config* cfg) {
  if (!m || !cfg) {
    set_error("nb_set_tile_config: NULL argument");
    return NB_EINVAL;
  }
  if (cfg->variant < NB_VARIANT_AUTO || cfg->variant > NB_VARIANT_REGISTER || cfg->stages < 0 ||
      cfg->stages > 6 || cfg->rows_per_stage < 0 || cfg->rows_per_stage > 48 ||
      cfg->rows_per_warp < 0 || cfg->rows_per_warp > 2) {
    set_error("nb_set_tile_config: variant in 0..2, stages in 0..6, rows_per_stage in 0..48, "
              "rows_per_warp in 0..2");
    return NB_EINVAL;
  }
  m->tile = *cfg;
  return NB_OK;
}

extern "C" nb_status nb_get_tile_config(const nb_model* m, nb_tile_config* cfg) {
  if (!m || !cfg) {
    set_error("nb_get_tile_config: NULL argument");
    return NB_EINVAL;
  }
  *cfg = m->tile;
  return NB_OK;
}

extern "C" nb_status nb_autotune_score(nb_model* m, const void* X, nb_dtype dtype, int64_t n,
                                       int64_t ld, const nb_aux* aux, void* cuda_stream,
                                       nb_tile_config* best, float* best_ms) {
  if (!m) {
    set_error("nb_autotune_score: NULL model");
    return NB_EINVAL;
  }
  const nb_tile_config keep = m->tile;
  if (m->kind != NB_MULTINOMIAL || m->C != 2 || n <= 0) {
    if (best) *best = keep;
    if (best_ms) *best_ms = 0.f;
    return NB_OK;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int es = elem_size(dtype);
  if (es == 0 || ld < m->F) {
    set_error("nb_autotune_score: bad dtype or ld");
    return NB_EINVAL;
  }
  const int64_t ld_bytes = ld * es;
  const int nvec_row = (m->F * es + 15) / 16;
  const bool same_order = dtype == NB_U8 || nvec_row > 64;

  std::vector<nb_tile_config> cand;
  // rows per warp changes the FP32 reduction tree, so it is varied only for u8
  const int rpw_max = dtype == NB_U8 ? 2 : 1;
  for (int rpw = 1; rpw <= rpw_max; ++rpw) {
    cand.push_back({NB_VARIANT_PIPELINED, 0, 0, rpw});
    for (int s : {2, 3, 4, 6}) {
      for (int rs : {8, 16, 24, 32, 48}) {
        if ((int64_t)rs * ld_bytes > 48 * 1024 || (int64_t)rs * ld_bytes < 4096) continue;
        cand.push_back({NB_VARIANT_PIPELINED, s, rs, rpw});
      }
    }
  }
  if (same_order) cand.push_back({NB_VARIANT_REGISTER, 0, 0, 0});

  void* scratch = nullptr;
  const size_t out_bytes = (size_t)n * (1 + 4 + 4 * m->C) + 64;
  NB_TRY_CUDA(cudaMallocAsync(&scratch, out_bytes, st), "cudaMallocAsync(autotune)");
  char* b = static_cast<char*>(scratch);
  float* margin = reinterpret_cast<float*>(b);
  float* logpost = reinterpret_cast<float*>(b + (size_t)n * 4);
  uint8_t* label = reinterpret_cast<uint8_t*>(b + (size_t)n * (4 + 4 * m->C));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  nb_score_opts opts{1, NB_RECHECK_LP, aux};
  float best_t = 1e30f;
  nb_tile_config best_c = keep;
  nb_status status = NB_OK;
  for (const nb_tile_config& c : cand) {
    m->tile = c;
    nb_status s = nb_score_group(m, X, dtype, n, ld, label, margin, logpost, &opts, st, nullptr);
    if (s == NB_EUNSUPPORTED) continue;
    if (s != NB_OK) {
      status = s;
      break;
    }
    // the fastest of a few repetitions (the least disturbed by other work)
    float t_min = 1e30f;
    const int reps = 5;
    for (int r = 0; r < reps; ++r) {
      cudaEventRecord(e0, st);
      s = nb_score_group(m, X, dtype, n, ld, label, margin, logpost, &opts, st, nullptr);
      cudaEventRecord(e1, st);
      if (s != NB_OK) break;
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      t_min = ms < t_min ? ms : t_min;
    }
    if (s != NB_OK) {
      status = s;
      break;
    }
    if (t_min < best_t) {
      best_t = t_min;
      best_c = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(scratch, st);
  cudaStreamSynchronize(st);
  if (status != NB_OK) {
    m->tile = keep;
    return status;
  }
  m->tile = best_c;
  if (best) *best = best_c;
  if (best_ms) *best_ms = best_t;
  return NB_OK;
}
