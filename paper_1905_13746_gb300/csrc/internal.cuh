// Internal declarations of the nbgpu library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nbgpu.h"

namespace nbg {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);
nb_status cuda_status(cudaError_t e, const char* what);

#define NB_TRY_CUDA(expr, what)                          \
  do {                                                   \
    cudaError_t e__ = (expr);                            \
    if (e__ != cudaSuccess) return ::nbg::cuda_status(e__, what); \
  } while (0)

// device status word bits (model / call error words)
enum : int {
  ST_BAD_LABEL = 1,       // a label outside [0, C)
  ST_BAD_VALUE = 2,       // negative, fractional or non-finite count
  ST_TIMEOUT = 4,         // a bounded wait gave up
  ST_BAD_TABLE = 8,       // non-finite parameter table
  ST_OVF_RANGE = 16,      // overflow column outside [0, F)
  ST_BAD_ROUTE = 32       // routing / gather input: negative size, group, label or column out of range
};

constexpr uint8_t kLabelRecheck = 255;   // internal marker in label[]

// Dynamic shared memory above this size is requested through the kernel's
// max-dynamic-shared-memory attribute; the default limit of 48 KB covers
// dynamic and static shared memory together, and the kernels declare a few
// static barriers.
constexpr int kSmemOptIn = 32 * 1024;

inline int elem_size(nb_dtype d) {
  switch (d) {
    case NB_F32: return 4;
    case NB_U16: return 2;
    case NB_BF16: return 2;
    case NB_U8: return 1;
    case NB_FP8E4M3: return 1;
  }
  return 0;
}

// ---------------------------------------------------------------------------
// two-class scalars produced on the device by the fit (one struct in HBM)
// ---------------------------------------------------------------------------
struct C2Header {
  float b;            // log pi_1 - log pi_0 (FP32)
  float maxabs;       // max_j |Delta_j| of the FP32 table
  float inv_scale;    // 2^-S: fixed-point step of the integer Delta table
  float maxabs_q;     // max_j |Delta_j| bound used with the fixed-point table
  double b64;         // FP64 b
  int32_t S;          // Delta_q = round(Delta * 2^S), |Delta_q| <= 2^22
  int32_t pad;
};

// fixed-point scalars of the many-class tensor-core tables (one struct in HBM)
struct TcHeader {
  float scale;        // 2^-S: step of the fixed-point weights Q = round(w 2^S)
  float tau_unit;     // 2^-(S+1): largest rounding error of one weight
  int32_t S;
  int32_t pad;
};

// tensor-core scorer limits: classes, features
constexpr int kTcMaxC = 64;
// classes of a Gaussian model's FP32 tables per feature: blocks of 4 (C <= 4)
// or 16, the class blocks of the CUDA-core scorer
__host__ __device__ constexpr int gauss_cpad(int C) { return C <= 4 ? 4 : ((C + 15) / 16) * 16; }
constexpr int kTcMaxF = 32768;
constexpr int kTcgMaxF = 8192;   // Gaussian tensor-core tables
constexpr int kTcgFS = 32;       // ... features per stage (a multiple of 8 dividing 32)

// scalars of the Gaussian tensor-core tables (one struct in HBM)
struct TcgHeader {
  int bad;            // a weight outside the FP16 range: the tables are not used
  float wsum;         // sum_j (max_c |B_cj| + max_c |A_cj|), rounded up
};

// ---------------------------------------------------------------------------
// model (library-owned)
// ---------------------------------------------------------------------------
struct ModelDev {
  // all pointers into one device allocation
  uint64_t* counts;    // C x F      (multinomial)
  uint64_t* nc;        // C
  double* p0;          // C x F      log theta (multinomial) | mu (Gaussian)
  double* p1;          // C x F      var (Gaussian)
  double* log_pi;      // C
  double* gconst;      // C          Gaussian: log pi_c - 1/2 sum_j log(2 pi var_cj)
  int* status;         // 1 int: ST_* bits raised while fitting (cleared by each fit)
  int* sstatus;        // 1 int: ST_* bits raised by scoring calls (kept until
                       // nb_model_check reports them)
  unsigned long long* fin;   // 4 words of the two-class fit finish (zero between fits)
  // two-class multinomial tables
  C2Header* c2;        // 1
  float* delta;        // F_pad      FP32 Delta, plain order
  int32_t* delta_q;    // F_pad      fixed-point Delta
  uint4* limbs;        // 3 * nvec8  int8 limbs of delta_q, interleaved (u8 path), then
                       //            F_pad packed words (limb l in byte l)
  float4* il[3];       // interleaved FP32 quads for 4/8/16 elements per vector
  // general-C tables (CUDA-core scorer)
  float* w;            // C x F_pad  centred weights log theta_cj - mean_c log theta_cj
  float* bias;         // C          log pi_c
  float* wmax;         // 1          max |w|
  // many-class tensor-core tables (3 <= C <= kTcMaxC), else nullptr
  uint8_t* tc_w;       // ceil(F/64) stages x 3*Cp x 64 FP16 limbs (MMA operand layout)
  int32_t* tc_q;       // C x F fixed-point weights
  TcHeader* tc_hdr;    // 1
  // Gaussian FP32 tables
  float* g_mu;         // F_pad x gauss_cpad(C), feature-major (classes past C: 0)
  float* g_ivar;       // same layout, 1 / var
  float* g_const;      // 2C         gconst in FP32, then a4_c = sum_j m^2 v (FP32 tables)
  // Gaussian tensor-core tables (3 <= C <= kTcMaxC, F <= kTcgMaxF), else nullptr;
  // the FP16 limbs of B and A go to tc_w
  float* tcg_kc;       // C          K_c
  float* tcg_ctr;      // F rounded up to kTcgFS: centres m_j
  float* tcg_bmax;     // ... max_c |B_cj|
  float* tcg_amax;     // ... max_c |A_cj|
  TcgHeader* tcg_hdr;  // 1
};

}  // namespace nbg

struct nb_model {
  nb_kind kind;
  int C;
  int F;
  int F_pad;        // F rounded up to a multiple of 16
  int nvec8;        // F_pad / 16 (u8 vectors of 16 bytes)
  double alpha;
  double var_smoothing;
  int device;
  nb_tile_config tile;   // scorer kernel configuration (autotuned or set)
  cudaStream_t stream;   // stream of the fit
  void* mem;
  size_t mem_bytes;
  nbg::ModelDev d;
};

namespace nbg {

// launchers implemented in fit.cu / score2.cu / recheck.cu / pack.cu
nb_status launch_fit_multinomial(nb_model* m, const void* X, nb_dtype dt,
                                 int64_t n, int64_t ld, const int32_t* y,
                                 const nb_aux* aux, const double* log_prior_dev,
                                 cudaStream_t st);
nb_status launch_fit_gaussian(nb_model* m, const float* X, int64_t n,
                              int64_t ld, const int32_t* y,
                              const double* log_prior_dev, cudaStream_t st);

struct ScoreOut {
  uint8_t* label;
  float* margin;
  float* logpost;
  int64_t* n_rechecked;
  int want_lp;
  int recheck;
  bool counted = false;   // the scorer counted its marked rows into n_rechecked
};

nb_status launch_score2(const nb_model* m, const void* X, nb_dtype dt,
                        int64_t n, int64_t ld, const nb_aux* aux,
                        const ScoreOut& o, cudaStream_t st);
nb_status launch_fit2_pipe(nb_model* m, const void* X, nb_dtype dt, int64_t n, int64_t ld,
                           const int32_t* y, const nb_aux* aux, cudaStream_t st);
struct S2Args;
nb_status launch_score2_pipe(const S2Args& a, nb_dtype dt, int stages, int rows_per_stage,
                             int rows_per_warp, int stage_entries, cudaStream_t st);
nb_status launch_score_general(const nb_model* m, const void* X, nb_dtype dt,
                               int64_t n, int64_t ld, const nb_aux* aux,
                               const ScoreOut& o, cudaStream_t st);
nb_status launch_recheck(const nb_model* m, const void* X, nb_dtype dt,
                         int64_t n, int64_t ld, const nb_aux* aux,
                         const ScoreOut& o, cudaStream_t st);

// many-class tensor-core scorer (score_tc.cu)
inline int tc_classes_padded(int C) { return (C + 15) / 16 * 16; }
inline size_t tc_w_bytes(int C, int F) {
  return (size_t)((F + 63) / 64) * 3 * tc_classes_padded(C) * 128;
}
inline bool tc_tables(nb_kind kind, int C, int F) {
  return kind == NB_MULTINOMIAL && C >= 3 && C <= kTcMaxC && F <= kTcMaxF;
}
bool tc_eligible(const nb_model* m, nb_dtype dt, const void* X, int64_t ld);
nb_status launch_derive_tc(nb_model* m, cudaStream_t st);

// many-class Gaussian tensor-core scorer (score_tcg.cu)
inline size_t tcg_w_bytes(int C, int F) {
  return (size_t)((F + kTcgFS - 1) / kTcgFS) * tc_classes_padded(C) * (16 * kTcgFS);
}
inline bool tcg_tables(nb_kind kind, int C, int F) {
  return kind == NB_GAUSSIAN && C >= 3 && C <= kTcMaxC && F <= kTcgMaxF;
}
bool tcg_eligible(const nb_model* m, const void* X, int64_t ld, int recheck);
nb_status launch_derive_tcg(nb_model* m, cudaStream_t st);
nb_status launch_score_tcg(const nb_model* m, const float* X, int64_t n, int64_t ld,
                           const ScoreOut& o, cudaStream_t st);
nb_status launch_score_tc(const nb_model* m, const void* X, nb_dtype dt, int64_t n, int64_t ld,
                          const nb_aux* aux, const ScoreOut& o, cudaStream_t st);

int num_sms();

// Launch k with programmatic stream serialisation (see pdl_wait()).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, args...);
}
// process-wide count of kernels this library has launched
void count_launch();

// Gaussian fit: rows per deterministic partial sum, features per block tile
constexpr int kGChunkRows = 256;
constexpr int kGTile = 64;
// features per block tile of a fit with C classes: 64 up to 32 classes, 32
// above (the block's shared partial sums, 8 (C + 1) tile doubles, must fit);
// the tile changes which block sums a feature, not the order of its sums
inline int gauss_tile(int C) { return C <= 32 ? kGTile : kGTile / 2; }
// rows per partial sum of a fit of n rows: 32 for small fits (more blocks in
// flight), else kGChunkRows; the partials are summed in chunk order, so the
// result depends only on n (every Gaussian fit path uses this rule)
inline int64_t gauss_chunk_rows(int64_t n) { return n <= 65536 ? 32 : kGChunkRows; }

// ST_* bits of a status word -> status code and error text (first error wins)
nb_status status_from_word(int w);

// Looks up the allocation-free re-fit's device scratch for the current device
// (noalloc.cu); under lazy module loading this is what commits it.
nb_status noalloc_scratch_prepare();

// Gaussian fit kernels (fit.cu)
__global__ void k_label_hist(const int32_t* y, int64_t n, int C, unsigned long long* nc,
                             int* status);
__global__ void k_gauss_partial(const float* X, int64_t ld, int64_t n, int F, int C,
                                const int32_t* y, int pass, const double* mu_c,
                                const double* mu_all, double* partial, int64_t chunk_rows,
                                int tile, int* status);
__global__ void k_gauss_reduce(const double* partial, int nchunk, int F, int C,
                               const unsigned long long* nc, int64_t n, int pass, double* mu_c,
                               double* mu_all, double* m2_c, double* m2_all);
__global__ void k_gauss_finalize(const double* m2_all, int F, int F_pad, int C,
                                 double var_smoothing, const unsigned long long* nc, int64_t n,
                                 int prior_given, const double* mu, double* var, double* log_pi,
                                 double* gconst, float* g_mu, float* g_ivar, float* g_const,
                                 int* status);

}  // namespace nbg
