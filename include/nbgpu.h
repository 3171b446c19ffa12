/*
 * nbgpu -- Naive Bayes fit and group scoring on one sm_103a GPU (C ABI).
 *
 * Method: Sahay & Chaudhari, "An Efficient Detection of Malware by Naive
 * Bayes Classifier Using GPGPU".
 *   Sec. 3  files are opcode-occurrence-count vectors, partitioned into
 *           size groups;
 *   Sec. 4  a Naive Bayes model is trained on labelled vectors; a file's
 *           posterior is P(C | a_1..a_n) = P(a_1..a_n | C) / P(a_1..a_n)
 *           with class-conditionally independent features (the single
 *           display equation), and the file is malware when the malware
 *           posterior is higher, otherwise benign (the decision rule below
 *           it); the files of a group are classified in parallel on the GPU.
 *
 * Readings used throughout (the paper leaves them open):
 *   - count features: multinomial event model, Laplace smoothing alpha
 *     (default 1): log theta_cj = log(N_cj + alpha) - log(N_c + alpha F);
 *   - real features: Gaussian class densities, maximum-likelihood variance
 *     plus eps = var_smoothing * max_j Var(x_.j);
 *   - prior: empirical n_c / n unless log priors are supplied;
 *   - ties go to the lowest class index (benign = 0 for two classes);
 *   - margin = (top score) - (second score), natural-log units, >= 0;
 *   - logpost_c = s_c - logsumexp_c(s), so the dropped evidence and the
 *     multinomial coefficient (class-independent) do not matter.
 *
 * Conventions
 *   - Every pointer named X, y, label, margin, logpost, ovf_*, row_exp,
 *     n_rechecked is a caller-owned DEVICE pointer unless stated otherwise.
 *     Models and servers are library-owned opaque handles.
 *   - Matrices are row-major, one row per file, leading dimension `ld`
 *     elements (ld >= F).  The buffer must be readable for n * ld elements.
 *     The fast paths need base and ld * element_size 16-byte aligned; other
 *     layouts take a slower, still exact, path.
 *   - Calls are asynchronous on the given CUDA stream (`cuda_stream` is a
 *     cudaStream_t; NULL = legacy default stream) unless documented.
 *   - No exception crosses the ABI.  Every call returns an nb_status; the
 *     message of the last failure on the calling thread is nb_last_error().
 *   - C <= 255 (labels are uint8; 255 is reserved as an internal marker).
 */
#ifndef NBGPU_H
#define NBGPU_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define NB_API __attribute__((visibility("default")))
#else
#define NB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NB_OK = 0,
  NB_EINVAL = 1,        /* bad argument or invalid data (e.g. a label >= C) */
  NB_ENOMEM = 2,        /* a device or host allocation failed */
  NB_ECUDA = 3,         /* a CUDA runtime call failed */
  NB_ETIMEOUT = 4,      /* a bounded wait ran out */
  NB_EUNSUPPORTED = 5,  /* valid request this build does not implement */
  NB_EBUSY = 6          /* no free slot or memory for the request */
} nb_status;

typedef enum { NB_MULTINOMIAL = 0, NB_GAUSSIAN = 1 } nb_kind;

/* Feature storage types.  Counts are exact in U16 (0..65535), in U8 (0..255,
 * or up to 255 + 65535 with the overflow list of nb_aux), in BF16 up to 256
 * and in FP8 E4M3 up to 16 (above, the per-row power-of-two scale of nb_aux
 * applies and values are rounded to the format). */
typedef enum {
  NB_F32 = 0,
  NB_U16 = 1,
  NB_U8 = 2,
  NB_BF16 = 3,
  NB_FP8E4M3 = 4
} nb_dtype;

/* Side arrays of the compact storage formats (all device pointers).
 *   NB_U8 overflow list: row i's entries are ovf_ptr[i] .. ovf_ptr[i+1]-1; an
 *     entry (ovf_col[k], ovf_add[k]) adds ovf_add[k] to the stored byte (255)
 *     of column ovf_col[k].  ovf_ptr has n+1 entries, ovf_ptr[0] = 0.
 *   NB_FP8E4M3 row scale: row i's values are multiplied by 2^row_exp[i]. */
typedef struct {
  const int64_t* ovf_ptr;
  const uint16_t* ovf_col;
  const uint16_t* ovf_add;
  const int8_t* row_exp;
} nb_aux;

typedef struct {
  double alpha;             /* multinomial smoothing (>= 0); 1 = Laplace */
  const double* log_prior;  /* HOST pointer to C log priors, or NULL = empirical */
  double var_smoothing;     /* Gaussian epsilon factor (>= 0), default 1e-9 */
  const nb_aux* aux;        /* side arrays of X's format, or NULL */
  int no_sync;              /* 0: nb_fit waits for the stream and reports
                               invalid data (labels outside [0,C), negative or
                               fractional counts) as NB_EINVAL; 1: fully
                               asynchronous, check later with nb_model_check */
} nb_fit_opts;

/* Recheck policy for rows whose FP32/fixed-point result might differ from
 * the FP64 definition:
 *   NB_RECHECK_OFF   -- no recheck of near-ties (labels may differ there);
 *                       rows that a fast path cannot compute at all are still
 *                       recomputed in FP64: a two-class u8 row whose stored
 *                       counts total 2^24 or more (its int32 limb sums could
 *                       wrap), tensor-core rows of 2^17 or more counts beyond
 *                       the scorer's exact-redo capacity (FP8 and BF16 rows:
 *                       all of them) and FP8 / BF16 rows outside the
 *                       tensor-core scorer's count check;
 *   NB_RECHECK_LABEL -- rows whose margin is within the rigorous error bound
 *                       of the fast path are recomputed in FP64, so every
 *                       label equals the FP64 decision;
 *   NB_RECHECK_LP    -- additionally rows whose log posteriors could be off
 *                       by more than 1e-5 * max(1, |logpost|).  */
typedef enum { NB_RECHECK_OFF = 0, NB_RECHECK_LABEL = 1, NB_RECHECK_LP = 2 } nb_recheck;

typedef struct {
  int want_logpost;     /* write logpost (n x C, float) when non-zero */
  nb_recheck recheck;   /* default NB_RECHECK_LP */
  const nb_aux* aux;    /* side arrays of X's format, or NULL */
} nb_score_opts;

typedef struct nb_model nb_model;
typedef struct nb_server nb_server;

/* Kernel configuration of a model's scorer.
 *   variant  two classes: NB_VARIANT_AUTO: TMA-pipelined kernel when the row
 *            fits a stage, else the register-streaming kernel;
 *            NB_VARIANT_PIPELINED / NB_VARIANT_REGISTER: force one.
 *            3..64 classes with U8, FP8E4M3 or BF16 storage, X 16-byte
 *            aligned and ld * element size a multiple of 16:
 *            NB_VARIANT_AUTO / NB_VARIANT_PIPELINED take the tensor-core
 *            scorer (fixed-point weights, exact accumulation; FP8 and BF16
 *            rows must hold counts: a row with a value that is not an integer
 *            below 1024 after its row scale, or with an FP8 row exponent
 *            other than 0 or 1, is recomputed in FP64 instead),
 *            NB_VARIANT_REGISTER the CUDA-core scorer.
 *            Gaussian, 3..64 classes, F <= 8192, X 16-byte aligned and ld a
 *            multiple of 4: NB_VARIANT_AUTO takes the tensor-core scorer
 *            (FP16 limbs, FP32 accumulation, rigorous per-row bound) in the
 *            label and OFF recheck modes and the CUDA-core scorer in the
 *            log-posterior mode (its bound leaves most rows to FP64 there);
 *            NB_VARIANT_PIPELINED takes the tensor-core scorer in every mode;
 *            NB_VARIANT_REGISTER the CUDA-core scorer.
 *   stages, rows_per_stage: pipeline depth and rows per shared-memory stage
 *            (0 = defaults: stages of 16-48 KB filling ~100-180 KB per block);
 *   rows_per_warp: 1 (32 lanes per row) or 2 (16 lanes per row, more table
 *            registers per lane); 0 = 1.
 * For u8 storage every configuration gives bit-identical results (exact
 * integer sums).  For the FP32 paths the two variants share the reduction
 * order when a row spans >= 64 sixteen-byte vectors; nb_autotune_score keeps
 * the variant fixed otherwise, so tuning never changes a result. */
typedef enum {
  NB_VARIANT_AUTO = 0,
  NB_VARIANT_PIPELINED = 1,
  NB_VARIANT_REGISTER = 2
} nb_variant;

typedef struct {
  int variant;
  int stages;
  int rows_per_stage;
  int rows_per_warp;
} nb_tile_config;

/* ---- fit -----------------------------------------------------------------
 * Train one model on n labelled files (Sec. 4, "trained the model").
 *   kind  NB_MULTINOMIAL: X holds counts (U8[+overflow], U16, F32, BF16,
 *         FP8E4M3 with integer values); N_cj is accumulated exactly in
 *         uint64, then log theta and log prior in FP64 on the device.
 *         NB_GAUSSIAN: X holds real values (F32); class means and MLE
 *         variances are computed in FP64 by two deterministic passes.
 *   y     int32 labels in [0, C) (device), n entries.
 *   C     2 <= C <= 255;  F >= 1.
 * On success *out owns device tables; free it with nb_model_free.  Errors:
 * NB_EINVAL (arguments, or invalid data when opts->no_sync == 0), NB_ENOMEM,
 * NB_ECUDA.  The call may allocate device memory. */
NB_API nb_status nb_fit(nb_kind kind, const void* X, nb_dtype dtype, int64_t n,
                 int32_t F, int64_t ld, const int32_t* y, int32_t C,
                 const nb_fit_opts* opts, void* cuda_stream, nb_model** out);

/* Re-trains an existing model in place on new data with the same F and C
 * (kind, C and F are the model's).  Allocates no model memory, so a training
 * loop or a timed benchmark step does not pay for cudaMalloc / cudaFree; the
 * count reduction still takes stream-ordered scratch (cudaMallocAsync).  The
 * model must not be in use by a score call on another stream meanwhile.
 * Same errors as nb_fit. */
NB_API nb_status nb_refit(nb_model* model, const void* X, nb_dtype dtype, int64_t n,
                   int64_t ld, const int32_t* y, const nb_fit_opts* opts,
                   void* cuda_stream);

/* Allocation-free re-fit of a Gaussian model (this entry point has no
 * counterpart in the paper; it is a deployment convenience).
 * Same work and the same bits as nb_refit on a Gaussian model (the same row
 * chunks and summation order), for callers that may not allocate device
 * memory when they re-train -- a thread held to a fixed memory budget, code
 * between a CUDA graph's instantiation and its replays, an embedded runtime
 * that forbids allocation after start-up.  Its scratch (per-chunk partial
 * sums) is a fixed 8 MiB device array inside the library.  The 8 MiB are
 * committed on a device when nb_fit first creates a Gaussian model there
 * (the library then looks up the array's address, which makes the CUDA
 * runtime load the array's module; with lazy module loading, the default,
 * merely loading the library commits nothing), or else at the first call of
 * this entry point on that device; they stay until the process exits.  Make
 * that first call, or the Gaussian nb_fit, before any stream capture.
 * Requests needing more than ceil(n/r) * (C+1) * F + 2F doubles <= 2^20, with
 * r = 32 rows per partial sum for n <= 65,536 and 256 above, are rejected
 * with NB_EINVAL (use nb_refit for those).  All calls share the array, so
 * calls that may run at the same time on the GPU (unordered streams) race;
 * order them.  X (F32, n x ld) and y are device pointers; opts->log_prior
 * (host), var_smoothing and no_sync act as for nb_refit (alpha and aux are
 * ignored); errors as nb_refit. */
NB_API nb_status nb_refit_gaussian_noalloc(nb_model* model, const float* X, int64_t n,
                                           int64_t ld, const int32_t* y,
                                           const nb_fit_opts* opts, void* cuda_stream);

/* Waits for the model's stream, then reports, in this order: NB_ETIMEOUT if
 * a bounded device wait ran out (in the last fit, or in a scoring call with
 * this model since the previous check: the outputs of that call are not
 * valid); NB_EINVAL if the last fit's data were invalid or a scoring call met
 * an overflow-list column outside [0, F).  Errors of scoring calls are kept
 * (a later re-fit does not clear them) until this call reports them, and
 * cleared then; errors of the fit are cleared by the next fit. */
NB_API nb_status nb_model_check(const nb_model* model);

/* Copies the exact multinomial counts N_cj (C x F) and n_c (C) to HOST
 * buffers (either may be NULL).  Synchronises the fit's stream. */
NB_API nb_status nb_model_counts(const nb_model* model, uint64_t* host_counts,
                          uint64_t* host_nc);

/* Copies the FP64 parameters to HOST buffers (any may be NULL):
 *   multinomial: p0 = log theta (C x F);  Gaussian: p0 = mu, p1 = var;
 *   log_pi (C). */
NB_API nb_status nb_model_params(const nb_model* model, double* host_p0,
                          double* host_p1, double* host_log_pi);

/* Shape of a model (any out pointer may be NULL). */
NB_API nb_status nb_model_info(const nb_model* model, int32_t* kind, int32_t* C,
                        int32_t* F);

NB_API void nb_model_free(nb_model* model);

/* ---- score ---------------------------------------------------------------
 * Classify n files (one group) with a fitted model (Sec. 4 posterior and
 * decision rule).  X has F = the model's F columns in `dtype`.
 *   label    uint8[n]   argmax class (ties -> lowest index)
 *   margin   float[n]   top-1 minus top-2 joint log score
 *   logpost  float[n*C] log posteriors, or NULL
 *   n_rechecked  device int64 (or NULL): receives the number of rows this
 *            call recomputed in FP64.
 * Two-class multinomial models use the difference form d = s_1 - s_0 =
 * b + sum_j x_j (log theta_1j - log theta_0j).  n may be 0.  Asynchronous. */
NB_API nb_status nb_score_group(const nb_model* model, const void* X, nb_dtype dtype,
                         int64_t n, int64_t ld, uint8_t* label, float* margin,
                         float* logpost, const nb_score_opts* opts,
                         void* cuda_stream, int64_t* n_rechecked);

/* The scorer nb_score_group launches for these arguments (before its FP64
 * recheck launch).  Host only: reads the model's shape and tile
 * configuration and the address and pitch of X, launches nothing. */
typedef enum {
  NB_PATH_TWO_CLASS = 0,      /* two-class difference-form scorer */
  NB_PATH_TENSOR = 1,         /* many-class multinomial tensor-core scorer */
  NB_PATH_TENSOR_GAUSS = 2,   /* many-class Gaussian tensor-core scorer */
  NB_PATH_GENERAL = 3         /* CUDA-core scorer (either kind) */
} nb_path;
/* Returns an nb_path, or -1 (and sets the last error) when model is NULL or
 * recheck is not an nb_recheck. */
NB_API int nb_score_path(const nb_model* model, const void* X, nb_dtype dtype, int64_t ld,
                         int recheck);

/* ---- batches of groups: one persistent launch per kernel family ----------
 * The paper scores files group by group, each group with its own model
 * (Sec. 3 size groups, Sec. 4 per-group models).  A batch scores many groups
 * of uneven size (1 to 10^5+ files) at once: the groups of two-class models
 * in one launch of the pipelined two-class kernel, the groups of many-class
 * models in one launch of the tensor-core kernel (U8, FP8E4M3 or BF16 rows
 * that nb_score_group would score there) and one of the general kernel (the
 * rest), then one FP64 recheck launch per family -- independent of the number
 * of groups.  Each row's arithmetic
 * is that of nb_score_group, so a group's results are the same bits alone
 * and inside any batch.
 *
 * nb_batch_create: models[0..n_models) (multinomial, all with the same F,
 *   n_models <= 128; the two-class models' tables, 3 bytes per feature (u8
 *   storage) or 4 (F32), must fit one block's shared memory together, else
 *   NB_EINVAL), the storage dtype of every group (two-class models: U8 or
 *   F32), the largest leading dimension a group will use, the largest number
 *   of groups per call, and the score options (want_logpost, recheck; aux is
 *   ignored -- each group carries its own).  Allocates the batch's device and
 *   pinned host work lists.
 * nb_batch_score: scores groups[0..n_groups) on the stream (asynchronous).
 *   X must be 16-byte aligned with ld * element size a multiple of 16.
 *   n_rechecked: device int64 or NULL.  Successive calls on one batch must be
 *   ordered (one stream); the host buffer of a call is reused two calls later,
 *   after waiting for that call's copy to finish.
 * nb_batch_capture: records the batch's launch sequence (work-list copy, the
 *   scoring launches, the recheck launches) into CUDA graphs on the stream
 *   (which must not be capturing already); later nb_batch_score calls replay
 *   them instead of launching -- the work list is read from device memory, so
 *   one graph serves every batch.
 * nb_batch_destroy: waits for the batch's work and frees it. */
typedef struct {
  int model;              /* slot in the batch's model list */
  const void* X;          /* n x ld elements of the batch's dtype (device) */
  int64_t n;
  int64_t ld;
  nb_aux aux;             /* the group's side arrays (zero when none) */
  uint8_t* label;         /* n */
  float* margin;          /* n */
  float* logpost;         /* n x C, or NULL when want_logpost is 0 */
} nb_group;

typedef struct nb_batch nb_batch;

NB_API nb_status nb_batch_create(const nb_model* const* models, int n_models, nb_dtype dtype,
                                 int64_t max_ld, int max_groups, const nb_score_opts* opts,
                                 nb_batch** out);
NB_API nb_status nb_batch_score(nb_batch* batch, const nb_group* groups, int n_groups,
                                void* cuda_stream, int64_t* n_rechecked);
NB_API nb_status nb_batch_capture(nb_batch* batch, void* cuda_stream);
NB_API void nb_batch_destroy(nb_batch* batch);

/* ---- serving: continuous batching of arriving groups ----------------------
 * The paper classifies the files of each group with the group's model
 * (Sec. 3, Sec. 4); a server keeps the models resident and classifies groups
 * as they arrive.  It owns a device memory budget and a host worker thread.
 * Groups are submitted with nb_classify_stream (asynchronous: it returns a
 * ticket at once) and admitted in arrival order while the budget has room for
 * their staged bytes; a group whose X is host memory is copied to the device
 * on a copy stream as soon as it is admitted.  Each step of the worker scores
 * the groups admitted since the last step (at most max_slots) in one batch
 * (nb_batch_*, replayed from a captured graph) while up to one earlier step
 * still runs on the GPU, copies results bound for host memory back, and
 * completes the tickets of finished steps.  Results equal nb_score_group on
 * the group alone.
 *
 * nb_server_create: models (multinomial, same F, <= 128), the storage dtype of
 *   submitted groups (dense rows, ld = F, no side arrays), the device memory
 *   budget in bytes for staged inputs and outputs (0 = 1 GiB), the most
 *   groups per step (max_slots, the batch size bound), score options.
 * nb_classify_stream: model_id = slot in models; X host or device (n x F);
 *   label / margin / logpost (n x C, or NULL) all device memory (written by
 *   the kernels), all page-locked host memory (written by copies), or host
 *   memory of any kind (staged in the server's page-locked pool and copied
 *   by the worker); they must stay valid until the ticket completes.
 *   NB_EBUSY if the group alone exceeds the budget; NB_EINVAL for outputs
 *   that mix device and host memory.
 * nb_wait: waits for a ticket; NB_ETIMEOUT after timeout_us (< 0: no limit).
 * nb_server_stats: latency percentiles (arrival to completion, microseconds)
 *   and files per second over the completed tickets (any pointer may be NULL).
 * nb_server_destroy: drains the queue, stops the worker, frees everything. */
NB_API nb_status nb_server_create(const nb_model* const* models, int n_models, nb_dtype dtype,
                                  size_t mem_budget, int max_slots, const nb_score_opts* opts,
                                  nb_server** out);
NB_API nb_status nb_classify_stream(nb_server* server, int model_id, const void* X, int64_t n,
                                    int32_t F, uint8_t* label, float* margin, float* logpost,
                                    uint64_t* ticket);
/* Submit `count` groups in one call (same rules as nb_classify_stream, one
 * entry per group in each array; logpost may be NULL).  arrival_us (or NULL
 * = now) gives each group's arrival time on nb_clock_us()'s clock, so a
 * caller replaying an arrival schedule in bursts gets latencies measured from
 * the scheduled arrivals.  On an error, groups before the failing one stay
 * submitted and *submitted tells how many. */
NB_API nb_status nb_classify_stream_batch(nb_server* server, int count, const int* model_ids,
                                          const void* const* X, const int64_t* n,
                                          uint8_t* const* label, float* const* margin,
                                          float* const* logpost, const double* arrival_us,
                                          uint64_t* tickets, int* submitted);
/* The servers' steady clock in microseconds. */
NB_API double nb_clock_us(void);
NB_API nb_status nb_wait(nb_server* server, uint64_t ticket, int64_t timeout_us);
NB_API nb_status nb_server_stats(nb_server* server, double* p50_us, double* p99_us,
                                 double* files_per_s);
NB_API void nb_server_destroy(nb_server* server);

/* ---- tile configuration and autotuning -----------------------------------
 * nb_set_tile_config / nb_get_tile_config: set or read a model's scorer
 * configuration (see nb_tile_config).
 * nb_autotune_score: times the candidate configurations of the model's scorer
 * on the caller's data (X as for nb_score_group; outputs go to scratch it
 * allocates and frees), sets the fastest on the model and returns it in *best
 * (and its time in ms in *best_ms, either may be NULL).  Synchronises the
 * stream; not for use inside stream capture.  Only two-class multinomial
 * models have choices; other models return their default. */
NB_API nb_status nb_set_tile_config(nb_model* model, const nb_tile_config* cfg);
NB_API nb_status nb_get_tile_config(const nb_model* model, nb_tile_config* cfg);
NB_API nb_status nb_autotune_score(nb_model* model, const void* X, nb_dtype dtype,
                                   int64_t n, int64_t ld, const nb_aux* aux,
                                   void* cuda_stream, nb_tile_config* best,
                                   float* best_ms);

/* ---- storage packing (supporting; not part of a timed score) ------------
 * U16 counts -> U8 plane + overflow list, in two calls:
 *   nb_pack_u8_count writes ovf_ptr (n+1 entries, device) and returns the
 *   total number of entries in *host_total (synchronises the stream);
 *   nb_pack_u8_fill writes plane (n x ld_out bytes), ovf_col and ovf_add.
 * Entries are ordered by row, then column. */
NB_API nb_status nb_pack_u8_count(const uint16_t* X, int64_t n, int32_t F, int64_t ld,
                           int64_t* ovf_ptr, int64_t* host_total,
                           void* cuda_stream);
NB_API nb_status nb_pack_u8_fill(const uint16_t* X, int64_t n, int32_t F, int64_t ld,
                          uint8_t* plane, int64_t ld_out,
                          const int64_t* ovf_ptr, uint16_t* ovf_col,
                          uint16_t* ovf_add, void* cuda_stream);
/* U16 or F32 non-negative values -> BF16 (round to nearest even). */
NB_API nb_status nb_pack_bf16(const void* X, nb_dtype src, int64_t n, int32_t F,
                       int64_t ld, uint16_t* out, int64_t ld_out,
                       void* cuda_stream);
/* U16 or F32 non-negative values -> FP8 E4M3 with a per-row exponent
 * e = max(0, ceil(log2(max_row / 448))), stored byte = E4M3(x / 2^e) (round
 * to nearest even). */
NB_API nb_status nb_pack_fp8(const void* X, nb_dtype src, int64_t n, int32_t F,
                      int64_t ld, uint8_t* out, int64_t ld_out,
                      int8_t* row_exp, void* cuda_stream);

/* ---- the group-wise method ------------------------------------------------
 * Sec. 3: files below 500 KB fall into 100 size groups of 5 KB; per group the
 * opcodes whose normalised occurrence differs most between malware and benign
 * files are kept (top k, k = 20..200 in Sec. 4).  Sec. 4: one model per
 * group on its k opcodes, except for groups with fewer than six training
 * files of either class, whose files take the next group's model.
 * Readings: size group g = min(floor(size / bin_bytes), n_bins - 1) (5120
 * and 100 in the paper; a larger file joins the last group); a group is
 * trained when every class has >= min_files files; an untrained group takes
 * the first trained group above it, else the nearest one below. */

/* HOST function.  class_counts: n_bins x C training files per (group,
 * class), host memory.  Writes model_of[g] (host, n_bins) = the group whose
 * model classifies group g's files.  NB_EINVAL when no group is trained. */
NB_API nb_status nb_group_fallback(const int64_t* class_counts, int32_t n_bins, int32_t C,
                                   int64_t min_files, int32_t* model_of);

/* Route n files by size and sort them by group, stably.
 *   sizes     int64[n] file sizes in bytes (device);
 *   model_of  int32[n_bins] (device) maps size groups to output groups
 *             [0, n_groups), or NULL: output group = size group (n_groups
 *             must equal n_bins);  n_groups <= 512;
 *   group     int32[n] (device): output group of each file;
 *   order     int64[n] (device, or NULL): files listed by group, in file
 *             order inside a group;  offsets int64[n_groups + 1] (device):
 *             group g is order[offsets[g] .. offsets[g+1]);
 *   y, C, class_counts: with labels y (device int32[n], classes < C) and
 *             class_counts (device int64[n_bins x C], n_bins * C <= 4096),
 *             the training files per (size group, class); else NULL;
 *   workspace device scratch of >= nb_route_workspace(n, n_groups) bytes;
 *   status    device int: the value 32 is or-ed in for a negative size
 *             (counted as 0), a model_of entry or a label out of range.
 * Three kernels, asynchronous on the stream. */
NB_API size_t nb_route_workspace(int64_t n, int32_t n_groups);
NB_API nb_status nb_route(const int64_t* sizes, int64_t n, int64_t bin_bytes, int32_t n_bins,
                          const int32_t* model_of, int32_t n_groups, const int32_t* y,
                          int32_t C, int32_t* group, int64_t* order, int64_t* offsets,
                          int64_t* class_counts, void* workspace, size_t workspace_bytes,
                          int* status, void* cuda_stream);

/* Top-k opcode selection of two-class multinomial models (fitted on a
 * group's training files over all opcodes).  With f_cj = N_cj / D_c, D_c the
 * class's total count (NB_SELECT_TOTAL) or number of files (NB_SELECT_FILES)
 * and f_c = 0 when D_c = 0, opcode j scores |f_1j - f_0j|, compared exactly
 * (128-bit integers over the common denominator); larger first, ties to the
 * lower index.  cols (device int32, n_models x k): model i's first k opcodes
 * in rank order.  n_models <= 128, 1 <= k <= F.  The models' fits must be
 * complete or ordered before the stream. */
typedef enum { NB_SELECT_TOTAL = 0, NB_SELECT_FILES = 1 } nb_select_norm;
NB_API nb_status nb_select_features(const nb_model* const* models, int32_t n_models,
                                    int32_t k, int32_t norm, int32_t* cols, void* cuda_stream);

/* Gather: out[r][t] = X[s][cols[g * k + t]] for t < k and 0 for k <= t <
 * ld_out, where s = order[r] (or r when order is NULL) and g = group[s] (or 0
 * when group is NULL; cols NULL: column t).  X: n_src source rows of F
 * elements (U8 or F32, row pitch ld); n output rows of pitch ld_out (U8: a
 * multiple of 4).  A source row outside [0, n_src) or a group outside [0,
 * n_groups) gives a zero row, a column outside [0, F) a zero; each raises the
 * value 32 in *status (device int).  All pointers device. */
NB_API nb_status nb_gather(const void* X, nb_dtype dtype, int64_t ld, int32_t F, int64_t n_src,
                           int64_t n,
                           const int64_t* order, const int32_t* group, int32_t n_groups,
                           const int32_t* cols, int32_t k, void* out, int64_t ld_out,
                           int* status, void* cuda_stream);

/* Group-wise classification of files given as full opcode histograms.
 * nb_groupwise_create: models[0..n_models) two-class multinomial, each on k
 *   opcodes (F = k), n_models <= 128; cols (host or device, n_models x k) the
 *   opcodes of each model in its feature order; model_of (host, n_bins) the
 *   model slot of each size group (for example nb_group_fallback's result
 *   renumbered to slots); bin_bytes; F_full the histogram width; dtype U8 or
 *   F32; max_files per call; score options.  Allocates all scratch.
 * nb_groupwise_classify: X (device, n x ld, ld >= F_full) full histograms,
 *   sizes (device int64[n]); label / margin / logpost (n x 2 or NULL) device,
 *   in the files' order.  U8 histograms with 16-byte aligned rows take one
 *   fused launch: every model's weights and opcode selection sit in shared
 *   memory, each row finds its model from its size and is scored on its
 *   selected counts straight from the streamed histogram, then the FP64
 *   recheck (two launches in all).  Otherwise -- F32 histograms, unaligned
 *   rows, or models whose tables exceed shared memory -- the files are routed
 *   (nb_route), each file's model's opcodes gathered into a dense matrix
 *   ordered by group (nb_gather), every group scored in one batched launch
 *   whose work list a kernel builds on the device, rechecked in FP64, and the
 *   results scattered back (eight launches).  No host synchronisation either
 *   way; every file's results equal nb_score_group of its model on its
 *   gathered row.  Asynchronous.  The models must not be re-fitted while the
 *   object exists (the fused path keeps a copy of their u8 tables).
 * nb_groupwise_status: reads (synchronously) the object's status word (32:
 *   a bad size or column was met).  nb_groupwise_destroy frees everything. */
typedef struct nb_groupwise nb_groupwise;
NB_API nb_status nb_groupwise_create(const nb_model* const* models, int32_t n_models,
                                     const int32_t* cols, int32_t k, const int32_t* model_of,
                                     int32_t n_bins, int64_t bin_bytes, int32_t F_full,
                                     nb_dtype dtype, int64_t max_files,
                                     const nb_score_opts* opts, nb_groupwise** out);
NB_API nb_status nb_groupwise_classify(nb_groupwise* gw, const void* X, int64_t ld,
                                       const int64_t* sizes, int64_t n, uint8_t* label,
                                       float* margin, float* logpost, void* cuda_stream,
                                       int64_t* n_rechecked);
NB_API nb_status nb_groupwise_status(nb_groupwise* gw, int* host_status);
NB_API void nb_groupwise_destroy(nb_groupwise* gw);

/* ---- errors / misc -------------------------------------------------------*/
NB_API const char* nb_last_error(void);
/* Number of CUDA kernels this library has launched in this process. */
NB_API uint64_t nb_kernel_launches(void);
NB_API const char* nb_version(void);

#ifdef __cplusplus
}
#endif
#endif /* NBGPU_H */
