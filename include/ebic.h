/* ebic.h -- C ABI of the GB300 (sm_103a) EBIC library.
 *
 * EBIC (arXiv 1801.03039) searches for order-preserving biclusters: a
 * bicluster is a series of column indices, and a row supports the series when
 * its values strictly rise along it (section "Motivation").  This library runs
 * the data-parallel core of the method on one GPU:
 *   - support counting and Eq. (1) fitness for a population of series
 *     (Step 4 of the "EBIC Algorithm" section), and
 *   - the whole generation loop of Steps 1-5 (elitism, tournament with the
 *     crowding penalty, mutation, crossover, tabu list, top-rank list),
 *     kept on the device between calls.
 *
 * Conventions shared by every entry point:
 *   - Matrices are row-major float32 [rows][cols] on the caller's side.
 *   - A population is given in CBF (Fig. 3): offsets[P + 1] (int32, offsets[0]
 *     = 0, non-decreasing, offsets[P] = total length) and cols[offsets[P]]
 *     (int32, 0-based column indices).  Fig. 3 stores only the P start
 *     offsets; this ABI adds offsets[P] so that every length is explicit.
 *   - Series lengths are 1 .. EBIC_MAX_EVAL_LEN for evaluation.  A column may
 *     repeat inside a series; such a series is supported by no row (the strict
 *     chain cannot pass the same value twice).  A length-1 series is supported
 *     by every row.
 *   - Every buffer the caller passes stays owned by the caller.  Inputs are
 *     only read, during the call (host variants) or until the work queued on
 *     the given stream has run (device variants).
 *   - Every call returns an ebic_status.  On EBIC_ERR_ARG nothing was written
 *     and no GPU work was queued.  ebic_last_error() gives a message for the
 *     last failing call on the calling thread.
 *   - A handle is bound to the CUDA device that was current when it was
 *     created.  A handle must not be used from two threads at once.
 *   - `void* stream` parameters take a cudaStream_t (NULL = legacy default).
 */
#ifndef EBIC_H_
#define EBIC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EBIC_ABI_VERSION 2
#define EBIC_MAX_EVAL_LEN 1024 /* longest series accepted by evaluation */
#define EBIC_MAX_EA_LEN 64     /* longest series the EA builds (len_max) */
#define EBIC_MAX_TOURNAMENT 4  /* largest tournament_k */

typedef struct ebic_ctx* ebic_handle;

typedef enum {
  EBIC_OK = 0,
  EBIC_ERR_ARG = 1,       /* invalid argument; nothing written */
  EBIC_ERR_CUDA = 2,      /* a CUDA call failed; see ebic_last_error() */
  EBIC_ERR_OOM = 3,       /* device allocation failed */
  EBIC_ERR_TIMEOUT = 4,   /* a bounded device wait gave up */
  EBIC_ERR_STATE = 5,     /* call out of order (e.g. step before init) */
  EBIC_ERR_CANCELLED = 6, /* reserved: run cancelled by the caller */
  EBIC_ERR_DEVICE = 7     /* a kernel flagged invalid device-side input */
} ebic_status;

/* Support path of the evaluation kernel. */
typedef enum {
  EBIC_PATH_AUTO = 0,    /* pick by the built-in cost model / autotuner */
  EBIC_PATH_GATHER = 1,  /* compare fp32 values read from the column-major matrix */
  EBIC_PATH_BITMASK = 2  /* AND precomputed pair bitmasks (needs the pair table) */
} ebic_path;

/* Which support enters |I| of Eq. (1). */
typedef enum {
  EBIC_SUPPORT_INC = 0,         /* rows rising along the series (the paper's search) */
  EBIC_SUPPORT_INC_PLUS_DEC = 1 /* rising plus falling rows */
} ebic_support_mode;

const char* ebic_last_error(void);
int32_t ebic_abi_version(void);
/* Number of CUDA kernels this library has launched in this process (all
 * handles, all threads); for measurement tools.  Library-internal memsets and
 * copies are not counted. */
uint64_t ebic_kernel_launches(void);
/* Read-bandwidth probe for measurement tools (no counterpart in the paper):
 * reads every byte of the device buffer d_buf (`bytes`, a multiple of 16) in
 * one kernel, once to warm the caches and then `reps` times, each timed with
 * CUDA events on `stream` (NULL: the legacy default stream; synchronises it).
 * *out_best_us = the fastest timed pass.  A buffer smaller than the L2 cache
 * gives the L2 read bandwidth, a larger one the HBM read bandwidth.  The
 * buffer is only read.  Allocates 4 bytes of device memory for the call. */
ebic_status ebic_probe_read_bandwidth(const void* d_buf, uint64_t bytes, int32_t reps,
                                      void* stream, float* out_best_us);

/* ---------------------------------------------------------------------------
 * Matrix.  Step 1 of the "EBIC Algorithm" section: the data is placed on the
 * GPU once.  The library keeps it column-major (each column padded to a
 * multiple of 128 rows with NaN, which no comparison passes), so that warps
 * walking rows read consecutive addresses, plus the table LN[m] = log(m)
 * (binary64, host libm) used by Eq. (1).
 *
 * ebic_load_matrix: host_rowmajor = rows x cols float32, row-major, host
 *   memory (pageable or pinned).  rows in [1, 2^26], cols in [1, 65535].  The
 *   data is copied; the caller keeps its buffer.  *out receives a new handle.
 * ebic_load_matrix_dev: the same from device memory, queued on `stream`.
 * ebic_free: releases the handle and all its device memory (NULL is ignored).
 * ------------------------------------------------------------------------- */
ebic_status ebic_load_matrix(const float* host_rowmajor, int32_t rows, int32_t cols,
                             ebic_handle* out);
ebic_status ebic_load_matrix_dev(const float* dev_rowmajor, int32_t rows, int32_t cols,
                                 void* stream, ebic_handle* out);
void ebic_free(ebic_handle h);

/* Shape queries. */
ebic_status ebic_matrix_shape(ebic_handle h, int32_t* rows, int32_t* cols);

/* ---------------------------------------------------------------------------
 * Pair bitmask table (derived from the pairwise count #{k : a_kp < a_kq} of
 * the "Motivation" section).  Layout: uint32 [cols][cols][words], words =
 * padded rows / 32; words 4b .. 4b + 3 of entry (p, q) cover rows 128b ..
 * 128b + 127, and bit l of word 4b + i is set iff row k = 128b + 4l + i has
 * a[k][p] < a[k][q] (IEEE; NaN and ties give 0; rows past the end give 0).
 * Size cols^2 * words * 4 bytes; the call fails with EBIC_ERR_OOM if that does
 * not fit.  Built on `stream`.  ebic_pair_table_bytes reports the size the
 * table would take (0 if not built yet in *built).
 * ------------------------------------------------------------------------- */
ebic_status ebic_build_pair_table(ebic_handle h, void* stream);
ebic_status ebic_pair_table_bytes(ebic_handle h, uint64_t* bytes, int32_t* built);
/* Copy words [w0, w0 + n) of entry (p, q) of the built table to host memory. */
ebic_status ebic_read_pair_words(ebic_handle h, int32_t p, int32_t q, int32_t w0, int32_t n,
                                 uint32_t* host_out);

/* Force a support path for later evaluations (EBIC_PATH_AUTO restores the
 * automatic choice).  EBIC_PATH_BITMASK builds the table if needed. */
ebic_status ebic_set_path(ebic_handle h, int32_t path);

/* Launch shape of later evaluations (set by the autotuner or by hand; every
 * field 0 = automatic).  Results never depend on these.
 *   kernel: bitmask path only -- 1 = one lane per 16-byte vector of a table
 *     entry (entries of at most 32 vectors, i.e. up to 4,096 rows), 2 = one
 *     warp per series part, 3 = staged: a persistent kernel in which one
 *     scout warp per group of warps copies the first dense_steps table rows
 *     of each series part into shared memory with bulk copies (the rows every
 *     128-row block still needs) and the group's other warps AND them and
 *     walk the remaining steps with per-vector loads and early exit; rising
 *     counts only (support mode EBIC_SUPPORT_INC, no falling counts), else
 *     the warp kernel runs.  4 = phased: a persistent kernel in which each
 *     CTA owns a fixed set of series and takes them in chunks of up to 32;
 *     each of its first warps owns a shared-memory slot, copies the first
 *     dense_steps table rows of one series at a time into it (cp.async),
 *     ANDs them and issues the next series' copies before loading the next
 *     steps of the 128-row blocks still alive; blocks alive after that are
 *     finished by the whole CTA at the end of the chunk; rising counts
 *     only, and only where two slots fit (else kernel 3's rules apply).  0 = lane kernel up
 *     to 2,048 rows, else warp kernel.
 *   vecs_per_part_bitmask / vecs_per_part_gather: 16-byte vectors of a table
 *     entry / of a column that one warp walks before the rest of the series
 *     goes to another warp (rounded to a multiple of 32).  For kernel 3,
 *     vecs_per_part_bitmask caps the vectors of one item (at most 256, the
 *     default cap; a series is cut into equal parts under the cap).
 *   batch_steps: AND steps fetched between two early-exit tests (4 or 8).
 *   vecs_per_lane: 16-byte vectors each lane of the warp kernel carries
 *     (1, 2 or 4; 4 only with batch_steps 4).  Series that need the falling
 *     count use batch_steps 4 and one vector per lane.
 *   dense_steps (kernels 3, 4): AND steps copied whole into shared memory,
 *     1..8 (0 = 4 for kernel 3, 5 for kernel 4).
 *   stages (kernel 3): items in flight per group, 2..4 (0 = 2); for kernel
 *     4 a cap on the slots, one per warp (0 = as many as fit, at most 32).
 *   groups (kernel 3): at most this many groups of warps per CTA (0 = as many
 *     as fit one CTA per SM).
 *   dynamic_rounds (kernel 3): groups take items in a fixed stride, except
 *     for this many last rounds of the even share plus the remainder, which
 *     they claim one at a time from a counter (1 .. 64; 0 or -1 = none,
 *     every item in the stride).
 *   vecs_per_lane also sets, for kernel 3, the 16-byte vectors each
 *     consumer thread carries: 1, 2 or 3 (0 = 2 for table entries over 64
 *     vectors; with 3 the remaining steps go two per batch). */
typedef struct {
  int32_t kernel;
  int32_t vecs_per_part_bitmask;
  int32_t vecs_per_part_gather;
  int32_t batch_steps;
  int32_t vecs_per_lane;
  int32_t dense_steps;
  int32_t stages;
  int32_t groups;
  int32_t dynamic_rounds;
} ebic_eval_tuning_t;
/* NULL restores the automatic choice. */
ebic_status ebic_set_eval_tuning(ebic_handle h, const ebic_eval_tuning_t* tuning);
ebic_status ebic_get_eval_tuning(ebic_handle h, ebic_eval_tuning_t* out);
/* Autotuner: evaluates the given device population (arguments as for
 * ebic_eval_population_dev, which it is) under a short list of launch shapes
 * for the handle's current path, timing each with CUDA events on `stream`, and
 * keeps the fastest for later evaluations.  Synchronises `stream`.  *chosen
 * and *best_us (nullable) receive the shape and its time per launch.
 * flags: 0 = time launches back to back (the table stays in L2 when it fits,
 * as in a generation loop); EBIC_TUNE_COLD_L2 = time each launch after the L2
 * has been emptied (an overwrite of one buffer of twice the L2 size, then a
 * read of another; both allocated for the call and freed), the case of a
 * table that other work evicts between passes.  Other bits: EBIC_ERR_ARG. */
#define EBIC_TUNE_COLD_L2 1
ebic_status ebic_autotune_eval(ebic_handle h, const int32_t* d_offsets, const int32_t* d_cols,
                               int32_t P, int32_t total_cols, int32_t sigma, int32_t support_mode,
                               uint32_t* d_inc, uint32_t* d_dec, double* d_fitness, void* stream,
                               int32_t flags, ebic_eval_tuning_t* chosen, float* best_us);

/* ---------------------------------------------------------------------------
 * Population evaluation: Step 4 of the "EBIC Algorithm" section with Eq. (1).
 * For each series s of the CBF population:
 *   inc[s] = #rows k with a[k][s0] < a[k][s1] < ... (strict, IEEE)
 *   dec[s] = #rows k with a[k][s0] > a[k][s1] > ...
 *   n      = inc (EBIC_SUPPORT_INC) or inc + dec (EBIC_SUPPORT_INC_PLUS_DEC)
 *   fitness[s] = 0 if n <= 1, else ldexp(LN[n - 1], min(n - sigma, 0)) * |s|
 *               (binary64; LN[m] = log(m) from the host libm)
 * Results are exact: counts are integers and the fitness is the same binary64
 * value a CPU evaluating the formula with that libm produces.
 *
 * ebic_eval_population: all buffers in host memory; synchronous.  offsets has
 *   P + 1 entries; cols offsets[P] entries; out_inc and out_fitness P entries;
 *   out_dec P entries or NULL.  P in [0, 2^24].  Invalid CBF (a column outside
 *   [0, cols), a length outside [1, EBIC_MAX_EVAL_LEN], offsets[0] != 0) gives
 *   EBIC_ERR_ARG with nothing written to the caller's buffers.  The offsets
 *   are checked before anything is queued; the column indices are checked on
 *   the host while the device evaluates (whose kernels bound-check them too;
 *   the device error flag this raises is cleared before the call returns).
 *   The results come back in one copy through a pinned stage of the handle.
 * ebic_eval_population_dev: the same with device buffers, queued on `stream`
 *   (asynchronous).  total_cols must equal offsets[P].  The CBF is validated on
 *   the device: an invalid series gets inc = dec = 0 and fitness = 0, and sets
 *   the handle's device error flag, which ebic_check_device_error() reports
 *   (EBIC_ERR_DEVICE) and clears.
 * ------------------------------------------------------------------------- */
ebic_status ebic_eval_population(ebic_handle h, const int32_t* offsets, const int32_t* cols,
                                 int32_t P, int32_t sigma, int32_t support_mode,
                                 uint32_t* out_inc, uint32_t* out_dec, double* out_fitness);
ebic_status ebic_eval_population_dev(ebic_handle h, const int32_t* d_offsets,
                                     const int32_t* d_cols, int32_t P, int32_t total_cols,
                                     int32_t sigma, int32_t support_mode, uint32_t* d_inc,
                                     uint32_t* d_dec, double* d_fitness, void* stream);
/* Synchronises the handle's work and reports/clears the device error flag. */
ebic_status ebic_check_device_error(ebic_handle h);

/* Evaluation that allocates nothing (the paper has no counterpart to this
 * entry point).  For callers that must not have a library allocate device
 * memory -- code inside a host framework that owns the device memory through
 * its own pool, or a latency-critical loop that cannot take the device
 * synchronisation an allocation may cause.  It computes the same inc and
 * fitness as ebic_eval_population_dev with EBIC_SUPPORT_INC and no dec
 * output, queued on `stream`; the caller owns every input and output.
 * Series split across warps keep their partial counts in one fixed static
 * device array of 16 bytes per series, EBIC_NOALLOC_MAX_SERIES series (1 MiB),
 * which every GPU that loads the library holds until the process exits.
 *   - P above EBIC_NOALLOC_MAX_SERIES gives EBIC_ERR_ARG (nothing queued).
 *   - It never builds the pair table: with the table already built (and the
 *     path not forced to gather) it uses it, otherwise the gather path.
 *   - Its launch shape is fixed (the warp kernel, 8 AND steps per exit test,
 *     the automatic split of series into parts): the handle's tuning, from
 *     ebic_set_eval_tuning or ebic_autotune_eval, does not apply to it.
 *   - The first call on each device looks up the array's device address with
 *     that device current; make that first call before any stream capture.
 *   - All calls share the array, which keeps the last call's contents (each
 *     call clears the part it uses first): calls that overlap on the GPU --
 *     from several streams, threads or handles at once -- race.
 *   - Invalid series are reported through ebic_check_device_error, as for
 *     ebic_eval_population_dev. */
#define EBIC_NOALLOC_MAX_SERIES 65536
ebic_status ebic_eval_population_dev_noalloc(ebic_handle h, const int32_t* d_offsets,
                                             const int32_t* d_cols, int32_t P,
                                             int32_t total_cols, int32_t sigma, uint32_t* d_inc,
                                             double* d_fitness, void* stream);

/* ---------------------------------------------------------------------------
 * Many problems in one launch (Step 4 repeated over independent problems, e.g.
 * restarts or datasets side by side).  A batch binds n (handle, population)
 * pairs; ebic_batch_eval then evaluates all of them -- rising support and
 * Eq. (1) fitness, exactly as ebic_eval_population_dev with
 * EBIC_SUPPORT_INC -- in one persistent launch that pulls (problem, series,
 * part) work items longest-first.  All handles must be on one device.
 * Flags:
 *   EBIC_BATCH_BUILD_TABLES  build each problem's pair table if it fits in
 *                            half the free device memory (cumulative);
 *   EBIC_BATCH_AUTOTUNE      time the gather and bitmask paths and a few part
 *                            sizes per problem (on the problem's own
 *                            population, writing its outputs) and keep the
 *                            fastest; otherwise bitmask where the table
 *                            exists, whole series per warp;
 *   EBIC_BATCH_GRAPH         capture the launch as a CUDA graph on the first
 *                            ebic_batch_eval and replay it afterwards.
 * The item buffers are caller-owned and must stay valid while the batch
 * exists.  ebic_batch_create synchronises `stream` and reads the offsets. */
typedef struct ebic_batch_ctx* ebic_batch;
typedef struct {
  const int32_t* d_offsets;  /* device, P + 1 entries */
  const int32_t* d_cols;     /* device, total_cols entries */
  int32_t P;
  int32_t total_cols;
  int32_t sigma;
  uint32_t* d_inc;           /* device, P entries (output) */
  double* d_fitness;         /* device, P entries (output) */
} ebic_batch_item_t;
#define EBIC_BATCH_AUTOTUNE 1
#define EBIC_BATCH_GRAPH 2
#define EBIC_BATCH_BUILD_TABLES 4
ebic_status ebic_batch_create(const ebic_handle* handles, const ebic_batch_item_t* items,
                              int32_t n, int32_t flags, void* stream, ebic_batch* out);
/* One evaluation of every problem, queued on `stream`. */
ebic_status ebic_batch_eval(ebic_batch b, void* stream);
/* The path (EBIC_PATH_*), vectors per part and parts per series chosen for a
 * problem; the total work items and the persistent grid size. */
ebic_status ebic_batch_describe(ebic_batch b, int32_t problem, int32_t* path,
                                int32_t* vecs_per_part, int32_t* parts, int64_t* work_items,
                                int32_t* grid);
void ebic_batch_free(ebic_batch b);

/* ---------------------------------------------------------------------------
 * Generation loop: Steps 1-5 of the "EBIC Algorithm" section, run entirely on
 * the device.  Semantics (identical to the library's reference reading):
 *   Step 1: distinct random series (length uniform in [len_min, len_max],
 *     distinct columns) until P are accepted; evaluate; build the top-rank list.
 *   Step 2: the best ceil(elite_frac * |list|) records start the new
 *     population; every column use raises that column's penalty count.
 *   Step 3: attempts until P individuals: tournament of tournament_k entrants
 *     from the previous population by f / penalty_base^theta (theta = mean
 *     penalty count of the entrant's columns; ties to the lower index); with
 *     probability p_crossover a second tournament and one-point crossover;
 *     then one of the four mutations (Fig. 1).  A child already evaluated in
 *     this run (tabu list) is a hit; more than P hits in one generation stops
 *     the run.
 *   Step 4: support and Eq. (1).
 *   Step 5: top-rank update by decreasing fitness: add unless an overlapping
 *     record of higher or equal fitness is listed (overlap = |a & b| /
 *     min(|a|, |b|) > overlap_tau); evict overlapping records of lower
 *     fitness; keep the toprank_size best.
 * Random numbers: Philox-4x32-10 (Salmon et al., SC'11), draw d of attempt j in
 * generation g = word d % 4 of Philox(counter (j, g, d / 4, 0), key = seed).
 * ------------------------------------------------------------------------- */
typedef struct {
  int32_t pop_size;        /* P >= 2 */
  int32_t len_min;         /* >= 1 */
  int32_t len_max;         /* len_min .. min(cols, EBIC_MAX_EA_LEN) */
  int32_t iterations;      /* Steps 2-5 passes run by ebic_run_generations */
  int32_t sigma;           /* Eq. (1) */
  int32_t toprank_size;    /* T >= 1 */
  int32_t tournament_k;    /* 1 .. EBIC_MAX_TOURNAMENT */
  int32_t support_mode;    /* ebic_support_mode */
  double overlap_tau;      /* in [0, 1] */
  double elite_frac;       /* in [0, 1]; the paper's value is 0.25 */
  double penalty_base;     /* >= 1; the paper's value is 1.2 */
  double p_crossover;      /* in [0, 1] */
  uint64_t seed;
} ebic_params_t;

typedef struct {
  int32_t generations_done;  /* Steps 2-5 passes completed */
  int32_t stop_reason;       /* 0 iterations reached, 1 tabu hits > P, 2 Step 1 failed */
  int64_t tabu_hits_total;
  int64_t attempts_total;
  int64_t evaluations_total;
  int32_t last_gen_hits;
  int32_t toprank_n;
  int64_t exact_tournaments; /* tournaments decided by the exact binary64 path */
} ebic_stats_t;

/* Fill *p with the defaults (P 100, len 2..6, sigma 10, T 100, k 2, tau 0.5,
 * elite 0.25, base 1.2, p_crossover 0.5, seed 0, 10 iterations). */
void ebic_default_params(ebic_params_t* p);

/* Step 1.  Allocates the run state on the device (population archive, tabu
 * hash table sized for (iterations + 1) * P series, penalty table) and runs
 * Step 1.  Replaces any earlier run of the handle.  The run evaluates with
 * the handle's launch shape when one was set with a nonzero kernel
 * (ebic_set_eval_tuning, ebic_autotune_eval), else with the shape the
 * autotuner picks on the initial population. */
ebic_status ebic_run_init(ebic_handle h, const ebic_params_t* p);
/* Steps 2-5, `generations` times (fewer if the tabu rule stops the run, or if
 * the archive is full: EBIC_ERR_STATE).  Synchronous. */
ebic_status ebic_run_step(ebic_handle h, int32_t generations, ebic_stats_t* stats);
/* Steps 2-5, `generations` times, queued on `stream` without waiting and
 * without reading anything back: generations after a stop do nothing, and
 * the caller learns where the run stands from ebic_run_step(h, 0, &stats) once
 * `stream` has been synchronised.  The run must not go past the generations
 * ebic_run_init sized it for (later generations are not written). */
ebic_status ebic_run_step_async(ebic_handle h, int32_t generations, void* stream);
/* One generation (Steps 2-5) as separate launches with CUDA events between
 * them; kernel_us[8] (nullable) receives the durations of: attempt
 * speculation (with screening: the whole records stage), the sequential
 * Step 3 builder, tabu insertion, Step 4 evaluation, Step 5 ranking; then,
 * with screening, the records stage split into candidate children, their
 * scores and the pick (zeros without screening).  Synchronous; for
 * measurement. */
ebic_status ebic_run_step_profiled(ebic_handle h, float* kernel_us);
/* In-graph timing of the Step 3 builder, for measurement.  Set before
 * ebic_run_init (it takes effect there; 0, the default, turns it off): the
 * captured generation then holds two event-record nodes around k_build, and
 * each replay by ebic_run_step / ebic_run_step_async points them at the next
 * of `slots` event pairs (a replay that reuses a pair first waits for the one
 * that used it).  EBIC_ERR_ARG unless 0 <= slots <= 2^20. */
ebic_status ebic_set_kernel_timing(ebic_handle h, int32_t slots);
/* Waits for every timed replay, then writes the mean k_build duration (us)
 * and the number of replays it covers since the run began or since the last
 * read with `reset` != 0, which starts the count again.  EBIC_ERR_STATE if the
 * run was started without timing. */
ebic_status ebic_read_kernel_timing(ebic_handle h, int32_t reset, double* mean_us,
                                    long long* count);
/* The current top-rank list as CBF: *inout_n = capacity in records on entry,
 * records written on return; offsets needs capacity + 1 entries and cols
 * capacity * len_max.  fitness / inc may be NULL. */
ebic_status ebic_get_toprank(ebic_handle h, int32_t* offsets, int32_t* cols, double* fitness,
                             uint32_t* inc, int32_t* inout_n);
/* The current population (P records) in the same form, with inc, dec and
 * fitness (each nullable). */
ebic_status ebic_get_population(ebic_handle h, int32_t* offsets, int32_t* cols, uint32_t* inc,
                                uint32_t* dec, double* fitness, int32_t* inout_n);
/* ebic_run_init + ebic_run_step(p->iterations) + ebic_get_toprank. */
ebic_status ebic_run_generations(ebic_handle h, const ebic_params_t* p, int32_t* out_offsets,
                                 int32_t* out_cols, double* out_fitness, int32_t* inout_n,
                                 ebic_stats_t* stats);

/* ---------------------------------------------------------------------------
 * Step 6 ("Prepare biclusters": the indices of the rows that match each
 * series of columns) and Step 7's expansion by negative trends.
 * EBIC_ROWS_RISING: the rows whose values rise strictly along the series (the
 * support of Step 4, as a list).  EBIC_ROWS_RISING_OR_FALLING: also the rows
 * that fall strictly along it (negative trends).  A one-column series matches
 * every row.  Step 7's expansion by "approximate" trends, which the paper does
 * not define, is ebic_extract_rows_approx below under a stated reading.
 *
 * offsets / cols: a CBF population as for ebic_eval_population (host).
 * row_offsets[P + 1] (host, int64) and rows (host): the row indices of series
 * i, ascending, are rows[row_offsets[i] .. row_offsets[i + 1]).
 * *inout_capacity: entries of `rows` on entry, entries written on return.  If
 * the rows do not fit, the call returns EBIC_ERR_ARG with the number needed in
 * *inout_capacity and writes nothing else (rows may be NULL to ask for it).
 * ------------------------------------------------------------------------- */
typedef enum {
  EBIC_ROWS_RISING = 0,
  EBIC_ROWS_RISING_OR_FALLING = 1
} ebic_rows_mode;
ebic_status ebic_extract_rows(ebic_handle h, const int32_t* offsets, const int32_t* cols,
                              int32_t P, int32_t mode, int64_t* row_offsets, int32_t* rows,
                              int64_t* inout_capacity);
/* Step 7's expansion by approximate trends, read as: a row follows a series
 * approximately when at most max_breaks of its L - 1 adjacent pairs do not
 * rise strictly (EBIC_ROWS_RISING_OR_FALLING: or at most max_breaks do not
 * fall strictly).  Ties and NaN break a pair in both directions.
 * max_breaks = 0 gives the rows of ebic_extract_rows.  Arguments, output and
 * errors as for ebic_extract_rows; EBIC_ERR_ARG unless 0 <= max_breaks <=
 * EBIC_MAX_EVAL_LEN. */
ebic_status ebic_extract_rows_approx(ebic_handle h, const int32_t* offsets, const int32_t* cols,
                                     int32_t P, int32_t max_breaks, int32_t mode,
                                     int64_t* row_offsets, int32_t* rows,
                                     int64_t* inout_capacity);

/* Recovery and relevance, Eq. (2)-(3): a bicluster is the set of cells rows x
 * columns and the Jaccard index of two biclusters is |e & f| / |e | f| over
 * cells.  recovery = mean over the E expected biclusters of the best index
 * against the F found ones; relevance = mean over the found ones of the best
 * against the expected ones (the paper's sums divided by their number of
 * terms).  Each bicluster is given as ascending, distinct row and column
 * indices in CSR form (host buffers: *_off[n + 1] int64 offsets into the
 * index arrays).  out_jaccard (nullable, host, E x F row-major) receives the
 * pairwise indices.  E or F = 0 gives 0 and 0.  Synchronous; runs on the
 * current device. */
ebic_status ebic_recovery_relevance(int32_t E, const int64_t* e_row_off, const int32_t* e_rows,
                                    const int64_t* e_col_off, const int32_t* e_cols, int32_t F,
                                    const int64_t* f_row_off, const int32_t* f_rows,
                                    const int64_t* f_col_off, const int32_t* f_cols,
                                    double* out_recovery, double* out_relevance,
                                    double* out_jaccard);

/* ---------------------------------------------------------------------------
 * Fitness surrogate and offspring screening.  The paper has no counterpart:
 * EBIC evaluates every child exactly (Step 4).  This is an optional
 * pre-screen: a small learned model predicts which of several candidate
 * children scores best, and only the chosen one goes on to Step 3's
 * acceptance and Step 4's exact evaluation, so every individual that enters a
 * population is still scored by Eq. (1) on exact support.
 *
 * Model: x[0:64] = sum over the series' columns of a learned 64-dimensional
 * column embedding, x[64] / x[65] = mean over the series' columns of the
 * column mean / population standard deviation of the matrix (NaN skipped),
 * x[66] = length / len_scale, x[67:80] = 0;  h1 = relu(x W1 + b1) (256),
 * h2 = relu(h1 W2 + b2) (256), y = h2 . w3 + b3.  y predicts the standardised
 * target (log1p(fitness) - mean) / sd, mean and sd taken over the training
 * set.  Operands bf16 on the tensor cores, fp32 accumulation, fp32 master
 * weights, Adam (beta1 0.9, beta2 0.999, eps 1e-8) on mean squared error.
 *
 * Parameter layout of the flat fp32 vector (ebic_surrogate_params):
 *   Emb [C][64] | W1 [80][256] | b1 [256] | W2 [256][256] | b2 [256] |
 *   w3 [256] | b3 [1]
 * ------------------------------------------------------------------------- */
typedef struct ebic_surrogate_ctx* ebic_surrogate;

/* A surrogate for the handle's matrix (column count and column statistics are
 * taken from it; the handle must outlive the surrogate).  Weights are
 * initialised from `seed` (embeddings N(0, 0.01), W1 / W2 He-scaled normal,
 * w3 N(0, 1/256), biases 0).  Column ids fit 16 bits (ebic_load_matrix
 * accepts at most 65,535 columns); the scoring kernel relies on it. */
ebic_status ebic_surrogate_create(ebic_handle h, int32_t len_scale, uint64_t seed,
                                  ebic_surrogate* out);
/* Releases the surrogate (NULL: nothing to do, EBIC_OK).  EBIC_ERR_STATE (and
 * nothing is released) while a run of some handle is screening with it:
 * detach it first with ebic_run_screen(h, NULL, 1, EBIC_SCREEN_OFF) or free
 * that handle. */
ebic_status ebic_surrogate_free(ebic_surrogate s);
/* Reads (write = 0) or replaces (write != 0) the fp32 parameters, layout
 * above.  *n_params = capacity on entry (ignored when host_params is NULL),
 * parameter count on return. */
ebic_status ebic_surrogate_params(ebic_surrogate s, float* host_params, int64_t* n_params,
                                  int32_t write);
/* The parameter gradients left by the last ebic_surrogate_step or training
 * step (same layout; n >= the parameter count). */
ebic_status ebic_surrogate_grads(ebic_surrogate s, float* host_grads, int64_t n);
/* Column mean and population standard deviation used as features (C each). */
ebic_status ebic_surrogate_colstats(ebic_surrogate s, float* host_mean, float* host_sd);
/* One forward + backward pass on explicit standardised targets (device
 * pointers): series r of the batch is row d_idx[b] (d_idx NULL: row b) of
 * d_seq[.][stride] / d_len; target d_target[r].  update != 0 also takes one Adam
 * step with learning rate lr.  *out_loss (nullable) = mean squared error before
 * the step.  Synchronous. */
ebic_status ebic_surrogate_step(ebic_surrogate s, const uint16_t* d_seq, const int32_t* d_len,
                                int32_t stride, const float* d_target, const int32_t* d_idx,
                                int32_t batch, float lr, int32_t update, float* out_loss);
/* Appends every evaluated individual of the handle's current run (series and
 * exact fitness) to the surrogate's training log.  *out_total (nullable) = log
 * size afterwards. */
ebic_status ebic_surrogate_log(ebic_surrogate s, ebic_handle h, int64_t* out_total);
/* Training on device arrays: n (series, fitness) pairs; targets standardised
 * over the n pairs; `steps` Adam steps on minibatches of `batch` rows drawn
 * uniformly with replacement (Philox-4x32-10 keyed by the creation seed and
 * the step number).  d_seq/d_len/d_fitness NULL: train on the log.  *out_loss
 * = minibatch loss of the last step.  Synchronous.  The call captures one
 * step as a CUDA graph and replays it `steps` times; the result equals that
 * of the same steps in any split across calls. */
ebic_status ebic_surrogate_train(ebic_surrogate s, const uint16_t* d_seq, const int32_t* d_len,
                                 int32_t stride, const double* d_fitness, int64_t n,
                                 int32_t steps, int32_t batch, float lr, float* out_loss);
/* The target standardisation of the last training call. */
ebic_status ebic_surrogate_target_norm(ebic_surrogate s, float* mean, float* sd);
/* Which kernel scores series (ebic_surrogate_predict and screening): 0 (the
 * default) = tiles of 128 series on the tcgen05 tensor cores, fp32
 * accumulators in tensor memory; 1 = tiles of 64 series on mma.sync.  Both
 * round the features and hidden activations to bf16 at the same points; they
 * differ only in the order of fp32 additions. */
ebic_status ebic_surrogate_forward_kernel(ebic_surrogate s, int32_t kind);
/* Which kernels run the six GEMMs of a training step: 0 (the default) = the
 * tcgen05 tensor cores with fp32 accumulators in tensor memory (operands that
 * are K-major in memory arrive by tensor copies or one bulk copy, the weight
 * gradients' MN-major operands are transposed in 8 x 8 blocks on the way into
 * shared memory); 1 = mma.sync tiles of 64 x 64.  Both round at the same
 * points (bf16 operands and stored activations, fp32 sums; split-K slices
 * summed in split order); they differ only in the order of fp32 additions.
 * EBIC_ERR_ARG for any other kind. */
ebic_status ebic_surrogate_train_kernel(ebic_surrogate s, int32_t kind);
/* Predicted standardised targets of n series (device pointers; d_out[n] fp32),
 * queued on `stream` (NULL: the surrogate's own stream, then synchronised). */
ebic_status ebic_surrogate_predict(ebic_surrogate s, const uint16_t* d_seq, const int32_t* d_len,
                                   int32_t stride, int64_t n, float* d_out, void* stream);

typedef enum {
  EBIC_SCREEN_OFF = 0,        /* plain EBIC */
  EBIC_SCREEN_SURROGATE = 1,  /* score candidates with the surrogate */
  EBIC_SCREEN_PSEUDO = 2      /* score candidates with Philox draws (testing the
                                 screening logic without a model) */
} ebic_screen_mode;

/* Screening for the next ebic_run_init of h.  Each attempt of Step 3 builds
 * `oversample` candidate children (1 .. 16) for its tournament outcome:
 * candidate v repeats the crossover cuts and the mutation with draws
 * 2k + 1 + 5v .. 2k + 5 + 5v (v = 0 is the plain child), and the candidate
 * with the highest score goes on (ties: lowest v).  Pseudo scores: candidate v
 * of tournament outcome c (= ta * k + tb; tb = 0 without crossover) scores
 * word 0 of Philox(counter (j, g, 65536 + c * oversample + v, 0), key = seed)
 * shifted right by 8.  oversample 1 or mode EBIC_SCREEN_OFF is plain EBIC.
 * The surrogate must stay alive while a run screens with it. */
ebic_status ebic_run_screen(ebic_handle h, ebic_surrogate s, int32_t oversample, int32_t mode);

#ifdef __cplusplus
}
#endif
#endif /* EBIC_H_ */
