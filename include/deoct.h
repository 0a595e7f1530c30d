/*
 * deoct.h -- C ABI of the GB300-native MH-DEOCT hot path.
 *
 * Method: Ren et al., "A GPU-Accelerated Moving-Horizon Algorithm for Training
 * Deep Classification Trees on Large Datasets" (arXiv 2311.06952).  Section
 * numbers, equations and algorithms below are the paper's.
 *
 * Conventions for every call:
 *  - Return value: DEOCT_OK (0) or a negative deoct_status; the message of the
 *    last failure on the calling thread is deoct_last_error_string().  No C++
 *    exception crosses this boundary.
 *  - Array arguments are DEVICE pointers owned by the caller unless the
 *    argument says "host".  The library never frees or keeps caller memory
 *    beyond the call (except through the queued stream work of an async call).
 *  - The library allocates only its own scratch, owned by the deoct_ctx and
 *    released by deoct_destroy.  A context must not be used by two host threads
 *    at once.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls marked "async" only enqueue work on it; calls marked
 *    "sync" return after that work has finished and report device-side errors
 *    (a bounded device wait that expired is DEOCT_ERR_TIMEOUT).
 *  - Sizes: n <= 2^24 samples per dataset (thresholds are packed in 24 bits),
 *    1 <= F <= 256 features, 1 <= K <= 255 classes, 1 <= depth <= 10,
 *    4 <= P <= 4096 individuals.  Violations return DEOCT_ERR_INVALID.
 */
#ifndef DEOCT_H_
#define DEOCT_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define DEOCT_API __attribute__((visibility("default")))
#else
#define DEOCT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DEOCT_OK = 0,
  DEOCT_ERR_INVALID = -1, /* bad argument, NaN feature, rank width too small, ... */
  DEOCT_ERR_OOM = -2,     /* device allocation of scratch failed */
  DEOCT_ERR_CUDA = -3,    /* a CUDA runtime call failed */
  DEOCT_ERR_TIMEOUT = -4, /* a bounded device-side wait ran out */
  DEOCT_ERR_BUDGET = -5   /* request exceeds the configured memory budget */
} deoct_status;

/* deoct_params.flags */
#define DEOCT_DITHER_M 0x1u /* M = rand(0,1) per (generation, individual), Section 3.3 */
#define DEOCT_BATCHED 0x2u  /* moving horizon: one batched launch per level */
#define DEOCT_CART_SEEDS 0x4u /* moving horizon: seed each DEOCT subtree with its greedy tree */
#define DEOCT_DE_SEEDS 0x8u   /* moving horizon: seed each DEOCT subtree from a full-depth DEOCT */

typedef struct deoct_ctx deoct_ctx;

/* A rank-encoded training set (Section 3.1 threshold sets, stored as ranks).
 *  ranks     [F][ld] feature-major, uint16 (rank_bytes = 2) or uint32 (4):
 *            ranks[p*ld + i] = number of distinct values of feature p below x_{i,p}.
 *            16-byte aligned base and ld*rank_bytes % 16 == 0 enable TMA
 *            staging; other layouts take a plain-load path.
 *  n_unique  [F] uint32, n_p of Section 3.1 (>= 1).
 *  labels    [n] uint8 class indices < K.
 * All three are device pointers owned by the caller. */
typedef struct {
  const void* ranks;
  int32_t rank_bytes;
  int64_t ld;
  const uint32_t* n_unique;
  const uint8_t* labels;
  int64_t n;
  int32_t F;
  int32_t K;
} deoct_dataset;

/* DE / moving-horizon knobs (Algorithm 2 and Algorithm 4 inputs).
 *  depth    tree depth D (DEOCT) or final depth (moving horizon)
 *  horizon  moving-horizon depth D_MH (Section 4); ignored by DEOCT calls
 *  pop, gens population size N and generations G (Algorithm 4)
 *  mut_f, cr mutation factor M and crossover probability CR (Eqs. mutation, crossover)
 *  alpha, n_min  complexity weight and minimum leaf size (Eq. opt_all, Section 3.2)
 *  flags    DEOCT_DITHER_M, DEOCT_BATCHED
 *  seed     Philox4x64-10 key word 0 (key word 1 is the stream id of a call) */
typedef struct {
  int32_t depth;
  int32_t horizon;
  int32_t pop;
  int32_t gens;
  float mut_f;
  float cr;
  double alpha;
  int32_t n_min;
  uint32_t flags;
  uint64_t seed;
} deoct_params;

/* Counters of kernel launches and (when timing is on) evaluator time. */
typedef struct {
  uint64_t launches;      /* every kernel this library launched */
  uint64_t eval_launches; /* population-evaluator launches */
  double eval_ms;         /* summed CUDA-event time of evaluator launches (timing on) */
  uint64_t eval_timed;    /* evaluator launches included in eval_ms */
} deoct_stats;

/* ---- context ------------------------------------------------------------ */

/* Create a context bound to CUDA device `device` (sync). *ctx receives it. */
DEOCT_API int deoct_create(deoct_ctx** ctx, int device);
/* Free the context's scratch (sync on the device).  NULL is accepted. */
DEOCT_API int deoct_destroy(deoct_ctx* ctx);
/* Message of the last failure on this thread ("" if none); static storage. */
DEOCT_API const char* deoct_last_error_string(void);
/* Library version string; static storage. */
DEOCT_API const char* deoct_version(void);
/* Enable (1) / disable (0) CUDA-event timing of every evaluator launch. */
DEOCT_API int deoct_set_timing(deoct_ctx* ctx, int enable);
/* Read the counters (sync on pending timing events) / reset them. */
DEOCT_API int deoct_get_stats(deoct_ctx* ctx, deoct_stats* out);
DEOCT_API int deoct_reset_stats(deoct_ctx* ctx);

/* Override the evaluator's launch shape (0 keeps the library's choice):
 *  S      samples per shared-memory tile (multiple of 128, 128..8192)
 *  TG     trees per job (tree group), 1..4096
 *  warps  warps per CTA, 1..32 (the streaming kernel, which evaluates groups of
 *         fewer than 16 trees, takes at most 16)
 *  grid   persistent CTAs (each walks an equal contiguous range of tiles)
 * Results do not depend on the shape; only speed does.  Invalid values are
 * DEOCT_ERR_INVALID; a shape whose tile does not fit in shared memory fails at
 * the next evaluation. */
DEOCT_API int deoct_set_eval_config(deoct_ctx* ctx, int32_t S, int32_t TG, int32_t warps, int32_t grid);
/* deoct_set_eval_streaming: with on != 0, every ballot-mode evaluation of
 * `ctx` (2^depth K <= 128) runs on the streaming kernel -- a producer warp
 * stages tiles into a ring of landing zones for the routing warps -- also for
 * groups of 16 or more trees, where the automatic choice is the re-laid kernel
 * (the batched level solve measures both).  Results are unchanged; 0 restores
 * the automatic choice.  sync. */
DEOCT_API int deoct_set_eval_streaming(deoct_ctx* ctx, int32_t on);

/* Self-test of the library's failure detection (no counterpart in the paper).
 * Every device-side wait of the library (the evaluator's mbarrier waits) is
 * bounded and, when it runs out, sets a bit in the context's status word that
 * the next sync call reports as DEOCT_ERR_TIMEOUT, leaving the context usable.
 * This call launches one warp that waits on an mbarrier nothing arrives on, for
 * `tries` hinted tries of up to ~1 us each (1 <= tries <= 2^20), then returns
 * what the sync check reports: DEOCT_ERR_TIMEOUT when the mechanism works.
 * sync. */
DEOCT_API int deoct_selftest_wait(deoct_ctx* ctx, int32_t tries, void* stream);

/* ---- a1: rank encoder ----------------------------------------------------
 * Section 3.1: the threshold set B_p of feature p is built from its sorted
 * unique values; a sample's position among them (its dense rank) decides every
 * threshold test, so the encoder emits ranks and n_p ("only need to generate
 * once").  Ranks are taken on the raw float32 values (monotone min-max scaling
 * leaves them unchanged); -0.0 equals +0.0.
 *  X          [n][F] float32 row-major (device, caller-owned)
 *  rank_bytes 2 (uint16 ranks, needs every n_p <= 65536) or 4
 *  ranks_out  [F][ld] (device); only columns 0..n-1 are written
 *  n_unique_out [F] uint32 (device)
 * sync.  DEOCT_ERR_INVALID on NaN, on n_p > 65536 with rank_bytes = 2 (the
 * outputs are then unspecified), or on bad sizes. */
DEOCT_API int deoct_encode(deoct_ctx* ctx, const float* X, int64_t n, int32_t F, int32_t rank_bytes,
                 void* ranks_out, int64_t ld, uint32_t* n_unique_out, void* stream);

/* As deoct_encode, and also writes the sorted distinct values of every feature
 * (the xhat_{1..n_p} of Section 3.1) to unique_out [F][ld] float32 (device;
 * entries n_p..ld-1 of a row are left untouched); unique_out may be NULL. */
DEOCT_API int deoct_encode_ex(deoct_ctx* ctx, const float* X, int64_t n, int32_t F,
                              int32_t rank_bytes, void* ranks_out, int64_t ld,
                              uint32_t* n_unique_out, float* unique_out, void* stream);

/* As deoct_encode_ex with the rank width chosen from the data: uint16 ranks
 * when every n_p <= 65536 (Section 3.1's threshold sets then fit 16 bits),
 * else uint32, written as [F][ld] of that width.  The width is decided from n_p
 * after the sort, before any rank is written, so no second pass is needed.
 *  ranks_out      device buffer of at least F * ld * 4 bytes (room for either width)
 *  ld             row stride in elements of the chosen width; >= n and a
 *                 multiple of 8 (rows stay 16-byte aligned at either width)
 *  rank_bytes_out host int32: 2 or 4, the width written
 * sync. */
DEOCT_API int deoct_encode_auto(deoct_ctx* ctx, const float* X, int64_t n, int32_t F,
                                void* ranks_out, int64_t ld, uint32_t* n_unique_out,
                                float* unique_out, int32_t* rank_bytes_out, void* stream);

/* ---- a2: decoding (Eq. aenc, Eq. benc) ------------------------------------
 * genes [P][2B] float32, individual s_r = [ahat_1..ahat_B, bhat_1..bhat_B],
 * B = 2^depth - 1.  a_t = floor(ahat_t) clamped to {0..F} (0 = no split);
 * theta_t = min(floor(bhat_t * (n_p + 1)), n_p - 1) for p = a_t - 1 (the rank
 * form of b_t = beta_{a_t, i}, i = floor(bhat_t (n_p+1)) + 1, where the last
 * threshold 1 of B_p routes like the one before it), theta_t = 0 when a_t = 0.
 *  a_out [P][B] uint16, theta_out [P][B] uint32 (device).  async. */
DEOCT_API int deoct_decode_population(deoct_ctx* ctx, const deoct_dataset* ds, const float* genes,
                            int32_t P, int32_t depth, uint16_t* a_out, uint32_t* theta_out,
                            void* stream);

/* ---- a3 + a4: population fitness evaluation (Algorithm 1, Section 3.2) ----
 * Every selected sample is routed through every tree (node t -> 2t if
 * rank[a_t - 1][i] < theta_t else 2t + 1; a_t = 0 -> right) and
 * counts[r][leaf][y_i] is incremented (the class count matrix Zhat).  Each
 * tree's misclassification count n - sum_leaf max_k Zhat (the loss identity
 * of Section 2) is returned in errors_out.
 *  sample_idx [n_sub] int32 indices into the dataset's samples, or NULL for
 *             all n samples (then n_sub must equal ds->n)
 *  a, theta   [P][B] decoded trees (a in {0..F}); a > F is DEOCT_ERR_INVALID
 *             reported by the next sync call, and the node then routes right
 *  counts_out [P][2^depth][K] uint32, or NULL
 *  errors_out [P] uint32, or NULL
 * One kernel launch when n_sub > 0: the trees are validated and packed as the
 * evaluator builds its node tables, and its last CTA writes errors_out and
 * counts_out from an accumulator in the context's scratch that is zero again
 * when the launch ends.  Calls on one context must therefore be ordered on one
 * stream (two streams sharing a context race on that scratch).  async. */
DEOCT_API int deoct_eval_population(deoct_ctx* ctx, const deoct_dataset* ds, const int32_t* sample_idx,
                          int64_t n_sub, const uint16_t* a, const uint32_t* theta, int32_t P,
                          int32_t depth, uint32_t* counts_out, uint32_t* errors_out,
                          void* stream);

/* ---- a5: DE (Algorithm 4) -------------------------------------------------
 * Random numbers: Philox4x64-10 (Salmon et al., SC'11) with key
 * (params->seed, stream_id) and counter (generation, individual, block, 0);
 * draw s of an individual is the (s % 8)-th 32-bit half (low first) of block
 * s / 8.  Per (g, r): draw 0 -> r1, 1 -> r2 (distinct from r and each other,
 * multiply-shift maps), 2 -> q_rand, 3 -> M when dithered, 4 + q -> rand(0,1)
 * of gene q; uniform = (draw >> 8) * 2^-24.  Gene arithmetic is float32 with
 * one rounding per operation: v = s_best + M (s_r1 - s_r2) (Eq. mutation),
 * clamped to [0, largest float below the gene bound]; u_q = v_q if
 * rand <= CR or q = q_rand else s_q (Eq. crossover); u replaces s iff
 * f(u) <= f(s) (Eq. selection); best = lowest index of the minimal fitness,
 * taken from the previous generation (Section 3.3).  Fitness is
 * f = errors + V + alpha * #splits in double (Section 3.2).
 *
 * deoct_de_init: S^1 of Algorithm 4 -- slots 0..S-1 take `seeds` [S][2B]
 * (device, nullable when S = 0), the others are uniform in the gene range
 * (generation tag 0, draw q for gene q); evaluates it.
 *  pop [P][2B] float32 out, fitness [P] double out, best [1] int32 out. async.
 * deoct_de_step: one generation g >= 1: trial population from (pop, best),
 * evaluation, selection; pop / fitness / best are updated in place. async. */
DEOCT_API int deoct_de_init(deoct_ctx* ctx, const deoct_dataset* ds, const int32_t* sample_idx,
                  int64_t n_sub, const deoct_params* params, uint64_t stream_id,
                  const float* seeds, int32_t S, float* pop, double* fitness, int32_t* best,
                  void* stream);
DEOCT_API int deoct_de_step(deoct_ctx* ctx, const deoct_dataset* ds, const int32_t* sample_idx,
                  int64_t n_sub, const deoct_params* params, uint64_t stream_id,
                  int32_t generation, float* pop, double* fitness, int32_t* best, void* stream);

/* DEOCT on one (sub)problem: deoct_de_init, then generations 1..G.  Writes the
 * best tree's decoded nodes to host arrays a_out [B] (uint16) and theta_out [B],
 * its fitness to *fitness_out (host), and, when pop_out is not NULL, the final
 * population [P][2B] to device memory.  sync. */
DEOCT_API int deoct_fit_subtree(deoct_ctx* ctx, const deoct_dataset* ds, const int32_t* sample_idx,
                      int64_t n_sub, const deoct_params* params, uint64_t stream_id,
                      const float* seeds, int32_t S, uint16_t* a_out, uint32_t* theta_out,
                      double* fitness_out, float* pop_out, void* stream);

/* ---- a6 / a7: moving-horizon DEOCT (Algorithm 2, Section 4) ---------------
 * Nodes are visited level by level (root depth 0).  A node whose sample set
 * X_t has more than n_min samples and at least two classes is solved with
 * horizon D_t = min(D_MH, D - depth(t)): D_t >= 2 by DEOCT of depth D_t on X_t
 * (Philox stream id = t, the node's 1-based BFS index; no warm starts), D_t = 1
 * by exhaustive depth-1 search (fewest fitness, then no split, lowest feature,
 * lowest threshold); the root node of the solution is kept.  Other nodes get
 * a_t = 0, theta_t = 0.  Thresholds are the global ranks.
 * DEOCT_BATCHED in params->flags solves all nodes of a level in one batched
 * launch per generation over a compacted sample index; otherwise each node is
 * a separate DEOCT (the plain per-node form).  Both give identical trees.
 * DEOCT_CART_SEEDS adds the CART warm start of Algorithm 2: slot 0 of each
 * DEOCT subtree's initial population is the greedy misclassification tree of
 * depth D_t on X_t (the depth-1 search applied top-down inside the subtree,
 * same solve rule and tie order), encoded as genes a + 1/2 and the float32
 * bhat nearest to (theta + 1/2)/(n_p + 1) that decodes to theta.
 * DEOCT_DE_SEEDS adds the DEOCT warm start of Algorithm 2: one DEOCT of the
 * full depth D on the whole set (Philox stream 0) runs first, and the subtree
 * of its best tree at node t (same shape and location) seeds node t's DEOCT.
 * With both flags the seeds are, in order, the DEOCT subtree and the greedy
 * subtree.
 *  a_out [2^D - 1] uint16, theta_out [2^D - 1] uint32, leaf_class_out [2^D]
 *  uint8 (Eq. opt_c on the whole set, lowest class on ties): host arrays.
 *  kind_out [2^D - 1] int32 (0 artificial, 1 depth-1 search, 2 DEOCT) and
 *  node_fit_out [2^D - 1] double: host, nullable.  sync. */
DEOCT_API int deoct_fit_moving_horizon(deoct_ctx* ctx, const deoct_dataset* ds, const deoct_params* params,
                             uint16_t* a_out, uint32_t* theta_out, uint8_t* leaf_class_out,
                             int32_t* kind_out, double* node_fit_out, void* stream);

/* Exhaustive depth-1 subtree (the bottom level of Algorithm 2): the
 * minimum-fitness tree among "no split" and every (feature p, theta in
 * 0..n_p-1) on the selected samples, first in the order (no split, p, theta).
 * Host outputs *a_out (0..F), *theta_out, *fitness_out.  sync. */
DEOCT_API int deoct_depth1_search(deoct_ctx* ctx, const deoct_dataset* ds, const int32_t* sample_idx,
                        int64_t n_sub, int32_t n_min, double alpha, uint16_t* a_out,
                        uint32_t* theta_out, double* fitness_out, void* stream);

/* ---- prediction with a fitted tree (raw feature values) --------------------
 * deoct_split_values: the raw-unit threshold of every node, from the sorted
 * distinct training values `unique` [F][ld] of deoct_encode_ex: for a_t >= 1
 * and theta_t >= 1, b_t = (xhat_{theta_t} + xhat_{theta_t + 1}) / 2 of feature
 * a_t (1-based xhat; the midpoints of the threshold set B_p, Section 3.1) in
 * double; theta_t = 0 gives the smallest training value (beta_{p,1} = 0 after
 * min-max scaling).  On training samples "x < b_t" routes exactly like
 * "rank < theta_t".  a, theta [B] in, b_out [B] double out (device). async.
 * deoct_predict: routes m samples X [m][F] float32 (device) through the tree
 * (x_{a_t} < b_t -> left, a_t = 0 -> right; Section 2) and writes the leaf
 * class (leaf_class [2^depth]) to pred_out [m] (nullable); with labels y [m]
 * it adds the number of correct predictions to *correct_out (device uint64,
 * zeroed first).  async. */
DEOCT_API int deoct_split_values(deoct_ctx* ctx, const float* unique, int64_t ld, const uint16_t* a,
                                 const uint32_t* theta, int32_t B, double* b_out, void* stream);
DEOCT_API int deoct_predict(deoct_ctx* ctx, const float* X, int64_t m, int32_t F, const uint16_t* a,
                            const double* b, int32_t depth, const uint8_t* leaf_class,
                            const uint8_t* y, uint8_t* pred_out, uint64_t* correct_out,
                            void* stream);

/* ---- a8: serving, continuous batching across jobs -------------------------
 * The paper solves one training problem at a time; a service fits many trees
 * at once.  An engine runs the DEOCT generations of the batched level solves
 * (Algorithm 2 with DEOCT_BATCHED, Algorithm 4) of every context attached to
 * it in shared launches: per tick, one evaluator launch and one DE-step launch
 * cover the problems of all resident jobs that share the rank width, the
 * subtree depth and the DE constants (population, M, CR, alpha, n_min,
 * dither).  A job's host thread still runs its own per-level work (histogram,
 * compaction, depth-1 search, initial population) on its own stream, then
 * hands the level's problems to the engine and waits; problems join at any
 * tick and leave after their own G generations.  Every problem keeps its
 * Philox key (seed, node id) and its own generation counter, so a job's tree
 * is identical alone and in any mix.
 *  deoct_engine_create   starts the engine (its own stream and host thread)
 *                        on `device`; deoct_engine_destroy stops it once the
 *                        submitted work is done (call it after every attached
 *                        context has finished its calls).
 *  deoct_engine_attach   routes the batched level solves of `ctx` through `e`
 *                        (NULL detaches).  Contexts stay single-threaded; the
 *                        engine may serve any number of them from as many host
 *                        threads.  Device errors in a shared launch are
 *                        returned to the jobs whose problems finish with it.
 *  deoct_engine_get_stats counters since creation. */
/* deoct_get_memory: the device bytes `ctx` holds (its scratch, grow-only until
 * deoct_destroy, plus its status word) and its pinned host staging bytes.
 * deoct_fit_scratch_bound: an upper bound of the device bytes by which `ctx`'s
 * scratch grows when it encodes an n x F set (rank_bytes 2 or 4, or 0 for the
 * widest choice of deoct_encode_auto) and fits it with
 * deoct_fit_moving_horizon under `params` (plain or batched, with or without
 * warm starts); with ctx NULL, the bytes a fresh context holds afterwards.  The
 * scratch is kept per buffer, so a context holding more bytes in total than a
 * request needs may still grow.  The caller's own arrays (features, ranks,
 * labels) are not included.  Neither call touches the GPU; ctx must not be in
 * use by another thread. */
DEOCT_API int deoct_get_memory(deoct_ctx* ctx, uint64_t* device_bytes, uint64_t* pinned_bytes);
/* deoct_release_scratch: frees every scratch buffer of `ctx` (the next calls
 * allocate again).  Synchronises the device.  sync. */
DEOCT_API int deoct_release_scratch(deoct_ctx* ctx);
/* deoct_set_scratch_limit (no counterpart in the paper: a serving budget): caps
 * the device bytes `ctx`'s scratch may hold, 0 = no cap (the default).  A call
 * whose scratch would grow past the cap fails with DEOCT_ERR_OOM before it
 * allocates or launches anything for that buffer; the context stays usable (raise
 * the cap, or release scratch, and call again).  Buffers already held above a
 * lowered cap are kept.  sync. */
DEOCT_API int deoct_set_scratch_limit(deoct_ctx* ctx, uint64_t bytes);
DEOCT_API int deoct_fit_scratch_bound(const deoct_ctx* ctx, int64_t n, int32_t F, int32_t K,
                                      int32_t rank_bytes, const deoct_params* params,
                                      uint64_t* bytes_out);

typedef struct deoct_engine deoct_engine;
typedef struct {
  uint64_t submissions;        /* level solves handed to the engine */
  uint64_t completed;          /* level solves returned */
  uint64_t ticks;              /* generations run (replays of the shared launches) */
  uint64_t launches;           /* kernel launches in those replays */
  uint64_t eval_launches;      /* of which evaluator launches */
  uint64_t shared_launches;    /* launches carrying problems of two or more jobs */
  uint64_t max_jobs_per_launch;
  uint64_t max_problems_per_launch;
} deoct_engine_stats;
DEOCT_API int deoct_engine_create(deoct_engine** out, int device);
DEOCT_API int deoct_engine_destroy(deoct_engine* e);
DEOCT_API int deoct_engine_attach(deoct_ctx* ctx, deoct_engine* e);
DEOCT_API int deoct_engine_get_stats(deoct_engine* e, deoct_engine_stats* out);

/* ---- evaluation without device allocation --------------------------------
 * The paper has no counterpart to this call; it exists for callers that cannot
 * allocate device memory -- a host framework that owns all device memory
 * through its own pool, or code that must not take the device-wide
 * synchronisation that cudaMalloc / cudaFree can cause.  It computes exactly
 * what deoct_eval_population computes, but needs no deoct_ctx and calls no
 * allocator: its scratch (packed trees, a status word, and the class counts
 * when counts_out is NULL) is one fixed array of DEOCT_NOALLOC_SCRATCH_BYTES
 * bytes inside the library, resident on every GPU that loads the library until
 * the process exits.
 *  - Runs on the current CUDA device.  The first call on a device looks up the
 *    array's device address (cudaGetSymbolAddress) and keeps it for the life of
 *    the process; make that first call before any stream capture.  The kept
 *    address does not survive cudaDeviceReset: a process that resets a device
 *    must not call this entry point on it afterwards.
 *  - Requests needing more scratch than the array holds (P * (2^depth - 1) * 4
 *    bytes of trees, plus P * 2^depth * K * 4 bytes of counts when counts_out is
 *    NULL, plus 256) return DEOCT_ERR_INVALID before any GPU work, and so does
 *    P outside 1..262144 (the limit of deoct_eval_population).
 *  - Every call shares the one array and each call clears what must start at
 *    zero; calls whose GPU work overlaps (other streams, other threads) race on
 *    it and must be serialised by the caller.
 *  - Device-side errors -- a tree naming a feature > F (it routes right), a
 *    sample_idx entry outside 0..n-1 (read as sample 0), a bounded device wait
 *    that expired -- cannot be returned by a later sync call, as there is no
 *    context.  Instead every errors_out entry of that call is set to 0xFFFFFFFF
 *    (no true error count reaches it, since n <= 2^24) and counts_out is not to
 *    be trusted.  With errors_out NULL such errors go unreported.
 * Arguments as deoct_eval_population.  async. */
#define DEOCT_NOALLOC_SCRATCH_BYTES (8u << 20)
DEOCT_API int deoct_eval_population_noalloc(const deoct_dataset* ds, const int32_t* sample_idx,
                                            int64_t n_sub, const uint16_t* a, const uint32_t* theta,
                                            int32_t P, int32_t depth, uint32_t* counts_out,
                                            uint32_t* errors_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DEOCT_H_ */
