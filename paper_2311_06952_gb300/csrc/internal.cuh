// internal.cuh -- declarations shared by the translation units of libdeoct.
#pragma once

#include "common.cuh"

namespace deoct {

// ---------------------------------------------------------------------------
// evaluator (eval.cu)
// ---------------------------------------------------------------------------
// One subproblem for the evaluator: a sample segment of a rank-encoded set and
// a population of packed trees whose class counts it accumulates.
struct EvalProb {
  const void* ranks;       // [F][ld] uint16 / uint32
  const uint8_t* labels;   // per sample (indexed like rank columns)
  const int32_t* idx;      // nullable: the segment lists column indices idx[start..start+count)
  const uint32_t* nodes;   // [P][B] packed (p << 24 | theta), see pack_node
  uint32_t* counts;        // [P][2^D][K], accumulated with atomics (caller zeroes)
  int64_t ld;
  int64_t ncols;           // columns of the rank rows (bound for idx entries)
  int64_t start;           // first sample of the segment (into idx, or a column)
  int64_t count;           // samples in the segment
  int32_t F, K, P, tma;    // tma: rank rows may be staged with 1-D bulk copies
  int32_t lab_tma = 0;     // labels + start is 16-byte aligned: labels staged by bulk copy too
  // nullable: the trees as given by the caller (a [P][B], 0 = no split; theta
  // [P][B]), validated and packed while a job's node table is built; `nodes`
  // is unused then
  const uint16_t* a16 = nullptr;
  const uint32_t* th32 = nullptr;
};
// A job is one tree group of one problem; its tiles are contiguous in the
// flattened tile order that the persistent CTAs split evenly.
struct EvalJob {
  int64_t tile_begin;
  int32_t prob, tree0, ntrees, ntiles;
};

struct EvalConfig {
  int S = 2048;     // samples per tile (multiple of 128)
  int TG = 256;     // trees per job
  int warps = 8;    // warps per CTA
  int grid = 0;     // CTAs (0: chosen from occupancy)
  int stream = 0;   // 1: the streaming kernel also for groups of 16+ trees (ballot mode)
};

// Evaluate several problems that share rank width W and depth D.  Either pass
// one problem in `single` (d_probs == nullptr: jobs derived arithmetically), or
// device arrays d_probs[nprob] / d_jobs[njobs] with host copies of the jobs'
// tile counts for planning.  Counts must be zeroed by the caller.
struct EvalPlan {
  EvalProb single;
  const EvalProb* d_probs = nullptr;
  const EvalJob* d_jobs = nullptr;
  int njobs = 0;
  int64_t total_tiles = 0;
  int Fmax = 0, Kmax = 0, Pmax = 0;
  int64_t max_count = 0;
  // single problem only: `single.counts` is an accumulator that is zero at
  // rest and `ticket` a zero-at-rest counter; the last CTA to finish writes
  // errors_out / counts_out (each nullable), zeroes both again
  uint32_t* ticket = nullptr;
  uint32_t* counts_out = nullptr;
  uint32_t* errors_out = nullptr;
  // multi-problem plans whose problems all read one rank array (the batched
  // level solve): that array, its row stride and width, so the launch can
  // describe it with one TMA tensor map (nullptr: no tensor map)
  const void* shared_ranks = nullptr;
  int64_t shared_ld = 0, shared_ncols = 0;
};

int eval_launch(deoct_ctx* ctx, int W, int D, const EvalPlan& plan, const EvalConfig& cfg,
                cudaStream_t stream);
// CTAs of a re-laid-kernel shape resident on one SM (shared memory and registers;
// 0 when the shape does not fit or runs on the streaming kernel).
int eval_ctas_per_sm(const deoct_ctx* ctx, int W, int D, int F, int K, const EvalConfig& c);
// Choose S / TG / warps for a workload shape (heuristic, tuned by measurement).
EvalConfig eval_choose_config(deoct_ctx* ctx, int W, int D, int F, int K, int P, int64_t n,
                              int nprob);
// build the job list for host-side problems (tile counts per problem)
void eval_build_jobs(const std::vector<int64_t>& counts, const std::vector<int>& pops, int S,
                     int TG, std::vector<EvalJob>* jobs, int64_t* total_tiles);
// errors[r] = n_valid - sum_leaf max_k counts (the loss identity of Section 2); with a
// non-null device status word that is non-zero when the kernel runs, every errors[r] is
// kErrorsInvalid instead
int launch_errors(deoct_ctx* ctx, const uint32_t* counts, int P, int L, int K, int64_t n_valid,
                  uint32_t* errors, cudaStream_t stream, const int* status = nullptr);
// The evaluator plan of one population on one (sub)set of a dataset, for the shape `cfg`:
// rank rows and labels are staged by bulk copies when the set is the whole dataset and the
// rows are 16-byte aligned (ranks base and row stride), else gathered with plain loads.
EvalPlan single_eval_plan(const deoct_dataset* ds, const int32_t* idx, int64_t n_sub,
                          const uint32_t* nodes, uint32_t* counts, int P, const EvalConfig& cfg);
// pack decoded (a, theta) into evaluator nodes, flagging a > F
int launch_pack_nodes(deoct_ctx* ctx, const uint16_t* a, const uint32_t* theta, int64_t count,
                      int F, uint32_t* nodes, cudaStream_t stream);

// ---------------------------------------------------------------------------
// DE (de.cu)
// ---------------------------------------------------------------------------
struct DEProb {
  float* pop;            // [P][2B]
  float* trial;          // [P][2B]
  double* fit;           // [P]
  double* fit_trial;     // [P]
  int32_t* best;         // [1]
  int32_t* gen;          // [1] generation counter (graph replay)
  uint32_t* nodes;       // [P][B] packed nodes of the population being evaluated
  uint32_t* counts;      // [P][2^D][K]
  const uint32_t* n_unique;
  const float* seeds;    // [S][2B] or nullptr
  int64_t n_valid;
  uint64_t seed;         // Philox key (seed, stream_id) of this problem's draws
  uint64_t stream_id;
  int32_t S, F, K;
  int32_t G;             // generations of this problem: trials are built for g <= G
};
// One DE launch: problems that share P, depth and the DE constants (each
// problem keeps its own data, Philox key and generation count).
struct DEArgs {
  DEProb single;
  const DEProb* probs;   // nullptr: use `single`
  int nprob;
  int P, depth;
  float M, CR;
  double alpha;
  int n_min, dither;
  int Kmax;              // the largest K of the launch's problems (0: not known)
  int* status;
  // nullable: kDePartBytes of scratch for the split steady-state step of one problem
  // with a large population (per-CTA argmin candidates, then the generation number)
  double* part_f = nullptr;
  int* part_i = nullptr;
  int* part_g = nullptr;
};
enum : int { DE_FIRST = 1, DE_SELECT = 2, DE_TRIAL = 4, DE_GEN_DEVICE = 8 };
// The split step: individuals per CTA and lanes per individual, and its scratch
// (kMaxPop / kDeWideR candidates of 8 + 4 bytes, then the generation number).
constexpr int kDeWideR = 32, kDeWideG = 8;
constexpr size_t kDePartBytes = 2048;
static_assert(kMaxPop / kDeWideR * 12 + 4 <= (int)kDePartBytes, "split-step scratch");

int de_launch_init(deoct_ctx* ctx, const DEArgs& a, cudaStream_t s);
// flags: DE_FIRST (fitness of the evaluated initial population), DE_SELECT
// (fitness of the evaluated trials + Eq. selection), DE_TRIAL (trial vectors of
// generation g), DE_GEN_DEVICE (g read from / advanced in prob.gen).
int de_launch_step(deoct_ctx* ctx, const DEArgs& a, int g, int flags, cudaStream_t s);
// decode the best individual: a_out [B], theta_out [B], *fit_out (device)
int launch_best_extract(deoct_ctx* ctx, const float* pop, const double* fit, const int32_t* best,
                        int depth, int F, const uint32_t* n_unique, uint16_t* a_out,
                        uint32_t* theta_out, double* fit_out, cudaStream_t s);
// decode genes [P][2B] -> a (uint16), theta (uint32)
int launch_decode(deoct_ctx* ctx, const float* genes, int P, int depth, int F,
                  const uint32_t* n_unique, uint16_t* a_out, uint32_t* theta_out,
                  cudaStream_t s);

// ---------------------------------------------------------------------------
// encoder (encode.cu)
// ---------------------------------------------------------------------------
// W = 2 or 4; W = 0 picks 2 when every n_p <= 65536, else 4 (reads n_p back: syncs s)
// and reports the width used in *W_used (nullable)
int encode_run(deoct_ctx* ctx, const float* X, int64_t n, int F, int W, void* ranks_out,
               int64_t ld, uint32_t* n_unique_out, float* unique_out, cudaStream_t s,
               int* W_used = nullptr);

// ---------------------------------------------------------------------------
// prediction (predict.cu)
// ---------------------------------------------------------------------------
int launch_split_values(deoct_ctx* ctx, const float* unique, int64_t ld, const uint16_t* a,
                        const uint32_t* theta, int B, double* b_out, cudaStream_t s);
int launch_predict(deoct_ctx* ctx, const float* X, int64_t m, int F, const uint16_t* a,
                   const double* b, int depth, const uint8_t* leaf_class, const uint8_t* y,
                   uint8_t* pred_out, unsigned long long* correct_out, cudaStream_t s);

// segmented LSD radix sort of uint32 keys with uint32 values; F segments of
// length n each, stored back to back.  Sorts `bits` low key bits.  On return
// *keys_out / *vals_out point at the sorted arrays (one of the two buffers).
int radix_sort_segments(deoct_ctx* ctx, uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1,
                        int64_t n, int F, int bits, uint32_t** keys_out, uint32_t** vals_out,
                        cudaStream_t s);

// ---------------------------------------------------------------------------
// moving horizon (mh.cu)
// ---------------------------------------------------------------------------
// engine.cu: run G generations of problems in steady state (trials of generation
// 1 built, counts zeroed) in the shared launches of engine `e`; returns when the
// last has completed.  W, Dt: rank width and subtree depth of the problems.
int engine_generations(deoct_engine* e, const void* owner, int W, int Dt, const DEArgs& a, int G,
                       const std::vector<DEProb>& dp, const std::vector<EvalProb>& ep);

size_t fit_scratch_bound(const deoct_ctx* ctx, int64_t n, int F, int K, int W, const deoct_params* prm);
int mh_run(deoct_ctx* ctx, const deoct_dataset* ds, const deoct_params* prm, uint16_t* a_out,
           uint32_t* th_out, uint8_t* leaf_class_out, int32_t* kind_out, double* node_fit_out,
           cudaStream_t s);
int depth1_run(deoct_ctx* ctx, const deoct_dataset* ds, const int32_t* sample_idx, int64_t n_sub,
               int n_min, double alpha, uint16_t* a_out, uint32_t* th_out, double* f_out,
               cudaStream_t s);

}  // namespace deoct
