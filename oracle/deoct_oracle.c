/*
 * deoct_oracle.c -- plain CPU oracle for the MH-DEOCT hot path
 * (Ren et al., "A GPU-Accelerated Moving-Horizon Algorithm for Training Deep
 * Classification Trees on Large Datasets", arXiv 2311.06952).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline / reference leg may load this library.  The product (the CUDA
 * library under paper_2311_06952_gb300/) never links, loads or calls it, and
 * this file includes nothing from there.
 *
 * Everything here is single-threaded, unblocked and unfused: each function is
 * the paper's definition or the paper's algorithm step by step, so that it can
 * be read against the paper by eye.  Build flags: -O2 -ffp-contract=off (no
 * fused multiply-add anywhere, so float arithmetic is IEEE round-to-nearest
 * per operation on x86-64 and aarch64 alike).
 *
 * Readings of points the paper leaves open are marked "Reading Cn" and match
 * the list kept in the design notes of the repository.
 *
 * Parity pins: every function below is checked by tests/test_oracle_*.py
 * against something other than itself (numpy.unique, numpy's Philox bit
 * generator, brute force over all trees, float-midpoint routing, invariants of
 * the loss, a numpy float32 restatement of the DE trial and initialisation).
 * The moving-horizon driver is pinned by special cases; the conventions it and
 * the DE step fix where the paper is silent are readings, not paper facts.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_INVALID (-1)
#define ORC_ERR_OOM (-2)

/* Threads of the OpenMP twins at the end of this file (1 = the plain loops). */
static int g_threads = 1;
void orc_eval_counts_omp(const uint32_t* ranks, int64_t n, int32_t F, const uint8_t* y,
                         int32_t K, const int32_t* idx, int64_t n_sub, const int32_t* a,
                         const uint32_t* theta, int32_t P, int32_t depth, uint32_t* counts);

/* ------------------------------------------------------------------------- */
/* Threshold sets as ranks (Section 3.1, "Decoding Tree Candidates").          */
/* ------------------------------------------------------------------------- */

static int cmp_float(const void* pa, const void* pb) {
  float a = *(const float*)pa, b = *(const float*)pb;
  return (a < b) ? -1 : (a > b) ? 1 : 0;
}

/* Section 3.1: the unique elements xhat_{1..n_p} of feature p, sorted
 * ascending, define the threshold set B_p.  We store, for every sample, the
 * 0-based index of its value among those unique elements (its dense rank), and
 * n_p.  Routing "x < beta_{p,i}" is then "rank < i-1" (see orc_decode).
 * Ranks are taken on the raw float32 values (Reading C2: monotone min-max
 * scaling does not change them); -0.0 is the same value as +0.0.
 * X is [n][F] row-major; ranks_out is [F][n]; returns ORC_ERR_INVALID on NaN. */
static int encode_feature(const float* X, int64_t n, int32_t F, int32_t p, float* col, float* uniq,
                          uint32_t* ranks_out, uint32_t* n_unique_out) {
  for (int64_t i = 0; i < n; ++i) {
    float v = X[i * F + p];
    if (isnan(v)) return ORC_ERR_INVALID;
    if (v == 0.0f) v = 0.0f; /* -0.0 and +0.0 are one value */
    col[i] = v;
  }
  memcpy(uniq, col, (size_t)n * sizeof(float));
  qsort(uniq, (size_t)n, sizeof(float), cmp_float);
  int64_t np = 0;
  for (int64_t i = 0; i < n; ++i)
    if (np == 0 || uniq[i] != uniq[np - 1]) uniq[np++] = uniq[i];
  n_unique_out[p] = (uint32_t)np;
  for (int64_t i = 0; i < n; ++i) {
    /* lower_bound: number of unique values strictly below col[i] */
    int64_t lo = 0, hi = np;
    while (lo < hi) {
      int64_t mid = lo + (hi - lo) / 2;
      if (uniq[mid] < col[i]) lo = mid + 1; else hi = mid;
    }
    ranks_out[(int64_t)p * n + i] = (uint32_t)lo;
  }
  return ORC_OK;
}

int orc_encode(const float* X, int64_t n, int32_t F, uint32_t* ranks_out,
               uint32_t* n_unique_out) {
  if (n <= 0 || F <= 0) return ORC_ERR_INVALID;
  float* col = (float*)malloc((size_t)n * sizeof(float));
  float* uniq = (float*)malloc((size_t)n * sizeof(float));
  if (!col || !uniq) { free(col); free(uniq); return ORC_ERR_OOM; }
  int rc = ORC_OK;
  for (int32_t p = 0; p < F && rc == ORC_OK; ++p)
    rc = encode_feature(X, n, F, p, col, uniq, ranks_out, n_unique_out);
  free(col);
  free(uniq);
  return rc;
}

/* ------------------------------------------------------------------------- */
/* Counter-based random numbers: Philox4x64-10 (Salmon, Moraes, Dror, Shaw,    */
/* "Parallel Random Numbers: As Easy as 1, 2, 3", SC'11).                      */
/* ------------------------------------------------------------------------- */

static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

/* One Philox4x64 round: two 64x64->128 multiplies by the published
 * multipliers, then the S-box permutation that xors the high halves with the
 * other two words and the round key.  The key is bumped by the published Weyl
 * constants between rounds; ten rounds in all. */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += W0; k1 += W1; }
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo64(M0, x0, &hi0, &lo0);
    mulhilo64(M1, x2, &hi1, &lo1);
    uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Reading C5: the DE draws of individual r in generation g are the 32-bit
 * halves of the Philox blocks with key (seed, stream) and counter
 * (g, r, block, 0); draw s lives in block s/8, word (s%8)/2, low half first. */
uint32_t orc_draw32(uint64_t seed, uint64_t stream, uint64_t g, uint64_t r, uint64_t s) {
  uint64_t ctr[4] = {g, r, s >> 3, 0}, key[2] = {seed, stream}, out[4];
  orc_philox4x64_10(ctr, key, out);
  uint64_t w = out[(s & 7) >> 1];
  return (s & 1) ? (uint32_t)(w >> 32) : (uint32_t)w;
}

/* A uniform float in [0,1): the top 24 bits of the draw times 2^-24 (exact). */
static float u01(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }
/* An integer in [0, m): multiply-shift of the 32-bit draw. */
static uint32_t below(uint32_t x, uint32_t m) {
  return (uint32_t)(((uint64_t)x * (uint64_t)m) >> 32);
}

/* ------------------------------------------------------------------------- */
/* Tree decoding (Section 3.1, Eq. aenc and Eq. benc).                          */
/* ------------------------------------------------------------------------- */

/* One branch node: a = floor(ahat) in {0..F} (0 = no split, Section 2);
 * for a >= 1 the threshold index i = floor(bhat*(n_p+1)) + 1 of Eq. benc
 * (n_p of the selected feature, Reading C3) selects beta_{a,i}.  In rank form
 * "x < beta_{a,i}" is "rank < theta" with theta = i - 1, and the last entry
 * (beta = 1 after min-max scaling) sends rank < n_p - 1 left (Reading C2), so
 * theta = min(floor(bhat*(n_p+1)), n_p - 1).  The product is exact in double
 * (24-bit float times an integer below 2^25).  a = 0 forces b = 0: theta = 0. */
static void decode_node(float ahat, float bhat, int32_t F, const uint32_t* n_unique,
                        int32_t* a_out, uint32_t* theta_out) {
  int32_t a = (int32_t)floorf(ahat);
  if (a < 0) a = 0;
  if (a > F) a = F;
  if (a == 0) { *a_out = 0; *theta_out = 0; return; }
  uint32_t np = n_unique[a - 1];
  double raw = floor((double)bhat * (double)((uint64_t)np + 1));
  if (raw < 0) raw = 0;
  if (raw > (double)np) raw = (double)np;
  uint32_t theta = (uint32_t)raw;
  if (theta > np - 1) theta = np - 1;
  *a_out = a;
  *theta_out = theta;
}

/* Individual s_r = [ahat_1..ahat_B, bhat_1..bhat_B] (Section 3.1); genes is
 * [P][2B]; a_out, theta_out are [P][B] (node t of tree r at r*B + t-1). */
void orc_decode(const float* genes, int32_t P, int32_t depth, int32_t F,
                const uint32_t* n_unique, int32_t* a_out, uint32_t* theta_out) {
  int32_t B = (1 << depth) - 1;
  for (int32_t r = 0; r < P; ++r)
    for (int32_t t = 0; t < B; ++t)
      decode_node(genes[(int64_t)r * 2 * B + t], genes[(int64_t)r * 2 * B + B + t], F,
                  n_unique, &a_out[(int64_t)r * B + t], &theta_out[(int64_t)r * B + t]);
}

/* ------------------------------------------------------------------------- */
/* Fitness evaluation (Section 3.2, Algorithm 1, Eq. opt_c, Eq. opt_all).       */
/* ------------------------------------------------------------------------- */

/* Routing rule of Section 2 / Algorithm 1: start at t = 1; at branch node t go
 * to 2t if x_{i,a_t} < b_t, else to 2t+1; a_t = 0 sends the sample right.
 * Returns the 0-based leaf index t - (B+1). */
static int32_t route(const uint32_t* ranks, int64_t n, int64_t i, const int32_t* a,
                     const uint32_t* theta, int32_t depth) {
  int32_t B = (1 << depth) - 1;
  int32_t t = 1;
  while (t <= B) {
    int32_t at = a[t - 1];
    int left = (at != 0) && (ranks[(int64_t)(at - 1) * n + i] < theta[t - 1]);
    t = left ? 2 * t : 2 * t + 1;
  }
  return t - (B + 1);
}

/* Class count matrix Zhat of Algorithm 1 (Eq. opt_c): counts[r][leaf][k] =
 * number of samples of class k that tree r assigns to leaf.  ranks is [F][n];
 * idx (nullable) restricts the sum to the samples idx[0..n_sub-1]. */
void orc_eval_counts(const uint32_t* ranks, int64_t n, int32_t F, const uint8_t* y,
                     int32_t K, const int32_t* idx, int64_t n_sub, const int32_t* a,
                     const uint32_t* theta, int32_t P, int32_t depth, uint32_t* counts) {
  (void)F;
  int32_t B = (1 << depth) - 1, L = 1 << depth;
  memset(counts, 0, (size_t)P * L * K * sizeof(uint32_t));
  int64_t m = idx ? n_sub : n;
  for (int32_t r = 0; r < P; ++r)
    for (int64_t j = 0; j < m; ++j) {
      int64_t i = idx ? idx[j] : j;
      int32_t leaf = route(ranks, n, i, a + (int64_t)r * B, theta + (int64_t)r * B, depth);
      counts[((int64_t)r * L + leaf) * K + y[i]] += 1;
    }
}

/* Soft-constrained DE fitness of Section 3.2:
 *   f = n - sum_leaf max_k zhat + alpha * #{t : a_t >= 1} + sum_leaf V_t,
 * V_t = 1 iff 0 < n_t < n_min.  The misclassification count is the right-hand
 * side of the loss identity at the end of Section 2 (Reading C4: a_t counts as
 * a split iff a_t >= 1).  errors_out, splits_out, v_out are nullable. */
void orc_fitness(const uint32_t* counts, const int32_t* a, int32_t P, int32_t depth,
                 int32_t K, int64_t n_sub, int32_t n_min, double alpha, double* fit_out,
                 uint32_t* errors_out, uint32_t* splits_out, uint32_t* v_out) {
  int32_t B = (1 << depth) - 1, L = 1 << depth;
  for (int32_t r = 0; r < P; ++r) {
    int64_t correct = 0;
    uint32_t v = 0, splits = 0;
    for (int32_t l = 0; l < L; ++l) {
      uint32_t mx = 0;
      int64_t nl = 0;
      for (int32_t k = 0; k < K; ++k) {
        uint32_t c = counts[((int64_t)r * L + l) * K + k];
        if (c > mx) mx = c;
        nl += c;
      }
      correct += mx;
      if (nl > 0 && nl < n_min) v += 1;
    }
    for (int32_t t = 0; t < B; ++t)
      if (a[(int64_t)r * B + t] >= 1) splits += 1;
    uint32_t errors = (uint32_t)(n_sub - correct);
    fit_out[r] = (double)((uint64_t)errors + v) + alpha * (double)splits;
    if (errors_out) errors_out[r] = errors;
    if (splits_out) splits_out[r] = splits;
    if (v_out) v_out[r] = v;
  }
}

/* Leaf class of Eq. opt_c: argmax_k zhat_t^k; ties and empty leaves take the
 * lowest class index (this choice does not change the fitness).  leaf_class is
 * [P][L]. */
void orc_leaf_classes(const uint32_t* counts, int32_t P, int32_t depth, int32_t K,
                      uint8_t* leaf_class) {
  int32_t L = 1 << depth;
  for (int32_t r = 0; r < P; ++r)
    for (int32_t l = 0; l < L; ++l) {
      int32_t best = 0;
      for (int32_t k = 1; k < K; ++k)
        if (counts[((int64_t)r * L + l) * K + k] > counts[((int64_t)r * L + l) * K + best])
          best = k;
      leaf_class[(int64_t)r * L + l] = (uint8_t)best;
    }
}

/* ------------------------------------------------------------------------- */
/* DEOCT: population DE with the previous generation's best                  */
/* (Section 3.3, Algorithm 4, Eq. mutation / crossover / selection).           */
/* ------------------------------------------------------------------------- */

typedef struct {
  int32_t depth, P, G;
  float M, CR;
  double alpha;
  int32_t n_min;
  uint64_t seed, stream;
  int32_t dither; /* 1: M = rand(0,1) per (g, r) as in Section 3.3 (Reading C7) */
} orc_de_params;

/* Gene range of Section 3.1: ahat in [0, F+1), bhat in [0, 1).  Reading C6:
 * a mutant outside the range is clamped to [0, largest float below the bound]. */
static float gene_hi(int32_t q, int32_t B, int32_t F) {
  float ub = (q < B) ? (float)(F + 1) : 1.0f;
  return nextafterf(ub, 0.0f);
}
static float clamp_gene(float v, float hi) {
  if (v < 0.0f) v = 0.0f;
  if (v > hi) v = hi;
  return v;
}

/* Evaluate a population of genes: decode (Eq. aenc/benc), count (Algorithm 1),
 * fitness (Section 3.2). */
static void eval_genes(const float* genes, int32_t P, const orc_de_params* prm,
                       const uint32_t* ranks, int64_t n, int32_t F, const uint32_t* n_unique,
                       const uint8_t* y, int32_t K, const int32_t* idx, int64_t n_sub,
                       int32_t* a, uint32_t* theta, uint32_t* counts, double* fit) {
  orc_decode(genes, P, prm->depth, F, n_unique, a, theta);
  if (g_threads > 1)
    orc_eval_counts_omp(ranks, n, F, y, K, idx, n_sub, a, theta, P, prm->depth, counts);
  else
    orc_eval_counts(ranks, n, F, y, K, idx, n_sub, a, theta, P, prm->depth, counts);
  orc_fitness(counts, a, P, prm->depth, K, idx ? n_sub : n, prm->n_min, prm->alpha, fit,
              NULL, NULL, NULL);
}

static int32_t argmin_first(const double* f, int32_t P) {
  int32_t b = 0;
  for (int32_t r = 1; r < P; ++r)
    if (f[r] < f[b]) b = r;
  return b;
}

/* One DE trial vector u_r^g (Eq. mutation with s_best of the previous
 * generation, Section 3.3; Eq. crossover).  Reading C5 fixes the draws:
 * slot 0 -> r1, slot 1 -> r2 (both distinct from r and from each other),
 * slot 2 -> q_rand, slot 3 -> M when dithered, slot 4+q -> rand(0,1) of gene q.
 * Reading C9: float32 arithmetic, one rounding per operation, no FMA. */
void orc_de_trial(const float* pop, int32_t P, int32_t B, int32_t F, int32_t best,
                  const orc_de_params* prm, int32_t g, int32_t r, float* u_out,
                  int32_t* r1_out, int32_t* r2_out, int32_t* qrand_out) {
  int32_t m = 2 * B;
  uint32_t x0 = orc_draw32(prm->seed, prm->stream, (uint64_t)g, (uint64_t)r, 0);
  uint32_t x1 = orc_draw32(prm->seed, prm->stream, (uint64_t)g, (uint64_t)r, 1);
  uint32_t x2 = orc_draw32(prm->seed, prm->stream, (uint64_t)g, (uint64_t)r, 2);
  uint32_t x3 = orc_draw32(prm->seed, prm->stream, (uint64_t)g, (uint64_t)r, 3);
  int32_t r1 = (int32_t)below(x0, (uint32_t)(P - 1));
  if (r1 >= r) r1 += 1;
  int32_t r2 = (int32_t)below(x1, (uint32_t)(P - 2));
  int32_t lo = r < r1 ? r : r1, hi = r < r1 ? r1 : r;
  if (r2 >= lo) r2 += 1;
  if (r2 >= hi) r2 += 1;
  int32_t qrand = (int32_t)below(x2, (uint32_t)m);
  float M = prm->dither ? u01(x3) : prm->M;
  const float* sb = pop + (int64_t)best * m;
  const float* s1 = pop + (int64_t)r1 * m;
  const float* s2 = pop + (int64_t)r2 * m;
  const float* sr = pop + (int64_t)r * m;
  for (int32_t q = 0; q < m; ++q) {
    float diff = s1[q] - s2[q];
    float scaled = M * diff;
    float v = sb[q] + scaled;
    float vc = clamp_gene(v, gene_hi(q, B, F));
    float rq = u01(orc_draw32(prm->seed, prm->stream, (uint64_t)g, (uint64_t)r, (uint64_t)(4 + q)));
    u_out[q] = (rq <= prm->CR || q == qrand) ? vc : sr[q];
  }
  if (r1_out) *r1_out = r1;
  if (r2_out) *r2_out = r2;
  if (qrand_out) *qrand_out = qrand;
}

/* Initial individual r (Algorithm 4, initialisation): the first S slots take
 * the warm starts, the others are uniform in the gene range, drawn with
 * generation tag 0 (draw q for gene q) and clamped as in Reading C6. */
static void init_individual(int32_t r, int32_t B, int32_t F, const orc_de_params* prm,
                            const float* seeds, int32_t S, float* out) {
  int32_t m = 2 * B;
  if (r < S) {
    for (int32_t q = 0; q < m; ++q) out[q] = seeds[(int64_t)r * m + q];
    return;
  }
  for (int32_t q = 0; q < m; ++q) {
    float ub = (q < B) ? (float)(F + 1) : 1.0f;
    float u = u01(orc_draw32(prm->seed, prm->stream, 0, (uint64_t)r, (uint64_t)q));
    float v = u * ub;
    out[q] = clamp_gene(v, gene_hi(q, B, F));
  }
}

/* Algorithm 4 (DEOCT).  Reading C12: one evaluation of S^1, then G
 * generations of trial / evaluate / select; Reading C10: u replaces s iff
 * f(u) <= f(s) (Eq. selection), best = lowest index among the minimal
 * fitness values, fixed for a whole generation (Section 3.3).
 * pop_out [P][2B], fit_out [P], best_out: the final S^{G+1}.
 * best_fit_hist [G+1] and pop_hist [(G+1)][P][2B] (nullable) record the state
 * after the initial evaluation and after every generation. */
int orc_de_run(const uint32_t* ranks, int64_t n, int32_t F, const uint32_t* n_unique,
               const uint8_t* y, int32_t K, const int32_t* idx, int64_t n_sub,
               const orc_de_params* prm, const float* seeds, int32_t S, float* pop_out,
               double* fit_out, int32_t* best_out, double* best_fit_hist, float* pop_hist,
               double* fit_hist) {
  int32_t P = prm->P, B = (1 << prm->depth) - 1, L = 1 << prm->depth, m = 2 * B;
  if (P < 4 || prm->depth < 1 || S < 0 || S > P) return ORC_ERR_INVALID;
  float* pop = pop_out;
  float* trial = (float*)malloc((size_t)P * m * sizeof(float));
  double* ft = (double*)malloc((size_t)P * sizeof(double));
  int32_t* a = (int32_t*)malloc((size_t)P * B * sizeof(int32_t));
  uint32_t* theta = (uint32_t*)malloc((size_t)P * B * sizeof(uint32_t));
  uint32_t* counts = (uint32_t*)malloc((size_t)P * L * K * sizeof(uint32_t));
  if (!trial || !ft || !a || !theta || !counts) {
    free(trial); free(ft); free(a); free(theta); free(counts);
    return ORC_ERR_OOM;
  }
  for (int32_t r = 0; r < P; ++r) init_individual(r, B, F, prm, seeds, S, pop + (int64_t)r * m);
  eval_genes(pop, P, prm, ranks, n, F, n_unique, y, K, idx, n_sub, a, theta, counts, fit_out);
  int32_t best = argmin_first(fit_out, P);
  if (best_fit_hist) best_fit_hist[0] = fit_out[best];
  if (pop_hist) memcpy(pop_hist, pop, (size_t)P * m * sizeof(float));
  if (fit_hist) memcpy(fit_hist, fit_out, (size_t)P * sizeof(double));
  for (int32_t g = 1; g <= prm->G; ++g) {
    for (int32_t r = 0; r < P; ++r)
      orc_de_trial(pop, P, B, F, best, prm, g, r, trial + (int64_t)r * m, NULL, NULL, NULL);
    eval_genes(trial, P, prm, ranks, n, F, n_unique, y, K, idx, n_sub, a, theta, counts, ft);
    for (int32_t r = 0; r < P; ++r)
      if (ft[r] <= fit_out[r]) {
        memcpy(pop + (int64_t)r * m, trial + (int64_t)r * m, (size_t)m * sizeof(float));
        fit_out[r] = ft[r];
      }
    best = argmin_first(fit_out, P);
    if (best_fit_hist) best_fit_hist[g] = fit_out[best];
    if (pop_hist) memcpy(pop_hist + (int64_t)g * P * m, pop, (size_t)P * m * sizeof(float));
    if (fit_hist) memcpy(fit_hist + (int64_t)g * P, fit_out, (size_t)P * sizeof(double));
  }
  *best_out = best;
  free(trial); free(ft); free(a); free(theta); free(counts);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Depth-1 subtree: exhaustive search ("CART with the misclassification loss"  */
/* at depth 1, Algorithm 2).                                                   */
/* ------------------------------------------------------------------------- */

/* Plain definition: every candidate depth-1 tree -- the no-split tree and
 * every (p, theta) with theta in {0..n_p-1}, the full decodable range -- is
 * scored with the fitness of Section 3.2 on the node's samples.  Reading: the
 * first minimum in the order (no split, then p ascending, then theta
 * ascending) wins.  For each feature the left-side class counts of all theta
 * come from one histogram over ranks and its running sum. */
int orc_depth1(const uint32_t* ranks, int64_t n, int32_t F, const uint32_t* n_unique,
               const uint8_t* y, int32_t K, const int32_t* idx, int64_t n_sub, int32_t n_min,
               double alpha, int32_t* a_out, uint32_t* theta_out, double* fit_out) {
  int64_t m = idx ? n_sub : n;
  int64_t* tot = (int64_t*)calloc((size_t)K, sizeof(int64_t));
  int64_t* left = (int64_t*)calloc((size_t)K, sizeof(int64_t));
  if (!tot || !left) { free(tot); free(left); return ORC_ERR_OOM; }
  for (int64_t j = 0; j < m; ++j) tot[y[idx ? idx[j] : j]] += 1;
  int64_t mx = 0;
  for (int32_t k = 0; k < K; ++k) if (tot[k] > mx) mx = tot[k];
  double best_f = (double)((m - mx) + ((m > 0 && m < n_min) ? 1 : 0));
  int32_t best_a = 0;
  uint32_t best_theta = 0;
  for (int32_t p = 0; p < F; ++p) {
    uint32_t np = n_unique[p];
    int64_t* hist = (int64_t*)calloc((size_t)np * K, sizeof(int64_t));
    if (!hist) { free(tot); free(left); return ORC_ERR_OOM; }
    for (int64_t j = 0; j < m; ++j) {
      int64_t i = idx ? idx[j] : j;
      hist[(int64_t)ranks[(int64_t)p * n + i] * K + y[i]] += 1;
    }
    for (int32_t k = 0; k < K; ++k) left[k] = 0;
    for (uint32_t theta = 0; theta < np; ++theta) {
      /* left = samples with rank < theta */
      if (theta > 0)
        for (int32_t k = 0; k < K; ++k) left[k] += hist[(int64_t)(theta - 1) * K + k];
      int64_t nl = 0, ml = 0, mr = 0;
      for (int32_t k = 0; k < K; ++k) {
        nl += left[k];
        if (left[k] > ml) ml = left[k];
        if (tot[k] - left[k] > mr) mr = tot[k] - left[k];
      }
      int64_t nr = m - nl;
      int64_t errors = m - ml - mr;
      int64_t v = ((nl > 0 && nl < n_min) ? 1 : 0) + ((nr > 0 && nr < n_min) ? 1 : 0);
      double f = (double)(errors + v) + alpha * 1.0;
      if (f < best_f) { best_f = f; best_a = p + 1; best_theta = theta; }
    }
    free(hist);
  }
  *a_out = best_a;
  *theta_out = best_theta;
  if (fit_out) *fit_out = best_f;
  free(tot);
  free(left);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Moving-horizon DEOCT (Section 4, Algorithm 2).                              */
/* ------------------------------------------------------------------------- */

typedef struct {
  int32_t depth, horizon, P, G;
  float M, CR;
  double alpha;
  int32_t n_min;
  uint64_t seed;
  int32_t dither;
  int32_t cart_seeds; /* 1: CART warm start of every DEOCT subtree */
  int32_t de_seeds;   /* 1: warm start from a full-depth DEOCT (Philox stream 0) */
} orc_mh_params;

/* Greedy misclassification tree of depth D on the samples idx[0..n_sub-1]
 * (Reading: the "CART solution" of Algorithm 2 is the exhaustive depth-1
 * search applied top-down; a node is split only if it has more than n_min
 * samples and two classes, as in Algorithm 2).  a_out, theta_out [2^D - 1]. */
int orc_greedy_tree(const uint32_t* ranks, int64_t n, int32_t F, const uint32_t* n_unique,
                    const uint8_t* y, int32_t K, const int32_t* idx, int64_t n_sub, int32_t depth,
                    int32_t n_min, double alpha, int32_t* a_out, uint32_t* theta_out) {
  int32_t B = (1 << depth) - 1;
  int64_t m = idx ? n_sub : n;
  int32_t* sub = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  uint8_t* seen = (uint8_t*)malloc((size_t)K);
  if (!sub || !seen) { free(sub); free(seen); return ORC_ERR_OOM; }
  for (int32_t t = 0; t < B; ++t) { a_out[t] = 0; theta_out[t] = 0; }
  int rc = ORC_OK;
  for (int32_t t = 1; t <= B && rc == ORC_OK; ++t) {
    int32_t d = 0;
    while ((1 << (d + 1)) <= t) ++d;
    int64_t nt = 0;
    for (int64_t j = 0; j < m; ++j) {
      int64_t i = idx ? idx[j] : j;
      int32_t u = 1;
      for (int32_t l = 0; l < d; ++l) {
        int32_t au = a_out[u - 1];
        int left = (au != 0) && (ranks[(int64_t)(au - 1) * n + i] < theta_out[u - 1]);
        u = left ? 2 * u : 2 * u + 1;
      }
      if (u == t) sub[nt++] = (int32_t)i;
    }
    memset(seen, 0, (size_t)K);
    int32_t ncls = 0;
    for (int64_t j = 0; j < nt; ++j)
      if (!seen[y[sub[j]]]) { seen[y[sub[j]]] = 1; ++ncls; }
    if (!(nt > n_min && ncls > 1)) continue;
    double f;
    rc = orc_depth1(ranks, n, F, n_unique, y, K, sub, nt, n_min, alpha, &a_out[t - 1],
                    &theta_out[t - 1], &f);
  }
  free(sub);
  free(seen);
  return rc;
}

/* Genes of a decoded node (inverse of Eq. aenc / Eq. benc): ahat = a + 1/2;
 * bhat = the float32 nearest (theta + 1/2) / (n_p + 1), moved one float at a
 * time until floor(bhat (n_p + 1)) = theta. */
static void node_genes(int32_t a, uint32_t theta, uint32_t np, float* ahat, float* bhat);

/* node_genes over m nodes: a [m], theta [m], np [m] (n_p of each node's
 * feature, 1 for a = 0) -> ahat [m], bhat [m]. */
void orc_node_genes(const int32_t* a, const uint32_t* theta, const uint32_t* np, int64_t m,
                    float* ahat, float* bhat) {
  for (int64_t i = 0; i < m; ++i) node_genes(a[i], theta[i], np[i], &ahat[i], &bhat[i]);
}

static void node_genes(int32_t a, uint32_t theta, uint32_t np, float* ahat, float* bhat) {
  *ahat = (float)a + 0.5f;
  if (a == 0) { *bhat = 0.0f; return; }
  double np1 = (double)np + 1.0;
  float b = (float)(((double)theta + 0.5) / np1);
  for (int it = 0; it < 64 && floor((double)b * np1) > (double)theta; ++it) b = nextafterf(b, 0.0f);
  for (int it = 0; it < 64 && floor((double)b * np1) < (double)theta; ++it) b = nextafterf(b, 1.0f);
  *bhat = b;
}

/* Algorithm 2 over the branch nodes t = 1..2^D-1 in BFS order.  For node t at
 * depth d (root d = 0, as in the Fig. 3 example of Section 4):
 *   - (X_t, Y_t) = the samples whose path from the root, through the splits
 *     fixed so far, reaches t;
 *   - if |X_t| > n_min and Y_t has at least two classes: D_t = min(D_MH, D-d);
 *     D_t >= 2 -> DEOCT of depth D_t on (X_t, Y_t), Philox stream = t, no warm
 *     starts (Reading C11); D_t = 1 -> exhaustive depth-1; keep the root node
 *     of the result (a DE root with a = 0 is kept as is, Reading C15);
 *   - otherwise the artificial node a_t = 0, b_t = 0.
 * Thresholds stay the global ones (Reading C14).  Outputs: a_out, theta_out
 * [2^D-1]; leaf_class_out [2^D] from Eq. opt_c on the whole training set;
 * kind_out [2^D-1] (nullable): 0 artificial, 1 depth-1 search, 2 DEOCT;
 * node_fit_out [2^D-1] (nullable): the solved subproblem's best fitness. */
int orc_mh(const uint32_t* ranks, int64_t n, int32_t F, const uint32_t* n_unique,
           const uint8_t* y, int32_t K, const orc_mh_params* prm, int32_t* a_out,
           uint32_t* theta_out, uint8_t* leaf_class_out, int32_t* kind_out,
           double* node_fit_out) {
  int32_t D = prm->depth, B = (1 << D) - 1, L = 1 << D;
  if (D < 1 || prm->horizon < 1) return ORC_ERR_INVALID;
  int32_t* sub = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  uint8_t* seen = (uint8_t*)malloc((size_t)K);
  if (!sub || !seen) { free(sub); free(seen); return ORC_ERR_OOM; }
  for (int32_t t = 0; t < B; ++t) { a_out[t] = 0; theta_out[t] = 0; }
  int rc = ORC_OK;
  /* DEOCT warm start trees {(a, b)}^0 of Algorithm 2: the best tree of one
   * DEOCT of the full depth on the whole set */
  int32_t* wa = NULL;
  uint32_t* wth = NULL;
  if (prm->de_seeds && D >= 2 && prm->horizon >= 2) {
    orc_de_params fp;
    fp.depth = D; fp.P = prm->P; fp.G = prm->G; fp.M = prm->M; fp.CR = prm->CR;
    fp.alpha = prm->alpha; fp.n_min = prm->n_min; fp.seed = prm->seed; fp.stream = 0;
    fp.dither = prm->dither;
    float* fpop = (float*)malloc((size_t)prm->P * 2 * B * sizeof(float));
    double* ffit = (double*)malloc((size_t)prm->P * sizeof(double));
    wa = (int32_t*)malloc((size_t)B * sizeof(int32_t));
    wth = (uint32_t*)malloc((size_t)B * sizeof(uint32_t));
    if (!fpop || !ffit || !wa || !wth) rc = ORC_ERR_OOM;
    int32_t fbest = 0;
    if (rc == ORC_OK)
      rc = orc_de_run(ranks, n, F, n_unique, y, K, NULL, n, &fp, NULL, 0, fpop, ffit, &fbest, NULL,
                      NULL, NULL);
    if (rc == ORC_OK) orc_decode(fpop + (int64_t)fbest * 2 * B, 1, D, F, n_unique, wa, wth);
    free(fpop);
    free(ffit);
  }
  for (int32_t t = 1; t <= B && rc == ORC_OK; ++t) {
    int32_t d = 0;
    while ((1 << (d + 1)) <= t) ++d;
    /* induce (X_t, Y_t): route every sample d levels through the fixed nodes */
    int64_t nt = 0;
    for (int64_t i = 0; i < n; ++i) {
      int32_t u = 1;
      for (int32_t l = 0; l < d; ++l) {
        int32_t au = a_out[u - 1];
        int left = (au != 0) && (ranks[(int64_t)(au - 1) * n + i] < theta_out[u - 1]);
        u = left ? 2 * u : 2 * u + 1;
      }
      if (u == t) sub[nt++] = (int32_t)i;
    }
    memset(seen, 0, (size_t)K);
    int32_t nclass = 0;
    for (int64_t j = 0; j < nt; ++j)
      if (!seen[y[sub[j]]]) { seen[y[sub[j]]] = 1; ++nclass; }
    if (kind_out) kind_out[t - 1] = 0;
    if (node_fit_out) node_fit_out[t - 1] = 0.0;
    if (!(nt > prm->n_min && nclass > 1)) continue; /* artificial node */
    int32_t Dt = prm->horizon < D - d ? prm->horizon : D - d;
    if (Dt >= 2) {
      orc_de_params dp;
      dp.depth = Dt; dp.P = prm->P; dp.G = prm->G; dp.M = prm->M; dp.CR = prm->CR;
      dp.alpha = prm->alpha; dp.n_min = prm->n_min; dp.seed = prm->seed;
      dp.stream = (uint64_t)t; dp.dither = prm->dither;
      int32_t Bt = (1 << Dt) - 1;
      float* pop = (float*)malloc((size_t)prm->P * 2 * Bt * sizeof(float));
      double* fit = (double*)malloc((size_t)prm->P * sizeof(double));
      float* seed_genes = (float*)malloc((size_t)2 * 2 * Bt * sizeof(float));
      int32_t* ga = (int32_t*)malloc((size_t)Bt * sizeof(int32_t));
      uint32_t* gth = (uint32_t*)malloc((size_t)Bt * sizeof(uint32_t));
      if (!pop || !fit || !seed_genes || !ga || !gth) {
        free(pop); free(fit); free(seed_genes); free(ga); free(gth);
        rc = ORC_ERR_OOM;
        break;
      }
      int32_t S = 0;
      if (wa) { /* the warm-start tree's subtree with the same shape and location */
        float* g = seed_genes + (int64_t)S * 2 * Bt;
        for (int32_t r = 0, q = 0; r < Dt; ++r)
          for (int32_t j = 0; j < (1 << r); ++j, ++q) {
            int32_t gt = (t << r) + j;
            node_genes(wa[gt - 1], wth[gt - 1], wa[gt - 1] > 0 ? n_unique[wa[gt - 1] - 1] : 1u,
                       &g[q], &g[Bt + q]);
          }
        S += 1;
      }
      if (prm->cart_seeds) { /* the CART solution of the subtree */
        float* g = seed_genes + (int64_t)S * 2 * Bt;
        rc = orc_greedy_tree(ranks, n, F, n_unique, y, K, sub, nt, Dt, prm->n_min, prm->alpha, ga,
                             gth);
        for (int32_t q = 0; q < Bt && rc == ORC_OK; ++q)
          node_genes(ga[q], gth[q], ga[q] > 0 ? n_unique[ga[q] - 1] : 1u, &g[q], &g[Bt + q]);
        S += 1;
      }
      int32_t best = 0;
      if (rc == ORC_OK)
        rc = orc_de_run(ranks, n, F, n_unique, y, K, sub, nt, &dp, S ? seed_genes : NULL, S, pop,
                        fit, &best, NULL, NULL, NULL);
      free(seed_genes);
      free(ga);
      free(gth);
      if (rc == ORC_OK) {
        int32_t a1;
        uint32_t th1;
        decode_node(pop[(int64_t)best * 2 * Bt + 0], pop[(int64_t)best * 2 * Bt + Bt], F,
                    n_unique, &a1, &th1);
        a_out[t - 1] = a1;
        theta_out[t - 1] = th1;
        if (kind_out) kind_out[t - 1] = 2;
        if (node_fit_out) node_fit_out[t - 1] = fit[best];
      }
      free(pop);
      free(fit);
    } else {
      int32_t a1;
      uint32_t th1;
      double f1;
      rc = orc_depth1(ranks, n, F, n_unique, y, K, sub, nt, prm->n_min, prm->alpha, &a1, &th1,
                      &f1);
      if (rc == ORC_OK) {
        a_out[t - 1] = a1;
        theta_out[t - 1] = th1;
        if (kind_out) kind_out[t - 1] = 1;
        if (node_fit_out) node_fit_out[t - 1] = f1;
      }
    }
  }
  free(wa);
  free(wth);
  if (rc == ORC_OK) {
    uint32_t* counts = (uint32_t*)malloc((size_t)L * K * sizeof(uint32_t));
    if (!counts) rc = ORC_ERR_OOM;
    else {
      if (g_threads > 1) orc_eval_counts_omp(ranks, n, F, y, K, NULL, n, a_out, theta_out, 1, D, counts);
      else orc_eval_counts(ranks, n, F, y, K, NULL, n, a_out, theta_out, 1, D, counts);
      orc_leaf_classes(counts, 1, D, K, leaf_class_out);
      free(counts);
    }
  }
  free(sub);
  free(seen);
  return rc;
}

/* ------------------------------------------------------------------------- */
/* Prediction with a fitted tree on raw values (Section 2 routing with the     */
/* threshold set B_p of Section 3.1 in raw units).                             */
/* ------------------------------------------------------------------------- */

/* b_t for node t: with u = the sorted distinct values of feature a_t - 1,
 * theta_t >= 1 -> (u[theta_t - 1] + u[theta_t]) / 2 (a midpoint of B_p),
 * theta_t = 0 -> u[0] (beta_1 = 0 after min-max scaling); a_t = 0 -> 0. */
int orc_split_values(const float* X, int64_t n, int32_t F, const int32_t* a, const uint32_t* theta,
                     int32_t B, double* b_out) {
  float* col = (float*)malloc((size_t)n * sizeof(float));
  if (!col) return ORC_ERR_OOM;
  for (int32_t t = 0; t < B; ++t) {
    if (a[t] == 0) { b_out[t] = 0.0; continue; }
    int32_t p = a[t] - 1;
    if (p >= F) { free(col); return ORC_ERR_INVALID; }
    for (int64_t i = 0; i < n; ++i) {
      float v = X[i * F + p];
      if (v == 0.0f) v = 0.0f;
      col[i] = v;
    }
    qsort(col, (size_t)n, sizeof(float), cmp_float);
    int64_t np = 0;
    for (int64_t i = 0; i < n; ++i)
      if (np == 0 || col[i] != col[np - 1]) col[np++] = col[i];
    if ((int64_t)theta[t] >= np) { free(col); return ORC_ERR_INVALID; }
    b_out[t] = theta[t] == 0 ? (double)col[0]
                             : ((double)col[theta[t] - 1] + (double)col[theta[t]]) * 0.5;
  }
  free(col);
  return ORC_OK;
}

/* Route every row of X [m][F] (x_{a_t} < b_t -> left, a_t = 0 -> right) and
 * output its leaf's class. */
void orc_predict(const float* X, int64_t m, int32_t F, const int32_t* a, const double* b,
                 int32_t depth, const uint8_t* leaf_class, uint8_t* pred) {
  int32_t B = (1 << depth) - 1;
  for (int64_t i = 0; i < m; ++i) {
    int32_t t = 1;
    while (t <= B) {
      int32_t at = a[t - 1];
      int left = (at != 0) && ((double)X[i * F + (at - 1)] < b[t - 1]);
      t = left ? 2 * t : 2 * t + 1;
    }
    pred[i] = leaf_class[t - (B + 1)];
  }
}

/* ------------------------------------------------------------------------- */
/* OpenMP twins for timing and for checking full-size workloads.  They compute */
/* exactly what the plain functions above compute (integer counts and sorts,   */
/* independent per feature or per (tree, sample chunk)), and tests check them  */
/* bit for bit against those functions.  With g_threads = 1 nothing here runs. */
/* ------------------------------------------------------------------------- */

/* Threads used by orc_encode_omp, orc_eval_counts_omp and, through them, by
 * orc_de_run and orc_mh (n < 1 means 1).  Returns the previous setting. */
int orc_set_threads(int n) {
  int old = g_threads;
  g_threads = n < 1 ? 1 : n;
  return old;
}

/* orc_encode with the features spread over the threads. */
int orc_encode_omp(const float* X, int64_t n, int32_t F, uint32_t* ranks_out,
                   uint32_t* n_unique_out) {
  if (n <= 0 || F <= 0) return ORC_ERR_INVALID;
  int rc = ORC_OK;
#pragma omp parallel num_threads(g_threads)
  {
    float* col = (float*)malloc((size_t)n * sizeof(float));
    float* uniq = (float*)malloc((size_t)n * sizeof(float));
    int mine = (col && uniq) ? ORC_OK : ORC_ERR_OOM;
#pragma omp for schedule(dynamic, 1)
    for (int32_t p = 0; p < F; ++p)
      if (mine == ORC_OK) mine = encode_feature(X, n, F, p, col, uniq, ranks_out, n_unique_out);
    free(col);
    free(uniq);
#pragma omp critical
    if (mine != ORC_OK && rc == ORC_OK) rc = mine;
  }
  return rc;
}

/* orc_eval_counts with the (tree, chunk of 2^16 samples) pairs spread over the
 * threads: each pair counts into its own zeroed array, added to counts[r]. */
void orc_eval_counts_omp(const uint32_t* ranks, int64_t n, int32_t F, const uint8_t* y,
                         int32_t K, const int32_t* idx, int64_t n_sub, const int32_t* a,
                         const uint32_t* theta, int32_t P, int32_t depth, uint32_t* counts) {
  (void)F;
  const int32_t B = (1 << depth) - 1, L = 1 << depth;
  const int64_t LK = (int64_t)L * K, CH = (int64_t)1 << 16;
  memset(counts, 0, (size_t)P * LK * sizeof(uint32_t));
  const int64_t m = idx ? n_sub : n;
  const int64_t nch = (m + CH - 1) / CH, items = (int64_t)P * nch;
  if (items == 0) return;
#pragma omp parallel num_threads(g_threads)
  {
    uint32_t* loc = (uint32_t*)malloc((size_t)LK * sizeof(uint32_t));
#pragma omp for schedule(dynamic, 1)
    for (int64_t it = 0; it < items; ++it) {
      const int32_t r = (int32_t)(it / nch);
      const int64_t j0 = (it % nch) * CH, j1 = j0 + CH < m ? j0 + CH : m;
      const int32_t* ar = a + (int64_t)r * B;
      const uint32_t* tr = theta + (int64_t)r * B;
      if (loc) {
        memset(loc, 0, (size_t)LK * sizeof(uint32_t));
        for (int64_t j = j0; j < j1; ++j) {
          int64_t i = idx ? idx[j] : j;
          loc[(int64_t)route(ranks, n, i, ar, tr, depth) * K + y[i]] += 1;
        }
        for (int64_t e = 0; e < LK; ++e)
          if (loc[e]) {
#pragma omp atomic
            counts[(int64_t)r * LK + e] += loc[e];
          }
      } else {
        for (int64_t j = j0; j < j1; ++j) {
          int64_t i = idx ? idx[j] : j;
          int64_t e = (int64_t)r * LK + (int64_t)route(ranks, n, i, ar, tr, depth) * K + y[i];
#pragma omp atomic
          counts[e] += 1;
        }
      }
    }
    free(loc);
  }
}
