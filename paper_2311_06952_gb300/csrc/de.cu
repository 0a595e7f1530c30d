// de.cu -- device-side DEOCT step (Algorithm 4; Eqs. mutation, crossover,
// selection; the fitness of Section 3.2) and tree decoding (Eq. aenc, Eq. benc).
//
// One CTA per subproblem.  A step kernel does, in order and as its flags ask:
//   DE_FIRST  fitness of the just-evaluated initial population, best;
//   DE_SELECT fitness of the just-evaluated trials, Eq. selection, best;
//   DE_TRIAL  trial vectors of generation g from (population, best), their
//             decoded nodes for the evaluator, and zeroed class counts.
// So one generation is two launches: evaluator, step(SELECT|TRIAL); for one
// problem with more than 256 individuals the step(SELECT|TRIAL) is itself split
// over CTAs in two launches (de_select_wide_kernel, de_trial_wide_kernel).  Gene
// arithmetic is float32 with one rounding per operation (__fsub_rn, __fmul_rn,
// __fadd_rn); random numbers come from Philox4x64-10 keyed by (seed, stream).
#include "internal.cuh"

namespace deoct {

namespace {

__device__ __forceinline__ const DEProb& prob_of(const DEArgs& a) {
  return a.probs ? a.probs[blockIdx.x] : a.single;
}

// (double)e for 0 <= e < 2^53 (exact), built with integer operations only: the
// leading one sets the exponent, the bits below it the significand.
__device__ __forceinline__ double exact_double(int64_t e) {
  if (e <= 0) return 0.0;
  const int lz = __clzll(e);
  const uint64_t mant = ((uint64_t)e << (lz + 1)) >> 12;  // the 52 bits below the leading one
  return __longlong_as_double((long long)(((uint64_t)(1086 - lz) << 52) | mant));
}

// Fitness order.  With alpha >= 0 every fitness is a non-negative double (not
// -0), whose bit pattern as a signed 64-bit integer orders exactly like the
// value, so comparisons need no FP64 arithmetic; a negative alpha compares the
// doubles.
__device__ __forceinline__ bool fit_le(double x, double y, bool bits) {
  return bits ? __double_as_longlong(x) <= __double_as_longlong(y) : x <= y;
}
__device__ __forceinline__ bool fit_lt(double x, double y, bool bits) {
  return bits ? __double_as_longlong(x) < __double_as_longlong(y) : x < y;
}

__device__ __forceinline__ float clamp_gene(float v, float hi) {
  v = v < 0.0f ? 0.0f : v;
  return v > hi ? hi : v;
}

// block-wide argmin (lowest index among minimal values); result in *best_s.
// bits: compare in the order of fit_lt (see there)
__device__ void block_argmin(const double* __restrict__ fit, int P, int* best_s, double* red_f,
                             int* red_i, bool bits) {
  double bf = 0.0;
  int bi = -1;
  for (int r = threadIdx.x; r < P; r += blockDim.x) {
    double f = fit[r];
    if (bi < 0 || fit_lt(f, bf, bits)) {
      bf = f;
      bi = r;
    }
  }
  // warp reduce
  for (int off = 16; off > 0; off >>= 1) {
    double of = __shfl_down_sync(0xFFFFFFFFu, bf, off);
    int oi = __shfl_down_sync(0xFFFFFFFFu, bi, off);
    if (oi >= 0 && (bi < 0 || fit_lt(of, bf, bits) || (!fit_lt(bf, of, bits) && oi < bi))) {
      bf = of;
      bi = oi;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red_f[warp] = bf;
    red_i[warp] = bi;
  }
  __syncthreads();
  if (warp == 0) {  // the warps' winners, reduced by one warp in the same order
    const int nw = (blockDim.x + 31) >> 5;
    bf = lane < nw ? red_f[lane] : 0.0;
    bi = lane < nw ? red_i[lane] : -1;
    for (int off = 16; off > 0; off >>= 1) {
      double of = __shfl_down_sync(0xFFFFFFFFu, bf, off);
      int oi = __shfl_down_sync(0xFFFFFFFFu, bi, off);
      if (oi >= 0 && (bi < 0 || fit_lt(of, bf, bits) || (!fit_lt(bf, of, bits) && oi < bi))) {
        bf = of;
        bi = oi;
      }
    }
    if (lane == 0) *best_s = bi;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(1024) de_init_kernel(const DEArgs a) {
  const DEProb& pb = prob_of(a);
  const int P = a.P, D = a.depth, B = (1 << D) - 1, m = 2 * B, L = 1 << D;
  const float ub_a = (float)(pb.F + 1);
  const float hi_a = below_bound(ub_a), hi_b = below_bound(1.0f);
  for (int r = threadIdx.x; r < P; r += blockDim.x) {
    float* g = pb.pop + (int64_t)r * m;
    if (r < pb.S) {
      for (int q = 0; q < m; ++q) g[q] = pb.seeds[(int64_t)r * m + q];
    } else {
      U64x4 blk;
      for (int q = 0; q < m; ++q) {
        if ((q & 7) == 0) blk = philox4x64_10(0ull, (uint64_t)r, (uint64_t)(q >> 3), 0ull, pb.seed,
                                              pb.stream_id);
        const float u = u01(draw_from_block(blk, (uint32_t)q));
        const bool is_a = q < B;
        g[q] = clamp_gene(__fmul_rn(u, is_a ? ub_a : 1.0f), is_a ? hi_a : hi_b);
      }
    }
    for (int t = 0; t < B; ++t) {
      int av;
      uint32_t th;
      decode_gene_pair(g[t], g[B + t], pb.F, pb.n_unique, &av, &th);
      pb.nodes[(int64_t)r * B + t] = pack_node(av, th);
    }
  }
  uint32_t* cnt = pb.counts;
  const int64_t total = (int64_t)P * L * pb.K;
  for (int64_t e = threadIdx.x; e < total; e += blockDim.x) cnt[e] = 0;
  if (threadIdx.x == 0 && pb.gen) *pb.gen = 1;
}

// The fitness of Section 3.2 of individual r from its class counts,
//   f = (errors + V) + alpha * splits, errors = n - sum_leaf max_k count,
//   V = #{leaf : 0 < n_leaf < n_min}, splits = #{t : a_t >= 1} (ahat_t >= 1),
// by its group of G lanes (G a power of two that divides 32; `sub` the lane's
// place in the group, `gm` the group's lane mask): each lane takes leaves sub,
// sub + G, ... and genes sub, sub + G, ..., and the integer partial sums meet
// by shuffles, so every lane returns the same value.
__device__ double group_fitness(const uint32_t* __restrict__ c, const float* __restrict__ genes,
                                int B, int L, int K, int64_t n_valid, int n_min, double alpha,
                                int sub, int G, uint32_t gm) {
  long long correct = 0;
  uint32_t v = 0, splits = 0;
  // the lane's counts (leaves sub, sub + G, ..., every class), sixteen loads in
  // flight at a time: one after another they were a chain of memory round trips
  const int nc = ((L - sub + G - 1) / G) * K;
  int li = sub, ki = 0;  // leaf and class of the next count loaded
  uint32_t mx = 0;
  int64_t nl = 0;
  int kr = 0;            // classes of the current leaf reduced so far
  for (int e0 = 0; e0 < nc; e0 += 16) {
    uint32_t x[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      x[j] = e0 + j < nc ? c[li * K + ki] : 0u;
      if (++ki == K) {
        ki = 0;
        li += G;
      }
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (e0 + j < nc) {
        mx = x[j] > mx ? x[j] : mx;
        nl += x[j];
        if (++kr == K) {
          correct += mx;
          if (nl > 0 && nl < n_min) v += 1;
          mx = 0;
          nl = 0;
          kr = 0;
        }
      }
    }
  }
  for (int t = sub; t < B; t += G) splits += genes[t] >= 1.0f ? 1u : 0u;
  for (int o = G >> 1; o > 0; o >>= 1) {
    correct += __shfl_xor_sync(gm, correct, o);
    v += __shfl_xor_sync(gm, v, o);
    splits += __shfl_xor_sync(gm, splits, o);
  }
  const int64_t errors = n_valid - (int64_t)correct;
  // alpha = 0 (the default): the fitness is the integer errors + V, and
  // (errors + V) + 0 * splits is that integer exactly
  if (alpha == 0.0) return exact_double(errors + (int64_t)v);
  return __dadd_rn((double)(errors + (int64_t)v), __dmul_rn(alpha, (double)splits));
}

// Eq. selection of individual r by its group of G lanes: the fitness of its
// just-evaluated trial from the class counts; the trial replaces the individual
// when it is no worse (ties go to the trial).
__device__ __forceinline__ void select_individual(const DEArgs& a, const DEProb& pb, int r, int B,
                                                  int L, int K, int sub, int G, uint32_t gm,
                                                  bool bits) {
  const int m = 2 * B;
  const float* genes = pb.trial + (int64_t)r * m;
  const double f = group_fitness(pb.counts + (int64_t)r * L * K, genes, B, L, K, pb.n_valid,
                                 a.n_min, a.alpha, sub, G, gm);
  const double fr = pb.fit[r];
  __syncwarp(gm);  // every lane has read fit[r] before it is rewritten
  if (sub == 0) pb.fit_trial[r] = f;
  if (fit_le(f, fr, bits)) {
    float* dst = pb.pop + (int64_t)r * m;
    for (int q = sub; q < m; q += G) dst[q] = genes[q];
    if (sub == 0) pb.fit[r] = f;
  }
}

// Generation g's trial vector of individual r (Eqs. mutation and crossover) from
// the population and its best individual, stored with its decoded nodes.  Lane
// `sub` of the group takes consecutive genes, which share Philox blocks.
__device__ __forceinline__ void trial_individual(const DEArgs& a, const DEProb& pb, int r, int g,
                                                 int best, int B, int sub, int G, uint32_t gm) {
  const int P = a.P, m = 2 * B;
  const float ub_a = (float)(pb.F + 1);
  const float hi_a = below_bound(ub_a), hi_b = below_bound(1.0f);
  const float* sb = pb.pop + (int64_t)best * m;
  const int per = (m + G - 1) / G;
  // draws 0..7 come from block 0: r1, r2, q_rand, M, genes 0..3
  const U64x4 blk0 = philox4x64_10((uint64_t)g, (uint64_t)r, 0ull, 0ull, pb.seed, pb.stream_id);
  const uint32_t x0 = draw_from_block(blk0, 0), x1 = draw_from_block(blk0, 1);
  const uint32_t x2 = draw_from_block(blk0, 2), x3 = draw_from_block(blk0, 3);
  int r1 = (int)below(x0, (uint32_t)(P - 1));
  if (r1 >= r) r1 += 1;
  int r2 = (int)below(x1, (uint32_t)(P - 2));
  const int lo = r < r1 ? r : r1, hi = r < r1 ? r1 : r;
  if (r2 >= lo) r2 += 1;
  if (r2 >= hi) r2 += 1;
  const int qrand = (int)below(x2, (uint32_t)m);
  const float M = a.dither ? u01(x3) : a.M;
  const float* s1 = pb.pop + (int64_t)r1 * m;
  const float* s2 = pb.pop + (int64_t)r2 * m;
  const float* sr = pb.pop + (int64_t)r * m;
  float* u = pb.trial + (int64_t)r * m;
  U64x4 blk = blk0;
  uint32_t cur = 0;  // block held in blk
  const int q0 = sub * per, q1 = min(m, q0 + per);
  for (int q = q0; q < q1; ++q) {
    const uint32_t s = 4u + (uint32_t)q;
    if ((s >> 3) != cur) {
      cur = s >> 3;
      blk = philox4x64_10((uint64_t)g, (uint64_t)r, (uint64_t)cur, 0ull, pb.seed, pb.stream_id);
    }
    const float v = __fadd_rn(sb[q], __fmul_rn(M, __fsub_rn(s1[q], s2[q])));
    const float vc = clamp_gene(v, q < B ? hi_a : hi_b);
    const float rq = u01(draw_from_block(blk, s));
    u[q] = (rq <= a.CR || q == qrand) ? vc : sr[q];
  }
  __syncwarp(gm);  // the group's genes are written before they are decoded
  for (int t = sub; t < B; t += G) {
    int av;
    uint32_t th;
    decode_gene_pair(u[t], u[B + t], pb.F, pb.n_unique, &av, &th);
    pb.nodes[(int64_t)r * B + t] = pack_node(av, th);
  }
}

// One CTA per subproblem; each individual is worked on by a group of `lanes`
// consecutive threads (lanes x P <= blockDim.x, lanes <= 4), which shortens the
// chain of dependent loads one thread would walk alone.  Every value is the one a
// single thread computes: integer sums, the draws of a (generation,
// individual, block) Philox key, one rounding per float operation.
__global__ void __launch_bounds__(1024) de_step_kernel(const DEArgs a, int g_arg, int flags,
                                                       int lanes) {
  __shared__ double red_f[32];
  __shared__ int red_i[32];
  __shared__ int best_s;
  __shared__ int g_s;
  const DEProb& pb = prob_of(a);
  const int P = a.P, D = a.depth, B = (1 << D) - 1, m = 2 * B, L = 1 << D, K = pb.K;
  const int G = lanes;
  const int sub = threadIdx.x & (G - 1);
  const uint32_t gm = (G == 32 ? 0xFFFFFFFFu : ((1u << G) - 1u)) << ((threadIdx.x & 31) & ~(G - 1));
  const int r0 = threadIdx.x / G, rstep = blockDim.x / G;

  const bool bits = a.alpha >= 0.0;  // fitness order by bit patterns (see fit_lt)
  if (threadIdx.x == 0) g_s = (flags & DE_GEN_DEVICE) ? *pb.gen : g_arg;

  if (flags & (DE_FIRST | DE_SELECT)) {
    const bool first = (flags & DE_FIRST) != 0;
    for (int r = r0; r < P; r += rstep) {
      if (first) {
        const double f = group_fitness(pb.counts + (int64_t)r * L * K, pb.pop + (int64_t)r * m, B,
                                       L, K, pb.n_valid, a.n_min, a.alpha, sub, G, gm);
        if (sub == 0) pb.fit[r] = f;
      } else {
        select_individual(a, pb, r, B, L, K, sub, G, gm, bits);
      }
    }
    __syncthreads();
    block_argmin(pb.fit, P, &best_s, red_f, red_i, bits);
    if (threadIdx.x == 0) *pb.best = best_s;
  } else {
    if (threadIdx.x == 0) best_s = *pb.best;
    __syncthreads();
  }

  if (!(flags & DE_TRIAL)) return;
  const int g = g_s;
  if (g < 1 || g > pb.G) return;  // device-driven replay past the last generation
  const int best = best_s;
  for (int r = r0; r < P; r += rstep) trial_individual(a, pb, r, g, best, B, sub, G, gm);
  const int64_t total = (int64_t)P * L * K;
  for (int64_t e = threadIdx.x; e < total; e += blockDim.x) pb.counts[e] = 0;
  if (threadIdx.x == 0 && (flags & DE_GEN_DEVICE)) *pb.gen = g + 1;
}

// The steady-state step (Eq. selection of generation g - 1's trials, then
// generation g's trial vectors) when every individual has its own group of G
// lanes (P G <= 512) and a lane holds at most four consecutive genes (2B <= 4G).
// The general step waits on global memory once per gene or leaf in turn; here
// the loads an individual needs that do not wait for the argmin (its class
// counts, fitness, trial and population genes, and the genes of r1 and r2, whose
// draws need no memory) are issued together, the argmin reads the fitness from
// shared memory, and the decode reads the new genes and n_p there too.  The
// values are those of the general step: integer sums in any order, the same
// draws, one rounding per float operation, the same selection and argmin.
constexpr int kFastP = 256, kFastM = 16, kFastC = 16;

__global__ void __launch_bounds__(512) de_step_fast_kernel(const DEArgs a, int g_arg, int flags,
                                                          int G) {
  __shared__ double red_f[32];
  __shared__ int red_i[32];
  __shared__ int best_s;
  __shared__ double fit_s[kFastP];
  __shared__ unsigned char sel_s[kFastP];
  __shared__ float u_s[kFastP * kFastM];
  __shared__ uint32_t nu_s[kMaxF];
  const DEProb& pb = prob_of(a);
  const int P = a.P, B = (1 << a.depth) - 1, m = 2 * B, L = 1 << a.depth, K = pb.K;
  const int sub = threadIdx.x & (G - 1);
  const uint32_t gm = (G == 32 ? 0xFFFFFFFFu : ((1u << G) - 1u)) << ((threadIdx.x & 31) & ~(G - 1));
  const int r = threadIdx.x / G;
  const bool act = r < P;  // a whole group is active or not
  const bool bits = a.alpha >= 0.0;
  const int per = (m + G - 1) / G;
  const int q0 = sub * per, q1 = min(m, q0 + per);
  for (int f = threadIdx.x; f < pb.F; f += blockDim.x) nu_s[f] = pb.n_unique[f];

  // ---- this individual's own data (one round of loads) ----------------------
  // a lane's class counts: leaves sub, sub + G, ..., all K classes of each
  const int nc = ((L - sub + G - 1) / G) * K;  // at most kFastC (checked at launch)
  float tr[4], pr[4];
  uint32_t cv[kFastC];
  double fr = 0.0;
  if (act) {
    fr = pb.fit[r];
    const float* trg = pb.trial + (int64_t)r * m;
    const float* pog = pb.pop + (int64_t)r * m;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int q = q0 + j;
      tr[j] = q < q1 ? trg[q] : 0.0f;
      pr[j] = q < q1 ? pog[q] : 0.0f;
    }
    const uint32_t* c = pb.counts + (int64_t)r * L * K;
    int li = sub, ki = 0;  // leaf and class of the next count loaded
#pragma unroll
    for (int e = 0; e < kFastC; ++e) {
      cv[e] = e < nc ? c[li * K + ki] : 0u;
      if (++ki == K) {
        ki = 0;
        li += G;
      }
    }
  }

  // ---- generation g's draws and the genes of r1 and r2 (no memory needed for
  // the draws, so they run while the loads above are in flight) --------------
  const int g = (flags & DE_GEN_DEVICE) ? *pb.gen : g_arg;
  const bool trial = g >= 1 && g <= pb.G;
  int r1 = 0, r2 = 0, qrand = 0;
  float M = a.M, rq[4], t1[4], p1[4], t2[4], p2[4];
  if (act && trial) {
    const U64x4 blk0 = philox4x64_10((uint64_t)g, (uint64_t)r, 0ull, 0ull, pb.seed, pb.stream_id);
    const uint32_t x0 = draw_from_block(blk0, 0), x1 = draw_from_block(blk0, 1);
    const uint32_t x2 = draw_from_block(blk0, 2), x3 = draw_from_block(blk0, 3);
    r1 = (int)below(x0, (uint32_t)(P - 1));
    if (r1 >= r) r1 += 1;
    r2 = (int)below(x1, (uint32_t)(P - 2));
    const int lo = r < r1 ? r : r1, hi = r < r1 ? r1 : r;
    if (r2 >= lo) r2 += 1;
    if (r2 >= hi) r2 += 1;
    qrand = (int)below(x2, (uint32_t)m);
    if (a.dither) M = u01(x3);
    const float* t1g = pb.trial + (int64_t)r1 * m;
    const float* p1g = pb.pop + (int64_t)r1 * m;
    const float* t2g = pb.trial + (int64_t)r2 * m;
    const float* p2g = pb.pop + (int64_t)r2 * m;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int q = q0 + j;
      const bool in = q < q1;
      t1[j] = in ? t1g[q] : 0.0f;
      p1[j] = in ? p1g[q] : 0.0f;
      t2[j] = in ? t2g[q] : 0.0f;
      p2[j] = in ? p2g[q] : 0.0f;
    }
    // gene q draws s = q + 4 from block s / 8: a lane's four genes touch at most two
    U64x4 blk = blk0;
    uint32_t cur = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t s = 4u + (uint32_t)(q0 + j);
      if (q0 + j < q1 && (s >> 3) != cur) {
        cur = s >> 3;
        blk = philox4x64_10((uint64_t)g, (uint64_t)r, (uint64_t)cur, 0ull, pb.seed, pb.stream_id);
      }
      rq[j] = u01(draw_from_block(blk, s));
    }
  }

  // ---- the fitness of Section 3.2 from the counts (as group_fitness) ---------
  double f = 0.0;
  if (act) {
    long long correct = 0;
    uint32_t v = 0, splits = 0;
    uint32_t mx = 0;
    int64_t nl = 0;
    int kr = 0;  // classes of the current leaf reduced so far
#pragma unroll
    for (int e = 0; e < kFastC; ++e) {
      if (e < nc) {
        mx = cv[e] > mx ? cv[e] : mx;
        nl += cv[e];
        if (++kr == K) {
          correct += mx;
          if (nl > 0 && nl < a.n_min) v += 1;
          mx = 0;
          nl = 0;
          kr = 0;
        }
      }
    }
    if (a.alpha != 0.0) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (q0 + j < q1 && q0 + j < B) splits += tr[j] >= 1.0f ? 1u : 0u;
    }
    for (int o = G >> 1; o > 0; o >>= 1) {
      correct += __shfl_xor_sync(gm, correct, o);
      v += __shfl_xor_sync(gm, v, o);
      splits += __shfl_xor_sync(gm, splits, o);
    }
    const int64_t errors = pb.n_valid - (int64_t)correct;
    f = (a.alpha == 0.0) ? exact_double(errors + (int64_t)v)
                         : __dadd_rn((double)(errors + (int64_t)v), __dmul_rn(a.alpha, (double)splits));
  }

  // ---- Eq. selection, then the argmin over shared memory --------------------
  bool take = false;
  if (act) {
    __syncwarp(gm);  // every lane has read fit[r] before it is rewritten
    take = fit_le(f, fr, bits);  // ties go to the trial
    if (sub == 0) pb.fit_trial[r] = f;
    if (take) {
      float* dst = pb.pop + (int64_t)r * m;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (q0 + j < q1) dst[q0 + j] = tr[j];
      if (sub == 0) pb.fit[r] = f;
    }
    if (sub == 0) {
      fit_s[r] = take ? f : fr;
      sel_s[r] = take ? 1 : 0;
    }
  }
  __syncthreads();
  block_argmin(fit_s, P, &best_s, red_f, red_i, bits);
  if (threadIdx.x == 0) *pb.best = best_s;
  if (!trial) return;  // device-driven replay past the last generation

  // ---- generation g's trial vectors from the new population, decoded --------
  if (act) {
    const float ub_a = (float)(pb.F + 1);
    const float hi_a = below_bound(ub_a), hi_b = below_bound(1.0f);
    const float* sbg = pb.pop + (int64_t)best_s * m;  // the new population: copies are done
    const bool sel1 = sel_s[r1] != 0, sel2 = sel_s[r2] != 0;
    float* u = pb.trial + (int64_t)r * m;
    float* us = u_s + r * m;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int q = q0 + j;
      if (q < q1) {
        const float s1 = sel1 ? t1[j] : p1[j], s2 = sel2 ? t2[j] : p2[j];
        const float sr = take ? tr[j] : pr[j];
        const float v = __fadd_rn(sbg[q], __fmul_rn(M, __fsub_rn(s1, s2)));
        const float vc = clamp_gene(v, q < B ? hi_a : hi_b);
        const float uq = (rq[j] <= a.CR || q == qrand) ? vc : sr;
        u[q] = uq;
        us[q] = uq;
      }
    }
    __syncwarp(gm);  // the group's genes are in shared memory before they are decoded
    for (int t = sub; t < B; t += G) {
      int av;
      uint32_t th;
      decode_gene_pair(us[t], us[B + t], pb.F, nu_s, &av, &th);
      pb.nodes[(int64_t)r * B + t] = pack_node(av, th);
    }
  }
  const int64_t total = (int64_t)P * L * K;  // every count was read before the barrier
  for (int64_t e = threadIdx.x; e < total; e += blockDim.x) pb.counts[e] = 0;
  if (threadIdx.x == 0 && (flags & DE_GEN_DEVICE)) *pb.gen = g + 1;
}

// The steady-state step of one problem with a large population, split over CTAs
// of kDeWideR individuals (kDeWideG lanes each) in two launches: one CTA alone
// walks every individual through a chain of dependent loads, and at P = 1024
// that took 88 us a generation.  The first launch does Eq. selection and the
// argmin of each CTA's individuals; the second reduces those candidates to the
// best (lowest index among minimal fitness, as one CTA would find it, since the
// CTAs cover ascending index ranges), then builds the trials.  The values are
// those of the one-CTA step.
__global__ void __launch_bounds__(kDeWideR * kDeWideG) de_select_wide_kernel(const DEArgs a,
                                                                              int g_arg, int flags) {
  __shared__ double red_f[32];
  __shared__ int red_i[32];
  __shared__ int best_s;
  const DEProb& pb = a.single;
  const int P = a.P, B = (1 << a.depth) - 1, L = 1 << a.depth, K = pb.K;
  constexpr int G = kDeWideG;
  const int sub = threadIdx.x & (G - 1);
  const uint32_t gm = ((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1));
  const int r0 = blockIdx.x * kDeWideR, nr = min(kDeWideR, P - r0);
  const int r = r0 + (int)threadIdx.x / G;
  const bool bits = a.alpha >= 0.0;
  if (r < P) select_individual(a, pb, r, B, L, K, sub, G, gm, bits);  // whole groups only
  __syncthreads();
  block_argmin(pb.fit + r0, nr, &best_s, red_f, red_i, bits);
  if (threadIdx.x == 0) {
    a.part_f[blockIdx.x] = pb.fit[r0 + best_s];
    a.part_i[blockIdx.x] = r0 + best_s;
    // the generation is read here, before the second launch's first CTA advances it
    if (blockIdx.x == 0) *a.part_g = (flags & DE_GEN_DEVICE) ? *pb.gen : g_arg;
  }
}

__global__ void __launch_bounds__(kDeWideR * kDeWideG) de_trial_wide_kernel(const DEArgs a,
                                                                             int flags, int nblk) {
  __shared__ double red_f[32];
  __shared__ int red_i[32];
  __shared__ int best_s;
  const DEProb& pb = a.single;
  const int P = a.P, B = (1 << a.depth) - 1, L = 1 << a.depth, K = pb.K;
  constexpr int G = kDeWideG;
  const int sub = threadIdx.x & (G - 1);
  const uint32_t gm = ((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1));
  const int r0 = blockIdx.x * kDeWideR, nr = min(kDeWideR, P - r0);
  const int r = r0 + (int)threadIdx.x / G;
  block_argmin(a.part_f, nblk, &best_s, red_f, red_i, a.alpha >= 0.0);
  const int best = a.part_i[best_s];
  const int g = *a.part_g;
  const bool trial = g >= 1 && g <= pb.G;  // false: device-driven replay past the last generation
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *pb.best = best;
    if (trial && (flags & DE_GEN_DEVICE)) *pb.gen = g + 1;
  }
  if (!trial) return;
  if (r < P) trial_individual(a, pb, r, g, best, B, sub, G, gm);
  // this CTA's individuals' class counts, read by the first launch, zeroed for the next
  const int64_t e0 = (int64_t)r0 * L * K, e1 = (int64_t)(r0 + nr) * L * K;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) pb.counts[e] = 0;
}

__global__ void decode_kernel(const float* __restrict__ genes, int P, int B, int F,
                              const uint32_t* __restrict__ n_unique, uint16_t* __restrict__ a_out,
                              uint32_t* __restrict__ th_out) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)P * B) return;
  int64_t r = e / B;
  int t = (int)(e - r * B);
  int av;
  uint32_t th;
  decode_gene_pair(genes[r * 2 * B + t], genes[r * 2 * B + B + t], F, n_unique, &av, &th);
  a_out[e] = (uint16_t)av;
  th_out[e] = th;
}

__global__ void best_extract_kernel(const float* __restrict__ pop, const double* __restrict__ fit,
                                    const int32_t* __restrict__ best, int B, int F,
                                    const uint32_t* __restrict__ n_unique, uint16_t* __restrict__ a_out,
                                    uint32_t* __restrict__ th_out, double* __restrict__ fit_out) {
  const int b = *best;
  const float* g = pop + (int64_t)b * 2 * B;
  for (int t = threadIdx.x; t < B; t += blockDim.x) {
    int av;
    uint32_t th;
    decode_gene_pair(g[t], g[B + t], F, n_unique, &av, &th);
    a_out[t] = (uint16_t)av;
    th_out[t] = th;
  }
  if (threadIdx.x == 0) *fit_out = fit[b];
}

// Threads per individual in the step kernel: the largest power of two up to 4
// that keeps the CTA within 1024 threads (4 for P <= 256, 1 for P > 512).
// Measured on the moving-horizon workload (P = 128): 1 / 2 / 4 / 8 threads gave
// 0.2246 / 0.2215 / 0.2180 / 0.2212 s batched and 0.674 / 0.653 / 0.631 / 0.687 s
// plain (with 8, the CTA-wide argmin and barriers span 32 warps).
int lanes_for(int P) {
  int g = 1;
  while (g < 4 && P * g * 2 <= 1024) g *= 2;
  return g;
}

int block_for(int P) {
  int b = ((P + 31) / 32) * 32;
  if (b > 1024) b = 1024;
  if (b < 128) b = 128;
  return b;
}

}  // namespace

int de_launch_init(deoct_ctx* ctx, const DEArgs& a, cudaStream_t s) {
  const int nprob = a.probs ? a.nprob : 1;
  if (nprob <= 0) return DEOCT_OK;
  de_init_kernel<<<nprob, block_for(a.P), 0, s>>>(a);
  count_launch(ctx);
  return check_launch("de_init_kernel");
}

int de_launch_step(deoct_ctx* ctx, const DEArgs& a, int g, int flags, cudaStream_t s) {
  const int nprob = a.probs ? a.nprob : 1;
  if (nprob <= 0) return DEOCT_OK;
  const int lanes = lanes_for(a.P);
  const int m = 2 * ((1 << a.depth) - 1);
  const int L = 1 << a.depth;
  if ((flags & DE_SELECT) && (flags & DE_TRIAL) && !(flags & DE_FIRST) && a.P * lanes <= 512 &&
      a.P <= kFastP && m <= 4 * lanes && m <= kFastM && a.Kmax > 0 &&
      ((L + lanes - 1) / lanes) * a.Kmax <= kFastC) {
    de_step_fast_kernel<<<nprob, block_for(a.P * lanes), 0, s>>>(a, g, flags, lanes);
    count_launch(ctx);
    return check_launch("de_step_fast_kernel");
  }
  if ((flags & DE_SELECT) && (flags & DE_TRIAL) && !(flags & DE_FIRST) && !a.probs && a.part_f &&
      a.P > kFastP && a.P <= kMaxPop) {
    const int nblk = (a.P + kDeWideR - 1) / kDeWideR;
    de_select_wide_kernel<<<nblk, kDeWideR * kDeWideG, 0, s>>>(a, g, flags);
    count_launch(ctx);
    DEOCT_TRY(check_launch("de_select_wide_kernel"));
    de_trial_wide_kernel<<<nblk, kDeWideR * kDeWideG, 0, s>>>(a, flags, nblk);
    count_launch(ctx);
    return check_launch("de_trial_wide_kernel");
  }
  de_step_kernel<<<nprob, block_for(a.P * lanes), 0, s>>>(a, g, flags, lanes);
  count_launch(ctx);
  return check_launch("de_step_kernel");
}

int launch_best_extract(deoct_ctx* ctx, const float* pop, const double* fit, const int32_t* best,
                        int depth, int F, const uint32_t* n_unique, uint16_t* a_out,
                        uint32_t* theta_out, double* fit_out, cudaStream_t s) {
  best_extract_kernel<<<1, 256, 0, s>>>(pop, fit, best, (1 << depth) - 1, F, n_unique, a_out,
                                        theta_out, fit_out);
  count_launch(ctx);
  return check_launch("best_extract_kernel");
}

int launch_decode(deoct_ctx* ctx, const float* genes, int P, int depth, int F,
                  const uint32_t* n_unique, uint16_t* a_out, uint32_t* theta_out,
                  cudaStream_t s) {
  const int B = (1 << depth) - 1;
  const int64_t total = (int64_t)P * B;
  if (total <= 0) return DEOCT_OK;
  decode_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(genes, P, B, F, n_unique, a_out,
                                                               theta_out);
  count_launch(ctx);
  return check_launch("decode_kernel");
}

}  // namespace deoct
