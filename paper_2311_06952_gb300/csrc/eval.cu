// eval.cu -- population fitness evaluation (Algorithm 1, Section 3.2).
//
// Layout of the work: persistent CTAs split a flattened sequence of tiles
// (jobs x tiles; a job is one tree group of one subproblem) into equal
// contiguous ranges.  Per tile a CTA stages the feature-major rank rows of S
// samples in shared memory (1-D TMA bulk copies when the rows are aligned,
// plain loads for gathered subsets), so each sample is read from HBM once per
// tree group, and routes every sample through every tree of the job, whose
// nodes sit in shared memory.  Counting:
//  - ballot mode (2^D * K <= 128): the routing predicate of level d is a warp
//    ballot B_d over 32 samples; lane b owns bin b = leaf*K + k and adds
//    popc(Y_k & AND_d (B_d or ~B_d by bit d of leaf)) -- the class masks Y_k
//    are precomputed per tile, so counting costs no atomics;
//  - atomic mode (larger 2^D * K): per-warp shared histogram with atomics.
// Counts of a job accumulate in shared memory and reach HBM with one atomic
// add per (tree, bin) per CTA.
#include <algorithm>

#include "internal.cuh"

namespace deoct {

namespace {

template <int W>
struct RankT;
template <>
struct RankT<2> {
  typedef uint16_t T;
};
template <>
struct RankT<4> {
  typedef uint32_t T;
};

constexpr int kQMax = 4;  // ballot mode: bins per lane
constexpr int kU = 2;     // chunks of 32 samples interleaved per warp

struct EvalArgs {
  EvalProb single;
  const EvalProb* probs;
  const EvalJob* jobs;
  int njobs;
  int single_ntiles;  // tiles per job when `probs` is null
  int64_t total_tiles;
  int S, TG, Fmax, Kmax;
  int* status;
};

struct JobView {
  const EvalProb* p;
  int64_t tile;  // tile index within the job
  int32_t job, tree0, ntrees;
};

__device__ __forceinline__ void lookup_job(const EvalArgs& a, int64_t gt, JobView* v) {
  if (a.probs == nullptr) {
    int64_t job = gt / a.single_ntiles;
    v->p = &a.single;
    v->job = (int32_t)job;
    v->tile = gt - job * a.single_ntiles;
    v->tree0 = (int32_t)job * a.TG;
    int rem = a.single.P - v->tree0;
    v->ntrees = rem < a.TG ? rem : a.TG;
    return;
  }
  int lo = 0, hi = a.njobs - 1;  // last job with tile_begin <= gt
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (a.jobs[mid].tile_begin <= gt) lo = mid; else hi = mid - 1;
  }
  const EvalJob& j = a.jobs[lo];
  v->p = a.probs + j.prob;
  v->job = lo;
  v->tile = gt - j.tile_begin;
  v->tree0 = j.tree0;
  v->ntrees = j.ntrees;
}

__host__ __device__ __forceinline__ size_t align128(size_t x) { return (x + 127) & ~size_t(127); }

// shared-memory layout shared by host sizing and the kernel
struct SmemLayout {
  size_t tile, nodes, aux, cnt, total;
};
__host__ __device__ __forceinline__ SmemLayout smem_layout(int mode, int W, int D, int S, int TG,
                                                           int Fmax, int Kmax, int warps) {
  const int B = (1 << D) - 1, L = 1 << D;
  const int LK = L * Kmax;
  SmemLayout s;
  s.tile = 0;
  s.nodes = align128((size_t)Fmax * S * W);
  if (mode == 0) {
    const int Q = (LK + 31) / 32;
    s.aux = s.nodes + align128((size_t)TG * B * 8);
    s.cnt = s.aux + align128((size_t)S * Q * 4);
    s.total = s.cnt + align128((size_t)TG * LK * 4);
  } else {
    s.aux = s.nodes + align128((size_t)TG * B * 8);  // labels [S]
    s.cnt = s.aux + align128((size_t)S);             // per-warp histograms
    s.total = s.cnt + align128((size_t)warps * LK * 4);
  }
  return s;
}

template <int W, int D, int MODE>
__global__ void __launch_bounds__(512) eval_kernel(const EvalArgs a) {
  constexpr int B = (1 << D) - 1;
  constexpr int L = 1 << D;
  typedef typename RankT<W>::T RT;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;

  const int S = a.S;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const SmemLayout lay = smem_layout(MODE, W, D, S, a.TG, a.Fmax, a.Kmax, nw);
  unsigned char* tileb = smem + lay.tile;
  uint2* nodes_s = reinterpret_cast<uint2*>(smem + lay.nodes);
  uint32_t* aux32 = reinterpret_cast<uint32_t*>(smem + lay.aux);
  uint8_t* lab_s = smem + lay.aux;
  uint32_t* cnt_s = reinterpret_cast<uint32_t*>(smem + lay.cnt);

  const int64_t T = a.total_tiles;
  const int64_t t0 = (int64_t)blockIdx.x * T / gridDim.x;
  const int64_t t1 = (int64_t)(blockIdx.x + 1) * T / gridDim.x;
  if (t0 >= t1) return;

  if (threadIdx.x == 0) {
    mbar_init(&mbar, 1);
    fence_mbar_init();
  }
  if (MODE == 1) {
    const int LK = L * a.Kmax;
    for (int e = threadIdx.x; e < nw * LK; e += blockDim.x) cnt_s[e] = 0;
  }
  __syncthreads();

  uint32_t phase = 0;
  int cur_job = -1;
  JobView jv;
  int K = 0, LK = 0, Q = 0;
  // ballot mode per-lane constants: for bin b = lane + 32q, the mask that
  // selects "went right" (bit set) or "went left" at level d
  uint32_t cst[kQMax][D];

  auto flush = [&](const JobView& v) {
    if (MODE == 0) {
      uint32_t* dst = v.p->counts + (int64_t)v.tree0 * LK;
      for (int e = threadIdx.x; e < v.ntrees * LK; e += blockDim.x) {
        uint32_t c = cnt_s[e];
        if (c) atomicAdd(dst + e, c);
      }
    }
  };

  for (int64_t gt = t0; gt < t1; ++gt) {
    JobView nv;
    lookup_job(a, gt, &nv);
    if (nv.job != cur_job) {
      if (cur_job >= 0) flush(jv);
      __syncthreads();
      jv = nv;
      cur_job = nv.job;
      K = jv.p->K;
      LK = L * K;
      Q = (LK + 31) >> 5;
      // nodes of the job's trees -> {byte offset of the feature row in the tile, theta}
      const uint32_t* gn = jv.p->nodes + (int64_t)jv.tree0 * B;
      for (int e = threadIdx.x; e < jv.ntrees * B; e += blockDim.x) {
        uint32_t pk = gn[e];
        uint32_t f = pk >> 24;
        nodes_s[e] = make_uint2(f * (uint32_t)S * (uint32_t)W, pk & kThetaMask);
      }
      if (MODE == 0) {
        for (int e = threadIdx.x; e < jv.ntrees * LK; e += blockDim.x) cnt_s[e] = 0;
#pragma unroll
        for (int q = 0; q < kQMax; ++q) {
          int b = lane + 32 * q;
          int leaf = (b < LK) ? b / K : 0;
#pragma unroll
          for (int d = 0; d < D; ++d)
            cst[q][d] = ((leaf >> (D - 1 - d)) & 1) ? 0u : 0xFFFFFFFFu;
        }
      }
    }
    jv.tile = nv.tile;  // the tile changes every iteration, the job only sometimes
    const EvalProb& P = *jv.p;
    const int64_t s0 = P.start + jv.tile * (int64_t)S;
    const int64_t rem = P.start + P.count - s0;
    const int ns = rem < S ? (int)rem : S;
    const int nch = (ns + 31) >> 5;
    const int nchU = (nch + kU - 1) / kU * kU;

    // ---- stage rank rows -------------------------------------------------
    if (P.tma) {
      if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        const uint32_t bytes = ((uint32_t)ns * W + 15u) & ~15u;
        mbar_arrive_expect_tx(&mbar, bytes * (uint32_t)P.F);
        const unsigned char* src = static_cast<const unsigned char*>(P.ranks);
        for (int f = 0; f < P.F; ++f)
          bulk_g2s(tileb + (size_t)f * S * W, src + ((int64_t)f * P.ld + s0) * W, bytes, &mbar);
      }
    } else {
      const RT* src = static_cast<const RT*>(P.ranks);
      RT* dst = reinterpret_cast<RT*>(tileb);
      for (int e = threadIdx.x; e < P.F * S; e += blockDim.x) {
        int f = e / S, j = e - f * S;
        if (j < ns) {
          int64_t col = P.idx ? (int64_t)P.idx[s0 + j] : s0 + j;
          if ((uint64_t)col >= (uint64_t)P.ncols) {
            atomicOr(a.status, ST_BAD_INDEX);
            col = 0;
          }
          dst[e] = src[(int64_t)f * P.ld + col];
        }
      }
    }
    // ---- labels: class masks (ballot) or per-sample labels (atomic) -------
    if (MODE == 0) {
      for (int c = warp; c < nchU; c += nw) {
        int j = c * 32 + lane;
        uint32_t y = 0xFFu;
        if (j < ns) {
          int64_t col = P.idx ? (int64_t)P.idx[s0 + j] : s0 + j;
          if ((uint64_t)col >= (uint64_t)P.ncols) col = 0;
          y = P.labels[col];
        }
        uint32_t mine[kQMax] = {0u, 0u, 0u, 0u};
        for (int k = 0; k < K; ++k) {
          uint32_t m = __ballot_sync(0xFFFFFFFFu, y == (uint32_t)k);
#pragma unroll
          for (int q = 0; q < kQMax; ++q) {
            int b = lane + 32 * q;
            if (b < LK && (b % K) == k) mine[q] = m;
          }
        }
#pragma unroll
        for (int q = 0; q < kQMax; ++q)
          if (q < Q) aux32[(c * Q + q) * 32 + lane] = mine[q];
      }
    } else {
      for (int j = threadIdx.x; j < nchU * 32; j += blockDim.x) {
        uint8_t y = 0xFF;
        if (j < ns) {
          int64_t col = P.idx ? (int64_t)P.idx[s0 + j] : s0 + j;
          if ((uint64_t)col >= (uint64_t)P.ncols) col = 0;
          y = P.labels[col];
        }
        lab_s[j] = y;
      }
    }
    int ok = 1;
    if (P.tma) ok = mbar_wait_bounded(&mbar, phase, a.status) ? 1 : 0;
    phase ^= (P.tma ? 1u : 0u);
    if (__syncthreads_or(!ok)) {
      // timed out (status recorded): give the copies in flight one more bounded
      // wait before the CTA leaves
      if (threadIdx.x == 0) mbar_wait_bounded(&mbar, phase ^ 1u, a.status);
      __syncthreads();
      return;
    }

    // ---- route + count ---------------------------------------------------
    const unsigned char* tb = tileb;
    for (int i = warp; i < jv.ntrees; i += nw) {
      const uint2* tn = nodes_s + i * B - 1;  // tn[t] = node t (1-based)
      const uint2 n1 = tn[1];
      uint2 n2 = n1, n3 = n1;
      if (D >= 2) {
        n2 = tn[2];
        n3 = tn[3];
      }
      if (MODE == 0) {
        uint32_t cnt[kQMax] = {0u, 0u, 0u, 0u};
        for (int c = 0; c < nchU; c += kU) {
          uint32_t bal[kU][D];
          uint32_t t[kU];
          const uint32_t jb0 = (uint32_t)(c * 32 + lane) * W;
#pragma unroll
          for (int u = 0; u < kU; ++u) {
            const uint32_t jb = jb0 + u * 32 * W;
            uint32_t rv = *reinterpret_cast<const RT*>(tb + n1.x + jb);
            uint32_t g = rv >= n1.y;
            bal[u][0] = __ballot_sync(0xFFFFFFFFu, g);
            t[u] = 2 + g;
            if (D >= 2) {
              uint32_t ro = g ? n3.x : n2.x;
              uint32_t th = g ? n3.y : n2.y;
              uint32_t rv1 = *reinterpret_cast<const RT*>(tb + ro + jb);
              uint32_t g1 = rv1 >= th;
              bal[u][1 < D ? 1 : 0] = __ballot_sync(0xFFFFFFFFu, g1);
              t[u] = 2 * t[u] + g1;
            }
          }
#pragma unroll
          for (int d = 2; d < D; ++d) {
#pragma unroll
            for (int u = 0; u < kU; ++u) {
              const uint32_t jb = jb0 + u * 32 * W;
              const uint2 nd = tn[t[u]];
              uint32_t rv = *reinterpret_cast<const RT*>(tb + nd.x + jb);
              uint32_t g = rv >= nd.y;
              bal[u][d] = __ballot_sync(0xFFFFFFFFu, g);
              t[u] = 2 * t[u] + g;
            }
          }
#pragma unroll
          for (int u = 0; u < kU; ++u) {
#pragma unroll
            for (int q = 0; q < kQMax; ++q) {
              if (q < Q) {
                uint32_t m = aux32[((c + u) * Q + q) * 32 + lane];
#pragma unroll
                for (int d = 0; d < D; ++d) m &= bal[u][d] ^ cst[q][d];
                cnt[q] += __popc(m);
              }
            }
          }
        }
#pragma unroll
        for (int q = 0; q < kQMax; ++q) {
          int b = lane + 32 * q;
          if (q < Q && b < LK) cnt_s[i * LK + b] += cnt[q];
        }
      } else {
        uint32_t* hw = cnt_s + warp * (L * a.Kmax);
        for (int c = 0; c < nch; ++c) {
          const uint32_t j = (uint32_t)(c * 32 + lane);
          const uint32_t jb = j * W;
          uint32_t t = 1;
#pragma unroll
          for (int d = 0; d < D; ++d) {
            const uint2 nd = tn[t];
            uint32_t rv = *reinterpret_cast<const RT*>(tb + nd.x + jb);
            t = 2 * t + (rv >= nd.y ? 1u : 0u);
          }
          uint32_t y = lab_s[j];
          if (y < (uint32_t)K) atomicAdd(hw + (t - L) * K + y, 1u);
        }
        __syncwarp();
        uint32_t* dst = P.counts + (int64_t)(jv.tree0 + i) * LK;
        for (int b = lane; b < LK; b += 32) {
          uint32_t v = hw[b];
          if (v) {
            atomicAdd(dst + b, v);
            hw[b] = 0;
          }
        }
        __syncwarp();
      }
    }
    __syncthreads();
  }
  if (cur_job >= 0) flush(jv);
}

template <int W, int D, int MODE>
int launch_t(deoct_ctx* ctx, const EvalArgs& args, const EvalConfig& cfg, size_t smem,
             cudaStream_t s) {
  auto kern = eval_kernel<W, D, MODE>;
  if (smem > 48 * 1024) {
    DEOCT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
  }
  // all of the unified L1/shared array as shared memory, so that the occupancy
  // computed below is the residency the launch gets
  DEOCT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
  int grid = cfg.grid;
  if (grid <= 0) {
    int occ = 0;
    DEOCT_CUDA_TRY(
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, cfg.warps * 32, smem));
    if (occ < 1) return set_error(DEOCT_ERR_INVALID, "evaluator tile does not fit: %zu B smem", smem);
    grid = occ * ctx->num_sms;
  }
  if ((int64_t)grid > args.total_tiles) grid = (int)args.total_tiles;
  if (grid < 1) return DEOCT_OK;
  kern<<<grid, cfg.warps * 32, smem, s>>>(args);
  count_launch(ctx);
  return check_launch("eval_kernel");
}

template <int W, int D>
int dispatch_mode(deoct_ctx* ctx, int mode, const EvalArgs& args, const EvalConfig& cfg,
                  size_t smem, cudaStream_t s) {
  if (mode == 0) return launch_t<W, D, 0>(ctx, args, cfg, smem, s);
  return launch_t<W, D, 1>(ctx, args, cfg, smem, s);
}

template <int W>
int dispatch_depth(deoct_ctx* ctx, int D, int mode, const EvalArgs& args, const EvalConfig& cfg,
                   size_t smem, cudaStream_t s) {
  switch (D) {
    case 1: return dispatch_mode<W, 1>(ctx, mode, args, cfg, smem, s);
    case 2: return dispatch_mode<W, 2>(ctx, mode, args, cfg, smem, s);
    case 3: return dispatch_mode<W, 3>(ctx, mode, args, cfg, smem, s);
    case 4: return dispatch_mode<W, 4>(ctx, mode, args, cfg, smem, s);
    case 5: return dispatch_mode<W, 5>(ctx, mode, args, cfg, smem, s);
    case 6: return launch_t<W, 6, 1>(ctx, args, cfg, smem, s);
    case 7: return launch_t<W, 7, 1>(ctx, args, cfg, smem, s);
    case 8: return launch_t<W, 8, 1>(ctx, args, cfg, smem, s);
    case 9: return launch_t<W, 9, 1>(ctx, args, cfg, smem, s);
    case 10: return launch_t<W, 10, 1>(ctx, args, cfg, smem, s);
  }
  return set_error(DEOCT_ERR_INVALID, "depth %d outside 1..%d", D, kMaxDepth);
}

__global__ void errors_kernel(const uint32_t* __restrict__ counts, int P, int L, int K,
                              int64_t n_valid, uint32_t* __restrict__ errors) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= P) return;
  const uint32_t* c = counts + (int64_t)r * L * K;
  int64_t correct = 0;
  for (int l = 0; l < L; ++l) {
    uint32_t mx = 0;
    for (int k = 0; k < K; ++k) mx = max(mx, c[l * K + k]);
    correct += mx;
  }
  errors[r] = (uint32_t)(n_valid - correct);
}

__global__ void pack_nodes_kernel(const uint16_t* __restrict__ a, const uint32_t* __restrict__ th,
                                  int64_t count, int F, uint32_t* __restrict__ nodes,
                                  int* status) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  int av = a[e];
  uint32_t tv = th[e];
  if (av > F || (av > 0 && tv > kThetaMask)) {
    atomicOr(status, ST_BAD_NODE);
    av = 0;
  }
  nodes[e] = pack_node(av, tv);
}

}  // namespace

void eval_build_jobs(const std::vector<int64_t>& counts, const std::vector<int>& pops, int S,
                     int TG, std::vector<EvalJob>* jobs, int64_t* total_tiles) {
  jobs->clear();
  int64_t tb = 0;
  for (size_t p = 0; p < counts.size(); ++p) {
    if (counts[p] <= 0) continue;
    int32_t ntiles = (int32_t)((counts[p] + S - 1) / S);
    for (int t0 = 0; t0 < pops[p]; t0 += TG) {
      EvalJob j;
      j.tile_begin = tb;
      j.prob = (int32_t)p;
      j.tree0 = t0;
      j.ntrees = std::min(TG, pops[p] - t0);
      j.ntiles = ntiles;
      jobs->push_back(j);
      tb += ntiles;
    }
  }
  *total_tiles = tb;
}

static size_t eval_smem(int mode, int W, int D, int S, int TG, int F, int K, int warps) {
  return smem_layout(mode, W, D, S, TG, F, K, warps).total;
}

static int eval_mode(int D, int K) { return ((1 << D) * K <= 32 * kQMax && D <= 5) ? 0 : 1; }

EvalConfig eval_choose_config(deoct_ctx* ctx, int W, int D, int F, int K, int P, int64_t n,
                              int nprob) {
  EvalConfig c;
  const int mode = eval_mode(D, K);
  c.S = 2048;
  c.TG = std::min(P, 256);
  c.warps = 8;
  const int limit = std::min(ctx->max_smem_optin, 227 * 1024);
  // fit in shared memory (keep room for two CTAs per SM when possible)
  while (eval_smem(mode, W, D, c.S, c.TG, F, K, c.warps) > (size_t)limit / 2 &&
         (c.S > 512 || c.TG > 32)) {
    if (c.S > 512) c.S /= 2; else c.TG /= 2;
  }
  while (eval_smem(mode, W, D, c.S, c.TG, F, K, c.warps) > (size_t)limit && (c.S > 128 || c.TG > 1)) {
    if (c.S > 128) c.S /= 2; else c.TG = std::max(1, c.TG / 2);
  }
  // enough independent tiles to fill the GPU for small problems
  auto work = [&](int S, int TG) {
    int64_t per = (n / std::max(1, nprob) + S - 1) / S;
    return per * nprob * ((P + TG - 1) / TG);
  };
  while (work(c.S, c.TG) < 2 * (int64_t)ctx->num_sms && (c.S > 256 || c.TG > 16)) {
    if (c.S > 256) c.S /= 2; else c.TG = std::max(16, c.TG / 2);
  }
  if (ctx->force_S) c.S = ctx->force_S;
  if (ctx->force_TG) c.TG = std::min(ctx->force_TG, std::max(1, P));
  if (ctx->force_warps) c.warps = ctx->force_warps;
  if (ctx->force_grid) c.grid = ctx->force_grid;
  return c;
}

int eval_launch(deoct_ctx* ctx, int W, int D, const EvalPlan& plan, const EvalConfig& cfg,
                cudaStream_t stream) {
  if (plan.total_tiles <= 0) return DEOCT_OK;
  if (D < 1 || D > kMaxDepth) return set_error(DEOCT_ERR_INVALID, "depth %d", D);
  const int mode = eval_mode(D, plan.Kmax);
  EvalArgs a;
  a.single = plan.single;
  a.probs = plan.d_probs;
  a.jobs = plan.d_jobs;
  a.njobs = plan.njobs;
  a.single_ntiles = 0;
  if (plan.d_probs == nullptr)
    a.single_ntiles = (int)((plan.single.count + cfg.S - 1) / cfg.S);
  a.total_tiles = plan.total_tiles;
  a.S = cfg.S;
  a.TG = cfg.TG;
  a.Fmax = plan.Fmax;
  a.Kmax = plan.Kmax;
  a.status = ctx->d_status;
  const size_t smem = eval_smem(mode, W, D, cfg.S, cfg.TG, plan.Fmax, plan.Kmax, cfg.warps);
  if (smem > (size_t)ctx->max_smem_optin)
    return set_error(DEOCT_ERR_INVALID, "evaluator needs %zu B shared memory (F=%d)", smem,
                     plan.Fmax);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ctx->timing) {
    DEOCT_CUDA_TRY(cudaEventCreate(&e0));
    DEOCT_CUDA_TRY(cudaEventCreate(&e1));
    DEOCT_CUDA_TRY(cudaEventRecord(e0, stream));
  }
  int rc = (W == 2) ? dispatch_depth<2>(ctx, D, mode, a, cfg, smem, stream)
                    : dispatch_depth<4>(ctx, D, mode, a, cfg, smem, stream);
  if (rc != DEOCT_OK) return rc;
  ctx->eval_launches += 1;
  if (ctx->timing) {
    DEOCT_CUDA_TRY(cudaEventRecord(e1, stream));
    ctx->ev_pairs.push_back(e0);
    ctx->ev_pairs.push_back(e1);
  }
  return DEOCT_OK;
}

int launch_errors(deoct_ctx* ctx, const uint32_t* counts, int P, int L, int K, int64_t n_valid,
                  uint32_t* errors, cudaStream_t stream) {
  errors_kernel<<<(P + 127) / 128, 128, 0, stream>>>(counts, P, L, K, n_valid, errors);
  count_launch(ctx);
  return check_launch("errors_kernel");
}

int launch_pack_nodes(deoct_ctx* ctx, const uint16_t* a, const uint32_t* theta, int64_t count,
                      int F, uint32_t* nodes, cudaStream_t stream) {
  if (count <= 0) return DEOCT_OK;
  pack_nodes_kernel<<<(unsigned)((count + 255) / 256), 256, 0, stream>>>(a, theta, count, F, nodes,
                                                                         ctx->d_status);
  count_launch(ctx);
  return check_launch("pack_nodes_kernel");
}

}  // namespace deoct
