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

constexpr int kQMax = 4;  // ballot mode: up to 4 bins per lane (2^D * K <= 128)

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

// Shared-memory layout, shared by host sizing and the kernel:
//   tile    [F][S] ranks in the compute layout (see tile_offset)
//   stage   [F][S] TMA landing zone (uint16 only; the uint32 path lands in `tile`)
//   nodes   [TG][B] {shared address of the feature row, theta}
//   aux     ballot mode: class masks [S/32][Q][32]; atomic mode: labels [S]
//   cnt     job counts [TG][2^D K] (both modes)
struct SmemLayout {
  size_t tile, stage, nodes, aux, cnt, total;
};
__host__ __device__ __forceinline__ SmemLayout smem_layout(int mode, int W, int D, int S, int TG,
                                                           int Fmax, int Kmax, int warps) {
  const int B = (1 << D) - 1, L = 1 << D;
  const int LK = L * Kmax;
  const size_t rows = align128((size_t)Fmax * S * W);
  SmemLayout s;
  s.tile = 0;
  s.stage = rows;
  s.nodes = s.stage + (W == 2 ? rows : 0);
  s.aux = s.nodes + align128((size_t)TG * B * 8);
  if (mode == 0) {
    const int Q = (LK + 31) / 32;
    s.cnt = s.aux + align128((size_t)S * Q * 4);
    s.total = s.cnt + align128((size_t)TG * LK * 4);
  } else {
    s.cnt = s.aux + align128((size_t)S);
    s.total = s.cnt + align128((size_t)TG * LK * 4);
  }
  return s;
}

// Byte offset of sample j inside a feature row of the compute tile.  uint32
// ranks: natural order (lane l of a warp reads bank l).  uint16 ranks: the two
// chunks of 32 samples of a chunk pair share 32-bit words -- word l of pair p
// holds sample 64p+l (low half) and 64p+32+l (high half) -- so a warp reading
// one chunk touches 32 distinct banks whatever rows its lanes are on.
template <int W>
__device__ __forceinline__ uint32_t tile_offset(uint32_t j) {
  if (W == 4) return j * 4u;
  return (j >> 6) * 128u + (j & 31u) * 4u + ((j >> 5) & 1u) * 2u;
}
// offset between the two chunks of a pair for the same lane
template <int W>
struct PairGeom {
  static constexpr uint32_t kSecond = (W == 2) ? 2u : 128u;
  static constexpr uint32_t kPairStride = 64u * W;
};

template <int W>
__device__ __forceinline__ uint32_t lds_rank(uint32_t addr) {
  uint32_t v;
  if (W == 2) {
    unsigned short h;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(h) : "r"(addr));
    v = h;
  } else {
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
  }
  return v;
}
__device__ __forceinline__ uint2 lds_node(uint32_t addr) {
  uint2 v;
  asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(addr));
  return v;
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}

// Route 64 samples (the two chunks of pair p) of one tree and add the bin
// counts owned by this lane.  Ballot of level d = "went right" at depth d for
// the 32 samples of a chunk; bin b = leaf*K + k is owned by lane b % 32.
template <int W, int D, int Q>
__device__ __forceinline__ void route_pair(uint32_t jb, uint32_t row0, uint32_t th0, uint32_t row2,
                                           uint32_t th2, uint32_t row3, uint32_t th3, uint32_t tnb32,
                                           uint32_t tnb48, uint32_t ntnb, uint32_t ymA, uint32_t ymB,
                                           const uint32_t (&cst)[Q][D], uint32_t (&cnt)[Q]) {
  constexpr uint32_t SEC = PairGeom<W>::kSecond;
  uint32_t BA[D], BB[D];
  // level 0: the root is the same node for every lane
  const uint32_t ra0 = lds_rank<W>(row0 + jb);
  const uint32_t rb0 = lds_rank<W>(row0 + jb + SEC);
  const bool pa0 = ra0 >= th0, pb0 = rb0 >= th0;
  BA[0] = __ballot_sync(0xFFFFFFFFu, pa0);
  BB[0] = __ballot_sync(0xFFFFFFFFu, pb0);
  if (D >= 2) {
    // level 1: two candidate nodes held in registers
    const uint32_t rowa = pa0 ? row3 : row2, tha = pa0 ? th3 : th2;
    const uint32_t rowb = pb0 ? row3 : row2, thb = pb0 ? th3 : th2;
    const uint32_t ra1 = lds_rank<W>(rowa + jb);
    const uint32_t rb1 = lds_rank<W>(rowb + jb + SEC);
    const bool pa1 = ra1 >= tha, pb1 = rb1 >= thb;
    BA[1 < D ? 1 : 0] = __ballot_sync(0xFFFFFFFFu, pa1);
    BB[1 < D ? 1 : 0] = __ballot_sync(0xFFFFFFFFu, pb1);
    // shared address of node t = 4 + 2 p0 + p1
    uint32_t aa = (pa0 ? tnb48 : tnb32) + (pa1 ? 8u : 0u);
    uint32_t ab = (pb0 ? tnb48 : tnb32) + (pb1 ? 8u : 0u);
#pragma unroll
    for (int d = 2; d < D; ++d) {
      const uint2 na = lds_node(aa);
      const uint2 nb = lds_node(ab);
      const uint32_t ra = lds_rank<W>(na.x + jb);
      const uint32_t rb = lds_rank<W>(nb.x + jb + SEC);
      const bool pa = ra >= na.y, pb = rb >= nb.y;
      BA[d] = __ballot_sync(0xFFFFFFFFu, pa);
      BB[d] = __ballot_sync(0xFFFFFFFFu, pb);
      if (d + 1 < D) {  // node 2t + p: address 2 addr(t) - base + 8 p
        aa = 2u * aa + ntnb + (pa ? 8u : 0u);
        ab = 2u * ab + ntnb + (pb ? 8u : 0u);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    uint32_t ma = lds_u32(ymA + q * 128u);
    uint32_t mb = lds_u32(ymB + q * 128u);
#pragma unroll
    for (int d = 0; d < D; ++d) {
      ma &= BA[d] ^ cst[q][d];
      mb &= BB[d] ^ cst[q][d];
    }
    cnt[q] += __popc(ma) + __popc(mb);
  }
}

// Stage the rank rows of one tile.  TMA path: one elected thread issues a 1-D
// bulk copy per feature row into `dst` and arms the mbarrier.
__device__ __forceinline__ void issue_tile_tma(const EvalProb& P, int64_t s0, int ns, int S, int W,
                                               unsigned char* dst, uint64_t* bar) {
  fence_proxy_async_smem();
  const uint32_t bytes = ((uint32_t)ns * W + 15u) & ~15u;
  mbar_arrive_expect_tx(bar, bytes * (uint32_t)P.F);
  const unsigned char* src = static_cast<const unsigned char*>(P.ranks);
  for (int f = 0; f < P.F; ++f)
    bulk_g2s(dst + (size_t)f * S * W, src + ((int64_t)f * P.ld + s0) * W, bytes, bar);
}

template <int W, int D, int MODE, int Q>
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
  unsigned char* stageb = (W == 2) ? smem + lay.stage : tileb;
  uint2* nodes_s = reinterpret_cast<uint2*>(smem + lay.nodes);
  uint32_t* aux32 = reinterpret_cast<uint32_t*>(smem + lay.aux);
  uint8_t* lab_s = smem + lay.aux;
  uint32_t* cnt_s = reinterpret_cast<uint32_t*>(smem + lay.cnt);
  const uint32_t tile_sa = smem_u32(tileb);
  const uint32_t nodes_sa = smem_u32(nodes_s);
  const uint32_t aux_sa = smem_u32(aux32);

  const int64_t T = a.total_tiles;
  const int64_t t0 = (int64_t)blockIdx.x * T / gridDim.x;
  const int64_t t1 = (int64_t)(blockIdx.x + 1) * T / gridDim.x;
  if (t0 >= t1) return;

  if (threadIdx.x == 0) {
    mbar_init(&mbar, 1);
    fence_mbar_init();
  }
  __syncthreads();

  uint32_t phase = 0;
  int cur_job = -1;
  JobView jv;
  int K = 0, LK = 0;
  uint32_t cst[Q][D];  // ballot mode: per owned bin, "right" (0) or "left" (~0) at level d
  bool staged = false; // the current tile's rows are already in flight (prefetched)

  auto flush = [&](const JobView& v) {
    uint32_t* dst = v.p->counts + (int64_t)v.tree0 * LK;
    for (int e = threadIdx.x; e < v.ntrees * LK; e += blockDim.x) {
      uint32_t c = cnt_s[e];
      if (c) atomicAdd(dst + e, c);
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
      // nodes -> {shared address of the feature row in the tile, theta}
      const uint32_t* gn = jv.p->nodes + (int64_t)jv.tree0 * B;
      for (int e = threadIdx.x; e < jv.ntrees * B; e += blockDim.x) {
        uint32_t pk = gn[e];
        uint32_t f = pk >> 24;
        nodes_s[e] = make_uint2(tile_sa + f * (uint32_t)S * (uint32_t)W, pk & kThetaMask);
      }
      for (int e = threadIdx.x; e < jv.ntrees * LK; e += blockDim.x) cnt_s[e] = 0;
      if (MODE == 0) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
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
    const int npair = (nch + 1) >> 1;

    // ---- stage rank rows -------------------------------------------------
    if (P.tma) {
      if (!staged && threadIdx.x == 0) issue_tile_tma(P, s0, ns, S, W, stageb, &mbar);
    } else {
      const RT* src = static_cast<const RT*>(P.ranks);
      for (int e = threadIdx.x; e < P.F * S; e += blockDim.x) {
        int f = e / S, j = e - f * S;
        if (j < ns) {
          int64_t col = P.idx ? (int64_t)P.idx[s0 + j] : s0 + j;
          if ((uint64_t)col >= (uint64_t)P.ncols) {
            atomicOr(a.status, ST_BAD_INDEX);
            col = 0;
          }
          *reinterpret_cast<RT*>(tileb + (size_t)f * S * W + tile_offset<W>((uint32_t)j)) =
              src[(int64_t)f * P.ld + col];
        }
      }
    }
    staged = false;
    // ---- labels: class masks (ballot) or per-sample labels (atomic) -------
    if (MODE == 0) {
      for (int c = warp; c < 2 * npair; c += nw) {
        int j = c * 32 + lane;
        uint32_t y = 0xFFu;
        if (j < ns) {
          int64_t col = P.idx ? (int64_t)P.idx[s0 + j] : s0 + j;
          if ((uint64_t)col >= (uint64_t)P.ncols) col = 0;
          y = P.labels[col];
        }
        uint32_t mine[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) mine[q] = 0u;
        for (int k = 0; k < K; ++k) {
          uint32_t m = __ballot_sync(0xFFFFFFFFu, y == (uint32_t)k);
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            int b = lane + 32 * q;
            if (b < LK && (b % K) == k) mine[q] = m;
          }
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) aux32[(c * Q + q) * 32 + lane] = mine[q];
      }
    } else {
      for (int j = threadIdx.x; j < 2 * npair * 32; j += blockDim.x) {
        uint8_t y = 0xFF;
        if (j < ns) {
          int64_t col = P.idx ? (int64_t)P.idx[s0 + j] : s0 + j;
          if ((uint64_t)col >= (uint64_t)P.ncols) col = 0;
          y = P.labels[col];
        }
        lab_s[j] = y;
      }
    }
    if (P.tma) {
      int ok = mbar_wait_bounded(&mbar, phase, a.status) ? 1 : 0;
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {
        // timed out (status recorded): give the copies in flight one more
        // bounded wait before the CTA leaves
        if (threadIdx.x == 0) mbar_wait_bounded(&mbar, phase ^ 1u, a.status);
        __syncthreads();
        return;
      }
      if (W == 2) {
        // stage (natural order) -> tile (chunk-pair interleaved)
        const uint16_t* st = reinterpret_cast<const uint16_t*>(stageb);
        uint32_t* tw = reinterpret_cast<uint32_t*>(tileb);
        const int words = npair * 32;  // per row
        for (int e = threadIdx.x; e < P.F * words; e += blockDim.x) {
          int f = e / words, w = e - f * words;
          int pp = w >> 5, l = w & 31;
          const uint16_t* srow = st + (size_t)f * S + pp * 64 + l;
          tw[(size_t)f * (S / 2) + w] = (uint32_t)srow[0] | ((uint32_t)srow[32] << 16);
        }
        __syncthreads();
        // prefetch the next tile of this CTA into the free landing zone
        if (gt + 1 < t1) {
          JobView xv;
          lookup_job(a, gt + 1, &xv);
          const EvalProb& X = *xv.p;
          if (X.tma) {
            if (threadIdx.x == 0) {
              const int64_t xs0 = X.start + xv.tile * (int64_t)S;
              const int64_t xrem = X.start + X.count - xs0;
              issue_tile_tma(X, xs0, xrem < S ? (int)xrem : S, S, W, stageb, &mbar);
            }
            staged = true;
          }
        }
      }
    } else {
      __syncthreads();
    }

    // ---- route + count ---------------------------------------------------
    if (MODE == 0) {
      // ballot mode: a warp owns a tree and walks all chunk pairs of the tile
      for (int i = warp; i < jv.ntrees; i += nw) {
        const uint32_t tnb = nodes_sa + (uint32_t)(i * B - 1) * 8u;  // node t at tnb + 8t
        const uint2 n1 = nodes_s[i * B];
        uint2 n2 = n1, n3 = n1;
        if (D >= 2) {
          n2 = nodes_s[i * B + 1];
          n3 = nodes_s[i * B + 2];
        }
        uint32_t cnt[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) cnt[q] = 0u;
        const uint32_t ntnb = 0u - tnb;
        for (int pp = 0; pp < npair; ++pp) {
          const uint32_t jb = (uint32_t)pp * PairGeom<W>::kPairStride + (uint32_t)lane * 4u;
          const uint32_t ymA = aux_sa + ((uint32_t)(2 * pp) * Q * 32u + lane) * 4u;
          const uint32_t ymB = ymA + Q * 128u;
          route_pair<W, D, Q>(jb, n1.x, n1.y, n2.x, n2.y, n3.x, n3.y, tnb + 32u, tnb + 48u, ntnb,
                              ymA, ymB, cst, cnt);
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          int b = lane + 32 * q;
          if (b < LK) cnt_s[i * LK + b] += cnt[q];
        }
      }
    } else {
      // shared-atomic mode (many bins): all warps work on one tree at a time,
      // splitting its chunks, and add into the job's shared counts
      for (int i = 0; i < jv.ntrees; ++i) {
        const uint32_t tnb = nodes_sa + (uint32_t)(i * B - 1) * 8u;
        uint32_t* ci = cnt_s + i * LK;
        for (int c = warp; c < nch; c += nw) {
          const uint32_t j = (uint32_t)(c * 32 + lane);
          const uint32_t jo = tile_offset<W>(j);
          uint32_t t = 1;
#pragma unroll
          for (int d = 0; d < D; ++d) {
            const uint2 nd = lds_node(tnb + 8u * t);
            uint32_t rv = lds_rank<W>(nd.x + jo);
            t = 2 * t + (rv >= nd.y ? 1u : 0u);
          }
          const uint32_t y = lab_s[j];
          if (y < (uint32_t)K) atomicAdd(ci + (t - L) * K + y, 1u);
        }
      }
    }
    __syncthreads();
  }
  if (staged && threadIdx.x == 0) mbar_wait_bounded(&mbar, phase, a.status);  // never left in flight
  if (cur_job >= 0) flush(jv);
}

template <int W, int D, int MODE, int Q>
int launch_t(deoct_ctx* ctx, const EvalArgs& args, const EvalConfig& cfg, size_t smem,
             cudaStream_t s) {
  auto kern = eval_kernel<W, D, MODE, Q>;
  DEOCT_TRY(set_max_dynamic_smem(ctx, kern));
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
int dispatch_mode(deoct_ctx* ctx, int mode, int Q, const EvalArgs& args, const EvalConfig& cfg,
                  size_t smem, cudaStream_t s) {
  if (mode == 1) return launch_t<W, D, 1, 1>(ctx, args, cfg, smem, s);
  switch (Q) {
    case 1: return launch_t<W, D, 0, 1>(ctx, args, cfg, smem, s);
    case 2: return launch_t<W, D, 0, 2>(ctx, args, cfg, smem, s);
    case 3: return launch_t<W, D, 0, 3>(ctx, args, cfg, smem, s);
    default: return launch_t<W, D, 0, 4>(ctx, args, cfg, smem, s);
  }
}

template <int W>
int dispatch_depth(deoct_ctx* ctx, int D, int mode, int Q, const EvalArgs& args,
                   const EvalConfig& cfg, size_t smem, cudaStream_t s) {
  switch (D) {
    case 1: return dispatch_mode<W, 1>(ctx, mode, Q, args, cfg, smem, s);
    case 2: return dispatch_mode<W, 2>(ctx, mode, Q, args, cfg, smem, s);
    case 3: return dispatch_mode<W, 3>(ctx, mode, Q, args, cfg, smem, s);
    case 4: return dispatch_mode<W, 4>(ctx, mode, Q, args, cfg, smem, s);
    case 5: return dispatch_mode<W, 5>(ctx, mode, Q, args, cfg, smem, s);
    case 6: return launch_t<W, 6, 1, 1>(ctx, args, cfg, smem, s);
    case 7: return launch_t<W, 7, 1, 1>(ctx, args, cfg, smem, s);
    case 8: return launch_t<W, 8, 1, 1>(ctx, args, cfg, smem, s);
    case 9: return launch_t<W, 9, 1, 1>(ctx, args, cfg, smem, s);
    case 10: return launch_t<W, 10, 1, 1>(ctx, args, cfg, smem, s);
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
int eval_counting_mode(int D, int K) { return eval_mode(D, K); }

EvalConfig eval_choose_config(deoct_ctx* ctx, int W, int D, int F, int K, int P, int64_t n,
                              int nprob) {
  EvalConfig c;
  const int mode = eval_mode(D, K);
  const int limit = std::min(ctx->max_smem_optin, 227 * 1024) - 1024;  // room for static smem
  const size_t two_per_sm = (size_t)(ctx->smem_per_sm - 2 * 1024) / 2;  // 1 KB reserved per CTA
  auto work = [&](int S, int TG) {
    int64_t per = (n / std::max(1, nprob) + S - 1) / S;
    return per * nprob * ((P + TG - 1) / TG);
  };
  if (mode == 0) {
    // measured on GB300 (n = 1e7, F = 10, depth 4, P = 1024): 16 warps per CTA and
    // two CTAs per SM beat 8 warps by 1.5x; tiles of 1024 samples with 256 trees
    // per job were the fastest shape that leaves room for two CTAs
    c.S = 2048;
    c.TG = std::min(P, 256);
    c.warps = 16;
    while (eval_smem(mode, W, D, c.S, c.TG, F, K, c.warps) > two_per_sm && (c.S > 512 || c.TG > 32)) {
      if (c.S > 512) c.S /= 2; else c.TG /= 2;
    }
    while (eval_smem(mode, W, D, c.S, c.TG, F, K, c.warps) > (size_t)limit && (c.S > 128 || c.TG > 1)) {
      if (c.S > 128) c.S /= 2; else c.TG = std::max(1, c.TG / 2);
    }
    // enough independent tiles to fill the GPU for small problems
    while (work(c.S, c.TG) < 2 * (int64_t)ctx->num_sms && (c.S > 256 || c.TG > 16)) {
      if (c.S > 256) c.S /= 2; else c.TG = std::max(16, c.TG / 2);
    }
    c.warps = std::max(4, std::min(16, c.TG));  // a warp owns a tree
  } else {
    // shared-atomic mode: the 16 warps split the chunks of one tree at a time, so
    // the tile keeps at least 16 chunks and the job's counts ([TG][2^D K]) set TG
    c.S = 1024;
    c.warps = 16;
    c.TG = std::min(P, 256);
    while (eval_smem(mode, W, D, c.S, c.TG, F, K, c.warps) > two_per_sm && c.TG > 1) c.TG /= 2;
    while (eval_smem(mode, W, D, c.S, c.TG, F, K, c.warps) > (size_t)limit && c.S > 128) c.S /= 2;
    while (work(c.S, c.TG) < 2 * (int64_t)ctx->num_sms && c.TG > 1) c.TG /= 2;
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
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  DEOCT_CUDA_TRY(cudaStreamIsCapturing(stream, &cs));
  const bool timed = ctx->timing && cs == cudaStreamCaptureStatusNone;  // not inside graphs
  if (timed) {
    DEOCT_CUDA_TRY(cudaEventCreate(&e0));
    DEOCT_CUDA_TRY(cudaEventCreate(&e1));
    DEOCT_CUDA_TRY(cudaEventRecord(e0, stream));
  }
  const int Q = ((1 << D) * plan.Kmax + 31) / 32;
  int rc = (W == 2) ? dispatch_depth<2>(ctx, D, mode, Q, a, cfg, smem, stream)
                    : dispatch_depth<4>(ctx, D, mode, Q, a, cfg, smem, stream);
  if (rc != DEOCT_OK) return rc;
  ctx->eval_launches += 1;
  if (timed) {
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
