// eval_kernel.cuh -- building blocks of the population evaluator (Algorithm 1,
// Section 3.2), shared by its two kernels:
//  - eval.cu, the re-laid kernel: one landing zone per CTA whose uint16 rows
//    are re-laid into a chunk-pair-interleaved compute tile (no bank conflicts
//    when 16 warps route 16+ trees), and the shared-atomic counting mode;
//  - eval_stream.cu, the streaming kernel: a producer warp keeps a ring of
//    landing zones filled by bulk copies while routing warps work on earlier
//    tiles straight from the landing zone, in natural sample order (groups of
//    fewer than 16 trees, where HBM sets the pace).
//
// Work layout (both): persistent CTAs split a flattened sequence of tiles
// (jobs x tiles; a job is one tree group of one subproblem) into equal
// contiguous ranges; per tile a CTA stages the feature-major rank rows and the
// labels of S samples in shared memory (1-D bulk copies when aligned, plain
// loads for gathered subsets), so each sample is read from HBM once per tree
// group.  Counting (ballot mode, 2^D K <= 128): the routing predicate of level
// d is a warp ballot B_d over 32 samples; lane b owns bin b = leaf K + k and
// adds popc(Y_k & AND_d (B_d or ~B_d by bit d of leaf)), with the class masks
// Y_k computed once per tile.  Job counts accumulate in shared memory and
// reach HBM with one atomic add per (tree, bin) per CTA.
#pragma once

#include <algorithm>
#include <type_traits>

#include "internal.cuh"

namespace deoct {
namespace evk {

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

constexpr int kQMax = 4;       // ballot mode: up to 4 bins per lane (2^D * K <= 128)
constexpr int kMaxStages = 3;  // streaming kernel: landing zones per CTA
// Streaming kernel: groups of fewer trees than this route pair-sliced (every
// warp its own chunk pairs of every tree, no CTA barrier per tile) on tiles of
// 2048 samples; larger groups share the tile's class masks and split trees over
// warps, with two barriers per tile, on tiles of 1024.  Measured on GB300
// (n = 1e7, depth 4): pair slicing 10% faster for one tree, 5% for two, even at
// four and 11% slower at eight; 2048-sample tiles 8% faster for one to three
// trees, 1-9% slower for four to twelve.
constexpr int kPairSliceTrees = 4;

struct EvalArgs {
  // the rank rows of every problem as one 2-D TMA tensor ([F] rows x width
  // columns, boxes of tmap_box columns x F rows), valid when tmap_box > 0
  CUtensorMap tmap;
  int tmap_box;
  EvalProb single;
  const EvalProb* probs;
  const EvalJob* jobs;
  int njobs;
  int single_ntiles;  // tiles per job when `probs` is null
  int64_t total_tiles;
  int S, TG, Fmax, Kmax;
  int lab_stage;         // the layout has label landing zones (else plain label loads)
  int nstage;            // streaming kernel: landing zones in the ring
  int* status;
  uint32_t* ticket;      // single problem finished by its last CTA (see EvalPlan)
  uint32_t* counts_out;
  uint32_t* errors_out;
};

struct JobView {
  const EvalProb* p;
  int32_t tile;    // tile index within the job (< 2^24 / 128)
  int32_t ntiles;  // tiles of the job
  int32_t job, tree0, ntrees;
};

__device__ __forceinline__ void lookup_job(const EvalArgs& a, int64_t gt, JobView* v) {
  if (a.probs == nullptr) {
    int64_t job = gt / a.single_ntiles;
    v->p = &a.single;
    v->job = (int32_t)job;
    v->tile = (int32_t)(gt - job * a.single_ntiles);
    v->ntiles = a.single_ntiles;
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
  v->tile = (int32_t)(gt - j.tile_begin);
  v->ntiles = j.ntiles;
  v->tree0 = j.tree0;
  v->ntrees = j.ntrees;
}

// The job and tile of flattened tile gt + 1, given those of gt: a search only
// at job boundaries.
__device__ __forceinline__ void advance_job(const EvalArgs& a, int64_t gt_next, JobView* v) {
  if (++v->tile >= v->ntiles) lookup_job(a, gt_next, v);
}

__host__ __device__ __forceinline__ size_t align128(size_t x) { return (x + 127) & ~size_t(127); }

// Bin slots per lane in ballot mode, ceil(2^D K / 32), three rounded up to four
// from depth 2 on: four slots take the class-major map (one class and the lower
// levels shared by a lane's bins), three would keep one class per bin.
__host__ __device__ __forceinline__ int bins_per_lane(int D, int LK) {
  const int q = (LK + 31) / 32;
  return (q == 3 && D >= 2) ? 4 : q;
}

// Shared-memory layout of the re-laid kernel (host sizing and kernel agree):
//   tile    [F][S] ranks in the compute layout (see tile_offset)
//   stage   [F][S] TMA landing zone (uint16 only; the uint32 path lands in `tile`)
//   nodes   [TG][B] {shared address of the feature row, theta}
//   aux     ballot mode: class masks [S/32][Q][32]; atomic mode: labels [S]
//   lab     [S] label landing zone of the bulk copy (absent when a forced
//           shape leaves no room for it; labels are then read with plain loads)
//   cnt     job counts [TG][2^D K] (both modes)
struct SmemLayout {
  size_t tile, stage, nodes, aux, lab, cnt, total;
};
__host__ __device__ __forceinline__ SmemLayout smem_layout(int mode, int W, int D, int S, int TG,
                                                           int Fmax, int Kmax, int warps,
                                                           int lab_stage = 1) {
  const int B = (1 << D) - 1, L = 1 << D;
  const int LK = L * Kmax;
  const size_t rows = align128((size_t)Fmax * S * W);
  SmemLayout s;
  s.tile = 0;
  s.stage = rows;
  s.nodes = s.stage + (W == 2 ? rows : 0);
  s.aux = s.nodes + align128((size_t)TG * B * 8);
  if (mode == 0) {
    const int Q = bins_per_lane(D, LK);
    s.lab = s.aux + align128((size_t)S * Q * 4);
  } else {
    s.lab = s.aux + align128((size_t)S);
  }
  s.cnt = s.lab + (lab_stage ? align128((size_t)S) : 0);
  s.total = s.cnt + align128((size_t)TG * LK * 4);
  return s;
}

// Shared-memory layout of the streaming kernel (ballot mode only):
//   stage s  [F][S] ranks (natural order), then [S] labels: landing zone s of
//            the ring, at s * sbytes
//   nodes, aux (class masks [S/32][Q][32]; the rows of a chunk pair belong to
//   the one routing warp that owns the pair), cnt as above
struct StreamLayout {
  size_t rbytes, sbytes, nodes, aux, cnt, total;
};
__host__ __device__ __forceinline__ StreamLayout stream_layout(int W, int D, int S, int TG,
                                                               int Fmax, int Kmax, int nstage,
                                                               int lab_stage) {
  const int B = (1 << D) - 1, L = 1 << D;
  const int LK = L * Kmax;
  const int Q = bins_per_lane(D, LK);
  StreamLayout s;
  s.rbytes = align128((size_t)Fmax * S * W);
  s.sbytes = s.rbytes + (lab_stage ? align128((size_t)S) : 0);
  s.nodes = (size_t)nstage * s.sbytes;
  s.aux = s.nodes + align128((size_t)TG * B * 8);
  s.cnt = s.aux + align128((size_t)S * Q * 4);
  s.total = s.cnt + align128((size_t)TG * LK * 4);
  return s;
}

// Byte offset of sample j inside a feature row of the re-laid compute tile.
// uint32 ranks: natural order (lane l of a warp reads bank l).  uint16 ranks:
// the two chunks of 32 samples of a chunk pair share 32-bit words -- word l of
// pair p holds sample 64p+l (low half) and 64p+32+l (high half) -- so a warp
// reading one chunk touches 32 distinct banks whatever rows its lanes are on.
template <int W>
__device__ __forceinline__ uint32_t tile_offset(uint32_t j) {
  if (W == 4) return j * 4u;
  return (j >> 6) * 128u + (j & 31u) * 4u + ((j >> 5) & 1u) * 2u;
}
// Where lane l finds the two samples of chunk pair p: at p * kPairStride +
// l * kLane and kSecond bytes further.  NAT: the two chunks are the first and
// the second 32 samples of the pair in natural order (the streaming kernel's
// uint32 tiles; for uint16 this geometry would put two lanes on one bank word).
// kShared: uint16 rows whose words each hold a sample of both chunks -- the
// re-laid tile (samples 64p + l and 64p + 32 + l) or the streaming kernel's
// landing zone read as even/odd chunks (64p + 2l and 64p + 2l + 1); the root is
// then read once for both chunks, the class masks of the pair sit side by
// side, and with few bins per lane the pair loop is unrolled by two.
template <int W, bool NAT>
struct PairGeom {
  static constexpr uint32_t kSecond = (W == 4) ? 128u : (NAT ? 64u : 2u);
  static constexpr uint32_t kPairStride = 64u * W;
  static constexpr uint32_t kLane = (W == 2 && NAT) ? 2u : 4u;
  static constexpr bool kShared = (W == 2 && !NAT);
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

// Barrier 1 among the first n threads (the consumer warps of the streaming
// kernel; barrier 0 is __syncthreads); the _or form also reduces a predicate.
__device__ __forceinline__ void bar_sync_n(int n) { asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory"); }
__device__ __forceinline__ int bar_or_n(int n, int pred) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.s32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, %2, p;\n\t"
      "selp.s32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(pred), "r"(n)
      : "memory");
  return r;
}

// The D level ballots of 64 samples (the two chunks of pair p) of one tree:
// BA[d] / BB[d] = "went right" at depth d for the 32 samples of chunk A / B.
// R32 (shared-word tiles, root theta <= 0xFFFF): one 32-bit load gives both
// chunks' root ranks, and th0 arrives shifted to the high half.
template <int W, int D, bool NAT, bool R32>
__device__ __forceinline__ void route_levels(uint32_t jb, uint32_t row0, uint32_t th0, uint32_t row2,
                                             uint32_t th2, uint32_t row3, uint32_t th3,
                                             uint32_t tnb32, uint32_t tnb48, uint32_t ntnb,
                                             uint32_t (&BA)[D], uint32_t (&BB)[D]) {
  constexpr uint32_t SEC = PairGeom<W, NAT>::kSecond;
  // level 0: the root is the same node for every lane
  bool pa0, pb0;
  if constexpr (R32) {
    // word = A | B << 16: B >= th <=> word >= th << 16, and A likewise
    // after shifting A into the high half
    const uint32_t w0 = lds_u32(row0 + jb);
    pa0 = (w0 << 16) >= th0;
    pb0 = w0 >= th0;
  } else {
    const uint32_t ra0 = lds_rank<W>(row0 + jb);
    const uint32_t rb0 = lds_rank<W>(row0 + jb + SEC);
    pa0 = ra0 >= th0;
    pb0 = rb0 >= th0;
  }
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
}

// The class-major map of bins to lanes, for Q = 2 and 4 bins per lane (depth
// at least log2 Q): with s = LK / Q = 2^(D - log2 Q) K, lane l < s owns bins
// q s + l (q < Q), all of class l % K and of leaf q 2^(D - log2 Q) + l / K, so
// they differ only in the top log2 Q levels and share the class mask and the
// levels below; lanes s..31 are idle.  Otherwise (Q = 1, 3) lane l owns bins
// l + 32 q, each with its own class.
template <int D, int Q>
__host__ __device__ constexpr bool class_major() {
  return (Q == 2 && D >= 1) || (Q == 4 && D >= 2);
}
// Bin of slot q of `lane` (-1: the slot is unused).
template <int D, int Q>
__device__ __forceinline__ int bin_of(int lane, int q, int LK) {
  if constexpr (class_major<D, Q>()) {
    const int s = LK / Q;
    return lane < s ? q * s + lane : -1;
  } else {
    const int b = lane + 32 * q;
    return b < LK ? b : -1;
  }
}

// Route 64 samples (the two chunks of pair p) of one tree and add the counts
// of the bins this lane owns (bin_of): the count of bin b = leaf K + k grows by
// popc(Y_k & AND_d (B_d or ~B_d)).  SC (the class-major map): the class mask
// and the levels below the top log2 Q are ANDed once for all bins of the lane.
template <int W, int D, int Q, bool NAT, bool R32, bool SC = false>
__device__ __forceinline__ void route_pair(uint32_t jb, uint32_t row0, uint32_t th0, uint32_t row2,
                                           uint32_t th2, uint32_t row3, uint32_t th3, uint32_t tnb32,
                                           uint32_t tnb48, uint32_t ntnb, uint32_t ymA, uint32_t ymB,
                                           const uint32_t (&cst)[Q][D], uint32_t (&cnt)[Q]) {
  uint32_t BA[D], BB[D];
  route_levels<W, D, NAT, R32>(jb, row0, th0, row2, th2, row3, th3, tnb32, tnb48, ntnb, BA, BB);
  constexpr int LQ = (Q == 4) ? 2 : 1;  // levels that tell a lane's bins apart
  if constexpr ((Q == 2 || Q == 4) && D >= LQ && SC) {
    {
      uint32_t ca, cb;
      if constexpr (PairGeom<W, NAT>::kShared) {
        const uint2 m2 = lds_node(ymA);
        ca = m2.x;
        cb = m2.y;
      } else {
        ca = lds_u32(ymA);
        cb = lds_u32(ymB);
      }
#pragma unroll
      for (int d = LQ; d < D; ++d) {
        ca &= BA[d] ^ cst[0][d];
        cb &= BB[d] ^ cst[0][d];
      }
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        uint32_t xa = ca, xb = cb;
#pragma unroll
        for (int d = 0; d < LQ; ++d) {  // bit LQ-1-d of q: right (1) or left (0) at level d
          const bool right = (q >> (LQ - 1 - d)) & 1;
          xa &= right ? BA[d] : ~BA[d];
          xb &= right ? BB[d] : ~BB[d];
        }
        cnt[q] += __popc(xa) + __popc(xb);
      }
      return;
    }
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    uint32_t ma, mb;
    if constexpr (PairGeom<W, NAT>::kShared) {  // [pair][q][lane][chunk]
      const uint2 m2 = lds_node(ymA + q * 256u);
      ma = m2.x;
      mb = m2.y;
    } else {  // [chunk][q][lane]
      ma = lds_u32(ymA + q * 128u);
      mb = lds_u32(ymB + q * 128u);
    }
#pragma unroll
    for (int d = 0; d < D; ++d) {
      ma &= BA[d] ^ cst[q][d];
      mb &= BB[d] ^ cst[q][d];
    }
    cnt[q] += __popc(ma) + __popc(mb);
  }
}

// Ballot mode: every tree of the job over the tile's npair chunk pairs.  A warp
// owns a tree and walks its pairs; a group with fewer trees than warps splits
// each tree's pairs over nw / ntrees warps.  jb0: byte offset of the tile's
// rows from the row addresses held in the node table.
template <int W, int D, int Q, bool NAT>
__device__ __forceinline__ void route_group(int nt, int npair, uint32_t jb0, const uint2* nodes_s,
                                            uint32_t nodes_sa, uint32_t aux_sa,
                                            const uint32_t (&cst)[Q][D], uint32_t* cnt_s, int LK,
                                            int lane, int warp, int nw) {
  constexpr int B = (1 << D) - 1;
  typedef PairGeom<W, NAT> G;
  typedef std::integral_constant<bool, class_major<D, Q>()> SCM;
  auto route_tree = [&](int i, int sl, int step) {
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
    if constexpr (G::kShared) {
      auto one = [&](int pp, auto r32, auto scc) {
        constexpr bool R32 = decltype(r32)::value;
        const uint32_t jb = jb0 + (uint32_t)pp * G::kPairStride + (uint32_t)lane * G::kLane;
        const uint32_t ym = aux_sa + ((uint32_t)pp * Q * 64u + (uint32_t)lane * 2u) * 4u;
        route_pair<W, D, Q, NAT, R32, decltype(scc)::value>(
            jb, n1.x, R32 ? (n1.y << 16) : n1.y, n2.x, n2.y, n3.x, n3.y, tnb + 32u, tnb + 48u, ntnb,
            ym, ym, cst, cnt);
      };
      auto walk = [&](auto r32, auto scc) {
        int pp = sl;
        // by two with one bin per lane, or two at depth <= 3 (measured: 3.8%
        // faster at depth 3, 1.5% slower at depth 4, where it spills)
        if constexpr (Q == 1 || (Q == 2 && D <= 3)) {
          for (; pp + step < npair; pp += 2 * step) {
            one(pp, r32, scc);
            one(pp + step, r32, scc);
          }
          if (pp < npair) one(pp, r32, scc);
        } else {
          for (; pp < npair; pp += step) one(pp, r32, scc);
        }
      };
      if (n1.y <= 0xFFFFu)
        walk(std::true_type{}, SCM{});
      else
        walk(std::false_type{}, SCM{});
    } else {
      auto walk = [&](auto scc) {
        for (int pp = sl; pp < npair; pp += step) {
          const uint32_t jb = jb0 + (uint32_t)pp * G::kPairStride + (uint32_t)lane * G::kLane;
          const uint32_t ymA = aux_sa + ((uint32_t)(2 * pp) * Q * 32u + lane) * 4u;
          const uint32_t ymB = ymA + Q * 128u;
          route_pair<W, D, Q, NAT, false, decltype(scc)::value>(jb, n1.x, n1.y, n2.x, n2.y, n3.x,
                                                                n3.y, tnb + 32u, tnb + 48u, ntnb,
                                                                ymA, ymB, cst, cnt);
        }
      };
      walk(SCM{});
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int b = bin_of<D, Q>(lane, q, LK);
      if (b >= 0) atomicAdd(&cnt_s[i * LK + b], cnt[q]);
    }
  };
  if (nt >= nw) {
    for (int i = warp; i < nt; i += nw) route_tree(i, 0, 1);
  } else {
    const int wpt = nw / nt;  // warps per tree
    for (int it = warp; it < nt * wpt; it += nw) route_tree(it / wpt, it % wpt, wpt);
  }
}

// A new job: node table {row_base + f S W, theta} (the trees as given are
// validated -- a > F, or a theta past the packed range, is flagged and
// evaluated as a no-split node), job counts zeroed, and in ballot mode the
// per-bin level masks cst.
template <int D, int Q, bool BALLOT>
__device__ __forceinline__ void setup_job(const JobView& jv, uint2* nodes_s, uint32_t* cnt_s,
                                          uint32_t row_base, int S, int W, int* status, int lane,
                                          int nthr, uint32_t (&cst)[Q][D], int* K_out,
                                          int* LK_out) {
  constexpr int B = (1 << D) - 1, L = 1 << D;
  const EvalProb& P = *jv.p;
  const int K = P.K, LK = L * K;
  if (P.a16) {
    const uint16_t* ga = P.a16 + (int64_t)jv.tree0 * B;
    const uint32_t* gth = P.th32 + (int64_t)jv.tree0 * B;
    for (int e = threadIdx.x; e < jv.ntrees * B; e += nthr) {
      int av = ga[e];
      uint32_t tv = gth[e];
      if (av > P.F || (av > 0 && tv > kThetaMask)) {
        atomicOr(status, ST_BAD_NODE);
        av = 0;
      }
      const uint32_t f = av > 0 ? (uint32_t)(av - 1) : 0u;
      nodes_s[e] = make_uint2(row_base + f * (uint32_t)S * (uint32_t)W, av > 0 ? tv : 0u);
    }
  } else {
    const uint32_t* gn = P.nodes + (int64_t)jv.tree0 * B;
    for (int e = threadIdx.x; e < jv.ntrees * B; e += nthr) {
      uint32_t pk = gn[e];
      uint32_t f = pk >> 24;
      nodes_s[e] = make_uint2(row_base + f * (uint32_t)S * (uint32_t)W, pk & kThetaMask);
    }
  }
  for (int e = threadIdx.x; e < jv.ntrees * LK; e += nthr) cnt_s[e] = 0;
  if (BALLOT) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int b = bin_of<D, Q>(lane, q, LK);
      const int leaf = b >= 0 ? b / K : 0;
#pragma unroll
      for (int d = 0; d < D; ++d) cst[q][d] = ((leaf >> (D - 1 - d)) & 1) ? 0u : 0xFFFFFFFFu;
    }
  }
  *K_out = K;
  *LK_out = LK;
}

// Labels of a tile that its bulk copy brings: the 16-byte multiple prefix
// (the rest is read with plain loads, so nothing past the label array is read).
__device__ __forceinline__ int tma_label_bytes(const EvalProb& P, int ns, int lab_stage) {
  return (lab_stage && P.tma && P.lab_tma) ? (ns & ~15) : 0;
}

// Stage the rank rows (and labels) of one tile, called by all lanes of one
// warp: lane 0 arms the mbarrier with the byte total, then the lanes issue the
// 1-D bulk copies (one per feature row into `dst`, one for the labels into
// `labdst`) side by side.
__device__ __forceinline__ void issue_tile_tma(const EvalProb& P, int64_t s0, int ns, int S, int W,
                                               unsigned char* dst, unsigned char* labdst,
                                               int lab_stage, uint64_t* bar, int lane) {
  fence_proxy_async_smem();
  const uint32_t bytes = ((uint32_t)ns * W + 15u) & ~15u;
  const uint32_t lbytes = (uint32_t)tma_label_bytes(P, ns, lab_stage);
  if (lane == 0) mbar_arrive_expect_tx(bar, bytes * (uint32_t)P.F + lbytes);
  __syncwarp();
  const unsigned char* src = static_cast<const unsigned char*>(P.ranks);
  const int ncopy = P.F + (lbytes ? 1 : 0);
  for (int c = lane; c < ncopy; c += 32) {
    if (c < P.F)
      bulk_g2s(dst + (size_t)c * S * W, src + ((int64_t)c * P.ld + s0) * W, bytes, bar);
    else
      bulk_g2s(labdst, P.labels + s0, lbytes, bar);
  }
}

// The same copies issued by the whole CTA (called by every thread): thread 0
// arms the mbarrier, and after a CTA barrier lane l of warp w issues copy
// w + nw l.  Issuing a copy costs its warp ~100 cycles, so the F row copies of
// a wide uint32 tile no longer keep warp 0 (and with it the tile's end
// barrier) behind the other warps.
__device__ __forceinline__ void issue_tile_rows_cta(const EvalProb& P, int64_t s0, int ns, int S, int W,
                                                    unsigned char* dst, unsigned char* labdst,
                                                    int lab_stage, uint64_t* bar, int lane, int warp,
                                                    int nw) {
  const uint32_t bytes = ((uint32_t)ns * W + 15u) & ~15u;
  const uint32_t lbytes = (uint32_t)tma_label_bytes(P, ns, lab_stage);
  if (threadIdx.x == 0) mbar_arrive_expect_tx(bar, bytes * (uint32_t)P.F + lbytes);
  __syncthreads();  // armed before any copy can complete
  const unsigned char* src = static_cast<const unsigned char*>(P.ranks);
  const int ncopy = P.F + (lbytes ? 1 : 0);
  for (int c = warp + nw * lane; c < ncopy; c += 32 * nw) {
    fence_proxy_async_smem();
    if (c < P.F)
      bulk_g2s(dst + (size_t)c * S * W, src + ((int64_t)c * P.ld + s0) * W, bytes, bar);
    else
      bulk_g2s(labdst, P.labels + s0, lbytes, bar);
  }
}

// Stage a tile through the tensor map: boxes of tmap_box samples x F rows land
// box-major -- box b at dst + b Fmax tmap_box W bytes, row f of a box at
// f tmap_box W bytes (one box of the whole tile is the natural [F][S] order) --
// one 2-D copy per box; the labels by one 1-D copy.  Called by all lanes of
// one warp.
__device__ __forceinline__ void issue_tile_boxes(const EvalArgs& a, const EvalProb& P, int64_t s0,
                                                 int ns, int W, unsigned char* dst,
                                                 unsigned char* labdst, uint64_t* bar, int lane) {
  fence_proxy_async_smem();
  const int BX = a.tmap_box;
  const int nbox = (ns + BX - 1) / BX;
  const uint32_t boxbytes = (uint32_t)BX * (uint32_t)P.F * (uint32_t)W;
  const uint32_t lbytes = (uint32_t)tma_label_bytes(P, ns, a.lab_stage);
  if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)nbox * boxbytes + lbytes);
  __syncwarp();
  const int ncopy = nbox + (lbytes ? 1 : 0);
  for (int c = lane; c < ncopy; c += 32) {
    if (c < nbox)
      bulk_tensor_2d_g2s(dst + (size_t)c * a.Fmax * BX * W, &a.tmap, (int)(s0 + (int64_t)c * BX), 0, bar);
    else
      bulk_g2s(labdst, P.labels + s0, lbytes, bar);
  }
}

// Label of tile sample j: landed by the bulk copy, else read (through the
// subset index when there is one); 0xFF past the end of the tile.
__device__ __forceinline__ uint32_t tile_label(const EvalProb& P, const uint8_t* lab_land,
                                               int lab_done, int64_t s0, int j, int ns) {
  if (j < lab_done) return lab_land[j];
  if (j >= ns) return 0xFFu;
  int64_t col = P.idx ? (int64_t)P.idx[s0 + j] : s0 + j;
  if ((uint64_t)col >= (uint64_t)P.ncols) col = 0;  // flagged by the rank gather
  return P.labels[col];
}

// Ballot mode: the class masks of the tile's chunks -- lane l's word q is the
// ballot of "label == class of bin l + 32 q" -- laid out [chunk][q][lane], or
// with PAIRED [pair][q][lane][chunk] (the two chunks of a pair side by side).
// EVENODD: chunk 2p holds the even and chunk 2p + 1 the odd samples of the
// 64-sample block p (lane l: samples 64p + 2l and 64p + 2l + 1), else chunk c
// holds samples 32c .. 32c + 31.
template <int D, int Q, bool PAIRED, bool EVENODD = false>
__device__ __forceinline__ void class_masks(const EvalProb& P, const uint8_t* lab_land, int lab_done,
                                            int64_t s0, int ns, int npair, int K, int LK, int lane,
                                            int warp, int nw, uint32_t* aux32) {
  int kq[Q];  // class of each bin this lane owns (-1: none)
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int b = bin_of<D, Q>(lane, q, LK);
    kq[q] = b >= 0 ? b % K : -1;
  }
  for (int c = warp; c < 2 * npair; c += nw) {
    const int j = EVENODD ? 64 * (c >> 1) + 2 * lane + (c & 1) : c * 32 + lane;
    const uint32_t y = tile_label(P, lab_land, lab_done, s0, j, ns);
    uint32_t mine[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) mine[q] = 0u;
    for (int k = 0; k < K; ++k) {
      uint32_t m = __ballot_sync(0xFFFFFFFFu, y == (uint32_t)k);
#pragma unroll
      for (int q = 0; q < Q; ++q)
        if (kq[q] == k) mine[q] = m;
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      if (PAIRED)
        aux32[((c >> 1) * Q + q) * 64 + lane * 2 + (c & 1)] = mine[q];
      else
        aux32[(c * Q + q) * 32 + lane] = mine[q];
    }
  }
}

// A job's shared counts into its problem's HBM counts (one atomic per nonzero
// bin), by threads 0..nthr-1.
__device__ __forceinline__ void flush_job(const JobView& v, const uint32_t* cnt_s, int LK, int nthr) {
  uint32_t* dst = v.p->counts + (int64_t)v.tree0 * LK;
  for (int e = threadIdx.x; e < v.ntrees * LK; e += nthr) {
    uint32_t c = cnt_s[e];
    if (c) atomicAdd(dst + e, c);
  }
}

// Last CTA of a single-problem launch: the counts copied out, errors per tree
// (n minus the sum over leaves of the majority count, the loss identity of
// Section 2), and the accumulator and ticket zeroed for the next launch.  The
// counts pass through the (now free) dynamic shared memory in chunks of whole
// trees, eight loads in flight per thread.
template <int D>
__device__ void finish_single(const EvalArgs& a, uint32_t* sm, size_t sm_bytes) {
  const EvalProb& P = a.single;
  constexpr int L = 1 << D;
  const int K = P.K, LK = L * K;
  uint32_t* acc = P.counts;
  const int per = (int)(sm_bytes / ((size_t)LK * 4));  // whole trees per chunk (>= 1)
  for (int r0 = 0; r0 < P.P; r0 += per) {
    const int nr = min(per, P.P - r0);
    const int64_t base = (int64_t)r0 * LK, ne = (int64_t)nr * LK;
    for (int64_t e0 = threadIdx.x; e0 < ne; e0 += 8 * (int64_t)blockDim.x) {
      uint32_t v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t e = e0 + (int64_t)u * blockDim.x;
        v[u] = e < ne ? __ldcg(acc + base + e) : 0u;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t e = e0 + (int64_t)u * blockDim.x;
        if (e < ne) {
          sm[e] = v[u];
          if (a.counts_out) a.counts_out[base + e] = v[u];
          acc[base + e] = 0u;
        }
      }
    }
    __syncthreads();
    if (a.errors_out) {
      for (int r = threadIdx.x; r < nr; r += blockDim.x) {
        const uint32_t* c = sm + (int64_t)r * LK;
        int64_t correct = 0;
        for (int l = 0; l < L; ++l) {
          uint32_t mx = 0;
          for (int k = 0; k < K; ++k) mx = max(mx, c[l * K + k]);
          correct += mx;
        }
        a.errors_out[r0 + r] = (uint32_t)(P.count - correct);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *a.ticket = 0u;
}

// Every CTA takes a ticket once its counts are visible device-wide; the last
// one finishes a single-problem launch (no-op without a ticket).
template <int D>
__device__ __forceinline__ void take_ticket(const EvalArgs& a, unsigned char* smem, size_t smem_bytes) {
  if (!a.ticket) return;
  __shared__ uint32_t s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(a.ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
  __syncthreads();
  if (s_last) {
    __threadfence();
    finish_single<D>(a, reinterpret_cast<uint32_t*>(smem), smem_bytes);
  }
}

// Launch one evaluator kernel instance: residency from the occupancy API with
// all of the unified L1/shared array as shared memory, the grid capped at the
// tile count.
template <typename Kern>
int launch_kernel(deoct_ctx* ctx, Kern kern, const EvalArgs& args, const EvalConfig& cfg,
                  size_t smem, cudaStream_t s, const char* name) {
  DEOCT_TRY(set_max_dynamic_smem(ctx, kern));
  DEOCT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
  int grid = cfg.grid;
  if (grid <= 0) {
    int occ = 0;
    DEOCT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, cfg.warps * 32, smem));
    if (occ < 1) return set_error(DEOCT_ERR_INVALID, "evaluator tile does not fit: %zu B smem", smem);
    grid = occ * ctx->num_sms;
  }
  if ((int64_t)grid > args.total_tiles) grid = (int)args.total_tiles;
  if (grid < 1) return DEOCT_OK;
  kern<<<grid, cfg.warps * 32, smem, s>>>(args);
  count_launch(ctx);
  return check_launch(name);
}

// eval_stream.cu: the streaming kernel for uint16 (W = 2) or uint32 (W = 4)
// ranks, depth 1..5, Q = 1..4 bins per lane.
int launch_stream(deoct_ctx* ctx, int W, int D, int Q, const EvalArgs& args, const EvalConfig& cfg,
                  size_t smem, cudaStream_t s);

}  // namespace evk
}  // namespace deoct
