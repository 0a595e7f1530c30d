// eval_stream.cu -- the streaming population evaluator (Algorithm 1, Section
// 3.2), ballot counting only.
//
// Warp-specialised: the last warp of the CTA stages tiles into a ring of
// `nstage` landing zones (rank rows + labels, 1-D bulk copies), the other warps
// route.  Each zone has a `full` mbarrier (the copies landed, or a plain
// arrival when the routing warps must gather the tile themselves) and an
// `empty` one that every routing warp arrives on once it is done with the
// zone.  Issuing a bulk copy costs the issuing warp ~100 cycles per copy
// (measured on GB300), which the producer warp spends off the routing warps'
// critical path; with two or three zones the copies of later tiles are in
// flight while a tile is routed.
//
// Each routing warp waits for the zone itself and releases it with its own
// arrival.  For groups of one to three trees the routing warps do not meet per
// tile at all: each owns the same chunk pairs of every tile (for every tree of
// the job) and computes the class masks of its own pairs.  Larger groups share
// the tile's class masks (two barriers per tile).  Job changes and gathered
// (subset-index) tiles also meet; every routing warp reaches each of these
// barriers at the same tile.  Trees route straight from the landing zone in the
// natural sample order the copies write (no re-layout pass; uint16 chunks take
// the even and the odd samples of a 64-sample block, so a pair's two samples
// of a row share one word).  This is the kernel for groups of fewer than 16
// trees, where HBM, not routing, sets the pace.
#include "eval_kernel.cuh"

namespace deoct {
namespace evk {
namespace {

// One routing warp's share of a tile: chunk pairs warp, warp + ncw, ... of
// every tree of the job.  The warp first writes the class masks of its pairs to
// entries of `aux` that no other warp touches, then routes each tree over its
// pairs from the landing zone and adds the bin counts to the job's shared
// counts with one atomic per (tree, bin) per tile.  Pair p covers samples
// 64p .. 64p + 63 of the zone.  With uint16 ranks its chunks are the even and
// the odd samples: lane l reads one word holding samples 64p + 2l and
// 64p + 2l + 1, the geometry of the re-laid tile (one root load per pair, no
// bank conflicts, masks [pair][q][lane][chunk]) without a re-layout pass.  With
// uint32 ranks they are the first and the second 32 samples (masks
// [chunk][q][lane]).  jb0: byte offset of the zone from the row addresses held
// in the node table.
template <int W, int D, int Q>
__device__ __forceinline__ void route_share(const EvalProb& P, int nt, int npair, uint32_t jb0,
                                            const uint2* nodes_s, uint32_t nodes_sa,
                                            uint32_t* aux32, uint32_t aux_sa,
                                            const uint8_t* lab_land, int lab_done, int64_t s0,
                                            int ns, int K, const int (&kq)[Q],
                                            const uint32_t (&cst)[Q][D], uint32_t* cnt_s, int LK,
                                            int lane, int warp, int ncw) {
  constexpr int B = (1 << D) - 1;
  constexpr bool EO = (W == 2);  // even/odd chunks on words shared by a pair
  typedef PairGeom<W, !EO> G;
  if (warp >= npair) return;
  typedef std::integral_constant<bool, class_major<D, Q>()> SCM;
  auto put = [&](int c, int q, uint32_t m) {
    if (EO)
      aux32[((c >> 1) * Q + q) * 64 + lane * 2 + (c & 1)] = m;
    else
      aux32[(c * Q + q) * 32 + lane] = m;
  };
  if (K == 2 && lab_done >= 64 * npair) {
    // two classes, every label of the tile landed: all bins of a lane have
    // class lane % 2 (bins lane + 32 q, or q s + lane with s even), so one
    // pair of ballots per chunk serves them
    const bool odd = lane & 1;
    for (int pp = warp; pp < npair; pp += ncw) {
      uint32_t ya, yb;
      if (EO) {
        const uint32_t l2 = *reinterpret_cast<const uint16_t*>(lab_land + 64 * pp + 2 * lane);
        ya = l2 & 0xFFu;
        yb = l2 >> 8;
      } else {
        ya = lab_land[64 * pp + lane];
        yb = lab_land[64 * pp + 32 + lane];
      }
      const uint32_t a1 = __ballot_sync(0xFFFFFFFFu, ya == 1u);
      const uint32_t a0 = __ballot_sync(0xFFFFFFFFu, ya == 0u);
      const uint32_t b1 = __ballot_sync(0xFFFFFFFFu, yb == 1u);
      const uint32_t b0 = __ballot_sync(0xFFFFFFFFu, yb == 0u);
      const uint32_t ma = odd ? a1 : a0, mb = odd ? b1 : b0;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        put(2 * pp, q, kq[q] >= 0 ? ma : 0u);
        put(2 * pp + 1, q, kq[q] >= 0 ? mb : 0u);
      }
    }
  } else {
    for (int c = 2 * warp; c < 2 * npair; c += (c & 1) ? 2 * ncw - 1 : 1) {
      const int j = EO ? 64 * (c >> 1) + 2 * lane + (c & 1) : c * 32 + lane;
      const uint32_t y = tile_label(P, lab_land, lab_done, s0, j, ns);
      uint32_t mine[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) mine[q] = 0u;
      for (int k = 0; k < K; ++k) {
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, y == (uint32_t)k);
#pragma unroll
        for (int q = 0; q < Q; ++q)
          if (kq[q] == k) mine[q] = m;
      }
#pragma unroll
      for (int q = 0; q < Q; ++q) put(c, q, mine[q]);
    }
  }
  __syncwarp();
  for (int i = 0; i < nt; ++i) {
    const uint32_t tnb = nodes_sa + (uint32_t)(i * B - 1) * 8u;  // node t at tnb + 8t
    const uint2 n1 = nodes_s[i * B];
    uint2 n2 = n1, n3 = n1;
    if (D >= 2) {
      n2 = nodes_s[i * B + 1];
      n3 = nodes_s[i * B + 2];
    }
    const uint32_t ntnb = 0u - tnb;
    uint32_t cnt[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) cnt[q] = 0u;
    auto walk = [&](auto r32, auto scc) {
      constexpr bool R32 = decltype(r32)::value;
      for (int pp = warp; pp < npair; pp += ncw) {
        const uint32_t jb = jb0 + (uint32_t)pp * G::kPairStride + (uint32_t)lane * G::kLane;
        uint32_t ymA, ymB;
        if (EO) {
          ymA = ymB = aux_sa + ((uint32_t)pp * Q * 64u + (uint32_t)lane * 2u) * 4u;
        } else {
          ymA = aux_sa + ((uint32_t)(2 * pp) * Q * 32u + lane) * 4u;
          ymB = ymA + Q * 128u;
        }
        route_pair<W, D, Q, !EO, R32, decltype(scc)::value>(
            jb, n1.x, R32 ? (n1.y << 16) : n1.y, n2.x, n2.y, n3.x, n3.y, tnb + 32u, tnb + 48u, ntnb,
            ymA, ymB, cst, cnt);
      }
    };
    if constexpr (EO) {
      if (n1.y <= 0xFFFFu)
        walk(std::true_type{}, SCM{});
      else
        walk(std::false_type{}, SCM{});
    } else {
      walk(std::false_type{}, SCM{});
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int b = bin_of<D, Q>(lane, q, LK);
      if (b >= 0) atomicAdd(&cnt_s[i * LK + b], cnt[q]);
    }
  }
}

template <int W, int D, int Q>
__global__ void __launch_bounds__(512, 2) eval_stream_kernel(const __grid_constant__ EvalArgs a) {
  typedef typename RankT<W>::T RT;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages];
  __shared__ volatile int s_abort;  // a routing warp's bounded wait ran out

  const int S = a.S, NS = a.nstage;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int ncw = (int)(blockDim.x >> 5) - 1;  // routing warps; warp ncw stages
  const int nct = ncw * 32;
  const StreamLayout lay = stream_layout(W, D, S, a.TG, a.Fmax, a.Kmax, NS, a.lab_stage);
  uint2* nodes_s = reinterpret_cast<uint2*>(smem + lay.nodes);
  uint32_t* aux32 = reinterpret_cast<uint32_t*>(smem + lay.aux);
  uint32_t* cnt_s = reinterpret_cast<uint32_t*>(smem + lay.cnt);
  const uint32_t stage0_sa = smem_u32(smem);
  const uint32_t nodes_sa = smem_u32(nodes_s);
  const uint32_t aux_sa = smem_u32(aux32);

  const int64_t T = a.total_tiles;
  const int64_t t0 = (int64_t)blockIdx.x * T / gridDim.x;
  const int64_t t1 = (int64_t)(blockIdx.x + 1) * T / gridDim.x;

  if (threadIdx.x == 0) {
    for (int z = 0; z < NS; ++z) {
      mbar_init(&full[z], 1);
      mbar_init(&empty[z], (uint32_t)ncw);
    }
    fence_mbar_init();
    s_abort = 0;
  }
  __syncthreads();

  int cur_job = -1;
  JobView jv;
  int LK = 0;
  if (warp == ncw) {
    // ---- producer: tile t0 + i into zone i % NS once the zone is free ------
    JobView pv;
    int64_t i = 0;
    uint32_t issued = 0;  // bit z: zone z was staged at least once
    int z = 0;            // i % NS
    uint32_t round = 0;   // i / NS
    for (int64_t pt = t0; pt < t1; ++pt, ++i) {
      if (round > 0) {
        int ok = 1;
        if (lane == 0) ok = mbar_wait_bounded(&empty[z], (round - 1) & 1u, a.status) ? 1 : 0;
        if (!__shfl_sync(0xFFFFFFFFu, ok, 0)) break;  // timed out (status recorded)
        mbar_try_wait(&empty[z], (round - 1) & 1u);   // every lane acquires (done at once)
      }
      if (pt == t0) {
        lookup_job(a, pt, &pv);
      } else {
        advance_job(a, pt, &pv);
      }
      const EvalProb& X = *pv.p;
      unsigned char* zone = smem + (size_t)z * lay.sbytes;
      if (X.tma) {
        const int64_t xs0 = X.start + pv.tile * (int64_t)S;
        const int64_t xrem = X.start + X.count - xs0;
        issue_tile_tma(X, xs0, xrem < S ? (int)xrem : S, S, W, zone, zone + lay.rbytes,
                       a.lab_stage, &full[z], lane);
      } else if (lane == 0) {
        mbar_arrive(&full[z]);  // the routing warps gather this tile themselves
      }
      issued |= 1u << z;
      __syncwarp();
      if (++z == NS) {
        z = 0;
        ++round;
      }
    }
    // every staged zone's last phase has completed (landed) before the CTA
    // leaves: waits that are already satisfied return at once
    if (lane == 0)
      for (int q = 0; q < NS; ++q)
        if (issued & (1u << q)) {
          // zone q was last staged in round r = the largest with r NS + q < i
          const uint32_t r = (uint32_t)((i - 1 - q) / NS);
          mbar_wait_bounded(&full[q], r & 1u, a.status);
        }
  } else {
    // ---- routing warps: their share of tile t0 + i from zone i % NS --------
    uint32_t cst[Q][D];  // per owned bin, "right" (0) or "left" (~0) at level d
    int kq[Q];           // class of each owned bin (-1: none)
    int K = 0;
    int z = 0;          // zone of tile gt: (gt - t0) % NS
    uint32_t ph = 0;    // parity of its phase: ((gt - t0) / NS) & 1
    bool dead = false;  // a bounded wait ran out: skip the work, keep the barriers
    for (int64_t gt = t0; gt < t1; ++gt) {
      JobView nv;  // job and tile of gt: a search at the first tile, then a step
      if (gt == t0) {
        lookup_job(a, gt, &nv);
      } else {
        nv = jv;
        advance_job(a, gt, &nv);
      }
      if (nv.job != cur_job) {
        bar_sync_n(nct);  // every routing warp is done with the previous job
        if (cur_job >= 0) flush_job(jv, cnt_s, LK, nct);
        bar_sync_n(nct);  // its counts are read before the new job zeroes them
        jv = nv;
        cur_job = nv.job;
        setup_job<D, Q, true>(jv, nodes_s, cnt_s, stage0_sa, S, W, a.status, lane, nct, cst, &K, &LK);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int b = bin_of<D, Q>(lane, q, LK);
          kq[q] = b >= 0 ? b % K : -1;
        }
        bar_sync_n(nct);  // node table and zeroed counts visible to every warp
      }
      jv.tile = nv.tile;
      const EvalProb& P = *jv.p;
      const int64_t s0 = P.start + jv.tile * (int64_t)S;
      const int64_t rem = P.start + P.count - s0;
      const int ns = rem < S ? (int)rem : S;
      const int npair = (((ns + 31) >> 5) + 1) >> 1;
      unsigned char* zone = smem + (size_t)z * lay.sbytes;
      const uint8_t* lab_land = zone + lay.rbytes;

      // lane 0 polls the zone's mbarrier; then every lane acquires the zone
      // through the completed phase (the test succeeds at once)
      if (!dead && s_abort) dead = true;
      if (!dead) {
        int ok = 1;
        if (lane == 0) ok = mbar_wait_bounded(&full[z], ph, a.status) ? 1 : 0;
        if (__shfl_sync(0xFFFFFFFFu, ok, 0)) {
          mbar_try_wait(&full[z], ph);
        } else {  // timed out (status recorded)
          dead = true;
          if (lane == 0) s_abort = 1;
        }
      }
      int lab_done = 0;
      if (P.tma) {
        lab_done = tma_label_bytes(P, ns, a.lab_stage);
      } else {
        // gathered subset or unaligned rows: the routing warps gather the
        // tile with plain loads in natural order, then meet
        if (!dead) {
          const RT* src = static_cast<const RT*>(P.ranks);
          for (int e = threadIdx.x; e < P.F * S; e += nct) {
            int f = e / S, jj = e - f * S;
            if (jj < ns) {
              int64_t col = P.idx ? (int64_t)P.idx[s0 + jj] : s0 + jj;
              if ((uint64_t)col >= (uint64_t)P.ncols) {
                atomicOr(a.status, ST_BAD_INDEX);
                col = 0;
              }
              reinterpret_cast<RT*>(zone + (size_t)f * S * W)[jj] = src[(int64_t)f * P.ld + col];
            }
          }
        }
        bar_sync_n(nct);
      }
      const uint32_t jb0 = (uint32_t)z * (uint32_t)lay.sbytes;
      if (jv.ntrees < kPairSliceTrees) {
        if (!dead)
          route_share<W, D, Q>(P, jv.ntrees, npair, jb0, nodes_s, nodes_sa, aux32, aux_sa, lab_land,
                               lab_done, s0, ns, K, kq, cst, cnt_s, LK, lane, warp, ncw);
      } else {
        // larger groups: the tile's class masks once, shared by every warp
        // (uint16: even/odd chunks on shared words, as in route_share)
        if (!dead)
          class_masks<D, Q, W == 2, W == 2>(P, lab_land, lab_done, s0, ns, npair, K, LK, lane, warp,
                                         ncw, aux32);
        bar_sync_n(nct);
        if (!dead)
          route_group<W, D, Q, W == 4>(jv.ntrees, npair, jb0, nodes_s, nodes_sa, aux_sa, cst, cnt_s,
                                       LK, lane, warp, ncw);
        bar_sync_n(nct);  // no warp rewrites the masks while another still reads them
      }
      __syncwarp();
      if (!dead && lane == 0) mbar_arrive(&empty[z]);  // this warp is done with zone z
      if (++z == NS) {
        z = 0;
        ph ^= 1u;
      }
    }
  }
  __syncthreads();
  if (cur_job >= 0) flush_job(jv, cnt_s, LK, nct);
  take_ticket<D>(a, smem, lay.total);
}

template <int W, int D>
int dispatch_q(deoct_ctx* ctx, int Q, const EvalArgs& args, const EvalConfig& cfg, size_t smem,
               cudaStream_t s) {
  switch (Q) {
    case 1: return launch_kernel(ctx, eval_stream_kernel<W, D, 1>, args, cfg, smem, s, "eval_stream_kernel");
    case 2: return launch_kernel(ctx, eval_stream_kernel<W, D, 2>, args, cfg, smem, s, "eval_stream_kernel");
    case 3:  // three slots only at depth 1 (bins_per_lane)
      if constexpr (D == 1)
        return launch_kernel(ctx, eval_stream_kernel<W, D, 3>, args, cfg, smem, s, "eval_stream_kernel");
      return launch_kernel(ctx, eval_stream_kernel<W, D, 4>, args, cfg, smem, s, "eval_stream_kernel");
    default: return launch_kernel(ctx, eval_stream_kernel<W, D, 4>, args, cfg, smem, s, "eval_stream_kernel");
  }
}

template <int W>
int dispatch_d(deoct_ctx* ctx, int D, int Q, const EvalArgs& args, const EvalConfig& cfg,
               size_t smem, cudaStream_t s) {
  switch (D) {
    case 1: return dispatch_q<W, 1>(ctx, Q, args, cfg, smem, s);
    case 2: return dispatch_q<W, 2>(ctx, Q, args, cfg, smem, s);
    case 3: return dispatch_q<W, 3>(ctx, Q, args, cfg, smem, s);
    case 4: return dispatch_q<W, 4>(ctx, Q, args, cfg, smem, s);
    case 5: return dispatch_q<W, 5>(ctx, Q, args, cfg, smem, s);
  }
  return set_error(DEOCT_ERR_INVALID, "streaming evaluator: depth %d outside 1..5", D);
}

}  // namespace

int launch_stream(deoct_ctx* ctx, int W, int D, int Q, const EvalArgs& args, const EvalConfig& cfg,
                  size_t smem, cudaStream_t s) {
  if (args.nstage < 1 || args.nstage > kMaxStages)
    return set_error(DEOCT_ERR_INVALID, "streaming evaluator: %d landing zones", args.nstage);
  return W == 2 ? dispatch_d<2>(ctx, D, Q, args, cfg, smem, s)
                : dispatch_d<4>(ctx, D, Q, args, cfg, smem, s);
}

}  // namespace evk
}  // namespace deoct
