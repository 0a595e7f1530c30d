// eval_stream.cu -- the streaming population evaluator (Algorithm 1, Section
// 3.2), ballot counting only.
//
// Warp-specialised: the last warp of the CTA stages tiles into a ring of
// `nstage` landing zones (rank rows + labels, 1-D bulk copies), the other warps
// route.  Each zone has a `full` mbarrier (the copies landed, or a plain
// arrival when the consumers must gather the tile themselves) and an `empty`
// one (the consumers are done with it).  Issuing a bulk copy costs the issuing
// warp ~100 cycles per copy (measured on GB300), which the producer warp
// spends off the routing warps' critical path; with two or three zones the
// copies of later tiles are in flight while a tile is routed.  Trees route
// straight from the landing zone in the natural sample order the copies write
// (no re-layout pass).  This is the kernel for groups of fewer than 16 trees,
// where HBM, not routing, sets the pace.
#include "eval_kernel.cuh"

namespace deoct {
namespace evk {
namespace {

template <int W, int D, int Q>
__global__ void __launch_bounds__(512, 2) eval_stream_kernel(const __grid_constant__ EvalArgs a) {
  typedef typename RankT<W>::T RT;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages];
  __shared__ uint8_t s_kind[kMaxStages];  // 1: zone's tile by bulk copy; 0: consumers gather it

  const int S = a.S, NS = a.nstage;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int ncw = (int)(blockDim.x >> 5) - 1;  // consumer warps; warp ncw stages
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
      mbar_init(&empty[z], 1);
    }
    fence_mbar_init();
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
        if (lane == 0) s_kind[z] = 1;
        __syncwarp();
        const int64_t xs0 = X.start + pv.tile * (int64_t)S;
        const int64_t xrem = X.start + X.count - xs0;
        issue_tile_tma(X, xs0, xrem < S ? (int)xrem : S, S, W, zone, zone + lay.rbytes,
                       a.lab_stage, &full[z], lane);
      } else if (lane == 0) {
        s_kind[z] = 0;
        mbar_arrive(&full[z]);
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
    // ---- consumers: route tile t0 + i from zone i % NS ---------------------
    uint32_t cst[Q][D];  // per owned bin, "right" (0) or "left" (~0) at level d
    int K = 0;
    int z = 0;        // zone of tile gt: (gt - t0) % NS
    uint32_t ph = 0;  // parity of its phase: ((gt - t0) / NS) & 1
    for (int64_t gt = t0; gt < t1; ++gt) {
      JobView nv;  // job and tile of gt: a search at the first tile, then a step
      if (gt == t0) {
        lookup_job(a, gt, &nv);
      } else {
        nv = jv;
        advance_job(a, gt, &nv);
      }
      if (nv.job != cur_job) {
        if (cur_job >= 0) flush_job(jv, cnt_s, LK, nct);
        bar_sync_n(nct);
        jv = nv;
        cur_job = nv.job;
        setup_job<D, Q, true>(jv, nodes_s, cnt_s, stage0_sa, S, W, a.status, lane, nct, cst, &K, &LK);
      }
      jv.tile = nv.tile;
      const EvalProb& P = *jv.p;
      const int64_t s0 = P.start + jv.tile * (int64_t)S;
      const int64_t rem = P.start + P.count - s0;
      const int ns = rem < S ? (int)rem : S;
      const int nch = (ns + 31) >> 5;
      const int npair = (nch + 1) >> 1;
      unsigned char* zone = smem + (size_t)z * lay.sbytes;
      const uint8_t* lab_land = zone + lay.rbytes;

      // one thread polls the zone's mbarrier while the others sleep in the
      // consumers' barrier; each then acquires the zone through the completed
      // phase (the test succeeds at once)
      int ok = 1;
      if (threadIdx.x == 0) ok = mbar_wait_bounded(&full[z], ph, a.status) ? 1 : 0;
      if (bar_or_n(nct, !ok)) break;  // timed out (status recorded)
      if (threadIdx.x != 0) mbar_try_wait(&full[z], ph);
      int lab_done = 0;
      if (s_kind[z]) {
        lab_done = tma_label_bytes(P, ns, a.lab_stage);
      } else {
        // gathered subset or unaligned rows: plain loads in natural order
        const RT* src = static_cast<const RT*>(P.ranks);
        for (int e = threadIdx.x; e < P.F * S; e += nct) {
          int f = e / S, j = e - f * S;
          if (j < ns) {
            int64_t col = P.idx ? (int64_t)P.idx[s0 + j] : s0 + j;
            if ((uint64_t)col >= (uint64_t)P.ncols) {
              atomicOr(a.status, ST_BAD_INDEX);
              col = 0;
            }
            reinterpret_cast<RT*>(zone + (size_t)f * S * W)[j] = src[(int64_t)f * P.ld + col];
          }
        }
      }
      class_masks<Q, false>(P, lab_land, lab_done, s0, ns, npair, K, LK, lane, warp, ncw, aux32);
      bar_sync_n(nct);
      route_group<W, D, Q, true>(jv.ntrees, npair, (uint32_t)z * (uint32_t)lay.sbytes, nodes_s,
                                 nodes_sa, aux_sa, cst, cnt_s, LK, lane, warp, ncw);
      bar_sync_n(nct);
      if (threadIdx.x == 0) mbar_arrive(&empty[z]);  // the producer may restage zone z
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
    case 3: return launch_kernel(ctx, eval_stream_kernel<W, D, 3>, args, cfg, smem, s, "eval_stream_kernel");
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
