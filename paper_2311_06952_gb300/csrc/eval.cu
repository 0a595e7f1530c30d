// eval.cu -- population fitness evaluation (Algorithm 1, Section 3.2): the
// re-laid kernel, the launch decision between it and the streaming kernel
// (eval_stream.cu), and the evaluator's small host-side helpers.
//
// The re-laid kernel stages each tile through one landing zone per CTA and,
// for uint16 ranks, re-lays the rows into a chunk-pair-interleaved compute
// tile so that 16 warps routing 16+ trees read shared memory without bank
// conflicts; the next tile's bulk copies fly while the current one is routed.
// It also holds the shared-atomic counting mode for 2^D K > 128 bins: all
// warps split each tree's chunks and add into the job's shared counts.
#include <cudaTypedefs.h>

#include "eval_kernel.cuh"

namespace deoct {

using namespace evk;

namespace {

template <int W, int D, int MODE, int Q>
__global__ void __launch_bounds__(1024, 1) eval_kernel(const __grid_constant__ EvalArgs a) {
  constexpr int B = (1 << D) - 1;
  constexpr int L = 1 << D;
  typedef typename RankT<W>::T RT;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;

  const int S = a.S;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const SmemLayout lay = smem_layout(MODE, W, D, S, a.TG, a.Fmax, a.Kmax, nw, a.lab_stage);
  unsigned char* tileb = smem + lay.tile;
  unsigned char* stageb = (W == 2) ? smem + lay.stage : tileb;
  uint2* nodes_s = reinterpret_cast<uint2*>(smem + lay.nodes);
  uint32_t* aux32 = reinterpret_cast<uint32_t*>(smem + lay.aux);
  uint8_t* lab_s = smem + lay.aux;
  unsigned char* lab_land = smem + lay.lab;
  uint32_t* cnt_s = reinterpret_cast<uint32_t*>(smem + lay.cnt);
  const uint32_t tile_sa = smem_u32(tileb);
  const uint32_t nodes_sa = smem_u32(nodes_s);
  const uint32_t aux_sa = smem_u32(aux32);

  const int64_t T = a.total_tiles;
  const int64_t t0 = (int64_t)blockIdx.x * T / gridDim.x;
  const int64_t t1 = (int64_t)(blockIdx.x + 1) * T / gridDim.x;

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

  for (int64_t gt = t0; gt < t1; ++gt) {
    JobView nv;  // job and tile of gt: a search at the first tile, then a step
    if (gt == t0) {
      lookup_job(a, gt, &nv);
    } else {
      nv = jv;
      advance_job(a, gt, &nv);
    }
    if (nv.job != cur_job) {
      if (cur_job >= 0) flush_job(jv, cnt_s, LK, blockDim.x);
      __syncthreads();
      jv = nv;
      cur_job = nv.job;
      setup_job<D, Q, MODE == 0>(jv, nodes_s, cnt_s, tile_sa, S, W, a.status, lane, blockDim.x, cst,
                                 &K, &LK);
    }
    jv.tile = nv.tile;  // the tile changes every iteration, the job only sometimes
    const EvalProb& P = *jv.p;
    const int64_t s0 = P.start + jv.tile * (int64_t)S;
    const int64_t rem = P.start + P.count - s0;
    const int ns = rem < S ? (int)rem : S;
    const int nch = (ns + 31) >> 5;
    const int npair = (nch + 1) >> 1;

    // ---- stage rank rows (and labels) ------------------------------------
    if (P.tma) {
      if (!staged) {  // (uniform across the CTA)
        if (a.tmap_box) {
          if (warp == 0) issue_tile_boxes(a, P, s0, ns, W, stageb, lab_land, &mbar, lane);
        } else {
          issue_tile_rows_cta(P, s0, ns, S, W, stageb, lab_land, a.lab_stage, &mbar, lane, warp, nw);
        }
      }
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
    if (P.tma) {
      // one thread polls the mbarrier while the others sleep in the CTA
      // barrier; each then acquires the landed bytes through the completed
      // phase (the test succeeds at once)
      int ok = 1;
      if (threadIdx.x == 0) ok = mbar_wait_bounded(&mbar, phase, a.status) ? 1 : 0;
      if (__syncthreads_or(!ok)) {
        // timed out (status recorded): give the copies in flight one more
        // bounded wait before the CTA leaves
        if (threadIdx.x == 0) mbar_wait_bounded(&mbar, phase, a.status);
        __syncthreads();
        break;  // the CTA still takes its ticket below
      }
      if (threadIdx.x != 0) mbar_try_wait(&mbar, phase);
      phase ^= 1u;
      if (W == 2) {
        // stage (natural order) -> tile (chunk-pair interleaved): a task is
        // four tile words of one row, from two 8-byte loads (samples 64p+4m..
        // +3 and 64p+32+4m..+3) and four byte permutes, one 16-byte store
        // (landing zone: natural rows [F][S], or box-major from the tensor map:
        // box b of BX samples at b Fmax BX, its row f at f BX -- a chunk pair
        // never straddles a box)
        const int quads = npair * 8;  // tasks per row
        const int tasks = P.F * quads;
        const int fstep = blockDim.x / quads, qstep = blockDim.x - fstep * quads;
        const int BX = a.tmap_box, lbx = BX ? __ffs(BX) - 1 : 0;
        int f = threadIdx.x / quads, q = threadIdx.x - f * quads;
        for (int e = threadIdx.x; e < tasks; e += blockDim.x) {
          const int pp = q >> 3, m = q & 7;
          const unsigned char* srow;
          if (BX) {
            const int j0 = pp * 64;
            srow = stageb + ((size_t)((j0 >> lbx) * a.Fmax + f) * BX + (j0 & (BX - 1))) * 2 + m * 8;
          } else {
            srow = stageb + (size_t)f * S * 2 + pp * 128 + m * 8;
          }
          const uint2 lo = *reinterpret_cast<const uint2*>(srow);
          const uint2 hi = *reinterpret_cast<const uint2*>(srow + 64);
          uint4 o;
          o.x = __byte_perm(lo.x, hi.x, 0x5410);
          o.y = __byte_perm(lo.x, hi.x, 0x7632);
          o.z = __byte_perm(lo.y, hi.y, 0x5410);
          o.w = __byte_perm(lo.y, hi.y, 0x7632);
          *reinterpret_cast<uint4*>(tileb + (size_t)f * S * 2 + pp * 128 + m * 16) = o;
          q += qstep;
          f += fstep;
          if (q >= quads) {
            q -= quads;
            ++f;
          }
        }
      }
    }
    // ---- labels: class masks (ballot) or per-sample labels (atomic) -------
    const int lab_done = tma_label_bytes(P, ns, a.lab_stage);
    if (MODE == 0) {
      class_masks<D, Q, PairGeom<W, false>::kShared>(P, lab_land, lab_done, s0, ns, npair, K, LK, lane,
                                                  warp, nw, aux32);
    } else {
      for (int j = threadIdx.x; j < 2 * npair * 32; j += blockDim.x)
        lab_s[j] = (uint8_t)tile_label(P, lab_land, lab_done, s0, j, ns);
    }
    __syncthreads();
    // prefetch the next tile of this CTA into the free landing zones (the
    // uint16 path routes from the re-laid tile, so its landing zone is free)
    if (W == 2 && P.tma && gt + 1 < t1) {
      JobView xv = jv;
      advance_job(a, gt + 1, &xv);
      const EvalProb& X = *xv.p;
      if (X.tma) {
        if (warp == 0) {
          const int64_t xs0 = X.start + xv.tile * (int64_t)S;
          const int64_t xrem = X.start + X.count - xs0;
          if (a.tmap_box)
            issue_tile_boxes(a, X, xs0, xrem < S ? (int)xrem : S, W, stageb, lab_land, &mbar, lane);
          else
            issue_tile_tma(X, xs0, xrem < S ? (int)xrem : S, S, W, stageb, lab_land,
                         a.lab_stage, &mbar, lane);
        }
        staged = true;
      }
    }

    // ---- route + count ---------------------------------------------------
    if (MODE == 0) {
      route_group<W, D, Q, false>(jv.ntrees, npair, 0u, nodes_s, nodes_sa, aux_sa, cst, cnt_s, LK,
                                  lane, warp, nw);
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
  if (cur_job >= 0) flush_job(jv, cnt_s, LK, blockDim.x);
  take_ticket<D>(a, smem, lay.total);
}

template <int W, int D, int MODE, int Q>
int launch_t(deoct_ctx* ctx, const EvalArgs& args, const EvalConfig& cfg, size_t smem,
             cudaStream_t s) {
  return launch_kernel(ctx, eval_kernel<W, D, MODE, Q>, args, cfg, smem, s, "eval_kernel");
}

template <int W, int D>
int dispatch_mode(deoct_ctx* ctx, int mode, int Q, const EvalArgs& args, const EvalConfig& cfg,
                  size_t smem, cudaStream_t s) {
  if (mode == 1) return launch_t<W, D, 1, 1>(ctx, args, cfg, smem, s);
  switch (Q) {
    case 1: return launch_t<W, D, 0, 1>(ctx, args, cfg, smem, s);
    case 2: return launch_t<W, D, 0, 2>(ctx, args, cfg, smem, s);
    case 3:  // three slots only at depth 1 (bins_per_lane)
      if constexpr (D == 1) return launch_t<W, D, 0, 3>(ctx, args, cfg, smem, s);
      return launch_t<W, D, 0, 4>(ctx, args, cfg, smem, s);
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
                              int64_t n_valid, uint32_t* __restrict__ errors,
                              const int* __restrict__ status) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= P) return;
  if (status != nullptr && *status != 0) {  // the counts are not to be trusted
    errors[r] = kErrorsInvalid;
    return;
  }
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

static int eval_mode(int D, int K) { return ((1 << D) * K <= 32 * kQMax && D <= 5) ? 0 : 1; }

// Ballot mode runs on the streaming kernel for groups of fewer than 16 trees
// (HBM sets the pace there).  Groups of 16+ trees keep the re-laid kernel: its
// single landing zone leaves room for twice the tile of the streaming ring
// (measured on GB300: HIGGS-shaped uint32 data, F = 28, ran 1.6x slower on the
// ring's smaller tiles).
static bool use_stream(int mode, int W, int TG, int force = 0) {
  (void)W;
  return mode == 0 && (TG < 16 || force);
}

// Landing zones the streaming kernel wants: three for small groups (HBM-bound),
// two for 16+ trees (the next tile flies while this one is routed).
static int want_stages(int TG) { return TG < 16 ? kMaxStages : 2; }

// Shared memory of a shape with `nstage` landing zones on the streaming kernel
// (0: as many as it wants; the re-laid kernel always has its tile and one
// landing zone).
static size_t eval_smem(int mode, int W, int D, int S, int TG, int F, int K, int warps,
                        int nstage = 0, int lab_stage = 1, int force_stream = 0) {
  if (use_stream(mode, W, TG, force_stream))
    return stream_layout(W, D, S, TG, F, K, nstage ? nstage : want_stages(TG), lab_stage).total;
  return smem_layout(mode, W, D, S, TG, F, K, warps, lab_stage).total;
}

int eval_ctas_per_sm(const deoct_ctx* ctx, int W, int D, int F, int K, const EvalConfig& c) {
  const int mode = eval_mode(D, K);
  if (use_stream(mode, W, c.TG, c.stream)) return 0;
  const size_t smem = eval_smem(mode, W, D, c.S, c.TG, F, K, c.warps);
  if (smem + 1024 > (size_t)ctx->max_smem_optin) return 0;
  const int by_smem = (int)((size_t)ctx->smem_per_sm / (smem + 1024));
  const int by_regs = 32 / std::max(1, c.warps);  // at most 64 registers a thread
  return std::min(by_smem, by_regs);
}

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
    c.warps = 16;
    if (P < 16) {
      // small groups run on the streaming kernel, where (measured on GB300,
      // n = 1e7, P = 1..12) 9 warps -- 8 routing warps and the producer -- and
      // tiles of 2048 samples (pair-sliced groups: a ring of two landing zones)
      // or 1024 (three zones) do best, at two or more CTAs per SM
      c.TG = P;
      const bool sliced = P < kPairSliceTrees;
      c.S = sliced ? 2048 : 1024;
      c.warps = 9;
      while (eval_smem(mode, W, D, c.S, c.TG, F, K, c.warps, sliced ? 2 : 0) > two_per_sm && c.S > 256)
        c.S /= 2;
      while (work(c.S, c.TG) < 2 * (int64_t)ctx->num_sms && c.S > 256) c.S /= 2;
    } else {
      // A warp owns a tree; 16 warps per CTA and two CTAs per SM (measured on
      // GB300: 1.5x faster than 8 warps).  Among the shapes that keep two CTAs
      // per SM, take the least estimated makespan: waves of work items (S
      // samples x TG trees) over the resident CTAs, each costing its S TG
      // evaluations plus a staging overhead worth about 7000 + 170 c
      // evaluations, c the bulk copies a tile takes (~100 cycles each to issue:
      // S / 256 tensor boxes for uint16 rows, F for uint32 rows -- their
      // one-box form for tiles of <= 256 samples measured no faster, as the
      // smaller tiles pay the rest of the overhead twice), fitted to shape
      // sweeps at n = 1e5, F = 20 and n = 1e7, F = 10.  Few large items leave
      // CTAs idle in the last wave; many small ones pay the overhead.
      const int64_t ncta = 2 * (int64_t)ctx->num_sms;
      double best = -1.0;
      for (int S : {2048, 1024, 512, 256})
        for (int TG : {256, 128, 64, 32, 16}) {
          const int tg = std::min(TG, P);
          if (tg < 16 || eval_smem(mode, W, D, S, tg, F, K, 16) > two_per_sm) continue;
          const int64_t items = work(S, tg);
          const double waves = (double)((items + ncta - 1) / ncta);
          const int copies = (W == 2) ? std::max(1, S / 256) : F;
          const double cost = waves * ((double)S * tg + 7000.0 + 170.0 * copies);
          if (best < 0 || cost < best) {
            best = cost;
            c.S = S;
            c.TG = tg;
          }
        }
      // One CTA of 32 warps per SM (a CTA twice as wide, so twice the trees and
      // samples per tile for the same staging and set-up): its work items cost
      // S TG evaluations plus about 25000 + 170 c, at 2.13 times the rate of a
      // 16-warp CTA, fitted to shape sweeps on GB300 (n = 1e7, uint16, depth 4:
      // 1024 x 256 with 16 warps 10.95 ms; 32 warps 10.88 ms at 1024 x 256, 10.43
      // at 2048 x 256, 10.29 at 2048 x 512; depth 3: 8.77 vs 7.80 ms; depth 5:
      // 11.68 vs 10.51 ms; identical counts)
      for (int S : {3072, 2048, 1536, 1024, 512})
        for (int TG : {512, 256, 128, 64, 32}) {
          const int tg = std::min(TG, P);
          if (tg < 16 || eval_smem(mode, W, D, S, tg, F, K, 32) > (size_t)limit) continue;
          const int64_t items = work(S, tg);
          const double waves = (double)((items + ctx->num_sms - 1) / ctx->num_sms);
          const int copies = (W == 2) ? std::max(1, S / 256) : F;
          const double cost = waves * ((double)S * tg + 25000.0 + 170.0 * copies) / 2.13;
          if (best < 0 || cost < best) {
            best = cost;
            c.S = S;
            c.TG = tg;
            c.warps = 32;
          }
        }
      if (best < 0) {  // nothing keeps two CTAs per SM: the largest shape that fits
        c.S = 2048;
        c.TG = std::min(P, 256);
        while (eval_smem(mode, W, D, c.S, c.TG, F, K, c.warps) > (size_t)limit && (c.S > 128 || c.TG > 16)) {
          if (c.S > 128) c.S /= 2; else c.TG = std::max(16, c.TG / 2);
        }
      }
    }
  } else {
    // shared-atomic mode: the 16 warps split the chunks of one tree at a time, so
    // the tile keeps at least 16 chunks (512 samples); the tile shrinks to that
    // before the group does, since every tree of a group reuses the staged tile
    // (wide uint32 data would otherwise end at one tree per group and restage
    // each tile once per tree), and the job's counts ([TG][2^D K]) set TG
    c.S = 1024;
    c.warps = 16;
    c.TG = std::min(P, 256);
    while (eval_smem(mode, W, D, c.S, c.TG, F, K, c.warps) > two_per_sm && c.S > 512) c.S /= 2;
    while (eval_smem(mode, W, D, c.S, c.TG, F, K, c.warps) > two_per_sm && c.TG > 1) c.TG /= 2;
    while (eval_smem(mode, W, D, c.S, c.TG, F, K, c.warps) > (size_t)limit && c.S > 128) c.S /= 2;
    while (work(c.S, c.TG) < 2 * (int64_t)ctx->num_sms && c.TG > 1) c.TG /= 2;
  }
  if (ctx->force_S) c.S = ctx->force_S;
  if (ctx->force_TG) c.TG = std::min(ctx->force_TG, std::max(1, P));
  if (ctx->force_warps) c.warps = ctx->force_warps;
  if (ctx->force_grid) c.grid = ctx->force_grid;
  if (ctx->force_stream) c.stream = 1;
  return c;
}

// cuTensorMapEncodeTiled from the driver (the runtime hands out its entry point).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// The rank rows of a plan as one 2-D tensor map ([F] rows of `ncols` columns,
// row stride ld), boxes of BX columns x F rows; false when the plan's problems
// do not share one TMA-able rank array or the driver declines.  uint16 tiles
// take boxes of 256 (or 128) samples (the re-layout reads them box-major);
// uint32 tiles route from the landing zone in natural order, so they take one
// box of the whole tile, which needs S <= 256.
static bool encode_rank_map(const EvalPlan& plan, int S, int W, EvalArgs* a) {
  const void* base = nullptr;
  int64_t ld = 0, ncols = 0;
  if (plan.d_probs == nullptr) {
    if (!plan.single.tma || plan.single.F != plan.Fmax) return false;
    base = plan.single.ranks;
    ld = plan.single.ld;
    ncols = plan.single.ncols;
  } else {
    if (!plan.shared_ranks) return false;
    base = plan.shared_ranks;
    ld = plan.shared_ld;
    ncols = plan.shared_ncols;
  }
  const int BX = (W == 4) ? S : ((S % 256 == 0) ? 256 : 128);
  if (BX > 256 || S % BX != 0 || plan.Fmax < 1 || plan.Fmax > 256 || ncols < 1) return false;
  if (reinterpret_cast<uintptr_t>(base) % 16 != 0 || (ld * W) % 16 != 0) return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)ncols, (cuuint64_t)plan.Fmax};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * W};
  const cuuint32_t box[2] = {(cuuint32_t)BX, (cuuint32_t)plan.Fmax};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(&a->tmap, W == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_UINT32,
                   2, const_cast<void*>(base), dims, strides,
                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return false;
  a->tmap_box = BX;
  return true;
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
  a.ticket = plan.d_probs == nullptr ? plan.ticket : nullptr;
  a.counts_out = plan.counts_out;
  a.errors_out = plan.errors_out;
  // Shared memory: the deepest landing-zone ring (streaming kernel: three
  // zones for small groups, two otherwise) that keeps two CTAs per SM, else
  // the deepest that fits one CTA; forced shapes that fit in no other way
  // drop the label landing zones (labels then come by plain loads).
  const bool streaming = use_stream(mode, W, cfg.TG, cfg.stream);
  const size_t cap = (size_t)ctx->max_smem_optin - 1024;  // room for the static shared memory
  const size_t two_per_sm = std::min(cap, (size_t)(ctx->smem_per_sm - 2 * 1024) / 2);
  auto need = [&](int ns, int lab) {
    return eval_smem(mode, W, D, cfg.S, cfg.TG, plan.Fmax, plan.Kmax, cfg.warps, ns, lab, cfg.stream);
  };
  const int want = streaming ? want_stages(cfg.TG) : 1;
  a.nstage = 0;
  a.lab_stage = 1;
  for (size_t lim : {two_per_sm, cap})
    for (int ns = want; ns >= 1 && a.nstage == 0; --ns)
      if (need(ns, 1) <= lim) a.nstage = ns;
  if (a.nstage == 0) {
    a.nstage = 1;
    a.lab_stage = 0;
  }
  const size_t smem = need(a.nstage, a.lab_stage);
  if (smem > cap)
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
  const int Q = bins_per_lane(D, (1 << D) * plan.Kmax);
  // re-laid kernel: a tile arrives as 2-D tensor boxes (uint16: S / BX boxes;
  // uint32: one box, tiles of at most 256 samples)
  a.tmap_box = 0;
  if (!streaming && (W == 2 || cfg.S <= 256)) encode_rank_map(plan, cfg.S, W, &a);
  EvalConfig scfg = cfg;  // the streaming kernel has a producer warp and >= 1 routing warp
  if (scfg.warps < 2) scfg.warps = 2;
  if (scfg.warps > 16) scfg.warps = 16;
  int rc = streaming ? launch_stream(ctx, W, D, Q, a, scfg, smem, stream)
           : (W == 2) ? dispatch_depth<2>(ctx, D, mode, Q, a, cfg, smem, stream)
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
                  uint32_t* errors, cudaStream_t stream, const int* status) {
  errors_kernel<<<(P + 127) / 128, 128, 0, stream>>>(counts, P, L, K, n_valid, errors, status);
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
