// mh.cu -- moving-horizon DEOCT (Algorithm 2, Section 4) and the exhaustive
// depth-1 search that Algorithm 2 uses at the bottom level.
//
// The tree is grown level by level.  Per level d the samples carry the id of
// the node they reached (node_of); a histogram of (node, class) decides which
// nodes are solved (more than n_min samples and at least two classes); the
// samples of solved nodes are compacted into contiguous, 16-sample-aligned
// segments (sample index, feature-major ranks, labels), so each node's subset
// is a TMA-able slice; then every solved node is solved with horizon
// D_t = min(D_MH, D - d):
//   D_t >= 2: DEOCT of depth D_t (Philox stream = node id), either
//     - plain: one DEOCT per node, each with its own launches, or
//     - batched: one multi-problem evaluator launch and one DE-step launch per
//       generation for all nodes of the level, replayed from a captured CUDA
//       graph, with the evaluator tile shape chosen by an autotuner;
//   D_t = 1: exhaustive depth-1 search: per feature, the (node, rank) keys of
//     the level are radix-sorted so each node's samples are in rank order, and
//     one CTA per (node, feature) sweeps the distinct ranks with running class
//     counts; the best split per node is reduced over features.
// Then the samples move one level down.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace deoct {

int run_deoct(deoct_ctx* ctx, const deoct_dataset* ds, const int32_t* idx, int64_t n_sub,
              const deoct_params* p, uint64_t stream_id, const float* seeds, int S, float* pop,
              double* fit, int32_t* best, cudaStream_t s);

namespace {

constexpr int kSegAlign = 16;  // samples; 32 bytes of uint16 ranks

__global__ void fill_i32_kernel(int32_t* __restrict__ p, int64_t n, int32_t v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// class histogram of the samples of each node of one level: hist[(t - base) * K + y]
__global__ void level_hist_kernel(const int32_t* __restrict__ node_of, const uint8_t* __restrict__ labels,
                                  int64_t n, int32_t base, int32_t nnodes, int K, int use_smem,
                                  uint32_t* __restrict__ hist) {
  extern __shared__ uint32_t h[];
  const int bins = nnodes * K;
  if (use_smem) {
    for (int e = threadIdx.x; e < bins; e += blockDim.x) h[e] = 0;
    __syncthreads();
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int t = node_of[i] - base;
    if (t < 0 || t >= nnodes) continue;
    int y = labels[i];
    if (y >= K) continue;
    if (use_smem) atomicAdd(&h[t * K + y], 1u);
    else atomicAdd(&hist[t * K + y], 1u);
  }
  if (use_smem) {
    __syncthreads();
    for (int e = threadIdx.x; e < bins; e += blockDim.x)
      if (h[e]) atomicAdd(&hist[e], h[e]);
  }
}

// one level down: node t -> 2t if rank[a_t - 1][i] < theta_t else 2t + 1
template <typename RT>
__global__ void route_level_kernel(int32_t* __restrict__ node_of, const RT* __restrict__ ranks,
                                   int64_t ld, int64_t n, int32_t base, int32_t nnodes,
                                   const uint32_t* __restrict__ lvl_nodes) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int t = node_of[i];
  int k = t - base;
  if (k < 0 || k >= nnodes) return;
  uint32_t pk = lvl_nodes[k];
  uint32_t f = pk >> 24, th = pk & kThetaMask;
  uint32_t r = ranks[(int64_t)f * ld + i];
  node_of[i] = 2 * t + (r < th ? 0 : 1);
}

// samples of solved nodes -> contiguous segments (order inside a segment is
// arbitrary: every consumer is order-independent)
__global__ void compact_kernel(const int32_t* __restrict__ node_of, int64_t n, int32_t base,
                               int32_t nnodes, const int32_t* __restrict__ slot_of,
                               const int64_t* __restrict__ seg_off, int32_t* __restrict__ cursor,
                               int32_t* __restrict__ idx_out, int32_t* __restrict__ pos_slot) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int m = -1;
  if (i < n) {
    int k = node_of[i] - base;
    if (k >= 0 && k < nnodes) m = slot_of[k];
  }
  const int lane = threadIdx.x & 31;
  const uint32_t peers = __match_any_sync(0xFFFFFFFFu, m);
  const int leader = __ffs(peers) - 1;
  int basepos = 0;
  if (m >= 0 && lane == leader) basepos = atomicAdd(&cursor[m], __popc(peers));
  basepos = __shfl_sync(0xFFFFFFFFu, basepos, leader);
  if (m >= 0) {
    int64_t pos = seg_off[m] + basepos + __popc(peers & ((1u << lane) - 1u));
    idx_out[pos] = (int32_t)i;
    pos_slot[pos] = m;
  }
}

// compacted rank rows and labels (padding: rank 0, label 0xFF)
template <typename RT>
__global__ void gather_kernel(const RT* __restrict__ ranks, int64_t ld, const uint8_t* __restrict__ labels,
                              const int32_t* __restrict__ idx, int64_t npad, RT* __restrict__ cranks,
                              int64_t cld, uint8_t* __restrict__ clabels) {
  int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int f = blockIdx.y;
  if (pos >= npad) return;
  int32_t i = idx[pos];
  cranks[(int64_t)f * cld + pos] = i >= 0 ? ranks[(int64_t)f * ld + i] : (RT)0;
  if (f == 0) clabels[pos] = i >= 0 ? labels[i] : (uint8_t)0xFF;
}

// class totals per segment slot
__global__ void seg_hist_kernel(const uint8_t* __restrict__ clabels, const int32_t* __restrict__ pos_slot,
                                int64_t npad, int K, uint32_t* __restrict__ tot) {
  int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= npad) return;
  int m = pos_slot[pos];
  int y = clabels[pos];
  if (m >= 0 && y < K) atomicAdd(&tot[(int64_t)m * K + y], 1u);
}

// depth-1 sort keys: (slot - s0) << 24 | rank for slots of the batch, else ~0
template <typename RT>
__global__ void d1_keys_kernel(const RT* __restrict__ cranks, int64_t cld, const uint8_t* __restrict__ clabels,
                               const int32_t* __restrict__ pos_slot, int64_t npad, int s0, int s1,
                               uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int f = blockIdx.y;
  if (pos >= npad) return;
  int m = pos_slot[pos];
  uint32_t key = 0xFFFFFFFFu, val = 0xFFu;
  if (m >= s0 && m < s1) {
    key = ((uint32_t)(m - s0) << 24) | ((uint32_t)cranks[(int64_t)f * cld + pos] & kThetaMask);
    val = clabels[pos];
  }
  keys[(int64_t)f * npad + pos] = key;
  vals[(int64_t)f * npad + pos] = val;
}

// One CTA per (node, feature): the node's samples in rank order; at every
// boundary between distinct ranks r_j < r_{j+1} the candidate theta = r_j + 1
// (the smallest threshold giving that partition) is scored with the fitness
// of Section 3.2.  Best (fitness, then theta) per (node, feature).
__global__ void d1_sweep_kernel(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                                int64_t npad, const int64_t* __restrict__ run_start,
                                const int64_t* __restrict__ cnt, const uint32_t* __restrict__ tot,
                                int K, const uint32_t* __restrict__ n_unique, int n_min, double alpha,
                                int F, double* __restrict__ best_f, uint32_t* __restrict__ best_th) {
  extern __shared__ uint32_t cs[];  // [blockDim.x][K] running class counts
  __shared__ double red_f[32];
  __shared__ uint32_t red_t[32];
  const int mb = blockIdx.x, p = blockIdx.y;
  const int NT = blockDim.x;
  const int64_t nm = cnt[mb];
  const uint32_t* kp = keys + (int64_t)p * npad + run_start[mb];
  const uint32_t* vp = vals + (int64_t)p * npad + run_start[mb];
  const uint32_t* T = tot + (int64_t)mb * K;
  const uint32_t np = n_unique[p];
  uint32_t* mine = cs + threadIdx.x * K;
  for (int k = 0; k < K; ++k) mine[k] = 0;
  const int64_t chunk = (nm + NT - 1) / NT;
  const int64_t e0 = (int64_t)threadIdx.x * chunk;
  const int64_t e1 = e0 + chunk < nm ? e0 + chunk : nm;
  for (int64_t e = e0; e < e1; ++e) {
    const uint32_t y = vp[e];
    if (y < (uint32_t)K) mine[y] += 1;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += NT) {  // exclusive scan over threads, per class
    uint32_t run = 0;
    for (int t = 0; t < NT; ++t) {
      uint32_t x = cs[t * K + k];
      cs[t * K + k] = run;
      run += x;
    }
  }
  __syncthreads();
  double bf = __longlong_as_double(0x7FF0000000000000LL);  // +inf
  uint32_t bt = 0xFFFFFFFFu;
  for (int64_t e = e0; e < e1; ++e) {
    const uint32_t y = vp[e];
    if (y < (uint32_t)K) mine[y] += 1;
    const uint32_t r = kp[e] & kThetaMask;
    const uint32_t rn = (e + 1 < nm) ? (kp[e + 1] & kThetaMask) : 0xFFFFFFFFu;
    if (rn == r) continue;
    const uint32_t th = r + 1;
    if (th >= np) continue;
    uint32_t ml = 0, mr = 0;
    for (int k = 0; k < K; ++k) {
      uint32_t l = mine[k], rr = T[k] - l;
      ml = l > ml ? l : ml;
      mr = rr > mr ? rr : mr;
    }
    const int64_t nl = e + 1, nr = nm - nl;
    const int64_t err = nm - (int64_t)ml - (int64_t)mr;
    const int64_t v = ((nl > 0 && nl < n_min) ? 1 : 0) + ((nr > 0 && nr < n_min) ? 1 : 0);
    const double f = __dadd_rn((double)(err + v), alpha);
    if (f < bf || (f == bf && th < bt)) {
      bf = f;
      bt = th;
    }
  }
  // block reduce: lowest fitness, then lowest theta
  for (int off = 16; off > 0; off >>= 1) {
    double of = __shfl_down_sync(0xFFFFFFFFu, bf, off);
    uint32_t ot = __shfl_down_sync(0xFFFFFFFFu, bt, off);
    if (of < bf || (of == bf && ot < bt)) {
      bf = of;
      bt = ot;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red_f[warp] = bf;
    red_t[warp] = bt;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (NT + 31) / 32; ++w)
      if (red_f[w] < bf || (red_f[w] == bf && red_t[w] < bt)) {
        bf = red_f[w];
        bt = red_t[w];
      }
    best_f[(int64_t)mb * F + p] = bf;
    best_th[(int64_t)mb * F + p] = bt;
  }
}

// per node: no split first, then the lowest feature among the minima
__global__ void d1_reduce_kernel(const double* __restrict__ best_f, const uint32_t* __restrict__ best_th,
                                 int M, int F, const int64_t* __restrict__ cnt,
                                 const uint32_t* __restrict__ tot, int K, int n_min,
                                 uint16_t* __restrict__ a_out, uint32_t* __restrict__ th_out,
                                 double* __restrict__ f_out) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const int64_t nm = cnt[m];
  uint32_t mx = 0;
  for (int k = 0; k < K; ++k) mx = max(mx, tot[(int64_t)m * K + k]);
  double f = (double)((nm - (int64_t)mx) + ((nm > 0 && nm < n_min) ? 1 : 0));
  int a = 0;
  uint32_t th = 0;
  for (int p = 0; p < F; ++p) {
    double bf = best_f[(int64_t)m * F + p];
    if (bf < f) {
      f = bf;
      a = p + 1;
      th = best_th[(int64_t)m * F + p];
    }
  }
  a_out[m] = (uint16_t)a;
  th_out[m] = th;
  f_out[m] = f;
}

// root node of each problem's best individual
__global__ void extract_roots_kernel(const DEProb* __restrict__ probs, int M, int B,
                                     uint16_t* __restrict__ a_out, uint32_t* __restrict__ th_out,
                                     double* __restrict__ f_out) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const DEProb& pb = probs[m];
  const int b = *pb.best;
  const float* g = pb.pop + (int64_t)b * 2 * B;
  int av;
  uint32_t th;
  decode_gene_pair(g[0], g[B], pb.F, pb.n_unique, &av, &th);
  a_out[m] = (uint16_t)av;
  th_out[m] = th;
  f_out[m] = pb.fit[b];
}

int launch_fill(deoct_ctx* ctx, int32_t* p, int64_t n, int32_t v, cudaStream_t s) {
  if (n <= 0) return DEOCT_OK;
  fill_i32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, n, v);
  count_launch(ctx);
  return check_launch("fill_i32_kernel");
}

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// host-pinned upload of a small array, ordered on the stream (the staging
// buffer is reused only after the stream has drained it)
template <typename T>
int upload(deoct_ctx* ctx, int slot, const std::vector<T>& host, T** dev, cudaStream_t s) {
  const size_t bytes = sizeof(T) * std::max<size_t>(1, host.size());
  DEOCT_TRY(scratch_get(ctx, slot, bytes, (void**)dev));
  if (host.empty()) return DEOCT_OK;
  DEOCT_CUDA_TRY(cudaStreamSynchronize(s));
  void* h = nullptr;
  DEOCT_TRY(pinned_get(ctx, bytes, &h));
  memcpy(h, host.data(), sizeof(T) * host.size());
  DEOCT_CUDA_TRY(cudaMemcpyAsync(*dev, h, sizeof(T) * host.size(), cudaMemcpyHostToDevice, s));
  DEOCT_CUDA_TRY(cudaStreamSynchronize(s));
  return DEOCT_OK;
}

template <typename T>
int download(deoct_ctx* ctx, const T* dev, size_t count, std::vector<T>* host, cudaStream_t s) {
  host->resize(count);
  if (count == 0) return DEOCT_OK;
  void* h = nullptr;
  DEOCT_TRY(pinned_get(ctx, sizeof(T) * count, &h));
  DEOCT_CUDA_TRY(cudaMemcpyAsync(h, dev, sizeof(T) * count, cudaMemcpyDeviceToHost, s));
  DEOCT_CUDA_TRY(cudaStreamSynchronize(s));
  memcpy(host->data(), h, sizeof(T) * count);
  return DEOCT_OK;
}

// A compacted set of node segments on the device.
struct Compacted {
  void* cranks = nullptr;   // [F][npad]
  uint8_t* clabels = nullptr;
  int32_t* idx = nullptr;
  int32_t* pos_slot = nullptr;
  int64_t npad = 0;
  std::vector<int64_t> seg_off, counts;
};

// Gather the samples listed in idx (already filled, -1 = padding) into the
// compacted rank rows and labels.
int gather_compacted(deoct_ctx* ctx, const deoct_dataset* ds, Compacted* c, cudaStream_t s,
                     int slot_ranks = SL_MH_RANKS, int slot_labels = SL_MH_LABELS) {
  const int W = ds->rank_bytes;
  DEOCT_TRY(scratch_get(ctx, slot_ranks, (size_t)ds->F * c->npad * W, &c->cranks));
  DEOCT_TRY(scratch_get(ctx, slot_labels, (size_t)c->npad, (void**)&c->clabels));
  dim3 g((unsigned)((c->npad + 255) / 256), ds->F);
  if (W == 2)
    gather_kernel<uint16_t><<<g, 256, 0, s>>>(static_cast<const uint16_t*>(ds->ranks), ds->ld, ds->labels,
                                              c->idx, c->npad, static_cast<uint16_t*>(c->cranks), c->npad,
                                              c->clabels);
  else
    gather_kernel<uint32_t><<<g, 256, 0, s>>>(static_cast<const uint32_t*>(ds->ranks), ds->ld, ds->labels,
                                              c->idx, c->npad, static_cast<uint32_t*>(c->cranks), c->npad,
                                              c->clabels);
  count_launch(ctx);
  return check_launch("gather_kernel");
}

// view of one segment as a dataset (16-sample aligned: TMA-able)
deoct_dataset segment_view(const deoct_dataset* ds, const Compacted& c, int m) {
  deoct_dataset v = *ds;
  v.ranks = static_cast<const unsigned char*>(c.cranks) + c.seg_off[m] * ds->rank_bytes;
  v.ld = c.npad;
  v.labels = c.clabels + c.seg_off[m];
  v.n = c.counts[m];
  return v;
}

// exhaustive depth-1 search for the segments [m0, m1) of a compacted set
int depth1_segments(deoct_ctx* ctx, const deoct_dataset* ds, const Compacted& c, int m0, int m1,
                    int n_min, double alpha, std::vector<uint16_t>* a, std::vector<uint32_t>* th,
                    std::vector<double>* f, cudaStream_t s) {
  const int F = ds->F, K = ds->K, W = ds->rank_bytes;
  const int64_t npad = c.npad;
  const int M = m1 - m0;
  uint32_t *k0, *k1, *v0, *v1, *tot, *bth;
  double* bf;
  int64_t *rs, *cn;
  DEOCT_TRY(scratch_get(ctx, SL_MH_D1KEYS, sizeof(uint32_t) * F * npad, (void**)&k0));
  DEOCT_TRY(scratch_get(ctx, SL_MH_D1VALS, sizeof(uint32_t) * F * npad, (void**)&v0));
  DEOCT_TRY(scratch_get(ctx, SL_MH_D1K1, sizeof(uint32_t) * F * npad, (void**)&k1));
  DEOCT_TRY(scratch_get(ctx, SL_MH_D1V1, sizeof(uint32_t) * F * npad, (void**)&v1));
  // per-slot class totals of all slots
  const int Mall = (int)c.counts.size();
  DEOCT_TRY(scratch_get(ctx, SL_MH_STATS, sizeof(uint32_t) * (size_t)Mall * K, (void**)&tot));
  DEOCT_CUDA_TRY(cudaMemsetAsync(tot, 0, sizeof(uint32_t) * (size_t)Mall * K, s));
  seg_hist_kernel<<<(unsigned)((npad + 255) / 256), 256, 0, s>>>(c.clabels, c.pos_slot, npad, K, tot);
  count_launch(ctx);
  DEOCT_TRY(check_launch("seg_hist_kernel"));
  const int kBatch = 255;
  a->resize(M);
  th->resize(M);
  f->resize(M);
  for (int b0 = m0; b0 < m1; b0 += kBatch) {
    const int b1 = std::min(m1, b0 + kBatch);
    const int Mb = b1 - b0;
    std::vector<int64_t> run_start(Mb), counts(Mb);
    int64_t acc = 0;
    for (int m = 0; m < Mb; ++m) {
      run_start[m] = acc;
      counts[m] = c.counts[b0 + m];
      acc += counts[m];
    }
    DEOCT_TRY(upload(ctx, SL_MH_SEG, run_start, &rs, s));
    DEOCT_TRY(upload(ctx, SL_MH_CURSOR, counts, &cn, s));
    dim3 g((unsigned)((npad + 255) / 256), F);
    if (W == 2)
      d1_keys_kernel<uint16_t><<<g, 256, 0, s>>>(static_cast<const uint16_t*>(c.cranks), npad, c.clabels,
                                                 c.pos_slot, npad, b0, b1, k0, v0);
    else
      d1_keys_kernel<uint32_t><<<g, 256, 0, s>>>(static_cast<const uint32_t*>(c.cranks), npad, c.clabels,
                                                 c.pos_slot, npad, b0, b1, k0, v0);
    count_launch(ctx);
    DEOCT_TRY(check_launch("d1_keys_kernel"));
    uint32_t *ks, *vs;
    DEOCT_TRY(radix_sort_segments(ctx, k0, v0, k1, v1, npad, F, 32, &ks, &vs, s));
    DEOCT_TRY(scratch_get(ctx, SL_MH_D1BEST, (sizeof(double) + sizeof(uint32_t)) * Mb * F + 64,
                          (void**)&bf));
    bth = reinterpret_cast<uint32_t*>(bf + (size_t)Mb * F);
    int NT = 256;
    while (NT > 32 && (size_t)NT * K * 4 > 96 * 1024) NT -= 32;
    const size_t sm = (size_t)NT * K * 4;
    DEOCT_TRY(set_max_dynamic_smem(ctx, d1_sweep_kernel));
    d1_sweep_kernel<<<dim3(Mb, F), NT, sm, s>>>(ks, vs, npad, rs, cn, tot + (size_t)b0 * K, K,
                                                ds->n_unique, n_min, alpha, F, bf, bth);
    count_launch(ctx);
    DEOCT_TRY(check_launch("d1_sweep_kernel"));
    unsigned char* dres;
    DEOCT_TRY(scratch_get(ctx, SL_D1_RESULT, (size_t)Mb * 16 + 64, (void**)&dres));
    double* df = reinterpret_cast<double*>(dres);
    uint32_t* dth = reinterpret_cast<uint32_t*>(dres + (size_t)Mb * 8);
    uint16_t* da = reinterpret_cast<uint16_t*>(dres + (size_t)Mb * 12);
    d1_reduce_kernel<<<(Mb + 127) / 128, 128, 0, s>>>(bf, bth, Mb, F, cn, tot + (size_t)b0 * K, K, n_min,
                                                      da, dth, df);
    count_launch(ctx);
    DEOCT_TRY(check_launch("d1_reduce_kernel"));
    std::vector<double> hf;
    std::vector<uint32_t> hth;
    std::vector<uint16_t> ha;
    DEOCT_TRY(download(ctx, df, Mb, &hf, s));
    DEOCT_TRY(download(ctx, dth, Mb, &hth, s));
    DEOCT_TRY(download(ctx, da, Mb, &ha, s));
    for (int m = 0; m < Mb; ++m) {
      (*a)[b0 - m0 + m] = ha[m];
      (*th)[b0 - m0 + m] = hth[m];
      (*f)[b0 - m0 + m] = hf[m];
    }
  }
  return DEOCT_OK;
}

// evaluator plan for the segments of a compacted set (one problem per node)
struct BatchedEval {
  std::vector<EvalProb> probs;
  std::vector<int> pops;
  EvalPlan plan;
};

int build_plan(deoct_ctx* ctx, BatchedEval* be, const EvalConfig& cfg, int F, int K, int P,
               cudaStream_t s) {
  std::vector<int64_t> counts(be->probs.size());
  int64_t mx = 0;
  for (size_t m = 0; m < be->probs.size(); ++m) {
    counts[m] = be->probs[m].count;
    mx = std::max(mx, counts[m]);
  }
  std::vector<EvalJob> jobs;
  int64_t total = 0;
  eval_build_jobs(counts, be->pops, cfg.S, cfg.TG, &jobs, &total);
  EvalJob* dj = nullptr;
  DEOCT_TRY(upload(ctx, SL_EVAL_JOBS, jobs, &dj, s));
  be->plan.d_jobs = dj;
  be->plan.njobs = (int)jobs.size();
  be->plan.total_tiles = total;
  be->plan.Fmax = F;
  be->plan.Kmax = K;
  be->plan.Pmax = P;
  be->plan.max_count = mx;
  if (!be->probs.empty()) {  // every segment reads the one compacted rank array
    be->plan.shared_ranks = be->probs[0].ranks;
    be->plan.shared_ld = be->probs[0].ld;
    be->plan.shared_ncols = be->probs[0].ncols;
  }
  return DEOCT_OK;
}

// root node (a, theta) and fitness of each problem's best individual -> host
int extract_roots(deoct_ctx* ctx, const DEProb* ddp, int M, int B, std::vector<uint16_t>* ra,
                  std::vector<uint32_t>* rth, std::vector<double>* rf, cudaStream_t s) {
  unsigned char* dres;
  DEOCT_TRY(scratch_get(ctx, SL_D1_RESULT, (size_t)M * 16 + 64, (void**)&dres));
  double* df = reinterpret_cast<double*>(dres);
  uint32_t* dth = reinterpret_cast<uint32_t*>(dres + (size_t)M * 8);
  uint16_t* da = reinterpret_cast<uint16_t*>(dres + (size_t)M * 12);
  extract_roots_kernel<<<(M + 127) / 128, 128, 0, s>>>(ddp, M, B, da, dth, df);
  count_launch(ctx);
  DEOCT_TRY(check_launch("extract_roots_kernel"));
  DEOCT_TRY(download(ctx, df, M, rf, s));
  DEOCT_TRY(download(ctx, dth, M, rth, s));
  DEOCT_TRY(download(ctx, da, M, ra, s));
  return DEOCT_OK;
}

int64_t nsum_of(const Compacted& c, int M) {
  int64_t t = 0;
  for (int m = 0; m < M; ++m) t += c.counts[m];
  return t;
}

uint64_t tune_key(int W, int D, int F, int K, int P, int64_t npad, int M) {
  auto lg = [](int64_t x) {
    int r = 0;
    while ((int64_t(1) << r) < x) ++r;
    return (uint64_t)r;
  };
  return ((uint64_t)W << 60) ^ ((uint64_t)D << 54) ^ ((uint64_t)F << 45) ^ ((uint64_t)K << 37) ^
         ((uint64_t)lg(P) << 32) ^ (lg(npad) << 24) ^ (lg(M) << 16);
}

// Batched DEOCT for all segments of a level: one evaluator launch and one DE
// step launch per generation, replayed from a captured CUDA graph.
int de_batched(deoct_ctx* ctx, const deoct_dataset* ds, const Compacted& c,
               const std::vector<int>& node_ids, int Dt, const deoct_params* prm,
               const float* d_seeds, int S, std::vector<uint16_t>* ra, std::vector<uint32_t>* rth,
               std::vector<double>* rf, cudaStream_t s) {
  const int M = (int)node_ids.size();
  const int P = prm->pop, B = (1 << Dt) - 1, L = 1 << Dt, m2 = 2 * B, K = ds->K, F = ds->F;
  const int W = ds->rank_bytes;
  // per-problem DE state, one block of device memory
  const size_t per = (size_t)P * m2 * 4 * 2 + (size_t)P * 8 * 2 + 16 + (size_t)P * B * 4 +
                     (size_t)P * L * K * 4;
  unsigned char* blk = nullptr;
  DEOCT_TRY(scratch_get(ctx, SL_MH_POP, per * M + 256 * (size_t)M, (void**)&blk));
  std::vector<DEProb> dp(M);
  BatchedEval be;
  be.probs.resize(M);
  be.pops.assign(M, P);
  for (int m = 0; m < M; ++m) {
    unsigned char* q = blk + (per + 256) * m;
    auto take = [&](size_t bytes) {
      unsigned char* r = q;
      q += (bytes + 15) & ~size_t(15);
      return r;
    };
    DEProb& d = dp[m];
    memset(&d, 0, sizeof(d));
    d.pop = reinterpret_cast<float*>(take((size_t)P * m2 * 4));
    d.trial = reinterpret_cast<float*>(take((size_t)P * m2 * 4));
    d.fit = reinterpret_cast<double*>(take((size_t)P * 8));
    d.fit_trial = reinterpret_cast<double*>(take((size_t)P * 8));
    d.best = reinterpret_cast<int32_t*>(take(4));
    d.gen = reinterpret_cast<int32_t*>(take(4));
    d.nodes = reinterpret_cast<uint32_t*>(take((size_t)P * B * 4));
    d.counts = reinterpret_cast<uint32_t*>(take((size_t)P * L * K * 4));
    d.n_unique = ds->n_unique;
    d.seeds = (d_seeds && S > 0) ? d_seeds + (size_t)m * S * m2 : nullptr;
    d.n_valid = c.counts[m];
    d.seed = prm->seed;
    d.stream_id = (uint64_t)node_ids[m];
    d.G = prm->gens;
    d.S = d.seeds ? S : 0;
    d.F = F;
    d.K = K;
    EvalProb& e = be.probs[m];
    e.ranks = c.cranks;
    e.labels = c.clabels;
    e.idx = nullptr;
    e.nodes = d.nodes;
    e.counts = d.counts;
    e.ld = c.npad;
    e.ncols = c.npad;
    e.start = c.seg_off[m];
    e.count = c.counts[m];
    e.F = F;
    e.K = K;
    e.P = P;
    e.tma = 1;
    e.lab_tma = (reinterpret_cast<uintptr_t>(c.clabels + e.start) % 16 == 0) ? 1 : 0;
  }
  DEProb* ddp = nullptr;
  EvalProb* dep = nullptr;
  DEOCT_TRY(upload(ctx, SL_DE_PROBS, dp, &ddp, s));
  DEOCT_TRY(upload(ctx, SL_EVAL_PROBS, be.probs, &dep, s));
  be.plan.d_probs = dep;
  DEArgs a;
  memset(&a, 0, sizeof(a));
  a.probs = ddp;
  a.nprob = M;
  a.P = P;
  a.depth = Dt;
  a.M = prm->mut_f;
  a.CR = prm->cr;
  a.alpha = prm->alpha;
  a.n_min = prm->n_min;
  a.dither = (prm->flags & DEOCT_DITHER_M) ? 1 : 0;
  a.Kmax = K;
  a.status = ctx->d_status;
  DEOCT_TRY(de_launch_init(ctx, a, s));

  if (ctx->engine) {
    // S^1 and the first trials here, then the G generations in the engine's
    // launches shared with other jobs
    EvalConfig cfg = eval_choose_config(ctx, W, Dt, F, K, P, std::max<int64_t>(1, nsum_of(c, M)), M);
    DEOCT_TRY(build_plan(ctx, &be, cfg, F, K, P, s));
    DEOCT_TRY(eval_launch(ctx, W, Dt, be.plan, cfg, s));
    DEOCT_TRY(de_launch_step(ctx, a, 0, DE_FIRST | DE_GEN_DEVICE | (prm->gens >= 1 ? DE_TRIAL : 0), s));
    DEOCT_CUDA_TRY(cudaStreamSynchronize(s));
    if (prm->gens >= 1) DEOCT_TRY(engine_generations(ctx->engine, ctx, W, Dt, a, prm->gens, dp, be.probs));
    return extract_roots(ctx, ddp, M, B, ra, rth, rf, s);
  }

  // ---- evaluator shape: autotuned once per workload class -------------------
  int64_t nsum = 0;
  for (int m = 0; m < M; ++m) nsum += c.counts[m];
  const uint64_t key = tune_key(W, Dt, F, K, P, c.npad, M);
  EvalConfig cfg = eval_choose_config(ctx, W, Dt, F, K, P, std::max<int64_t>(1, nsum / M), M);
  bool have = false;
  for (auto& kv : ctx->tuned)
    if (kv.first == key) {
      cfg.S = kv.second[0];
      cfg.TG = kv.second[1];
      cfg.warps = kv.second[2];
      cfg.stream = kv.second[3];
      have = true;
    }
  const bool forced = ctx->force_S || ctx->force_TG || ctx->force_warps || ctx->force_grid || ctx->force_stream;
  // timing some twenty candidate shapes three times each costs a few milliseconds,
  // which pays only on levels whose G + 1 evaluations are much longer than that:
  // from 2e10 tree-sample evaluations (~20 ms on GB300) on; smaller levels take the
  // chooser's shape
  const bool worth = (double)nsum * P * (prm->gens + 1) >= 2e10;
  if (!have && !forced && worth) {
    // candidates around the heuristic; each runs the real evaluation of S^1
    std::vector<EvalConfig> cands{cfg};  // the heuristic's own shape first
    for (int S : {256, 512, 1024, 2048})
      for (int TG : {cfg.TG, std::max(1, cfg.TG / 2), P}) {
        EvalConfig x = cfg;
        x.S = S;
        x.TG = std::min(TG, P);
        // ballot counting: a warp owns a tree (small groups split a tree's chunk
        // pairs over warps); shared atomics: warps split a tree's chunks
        x.warps = 16;
        bool dup = false;
        for (const EvalConfig& o : cands) dup = dup || (o.S == x.S && o.TG == x.TG && o.warps == x.warps);
        if (!dup) cands.push_back(x);
      }
    if (nsum >= 100000) {
      // large levels: the last wave of tiles leaves CTAs idle (up to 10% of a
      // uint32 launch at n = 1e6), so tile sizes between the powers of two join,
      // with 16 warps (one or two CTAs per SM) and 32 (one CTA): for each warp
      // count the two of least modelled makespan -- waves of tiles over the
      // resident CTAs, a wave costing its CTAs per SM x (S + 200) -- are timed
      for (int warps : {16, 32}) {
        std::vector<std::pair<double, EvalConfig>> model;
        for (int S = 256; S <= 2048; S += 128) {
          EvalConfig x = cfg;
          x.S = S;
          x.TG = std::min(cfg.TG, P);
          x.warps = warps;
          const int per_sm = eval_ctas_per_sm(ctx, W, Dt, F, K, x);
          if (per_sm < 1) continue;
          int64_t tiles = 0;
          for (int m = 0; m < M; ++m) tiles += (c.counts[m] + S - 1) / S;
          tiles *= (P + x.TG - 1) / x.TG;
          const int64_t slots = (int64_t)per_sm * ctx->num_sms;
          const double waves = (double)((tiles + slots - 1) / slots);
          model.push_back({waves * per_sm * (S + 200.0), x});
        }
        std::sort(model.begin(), model.end(),
                  [](const std::pair<double, EvalConfig>& u, const std::pair<double, EvalConfig>& v) {
                    return u.first < v.first;
                  });
        for (size_t i = 0; i < model.size() && i < 2; ++i) {
          const EvalConfig& x = model[i].second;
          bool dup = false;
          for (const EvalConfig& o : cands) dup = dup || (o.S == x.S && o.TG == x.TG && o.warps == x.warps);
          if (!dup) cands.push_back(x);
        }
      }
    }

    cudaEvent_t e0, e1;
    DEOCT_CUDA_TRY(cudaEventCreate(&e0));
    DEOCT_CUDA_TRY(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    EvalConfig best = cfg;
    const int saved_timing = ctx->timing;
    ctx->timing = 0;
    // the best of three timings per candidate: a single cold launch misranked
    // shapes that differ by a few percent (measured on GB300)
    for (const EvalConfig& x : cands) {
      DEOCT_TRY(build_plan(ctx, &be, x, F, K, P, s));
      float ms_x = 1e30f;
      bool ok = true;
      for (int rep = 0; rep < 3 && ok; ++rep) {
        for (int m = 0; m < M; ++m)
          DEOCT_CUDA_TRY(cudaMemsetAsync(dp[m].counts, 0, (size_t)P * L * K * 4, s));
        DEOCT_CUDA_TRY(cudaEventRecord(e0, s));
        int rc = eval_launch(ctx, W, Dt, be.plan, x, s);
        DEOCT_CUDA_TRY(cudaEventRecord(e1, s));
        if (rc != DEOCT_OK) {
          clear_error();
          cudaGetLastError();
          ok = false;
          break;
        }
        DEOCT_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0;
        DEOCT_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        ms_x = std::min(ms_x, ms);
      }
      if (ok && ms_x < best_ms) {
        best_ms = ms_x;
        best = x;
      }
    }
    ctx->timing = saved_timing;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cfg = best;
    ctx->tuned.push_back({key, {cfg.S, cfg.TG, cfg.warps, cfg.stream}});
    for (int m = 0; m < M; ++m)
      DEOCT_CUDA_TRY(cudaMemsetAsync(dp[m].counts, 0, (size_t)P * L * K * 4, s));
  }
  DEOCT_TRY(build_plan(ctx, &be, cfg, F, K, P, s));

  // ---- S^1, then G generations from one captured graph ---------------------
  DEOCT_TRY(eval_launch(ctx, W, Dt, be.plan, cfg, s));
  DEOCT_TRY(de_launch_step(ctx, a, 0, DE_FIRST | DE_GEN_DEVICE | (prm->gens >= 1 ? DE_TRIAL : 0), s));
  if (prm->gens >= 1) {
    if (!ctx->cap_stream)
      DEOCT_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const uint64_t l0 = ctx->launches, e0n = ctx->eval_launches;
    DEOCT_CUDA_TRY(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = eval_launch(ctx, W, Dt, be.plan, cfg, ctx->cap_stream);
    if (rc == DEOCT_OK)
      rc = de_launch_step(ctx, a, 0, DE_SELECT | DE_TRIAL | DE_GEN_DEVICE, ctx->cap_stream);
    cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &graph);
    if (rc != DEOCT_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ce != cudaSuccess)
      return set_error(DEOCT_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
    const uint64_t per_launch = ctx->launches - l0, per_eval = ctx->eval_launches - e0n;
    ctx->launches = l0;
    ctx->eval_launches = e0n;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    if (ce != cudaSuccess) {
      cudaGraphDestroy(graph);
      return set_error(DEOCT_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(ce));
    }
    for (int g = 1; g <= prm->gens; ++g) {
      ce = cudaGraphLaunch(exec, s);
      if (ce != cudaSuccess) break;
      ctx->launches += per_launch;
      ctx->eval_launches += per_eval;
    }
    cudaError_t ce2 = cudaStreamSynchronize(s);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return set_error(DEOCT_ERR_CUDA, "graph launch failed: %s", cudaGetErrorString(ce));
    if (ce2 != cudaSuccess) return set_error(DEOCT_ERR_CUDA, "generation loop failed: %s", cudaGetErrorString(ce2));
  }
  return extract_roots(ctx, ddp, M, B, ra, rth, rf, s);
}

// Plain form: one DEOCT (own launches) per node segment.
int de_plain(deoct_ctx* ctx, const deoct_dataset* ds, const Compacted& c,
             const std::vector<int>& node_ids, int Dt, const deoct_params* prm, const float* d_seeds,
             int S, std::vector<uint16_t>* ra, std::vector<uint32_t>* rth, std::vector<double>* rf,
             cudaStream_t s) {
  const int M = (int)node_ids.size();
  const int P = prm->pop, B = (1 << Dt) - 1;
  deoct_params dp = *prm;
  dp.depth = Dt;
  float* pop;
  double* fit;
  int32_t* best;
  DEOCT_TRY(scratch_get(ctx, SL_POP, (size_t)P * 2 * B * 4, (void**)&pop));
  DEOCT_TRY(scratch_get(ctx, SL_FIT, (size_t)P * 8, (void**)&fit));
  DEOCT_TRY(scratch_get(ctx, SL_BEST, 64, (void**)&best));
  unsigned char* dres;
  DEOCT_TRY(scratch_get(ctx, SL_D1_RESULT, (size_t)B * 6 + 64, (void**)&dres));
  double* df = reinterpret_cast<double*>(dres);
  uint32_t* dth = reinterpret_cast<uint32_t*>(dres + 8);
  uint16_t* da = reinterpret_cast<uint16_t*>(dres + 8 + (size_t)B * 4);
  ra->resize(M);
  rth->resize(M);
  rf->resize(M);
  for (int m = 0; m < M; ++m) {
    deoct_dataset v = segment_view(ds, c, m);
    const float* sd = (d_seeds && S > 0) ? d_seeds + (size_t)m * S * 2 * B : nullptr;
    DEOCT_TRY(run_deoct(ctx, &v, nullptr, v.n, &dp, (uint64_t)node_ids[m], sd, sd ? S : 0, pop, fit,
                        best, s));
    DEOCT_TRY(launch_best_extract(ctx, pop, fit, best, Dt, ds->F, ds->n_unique, da, dth, df, s));
    std::vector<double> hf;
    std::vector<uint32_t> hth;
    std::vector<uint16_t> ha;
    DEOCT_TRY(download(ctx, df, 1, &hf, s));
    DEOCT_TRY(download(ctx, dth, 1, &hth, s));
    DEOCT_TRY(download(ctx, da, 1, &ha, s));
    (*ra)[m] = ha[0];
    (*rth)[m] = hth[0];
    (*rf)[m] = hf[0];
  }
  return DEOCT_OK;
}

// ---- CART warm starts: greedy misclassification subtrees of every segment ----

// class histogram of (segment, subtree node) at one subtree depth
__global__ void sub_hist_kernel(const int32_t* __restrict__ pos_slot, const int32_t* __restrict__ sub_of,
                                const uint8_t* __restrict__ clabels, int64_t npad, int32_t base,
                                int32_t nsub, int K, uint32_t* __restrict__ hist) {
  int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= npad) return;
  const int m = pos_slot[pos];
  if (m < 0) return;
  const int k = sub_of[pos] - base;
  const int y = clabels[pos];
  if (k < 0 || k >= nsub || y >= K) return;
  atomicAdd(&hist[((int64_t)m * nsub + k) * K + y], 1u);
}

// positions of solved (segment, subtree node) pairs -> a new compacted set
__global__ void sub_compact_kernel(const int32_t* __restrict__ pos_slot, const int32_t* __restrict__ sub_of,
                                   const int32_t* __restrict__ idx, int64_t npad, int32_t base, int32_t nsub,
                                   const int32_t* __restrict__ slot2_of, const int64_t* __restrict__ seg_off2,
                                   int32_t* __restrict__ cursor2, int32_t* __restrict__ idx2,
                                   int32_t* __restrict__ pos_slot2) {
  int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int m2 = -1;
  if (pos < npad) {
    const int m = pos_slot[pos];
    if (m >= 0) {
      const int k = sub_of[pos] - base;
      if (k >= 0 && k < nsub) m2 = slot2_of[(int64_t)m * nsub + k];
    }
  }
  const int lane = threadIdx.x & 31;
  const uint32_t peers = __match_any_sync(0xFFFFFFFFu, m2);
  const int leader = __ffs(peers) - 1;
  int basepos = 0;
  if (m2 >= 0 && lane == leader) basepos = atomicAdd(&cursor2[m2], __popc(peers));
  basepos = __shfl_sync(0xFFFFFFFFu, basepos, leader);
  if (m2 >= 0) {
    const int64_t p2 = seg_off2[m2] + basepos + __popc(peers & ((1u << lane) - 1u));
    idx2[p2] = idx[pos];
    pos_slot2[p2] = m2;
  }
}

// one subtree level down inside every segment
template <typename RT>
__global__ void sub_route_kernel(const int32_t* __restrict__ pos_slot, int32_t* __restrict__ sub_of,
                                 const int32_t* __restrict__ idx, const RT* __restrict__ ranks, int64_t ld,
                                 int64_t npad, int32_t base, int32_t nsub,
                                 const uint32_t* __restrict__ packed) {
  int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= npad) return;
  const int m = pos_slot[pos];
  if (m < 0) return;
  const int t = sub_of[pos];
  const int k = t - base;
  if (k < 0 || k >= nsub) return;
  const uint32_t pk = packed[(int64_t)m * nsub + k];
  const uint32_t f = pk >> 24, th = pk & kThetaMask;
  const uint32_t r = ranks[(int64_t)f * ld + idx[pos]];
  sub_of[pos] = 2 * t + (r < th ? 0 : 1);
}

// genes of one decoded node: ahat = a + 1/2; bhat = the float32 nearest to
// (theta + 1/2) / (n_p + 1), nudged until floor(bhat (n_p + 1)) = theta
void encode_node_genes(int a, uint32_t theta, uint32_t np, float* ahat, float* bhat) {
  *ahat = (float)a + 0.5f;
  if (a == 0) {
    *bhat = 0.0f;
    return;
  }
  const double np1 = (double)np + 1.0;
  float b = (float)(((double)theta + 0.5) / np1);
  for (int it = 0; it < 64 && std::floor((double)b * np1) > (double)theta; ++it) b = std::nextafter(b, 0.0f);
  for (int it = 0; it < 64 && std::floor((double)b * np1) < (double)theta; ++it) b = std::nextafter(b, 1.0f);
  *bhat = b;
}

// Greedy depth-Dt subtree of every segment of c (CART warm starts of
// Algorithm 2): per subtree depth r, solved (segment, node) pairs get the
// exhaustive depth-1 split of their samples.  Result: genes [M][2B] (device).
int greedy_seeds(deoct_ctx* ctx, const deoct_dataset* ds, const Compacted& c, int Dt,
                 const deoct_params* prm, std::vector<float>* out_genes, cudaStream_t s) {
  const int M = (int)c.counts.size();
  const int B = (1 << Dt) - 1, K = ds->K;
  int32_t* sub_of;
  DEOCT_TRY(scratch_get(ctx, SL_MH_SUB, sizeof(int32_t) * c.npad, (void**)&sub_of));
  DEOCT_TRY(launch_fill(ctx, sub_of, c.npad, 1, s));
  std::vector<int> ga((size_t)M * B, 0);
  std::vector<uint32_t> gth((size_t)M * B, 0);
  for (int r = 0; r < Dt; ++r) {
    const int base = 1 << r, nsub = 1 << r;
    uint32_t* hist;
    const size_t hb = sizeof(uint32_t) * (size_t)M * nsub * K;
    DEOCT_TRY(scratch_get(ctx, SL_MH_SUBHIST, hb, (void**)&hist));
    DEOCT_CUDA_TRY(cudaMemsetAsync(hist, 0, hb, s));
    sub_hist_kernel<<<(unsigned)((c.npad + 255) / 256), 256, 0, s>>>(c.pos_slot, sub_of, c.clabels, c.npad,
                                                                     base, nsub, K, hist);
    count_launch(ctx);
    DEOCT_TRY(check_launch("sub_hist_kernel"));
    std::vector<uint32_t> hh;
    DEOCT_TRY(download(ctx, hist, (size_t)M * nsub * K, &hh, s));
    Compacted c2;
    std::vector<int32_t> slot2((size_t)M * nsub, -1);
    std::vector<int> pair_of;
    int64_t off = 0;
    for (int m = 0; m < M; ++m)
      for (int k = 0; k < nsub; ++k) {
        int64_t nt = 0;
        int ncls = 0;
        for (int y = 0; y < K; ++y) {
          const uint32_t v = hh[((size_t)m * nsub + k) * K + y];
          nt += v;
          ncls += v > 0 ? 1 : 0;
        }
        if (nt > prm->n_min && ncls > 1) {
          slot2[(size_t)m * nsub + k] = (int32_t)pair_of.size();
          pair_of.push_back(m * nsub + k);
          c2.seg_off.push_back(off);
          c2.counts.push_back(nt);
          off += round_up(nt, kSegAlign);
        }
      }
    std::vector<uint32_t> packed((size_t)M * nsub, 0);
    if (!pair_of.empty()) {
      c2.npad = std::max<int64_t>(off, kSegAlign);
      const int M2 = (int)pair_of.size();
      int32_t *dslot2, *dcur;
      int64_t* dseg2;
      DEOCT_TRY(upload(ctx, SL_MH_SEG, slot2, &dslot2, s));
      DEOCT_TRY(upload(ctx, SL_MH_STATS, c2.seg_off, &dseg2, s));
      DEOCT_TRY(scratch_get(ctx, SL_MH_CURSOR, sizeof(int32_t) * M2, (void**)&dcur));
      DEOCT_CUDA_TRY(cudaMemsetAsync(dcur, 0, sizeof(int32_t) * M2, s));
      DEOCT_TRY(scratch_get(ctx, SL_MH_IDX2, sizeof(int32_t) * c2.npad, (void**)&c2.idx));
      DEOCT_TRY(scratch_get(ctx, SL_MH_POS2, sizeof(int32_t) * c2.npad, (void**)&c2.pos_slot));
      DEOCT_TRY(launch_fill(ctx, c2.idx, c2.npad, -1, s));
      DEOCT_TRY(launch_fill(ctx, c2.pos_slot, c2.npad, -1, s));
      sub_compact_kernel<<<(unsigned)((c.npad + 255) / 256), 256, 0, s>>>(
          c.pos_slot, sub_of, c.idx, c.npad, base, nsub, dslot2, dseg2, dcur, c2.idx, c2.pos_slot);
      count_launch(ctx);
      DEOCT_TRY(check_launch("sub_compact_kernel"));
      DEOCT_TRY(gather_compacted(ctx, ds, &c2, s, SL_MH_RANKS2, SL_MH_LABELS2));
      std::vector<uint16_t> ra;
      std::vector<uint32_t> rth;
      std::vector<double> rf;
      DEOCT_TRY(depth1_segments(ctx, ds, c2, 0, M2, prm->n_min, prm->alpha, &ra, &rth, &rf, s));
      for (int j = 0; j < M2; ++j) {
        const int m = pair_of[j] / nsub, k = pair_of[j] % nsub;
        const int t = base + k;  // subtree node (1-based)
        ga[(size_t)m * B + t - 1] = ra[j];
        gth[(size_t)m * B + t - 1] = rth[j];
        packed[pair_of[j]] = ra[j] == 0 ? 0u : ((uint32_t)(ra[j] - 1) << 24) | (rth[j] & kThetaMask);
      }
    }
    if (r + 1 < Dt) {
      uint32_t* dpk;
      DEOCT_TRY(upload(ctx, SL_MH_CURSOR, packed, &dpk, s));
      const unsigned grid = (unsigned)((c.npad + 255) / 256);
      if (ds->rank_bytes == 2)
        sub_route_kernel<uint16_t><<<grid, 256, 0, s>>>(c.pos_slot, sub_of, c.idx,
                                                       static_cast<const uint16_t*>(ds->ranks), ds->ld,
                                                       c.npad, base, nsub, dpk);
      else
        sub_route_kernel<uint32_t><<<grid, 256, 0, s>>>(c.pos_slot, sub_of, c.idx,
                                                       static_cast<const uint32_t*>(ds->ranks), ds->ld,
                                                       c.npad, base, nsub, dpk);
      count_launch(ctx);
      DEOCT_TRY(check_launch("sub_route_kernel"));
    }
  }
  // genes of the greedy subtrees
  std::vector<uint32_t> nu;
  DEOCT_TRY(download(ctx, ds->n_unique, (size_t)ds->F, &nu, s));
  std::vector<float> genes((size_t)M * 2 * B);
  for (int m = 0; m < M; ++m)
    for (int t = 0; t < B; ++t) {
      const int a = ga[(size_t)m * B + t];
      const uint32_t th = gth[(size_t)m * B + t];
      encode_node_genes(a, th, a > 0 ? nu[a - 1] : 1u, &genes[(size_t)m * 2 * B + t],
                        &genes[(size_t)m * 2 * B + B + t]);
    }
  *out_genes = std::move(genes);
  return DEOCT_OK;
}

int launch_route(deoct_ctx* ctx, const deoct_dataset* ds, int32_t* node_of, int32_t base, int32_t nn,
                 const uint32_t* lvl, cudaStream_t s) {
  const unsigned grid = (unsigned)((ds->n + 255) / 256);
  if (ds->rank_bytes == 2)
    route_level_kernel<uint16_t><<<grid, 256, 0, s>>>(node_of, static_cast<const uint16_t*>(ds->ranks),
                                                      ds->ld, ds->n, base, nn, lvl);
  else
    route_level_kernel<uint32_t><<<grid, 256, 0, s>>>(node_of, static_cast<const uint32_t*>(ds->ranks),
                                                      ds->ld, ds->n, base, nn, lvl);
  count_launch(ctx);
  return check_launch("route_level_kernel");
}

int launch_level_hist(deoct_ctx* ctx, const deoct_dataset* ds, const int32_t* node_of, int32_t base,
                      int32_t nn, uint32_t* hist, cudaStream_t s) {
  const int bins = nn * ds->K;
  DEOCT_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * bins, s));
  const int use_smem = bins <= 12288 ? 1 : 0;
  int grid = (int)std::min<int64_t>((ds->n + 255) / 256, (int64_t)ctx->num_sms * 4);
  level_hist_kernel<<<grid, 256, use_smem ? bins * 4 : 0, s>>>(node_of, ds->labels, ds->n, base, nn,
                                                               ds->K, use_smem, hist);
  count_launch(ctx);
  return check_launch("level_hist_kernel");
}

}  // namespace

// Algorithm 2, level by level.
int mh_run(deoct_ctx* ctx, const deoct_dataset* ds, const deoct_params* prm, uint16_t* a_out,
           uint32_t* th_out, uint8_t* leaf_class_out, int32_t* kind_out, double* node_fit_out,
           cudaStream_t s) {
  const int D = prm->depth, H = prm->horizon, K = ds->K;
  const int B = (1 << D) - 1, Lf = 1 << D;
  const bool batched = (prm->flags & DEOCT_BATCHED) != 0;
  const int64_t n = ds->n;
  std::vector<uint16_t> a(B, 0);
  std::vector<uint32_t> th(B, 0);
  std::vector<int32_t> kind(B, 0);
  std::vector<double> nf(B, 0.0);
  int32_t* node_of;
  uint32_t* hist;
  DEOCT_TRY(scratch_get(ctx, SL_MH_NODEOF, sizeof(int32_t) * n, (void**)&node_of));
  DEOCT_TRY(scratch_get(ctx, SL_MH_HOSTBUF, sizeof(uint32_t) * (size_t)(2 * Lf) * K + 64, (void**)&hist));
  DEOCT_TRY(launch_fill(ctx, node_of, n, 1, s));
  // DEOCT warm start (Algorithm 2): one DEOCT of the full depth on the whole set
  std::vector<int> full_a;
  std::vector<uint32_t> full_th, nu_host;
  DEOCT_TRY(download(ctx, ds->n_unique, (size_t)ds->F, &nu_host, s));
  if ((prm->flags & DEOCT_DE_SEEDS) && D >= 2 && H >= 2) {
    deoct_params fp = *prm;
    fp.depth = D;
    float* pop;
    double* fit;
    int32_t* best;
    DEOCT_TRY(scratch_get(ctx, SL_POP, (size_t)prm->pop * 2 * B * 4, (void**)&pop));
    DEOCT_TRY(scratch_get(ctx, SL_FIT, (size_t)prm->pop * 8, (void**)&fit));
    DEOCT_TRY(scratch_get(ctx, SL_BEST, 64, (void**)&best));
    DEOCT_TRY(run_deoct(ctx, ds, nullptr, n, &fp, 0, nullptr, 0, pop, fit, best, s));
    unsigned char* dres;
    DEOCT_TRY(scratch_get(ctx, SL_D1_RESULT, (size_t)B * 6 + 64, (void**)&dres));
    double* df = reinterpret_cast<double*>(dres);
    uint32_t* dth = reinterpret_cast<uint32_t*>(dres + 8);
    uint16_t* da = reinterpret_cast<uint16_t*>(dres + 8 + (size_t)B * 4);
    DEOCT_TRY(launch_best_extract(ctx, pop, fit, best, D, ds->F, ds->n_unique, da, dth, df, s));
    std::vector<uint16_t> ha;
    DEOCT_TRY(download(ctx, dth, (size_t)B, &full_th, s));
    DEOCT_TRY(download(ctx, da, (size_t)B, &ha, s));
    full_a.assign(ha.begin(), ha.end());
  }
  const int64_t npad_max = round_up(n + (int64_t)kSegAlign * (Lf / 2), 64);
  Compacted c;
  DEOCT_TRY(scratch_get(ctx, SL_MH_IDX, sizeof(int32_t) * npad_max, (void**)&c.idx));
  DEOCT_TRY(scratch_get(ctx, SL_MISC, sizeof(int32_t) * npad_max, (void**)&c.pos_slot));
  for (int d = 0; d < D; ++d) {
    const int base = 1 << d, nn = 1 << d;
    DEOCT_TRY(launch_level_hist(ctx, ds, node_of, base, nn, hist, s));
    std::vector<uint32_t> hh;
    DEOCT_TRY(download(ctx, hist, (size_t)nn * K, &hh, s));
    std::vector<int32_t> slot_of(nn, -1);
    std::vector<int> solved;
    c.seg_off.clear();
    c.counts.clear();
    int64_t off = 0;
    for (int k = 0; k < nn; ++k) {
      int64_t nt = 0;
      int ncls = 0;
      for (int y = 0; y < K; ++y) {
        nt += hh[(size_t)k * K + y];
        ncls += hh[(size_t)k * K + y] > 0 ? 1 : 0;
      }
      if (nt > prm->n_min && ncls > 1) {  // Algorithm 2: |X_t| > n_min and >= 2 classes
        slot_of[k] = (int32_t)solved.size();
        solved.push_back(base + k);
        c.seg_off.push_back(off);
        c.counts.push_back(nt);
        off += round_up(nt, kSegAlign);
      }
    }
    const int M = (int)solved.size();
    if (M > 0) {
      c.npad = std::max<int64_t>(off, kSegAlign);
      const int Dt = std::min(H, D - d);
      int32_t* dslot;
      int64_t* dseg;
      int32_t* dcur;
      DEOCT_TRY(upload(ctx, SL_MH_SEG, slot_of, &dslot, s));
      DEOCT_TRY(upload(ctx, SL_MH_STATS, c.seg_off, &dseg, s));
      DEOCT_TRY(scratch_get(ctx, SL_MH_CURSOR, sizeof(int32_t) * M, (void**)&dcur));
      DEOCT_CUDA_TRY(cudaMemsetAsync(dcur, 0, sizeof(int32_t) * M, s));
      DEOCT_TRY(launch_fill(ctx, c.idx, c.npad, -1, s));
      DEOCT_TRY(launch_fill(ctx, c.pos_slot, c.npad, -1, s));
      compact_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(node_of, n, base, nn, dslot, dseg, dcur,
                                                                c.idx, c.pos_slot);
      count_launch(ctx);
      DEOCT_TRY(check_launch("compact_kernel"));
      DEOCT_TRY(gather_compacted(ctx, ds, &c, s));
      std::vector<uint16_t> ra;
      std::vector<uint32_t> rth;
      std::vector<double> rf;
      int kd;
      if (Dt >= 2) {
        kd = 2;
        // warm starts of Algorithm 2, per node in this order: the subtree of the
        // full-depth DEOCT at the node's location, then the greedy (CART) subtree
        const int Bt = (1 << Dt) - 1;
        const bool de_ws = !full_a.empty(), cart_ws = (prm->flags & DEOCT_CART_SEEDS) != 0;
        const int S = (de_ws ? 1 : 0) + (cart_ws ? 1 : 0);
        float* seeds = nullptr;
        if (S > 0) {
          std::vector<float> cart;
          if (cart_ws) DEOCT_TRY(greedy_seeds(ctx, ds, c, Dt, prm, &cart, s));
          std::vector<float> all((size_t)M * S * 2 * Bt);
          for (int m = 0; m < M; ++m) {
            float* dst = &all[(size_t)m * S * 2 * Bt];
            if (de_ws) {
              const int t = solved[m];
              for (int r = 0, q = 0; r < Dt; ++r)
                for (int j = 0; j < (1 << r); ++j, ++q) {
                  const int gt = (t << r) + j;  // global BFS index of subtree node q + 1
                  const int av = full_a[gt - 1];
                  encode_node_genes(av, full_th[gt - 1], av > 0 ? nu_host[av - 1] : 1u, &dst[q],
                                    &dst[Bt + q]);
                }
              dst += 2 * Bt;
            }
            if (cart_ws) memcpy(dst, &cart[(size_t)m * 2 * Bt], sizeof(float) * 2 * Bt);
          }
          DEOCT_TRY(upload(ctx, SL_MH_SEEDS, all, &seeds, s));
        }
        if (batched) DEOCT_TRY(de_batched(ctx, ds, c, solved, Dt, prm, seeds, S, &ra, &rth, &rf, s));
        else DEOCT_TRY(de_plain(ctx, ds, c, solved, Dt, prm, seeds, S, &ra, &rth, &rf, s));
      } else {
        kd = 1;
        if (batched) {
          DEOCT_TRY(depth1_segments(ctx, ds, c, 0, M, prm->n_min, prm->alpha, &ra, &rth, &rf, s));
        } else {
          ra.resize(M);
          rth.resize(M);
          rf.resize(M);
          for (int m = 0; m < M; ++m) {
            std::vector<uint16_t> a1;
            std::vector<uint32_t> t1;
            std::vector<double> f1;
            DEOCT_TRY(depth1_segments(ctx, ds, c, m, m + 1, prm->n_min, prm->alpha, &a1, &t1, &f1, s));
            ra[m] = a1[0];
            rth[m] = t1[0];
            rf[m] = f1[0];
          }
        }
      }
      for (int m = 0; m < M; ++m) {
        const int t = solved[m];
        a[t - 1] = ra[m];
        th[t - 1] = rth[m];
        nf[t - 1] = rf[m];
        kind[t - 1] = kd;
      }
    }
    // move every sample one level down
    std::vector<uint32_t> lvl(nn);
    for (int k = 0; k < nn; ++k) {
      const int t = base + k;
      lvl[k] = a[t - 1] == 0 ? 0u : ((uint32_t)(a[t - 1] - 1) << 24) | (th[t - 1] & kThetaMask);
    }
    uint32_t* dl;
    DEOCT_TRY(upload(ctx, SL_MH_CURSOR, lvl, &dl, s));
    DEOCT_TRY(launch_route(ctx, ds, node_of, base, nn, dl, s));
  }
  // leaf classes (Eq. opt_c): histogram of the leaves, lowest class on ties
  DEOCT_TRY(launch_level_hist(ctx, ds, node_of, Lf, Lf, hist, s));
  std::vector<uint32_t> hh;
  DEOCT_TRY(download(ctx, hist, (size_t)Lf * K, &hh, s));
  DEOCT_TRY(check_status(ctx, s));
  for (int l = 0; l < Lf; ++l) {
    int bk = 0;
    for (int k = 1; k < K; ++k)
      if (hh[(size_t)l * K + k] > hh[(size_t)l * K + bk]) bk = k;
    leaf_class_out[l] = (uint8_t)bk;
  }
  memcpy(a_out, a.data(), sizeof(uint16_t) * B);
  memcpy(th_out, th.data(), sizeof(uint32_t) * B);
  if (kind_out) memcpy(kind_out, kind.data(), sizeof(int32_t) * B);
  if (node_fit_out) memcpy(node_fit_out, nf.data(), sizeof(double) * B);
  return DEOCT_OK;
}

// The largest request of every scratch slot on the path of deoct_encode_auto
// (or deoct_encode of width W) followed by deoct_fit_moving_horizon on an n x F
// set; mirrors the allocation sites above and in encode.cu.  A context that
// holds have[s] bytes in slot s grows it to need + need / 8 (scratch_get's
// headroom) when need > have[s]; with ctx == nullptr every slot starts empty.
size_t fit_scratch_bound(const deoct_ctx* ctx, int64_t n, int F, int K, int W, const deoct_params* prm) {
  std::vector<size_t> slot(SL_COUNT, 0);
  auto need = [&](int sl, double bytes) { slot[sl] = std::max(slot[sl], (size_t)bytes); };
  const int D = prm->depth, H = std::max(1, prm->horizon), P = std::max(prm->pop, 1);
  const int Lf = 1 << D, nn = Lf / 2;  // at most 2^(D-1) nodes on a level
  const double nF = (double)n * F;
  const int64_t tiles = (n + 2047) / 2048;
  // encoder
  for (int sl : {SL_ENC_K0, SL_ENC_K1, SL_ENC_V0, SL_ENC_V1}) need(sl, 4.0 * nF);
  need(SL_ENC_TILE, 4.0 * F * tiles);
  need(SL_ENC_HIST, 4.0 * F * 256 * tiles);
  need(SL_ENC_TOT, 4.0 * F * 256);
  // moving horizon: level state and compacted segments
  const int64_t npad = round_up(n + (int64_t)kSegAlign * nn, 64);
  const int64_t ptiles = (npad + 2047) / 2048;
  need(SL_MH_NODEOF, 4.0 * n);
  need(SL_MH_HOSTBUF, 4.0 * 2 * Lf * K + 64);
  need(SL_MH_IDX, 4.0 * npad);
  need(SL_MISC, std::max(4.0 * npad, 8.0 + 6.0 * (Lf - 1) + 80));
  need(SL_MH_RANKS, (double)F * npad * W);
  need(SL_MH_LABELS, (double)npad);
  for (int sl : {SL_MH_D1KEYS, SL_MH_D1VALS, SL_MH_D1K1, SL_MH_D1V1}) need(sl, 4.0 * F * npad);
  need(SL_ENC_HIST, 4.0 * F * 256 * ptiles);
  // DEOCT subproblems of a level (subtree depth <= min(horizon, D)); the greedy
  // warm starts work on (node, subtree node) pairs: at most nn * L / 2 of them
  const int Dt = std::min(H, D), B = (1 << Dt) - 1, L = 1 << Dt;
  const double pairs = (double)nn * std::max(1, L / 2);
  need(SL_MH_STATS, std::max(8.0 * pairs, 4.0 * pairs * K));
  need(SL_MH_SEG, std::max(4.0 * pairs, 8.0 * 255));
  need(SL_MH_CURSOR, std::max(4.0 * pairs, 8.0 * 255));
  need(SL_MH_D1BEST, 12.0 * 255 * F + 64);
  need(SL_D1_RESULT, std::max(16.0 * std::max<double>(pairs, 255) + 64, 6.0 * (Lf - 1) + 64));
  const double per = (double)P * 2 * B * 4 * 2 + (double)P * 8 * 2 + 16 + (double)P * B * 4 +
                     (double)P * L * K * 4 + 6 * 15 + 256;
  need(SL_MH_POP, per * nn);
  need(SL_DE_PROBS, (double)sizeof(DEProb) * nn);
  need(SL_EVAL_PROBS, (double)sizeof(EvalProb) * nn);
  need(SL_EVAL_JOBS, (double)sizeof(EvalJob) * nn * (P + 1) * std::max<int64_t>(1, 1 + n / 128 / nn));
  // plain form and warm starts: one DEOCT's buffers, the seeds, the greedy subtrees
  const int Bf = Lf - 1;
  need(SL_POP, 4.0 * P * 2 * Bf);
  need(SL_FIT, 8.0 * P);
  need(SL_BEST, 64);
  need(SL_POP_TRIAL, 4.0 * P * 2 * Bf);
  need(SL_FIT_TRIAL, 8.0 * P);
  need(SL_NODES, 4.0 * P * Bf);
  need(SL_COUNTS, 4.0 * P * Lf * K);
  need(SL_GEN, 4);
  need(SL_DE_PART, kDePartBytes);
  need(SL_MH_SEEDS, 4.0 * 2 * nn * 2 * B);
  need(SL_MH_SUB, 4.0 * npad);
  need(SL_MH_SUBHIST, 4.0 * pairs * K);
  need(SL_MH_IDX2, 4.0 * npad);
  need(SL_MH_POS2, 4.0 * npad);
  need(SL_MH_RANKS2, (double)F * npad * W);
  need(SL_MH_LABELS2, (double)npad);
  size_t total = 0;
  for (int i = 0; i < SL_COUNT; ++i) {
    const size_t have = ctx ? ctx->scratch[i].bytes : 0;
    if (slot[i] > have) total += slot[i] + slot[i] / 8 - have;
  }
  return total;
}

// exhaustive depth-1 search on one sample subset
int depth1_run(deoct_ctx* ctx, const deoct_dataset* ds, const int32_t* sample_idx, int64_t n_sub,
               int n_min, double alpha, uint16_t* a_out, uint32_t* th_out, double* f_out,
               cudaStream_t s) {
  Compacted c;
  c.npad = round_up(std::max<int64_t>(n_sub, 1), kSegAlign);
  c.seg_off = {0};
  c.counts = {n_sub};
  DEOCT_TRY(scratch_get(ctx, SL_MH_IDX, sizeof(int32_t) * c.npad, (void**)&c.idx));
  DEOCT_TRY(scratch_get(ctx, SL_MISC, sizeof(int32_t) * c.npad, (void**)&c.pos_slot));
  DEOCT_TRY(launch_fill(ctx, c.idx, c.npad, -1, s));
  DEOCT_TRY(launch_fill(ctx, c.pos_slot, c.npad, -1, s));
  if (n_sub > 0) {
    if (sample_idx) {
      DEOCT_CUDA_TRY(cudaMemcpyAsync(c.idx, sample_idx, sizeof(int32_t) * n_sub, cudaMemcpyDeviceToDevice, s));
    } else {
      std::vector<int32_t> iota(n_sub);
      for (int64_t i = 0; i < n_sub; ++i) iota[i] = (int32_t)i;
      int32_t* tmp;
      DEOCT_TRY(upload(ctx, SL_MH_SEG, iota, &tmp, s));
      DEOCT_CUDA_TRY(cudaMemcpyAsync(c.idx, tmp, sizeof(int32_t) * n_sub, cudaMemcpyDeviceToDevice, s));
    }
    DEOCT_TRY(launch_fill(ctx, c.pos_slot, n_sub, 0, s));
  }
  DEOCT_TRY(gather_compacted(ctx, ds, &c, s));
  std::vector<uint16_t> a;
  std::vector<uint32_t> th;
  std::vector<double> f;
  DEOCT_TRY(depth1_segments(ctx, ds, c, 0, 1, n_min, alpha, &a, &th, &f, s));
  DEOCT_TRY(check_status(ctx, s));
  *a_out = a[0];
  *th_out = th[0];
  *f_out = f[0];
  return DEOCT_OK;
}

}  // namespace deoct
