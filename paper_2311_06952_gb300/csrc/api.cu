// api.cu -- the C ABI of include/deoct.h: context, validation, and the host
// orchestration of encoder, evaluator and DE kernels on the caller's stream.
#include <cstring>
#include <string>

#include "internal.cuh"

namespace deoct {

static thread_local std::string g_last_error;

int set_error(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}
void clear_error() { g_last_error.clear(); }

int check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return set_error(DEOCT_ERR_CUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
  return DEOCT_OK;
}

int scratch_get(deoct_ctx* ctx, int slot, size_t bytes, void** out) {
  Scratch& s = ctx->scratch[slot];
  if (bytes == 0) bytes = 16;
  if (s.bytes < bytes) {
    size_t want = bytes + bytes / 8;  // headroom against repeated growth
    if (ctx->scratch_limit) {  // the buffer's growth must keep the total within the limit
      size_t others = 0;
      for (int i = 0; i < SL_COUNT; ++i)
        if (i != slot) others += ctx->scratch[i].bytes;
      if (others + bytes > ctx->scratch_limit)
        return set_error(DEOCT_ERR_OOM,
                         "scratch of %zu bytes would pass the context's limit of %zu bytes (%zu held "
                         "in other buffers)", bytes, (size_t)ctx->scratch_limit, others);
      want = std::min(want, (size_t)ctx->scratch_limit - others);
    }
    if (s.ptr) {
      DEOCT_CUDA_TRY(cudaFree(s.ptr));  // synchronises the device: no pending use
      s.ptr = nullptr;
      s.bytes = 0;
    }
    cudaError_t e = cudaMalloc(&s.ptr, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      s.ptr = nullptr;
      return set_error(DEOCT_ERR_OOM, "scratch allocation of %zu bytes failed: %s", want,
                       cudaGetErrorString(e));
    }
    s.bytes = want;
  }
  *out = s.ptr;
  return DEOCT_OK;
}

int pinned_get(deoct_ctx* ctx, size_t bytes, void** out) {
  if (ctx->h_pinned_bytes < bytes) {
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    ctx->h_pinned = nullptr;
    ctx->h_pinned_bytes = 0;
    DEOCT_CUDA_TRY(cudaMallocHost(&ctx->h_pinned, bytes));
    ctx->h_pinned_bytes = bytes;
  }
  *out = ctx->h_pinned;
  return DEOCT_OK;
}

int check_status(deoct_ctx* ctx, cudaStream_t stream) {
  int st = 0;
  DEOCT_CUDA_TRY(cudaMemcpyAsync(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, stream));
  DEOCT_CUDA_TRY(cudaStreamSynchronize(stream));
  if (st == 0) return DEOCT_OK;
  DEOCT_CUDA_TRY(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), stream));
  DEOCT_CUDA_TRY(cudaStreamSynchronize(stream));
  if (st & ST_TIMEOUT) return set_error(DEOCT_ERR_TIMEOUT, "a bounded device wait expired");
  if (st & ST_NAN) return set_error(DEOCT_ERR_INVALID, "NaN in the feature matrix");
  if (st & ST_BAD_NODE) return set_error(DEOCT_ERR_INVALID, "a tree names a feature > F");
  if (st & ST_BAD_INDEX) return set_error(DEOCT_ERR_INVALID, "a sample index is out of range");
  return set_error(DEOCT_ERR_CUDA, "device status 0x%x", st);
}

int validate_dataset(const deoct_dataset* ds) {
  if (!ds) return set_error(DEOCT_ERR_INVALID, "dataset is NULL");
  if (!ds->ranks || !ds->n_unique || !ds->labels)
    return set_error(DEOCT_ERR_INVALID, "dataset pointers must not be NULL");
  if (ds->rank_bytes != 2 && ds->rank_bytes != 4)
    return set_error(DEOCT_ERR_INVALID, "rank_bytes must be 2 or 4 (got %d)", ds->rank_bytes);
  if (ds->n < 1 || ds->n > kMaxN)
    return set_error(DEOCT_ERR_INVALID, "n = %lld outside 1..2^24", (long long)ds->n);
  if (ds->ld < ds->n) return set_error(DEOCT_ERR_INVALID, "ld < n");
  if (ds->F < 1 || ds->F > kMaxF) return set_error(DEOCT_ERR_INVALID, "F = %d outside 1..256", ds->F);
  if (ds->K < 1 || ds->K > kMaxK) return set_error(DEOCT_ERR_INVALID, "K = %d outside 1..255", ds->K);
  return DEOCT_OK;
}

static int validate_subset(const deoct_dataset* ds, const int32_t* idx, int64_t n_sub) {
  if (idx == nullptr && n_sub != ds->n)
    return set_error(DEOCT_ERR_INVALID, "without sample_idx n_sub must equal n");
  if (n_sub < 0 || n_sub > kMaxN) return set_error(DEOCT_ERR_INVALID, "n_sub out of range");
  return DEOCT_OK;
}

static int validate_params(const deoct_params* p, bool need_pop) {
  if (!p) return set_error(DEOCT_ERR_INVALID, "params is NULL");
  if (p->depth < 1 || p->depth > kMaxDepth)
    return set_error(DEOCT_ERR_INVALID, "depth %d outside 1..%d", p->depth, kMaxDepth);
  if (need_pop && (p->pop < kMinPop || p->pop > kMaxPop))
    return set_error(DEOCT_ERR_INVALID, "population %d outside %d..%d", p->pop, kMinPop, kMaxPop);
  if (p->gens < 0) return set_error(DEOCT_ERR_INVALID, "gens < 0");
  if (p->n_min < 0) return set_error(DEOCT_ERR_INVALID, "n_min < 0");
  if (!(p->cr >= 0.0f && p->cr <= 1.0f)) return set_error(DEOCT_ERR_INVALID, "cr outside [0,1]");
  if (!(p->mut_f == p->mut_f)) return set_error(DEOCT_ERR_INVALID, "mut_f is NaN");
  if (!(p->alpha == p->alpha)) return set_error(DEOCT_ERR_INVALID, "alpha is NaN");
  return DEOCT_OK;
}

EvalPlan single_eval_plan(const deoct_dataset* ds, const int32_t* idx, int64_t n_sub,
                          const uint32_t* nodes, uint32_t* counts, int P, const EvalConfig& cfg) {
  EvalPlan plan;
  EvalProb& p = plan.single;
  p.ranks = ds->ranks;
  p.labels = ds->labels;
  p.idx = idx;
  p.nodes = nodes;
  p.counts = counts;
  p.ld = ds->ld;
  p.ncols = ds->n;
  p.start = 0;
  p.count = n_sub;
  p.F = ds->F;
  p.K = ds->K;
  p.P = P;
  const bool aligned = (reinterpret_cast<uintptr_t>(ds->ranks) % 16 == 0) &&
                       ((ds->ld * ds->rank_bytes) % 16 == 0);
  p.tma = (idx == nullptr && aligned) ? 1 : 0;
  p.lab_tma = (p.tma && reinterpret_cast<uintptr_t>(ds->labels) % 16 == 0) ? 1 : 0;
  plan.total_tiles = ((n_sub + cfg.S - 1) / cfg.S) * (int64_t)((P + cfg.TG - 1) / cfg.TG);
  plan.Fmax = ds->F;
  plan.Kmax = ds->K;
  plan.Pmax = P;
  plan.max_count = n_sub;
  return plan;
}

// evaluate one population on one (sub)set: counts must be zero beforehand
static int eval_single(deoct_ctx* ctx, const deoct_dataset* ds, const int32_t* idx, int64_t n_sub,
                       const uint32_t* nodes, uint32_t* counts, int P, int depth,
                       cudaStream_t s) {
  if (n_sub == 0) return DEOCT_OK;
  EvalConfig cfg = eval_choose_config(ctx, ds->rank_bytes, depth, ds->F, ds->K, P, n_sub, 1);
  EvalPlan plan = single_eval_plan(ds, idx, n_sub, nodes, counts, P, cfg);
  return eval_launch(ctx, ds->rank_bytes, depth, plan, cfg, s);
}

// One evaluation of caller-given trees in a single launch: the evaluator packs
// the trees while building its node tables and its last CTA writes errors and
// counts (see EvalPlan::ticket).  The accumulator slot is zero at rest: it is
// zeroed when (re)allocated and by every launch that used it.
static int eval_single_fused(deoct_ctx* ctx, const deoct_dataset* ds, const int32_t* idx,
                             int64_t n_sub, const uint16_t* a, const uint32_t* theta, int P,
                             int depth, uint32_t* counts_out, uint32_t* errors_out,
                             cudaStream_t s) {
  const size_t L = (size_t)1 << depth;
  const size_t bytes = 16 + sizeof(uint32_t) * (size_t)P * L * ds->K;
  const bool grows = ctx->scratch[SL_EVAL_ACC].bytes < bytes;
  uint32_t* base = nullptr;
  DEOCT_TRY(scratch_get(ctx, SL_EVAL_ACC, bytes, (void**)&base));
  if (grows) DEOCT_CUDA_TRY(cudaMemsetAsync(base, 0, ctx->scratch[SL_EVAL_ACC].bytes, s));
  EvalConfig cfg = eval_choose_config(ctx, ds->rank_bytes, depth, ds->F, ds->K, P, n_sub, 1);
  EvalPlan plan = single_eval_plan(ds, idx, n_sub, nullptr, base + 4, P, cfg);
  plan.single.a16 = a;
  plan.single.th32 = theta;
  plan.ticket = base;
  plan.counts_out = counts_out;
  plan.errors_out = errors_out;
  return eval_launch(ctx, ds->rank_bytes, depth, plan, cfg, s);
}

struct DEBuffers {
  float* trial;
  double* fit_trial;
  uint32_t* nodes;
  uint32_t* counts;
  int32_t* gen;
  unsigned char* part;  // kDePartBytes: the split step's argmin candidates and generation
};

static int de_buffers(deoct_ctx* ctx, const deoct_dataset* ds, const deoct_params* p, DEBuffers* b) {
  const size_t P = (size_t)p->pop, B = ((size_t)1 << p->depth) - 1, L = (size_t)1 << p->depth;
  DEOCT_TRY(scratch_get(ctx, SL_POP_TRIAL, P * 2 * B * sizeof(float), (void**)&b->trial));
  DEOCT_TRY(scratch_get(ctx, SL_FIT_TRIAL, P * sizeof(double), (void**)&b->fit_trial));
  DEOCT_TRY(scratch_get(ctx, SL_NODES, P * B * sizeof(uint32_t), (void**)&b->nodes));
  DEOCT_TRY(scratch_get(ctx, SL_COUNTS, P * L * ds->K * sizeof(uint32_t), (void**)&b->counts));
  DEOCT_TRY(scratch_get(ctx, SL_GEN, sizeof(int32_t), (void**)&b->gen));
  DEOCT_TRY(scratch_get(ctx, SL_DE_PART, kDePartBytes, (void**)&b->part));
  return DEOCT_OK;
}

static DEArgs de_args(const deoct_dataset* ds, const deoct_params* p, int64_t n_sub,
                      uint64_t stream_id, const DEBuffers& b, float* pop, double* fit,
                      int32_t* best, const float* seeds, int S, int* status) {
  DEArgs a;
  memset(&a, 0, sizeof(a));
  DEProb& d = a.single;
  d.pop = pop;
  d.trial = b.trial;
  d.fit = fit;
  d.fit_trial = b.fit_trial;
  d.best = best;
  d.gen = b.gen;
  d.nodes = b.nodes;
  d.counts = b.counts;
  d.n_unique = ds->n_unique;
  d.seeds = seeds;
  d.n_valid = n_sub;
  d.seed = p->seed;
  d.stream_id = stream_id;
  d.G = p->gens;
  d.S = S;
  d.F = ds->F;
  d.K = ds->K;
  a.probs = nullptr;
  a.nprob = 1;
  a.P = p->pop;
  a.depth = p->depth;
  a.M = p->mut_f;
  a.CR = p->cr;
  a.alpha = p->alpha;
  a.n_min = p->n_min;
  a.dither = (p->flags & DEOCT_DITHER_M) ? 1 : 0;
  a.Kmax = ds->K;
  a.status = status;
  const int nblk = kMaxPop / kDeWideR;
  a.part_f = reinterpret_cast<double*>(b.part);
  a.part_i = reinterpret_cast<int*>(b.part + sizeof(double) * nblk);
  a.part_g = reinterpret_cast<int*>(b.part + (sizeof(double) + sizeof(int)) * nblk);
  return a;
}

// Algorithm 4 on one (sub)problem, device-resident: S^1, then G generations.
int run_deoct(deoct_ctx* ctx, const deoct_dataset* ds, const int32_t* idx, int64_t n_sub,
              const deoct_params* p, uint64_t stream_id, const float* seeds, int S, float* pop,
              double* fit, int32_t* best, cudaStream_t s) {
  DEBuffers b;
  DEOCT_TRY(de_buffers(ctx, ds, p, &b));
  DEArgs a = de_args(ds, p, n_sub, stream_id, b, pop, fit, best, seeds, S, ctx->d_status);
  DEOCT_TRY(de_launch_init(ctx, a, s));
  DEOCT_TRY(eval_single(ctx, ds, idx, n_sub, b.nodes, b.counts, p->pop, p->depth, s));
  // The generation number lives on the device (set to 1 by the init kernel and
  // advanced by every trial step), so every generation is the same pair of
  // launches: captured once as a CUDA graph and replayed G times.  With
  // per-launch timing on, the launches are issued directly so that each
  // evaluator launch gets its own events.
  DEOCT_TRY(de_launch_step(ctx, a, 0, DE_FIRST | DE_GEN_DEVICE | (p->gens >= 1 ? DE_TRIAL : 0), s));
  if (p->gens < 1) return DEOCT_OK;
  if (ctx->timing || p->gens < 3) {
    for (int g = 1; g <= p->gens; ++g) {
      DEOCT_TRY(eval_single(ctx, ds, idx, n_sub, b.nodes, b.counts, p->pop, p->depth, s));
      DEOCT_TRY(de_launch_step(ctx, a, 0, DE_SELECT | DE_TRIAL | DE_GEN_DEVICE, s));
    }
    return DEOCT_OK;
  }
  if (!ctx->cap_stream)
    DEOCT_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  const uint64_t l0 = ctx->launches, e0 = ctx->eval_launches;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  DEOCT_CUDA_TRY(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = eval_single(ctx, ds, idx, n_sub, b.nodes, b.counts, p->pop, p->depth, ctx->cap_stream);
  if (rc == DEOCT_OK) rc = de_launch_step(ctx, a, 0, DE_SELECT | DE_TRIAL | DE_GEN_DEVICE, ctx->cap_stream);
  cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &graph);
  const uint64_t per_launch = ctx->launches - l0, per_eval = ctx->eval_launches - e0;
  ctx->launches = l0;
  ctx->eval_launches = e0;
  if (rc != DEOCT_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (ce != cudaSuccess) return set_error(DEOCT_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
  ce = cudaGraphInstantiate(&exec, graph, 0);
  if (ce != cudaSuccess) {
    cudaGraphDestroy(graph);
    return set_error(DEOCT_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(ce));
  }
  for (int g = 1; g <= p->gens && ce == cudaSuccess; ++g) {
    ce = cudaGraphLaunch(exec, s);
    ctx->launches += per_launch;
    ctx->eval_launches += per_eval;
  }
  // the graph may be destroyed once its launches are queued
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) return set_error(DEOCT_ERR_CUDA, "graph launch failed: %s", cudaGetErrorString(ce));
  return DEOCT_OK;
}

}  // namespace deoct

using namespace deoct;

#define API_BEGIN \
  clear_error();  \
  try {
#define API_END                                                          \
  }                                                                      \
  catch (const std::exception& e) {                                      \
    return set_error(DEOCT_ERR_INVALID, "internal exception: %s", e.what()); \
  }                                                                      \
  catch (...) {                                                          \
    return set_error(DEOCT_ERR_INVALID, "internal exception");           \
  }

#define CTX_CHECK(ctx)                                                            \
  do {                                                                            \
    if (!(ctx)) return set_error(DEOCT_ERR_INVALID, "context is NULL");           \
    DEOCT_CUDA_TRY(cudaSetDevice((ctx)->device));                                 \
  } while (0)

extern "C" {

const char* deoct_last_error_string(void) { return g_last_error.c_str(); }

const char* deoct_version(void) { return "deoct-gb300 0.1 (sm_103a)"; }

int deoct_create(deoct_ctx** out, int device) {
  API_BEGIN
  if (!out) return set_error(DEOCT_ERR_INVALID, "out is NULL");
  *out = nullptr;
  DEOCT_CUDA_TRY(cudaSetDevice(device));
  int major = 0, minor = 0;
  DEOCT_CUDA_TRY(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device));
  DEOCT_CUDA_TRY(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device));
  if (!(major == 10 && minor == 3))
    return set_error(DEOCT_ERR_CUDA, "libdeoct is built for sm_103a (GB300); device %d is sm_%d%d",
                     device, major, minor);
  deoct_ctx* ctx = new deoct_ctx();
  ctx->device = device;
  DEOCT_CUDA_TRY(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device));
  DEOCT_CUDA_TRY(
      cudaDeviceGetAttribute(&ctx->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  DEOCT_CUDA_TRY(
      cudaDeviceGetAttribute(&ctx->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device));
  cudaError_t e = cudaMalloc(&ctx->d_status, sizeof(int));
  if (e != cudaSuccess) {
    delete ctx;
    return set_error(DEOCT_ERR_OOM, "status word allocation failed: %s", cudaGetErrorString(e));
  }
  DEOCT_CUDA_TRY(cudaMemset(ctx->d_status, 0, sizeof(int)));
  *out = ctx;
  return DEOCT_OK;
  API_END
}

int deoct_destroy(deoct_ctx* ctx) {
  API_BEGIN
  if (!ctx) return DEOCT_OK;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (int i = 0; i < SL_COUNT; ++i)
    if (ctx->scratch[i].ptr) cudaFree(ctx->scratch[i].ptr);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
  for (cudaEvent_t ev : ctx->ev_pairs) cudaEventDestroy(ev);
  delete ctx;
  return DEOCT_OK;
  API_END
}

int deoct_set_timing(deoct_ctx* ctx, int enable) {
  API_BEGIN
  CTX_CHECK(ctx);
  ctx->timing = enable ? 1 : 0;
  return DEOCT_OK;
  API_END
}

int deoct_get_stats(deoct_ctx* ctx, deoct_stats* out) {
  API_BEGIN
  CTX_CHECK(ctx);
  if (!out) return set_error(DEOCT_ERR_INVALID, "out is NULL");
  for (size_t i = 0; i + 1 < ctx->ev_pairs.size(); i += 2) {
    DEOCT_CUDA_TRY(cudaEventSynchronize(ctx->ev_pairs[i + 1]));
    float ms = 0.0f;
    DEOCT_CUDA_TRY(cudaEventElapsedTime(&ms, ctx->ev_pairs[i], ctx->ev_pairs[i + 1]));
    ctx->eval_ms += ms;
    ctx->eval_timed += 1;
    cudaEventDestroy(ctx->ev_pairs[i]);
    cudaEventDestroy(ctx->ev_pairs[i + 1]);
  }
  ctx->ev_pairs.clear();
  out->launches = ctx->launches;
  out->eval_launches = ctx->eval_launches;
  out->eval_ms = ctx->eval_ms;
  out->eval_timed = ctx->eval_timed;
  return DEOCT_OK;
  API_END
}

int deoct_reset_stats(deoct_ctx* ctx) {
  API_BEGIN
  CTX_CHECK(ctx);
  for (cudaEvent_t ev : ctx->ev_pairs) cudaEventDestroy(ev);
  ctx->ev_pairs.clear();
  ctx->launches = 0;
  ctx->eval_launches = 0;
  ctx->eval_ms = 0.0;
  ctx->eval_timed = 0;
  return DEOCT_OK;
  API_END
}

int deoct_get_memory(deoct_ctx* ctx, uint64_t* device_bytes, uint64_t* pinned_bytes) {
  API_BEGIN
  if (!ctx) return set_error(DEOCT_ERR_INVALID, "context is NULL");
  uint64_t d = ctx->d_status ? sizeof(int) : 0;
  for (int i = 0; i < SL_COUNT; ++i) d += ctx->scratch[i].bytes;
  if (device_bytes) *device_bytes = d;
  if (pinned_bytes) *pinned_bytes = ctx->h_pinned_bytes;
  return DEOCT_OK;
  API_END
}

int deoct_set_scratch_limit(deoct_ctx* ctx, uint64_t bytes) {
  API_BEGIN
  CTX_CHECK(ctx);
  ctx->scratch_limit = bytes;
  return DEOCT_OK;
  API_END
}

int deoct_release_scratch(deoct_ctx* ctx) {
  API_BEGIN
  CTX_CHECK(ctx);
  for (int i = 0; i < SL_COUNT; ++i)
    if (ctx->scratch[i].ptr) {
      DEOCT_CUDA_TRY(cudaFree(ctx->scratch[i].ptr));  // synchronises the device
      ctx->scratch[i].ptr = nullptr;
      ctx->scratch[i].bytes = 0;
    }
  return DEOCT_OK;
  API_END
}

int deoct_fit_scratch_bound(const deoct_ctx* ctx, int64_t n, int32_t F, int32_t K, int32_t rank_bytes,
                            const deoct_params* params, uint64_t* bytes_out) {
  API_BEGIN
  if (!params || !bytes_out) return set_error(DEOCT_ERR_INVALID, "NULL argument");
  if (n < 1 || n > kMaxN || F < 1 || F > kMaxF || K < 1 || K > kMaxK)
    return set_error(DEOCT_ERR_INVALID, "bad n, F or K");
  if (rank_bytes != 0 && rank_bytes != 2 && rank_bytes != 4)
    return set_error(DEOCT_ERR_INVALID, "rank_bytes must be 0, 2 or 4");
  if (params->depth < 1 || params->depth > kMaxDepth) return set_error(DEOCT_ERR_INVALID, "bad depth");
  *bytes_out = (uint64_t)fit_scratch_bound(ctx, n, F, K, rank_bytes == 2 ? 2 : 4, params) +
               (ctx ? 0 : sizeof(int));
  return DEOCT_OK;
  API_END
}

int deoct_set_eval_config(deoct_ctx* ctx, int32_t S, int32_t TG, int32_t warps, int32_t grid) {
  API_BEGIN
  CTX_CHECK(ctx);
  if (S != 0 && (S < 128 || S > 8192 || S % 128 != 0))
    return set_error(DEOCT_ERR_INVALID, "S = %d: want a multiple of 128 in 128..8192", S);
  if (TG < 0 || TG > kMaxPop) return set_error(DEOCT_ERR_INVALID, "TG = %d out of range", TG);
  if (warps < 0 || warps > 32) return set_error(DEOCT_ERR_INVALID, "warps = %d out of range", warps);
  if (grid < 0) return set_error(DEOCT_ERR_INVALID, "grid < 0");
  ctx->force_S = S;
  ctx->force_TG = TG;
  ctx->force_warps = warps;
  ctx->force_grid = grid;
  return DEOCT_OK;
  API_END
}

int deoct_set_eval_streaming(deoct_ctx* ctx, int32_t on) {
  API_BEGIN
  CTX_CHECK(ctx);
  ctx->force_stream = on ? 1 : 0;
  return DEOCT_OK;
  API_END
}

namespace deoct {
namespace {
// One warp waits on an mbarrier that nothing arrives on: lane 0's bounded wait
// runs out and records ST_TIMEOUT.
__global__ void selftest_wait_kernel(uint32_t tries, int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncwarp();
  if (threadIdx.x == 0) mbar_wait_tries(&bar, 0u, tries, status);
  __syncwarp();
}
}  // namespace
}  // namespace deoct

int deoct_selftest_wait(deoct_ctx* ctx, int32_t tries, void* stream) {
  API_BEGIN
  CTX_CHECK(ctx);
  if (tries < 1 || tries > (1 << 20)) return set_error(DEOCT_ERR_INVALID, "tries = %d", tries);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  selftest_wait_kernel<<<1, 32, 0, s>>>((uint32_t)tries, ctx->d_status);
  count_launch(ctx);
  DEOCT_TRY(check_launch("selftest_wait_kernel"));
  return check_status(ctx, s);
  API_END
}

int deoct_encode(deoct_ctx* ctx, const float* X, int64_t n, int32_t F, int32_t rank_bytes,
                 void* ranks_out, int64_t ld, uint32_t* n_unique_out, void* stream) {
  return deoct_encode_ex(ctx, X, n, F, rank_bytes, ranks_out, ld, n_unique_out, nullptr, stream);
}

int deoct_encode_ex(deoct_ctx* ctx, const float* X, int64_t n, int32_t F, int32_t rank_bytes,
                    void* ranks_out, int64_t ld, uint32_t* n_unique_out, float* unique_out,
                    void* stream) {
  API_BEGIN
  CTX_CHECK(ctx);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!X || !ranks_out || !n_unique_out) return set_error(DEOCT_ERR_INVALID, "NULL pointer");
  if (n < 1 || n > kMaxN) return set_error(DEOCT_ERR_INVALID, "n = %lld outside 1..2^24", (long long)n);
  if (F < 1 || F > kMaxF) return set_error(DEOCT_ERR_INVALID, "F = %d outside 1..256", F);
  if (rank_bytes != 2 && rank_bytes != 4) return set_error(DEOCT_ERR_INVALID, "rank_bytes must be 2 or 4");
  if (ld < n) return set_error(DEOCT_ERR_INVALID, "ld < n");
  DEOCT_TRY(encode_run(ctx, X, n, F, rank_bytes, ranks_out, ld, n_unique_out, unique_out, s));
  DEOCT_TRY(check_status(ctx, s));
  if (rank_bytes == 2) {
    uint32_t* h = nullptr;
    DEOCT_TRY(pinned_get(ctx, sizeof(uint32_t) * F, (void**)&h));
    DEOCT_CUDA_TRY(cudaMemcpyAsync(h, n_unique_out, sizeof(uint32_t) * F, cudaMemcpyDeviceToHost, s));
    DEOCT_CUDA_TRY(cudaStreamSynchronize(s));
    for (int f = 0; f < F; ++f)
      if (h[f] > 65536u)
        return set_error(DEOCT_ERR_INVALID, "feature %d has %u distinct values: needs rank_bytes = 4",
                         f, h[f]);
  }
  return DEOCT_OK;
  API_END
}

int deoct_encode_auto(deoct_ctx* ctx, const float* X, int64_t n, int32_t F, void* ranks_out,
                      int64_t ld, uint32_t* n_unique_out, float* unique_out,
                      int32_t* rank_bytes_out, void* stream) {
  API_BEGIN
  CTX_CHECK(ctx);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!X || !ranks_out || !n_unique_out || !rank_bytes_out)
    return set_error(DEOCT_ERR_INVALID, "NULL pointer");
  if (n < 1 || n > kMaxN) return set_error(DEOCT_ERR_INVALID, "n = %lld outside 1..2^24", (long long)n);
  if (F < 1 || F > kMaxF) return set_error(DEOCT_ERR_INVALID, "F = %d outside 1..256", F);
  if (ld < n || ld % 8 != 0) return set_error(DEOCT_ERR_INVALID, "ld must be >= n and a multiple of 8");
  int W = 0;
  DEOCT_TRY(encode_run(ctx, X, n, F, 0, ranks_out, ld, n_unique_out, unique_out, s, &W));
  DEOCT_TRY(check_status(ctx, s));
  *rank_bytes_out = W;
  return DEOCT_OK;
  API_END
}

int deoct_split_values(deoct_ctx* ctx, const float* unique, int64_t ld, const uint16_t* a,
                       const uint32_t* theta, int32_t B, double* b_out, void* stream) {
  API_BEGIN
  CTX_CHECK(ctx);
  if (!unique || !a || !theta || !b_out) return set_error(DEOCT_ERR_INVALID, "NULL pointer");
  if (B < 1 || B > (1 << kMaxDepth) - 1) return set_error(DEOCT_ERR_INVALID, "B = %d out of range", B);
  if (ld < 1) return set_error(DEOCT_ERR_INVALID, "ld < 1");
  return launch_split_values(ctx, unique, ld, a, theta, B, b_out, static_cast<cudaStream_t>(stream));
  API_END
}

int deoct_predict(deoct_ctx* ctx, const float* X, int64_t m, int32_t F, const uint16_t* a,
                  const double* b, int32_t depth, const uint8_t* leaf_class, const uint8_t* y,
                  uint8_t* pred_out, uint64_t* correct_out, void* stream) {
  API_BEGIN
  CTX_CHECK(ctx);
  if (!X || !a || !b || !leaf_class) return set_error(DEOCT_ERR_INVALID, "NULL pointer");
  if (m < 0 || F < 1 || F > kMaxF) return set_error(DEOCT_ERR_INVALID, "bad m or F");
  if (depth < 1 || depth > kMaxDepth) return set_error(DEOCT_ERR_INVALID, "depth out of range");
  if (correct_out && !y) return set_error(DEOCT_ERR_INVALID, "correct_out needs labels y");
  return launch_predict(ctx, X, m, F, a, b, depth, leaf_class, y, pred_out,
                        reinterpret_cast<unsigned long long*>(correct_out),
                        static_cast<cudaStream_t>(stream));
  API_END
}

int deoct_decode_population(deoct_ctx* ctx, const deoct_dataset* ds, const float* genes, int32_t P,
                            int32_t depth, uint16_t* a_out, uint32_t* theta_out, void* stream) {
  API_BEGIN
  CTX_CHECK(ctx);
  DEOCT_TRY(validate_dataset(ds));
  if (!genes || !a_out || !theta_out) return set_error(DEOCT_ERR_INVALID, "NULL pointer");
  if (P < 0 || P > kMaxPop * 64) return set_error(DEOCT_ERR_INVALID, "P out of range");
  if (depth < 1 || depth > kMaxDepth) return set_error(DEOCT_ERR_INVALID, "depth out of range");
  return launch_decode(ctx, genes, P, depth, ds->F, ds->n_unique, a_out, theta_out,
                       static_cast<cudaStream_t>(stream));
  API_END
}

int deoct_eval_population(deoct_ctx* ctx, const deoct_dataset* ds, const int32_t* sample_idx,
                          int64_t n_sub, const uint16_t* a, const uint32_t* theta, int32_t P,
                          int32_t depth, uint32_t* counts_out, uint32_t* errors_out, void* stream) {
  API_BEGIN
  CTX_CHECK(ctx);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DEOCT_TRY(validate_dataset(ds));
  DEOCT_TRY(validate_subset(ds, sample_idx, n_sub));
  if (!a || !theta) return set_error(DEOCT_ERR_INVALID, "NULL tree arrays");
  if (P < 1 || P > kMaxPop * 64) return set_error(DEOCT_ERR_INVALID, "P = %d out of range", P);
  if (depth < 1 || depth > kMaxDepth) return set_error(DEOCT_ERR_INVALID, "depth out of range");
  const int B = (1 << depth) - 1, L = 1 << depth;
  if (n_sub > 0)
    return eval_single_fused(ctx, ds, sample_idx, n_sub, a, theta, P, depth, counts_out, errors_out, s);
  // empty set: the trees are still validated; counts and errors are zero
  uint32_t* nodes = nullptr;
  DEOCT_TRY(scratch_get(ctx, SL_PACKED, sizeof(uint32_t) * (size_t)P * B, (void**)&nodes));
  uint32_t* counts = counts_out;
  if (!counts) DEOCT_TRY(scratch_get(ctx, SL_COUNTS, sizeof(uint32_t) * (size_t)P * L * ds->K, (void**)&counts));
  DEOCT_TRY(launch_pack_nodes(ctx, a, theta, (int64_t)P * B, ds->F, nodes, s));
  DEOCT_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (size_t)P * L * ds->K, s));
  DEOCT_TRY(eval_single(ctx, ds, sample_idx, n_sub, nodes, counts, P, depth, s));
  if (errors_out) DEOCT_TRY(launch_errors(ctx, counts, P, L, ds->K, n_sub, errors_out, s));
  return DEOCT_OK;
  API_END
}

int deoct_de_init(deoct_ctx* ctx, const deoct_dataset* ds, const int32_t* sample_idx, int64_t n_sub,
                  const deoct_params* params, uint64_t stream_id, const float* seeds, int32_t S,
                  float* pop, double* fitness, int32_t* best, void* stream) {
  API_BEGIN
  CTX_CHECK(ctx);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DEOCT_TRY(validate_dataset(ds));
  DEOCT_TRY(validate_subset(ds, sample_idx, n_sub));
  DEOCT_TRY(validate_params(params, true));
  if (!pop || !fitness || !best) return set_error(DEOCT_ERR_INVALID, "NULL output");
  if (S < 0 || S > params->pop || (S > 0 && !seeds)) return set_error(DEOCT_ERR_INVALID, "bad seeds");
  DEBuffers b;
  DEOCT_TRY(de_buffers(ctx, ds, params, &b));
  DEArgs a = de_args(ds, params, n_sub, stream_id, b, pop, fitness, best, seeds, S, ctx->d_status);
  DEOCT_TRY(de_launch_init(ctx, a, s));
  DEOCT_TRY(eval_single(ctx, ds, sample_idx, n_sub, b.nodes, b.counts, params->pop, params->depth, s));
  return de_launch_step(ctx, a, 0, DE_FIRST, s);
  API_END
}

int deoct_de_step(deoct_ctx* ctx, const deoct_dataset* ds, const int32_t* sample_idx, int64_t n_sub,
                  const deoct_params* params, uint64_t stream_id, int32_t generation, float* pop,
                  double* fitness, int32_t* best, void* stream) {
  API_BEGIN
  CTX_CHECK(ctx);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DEOCT_TRY(validate_dataset(ds));
  DEOCT_TRY(validate_subset(ds, sample_idx, n_sub));
  DEOCT_TRY(validate_params(params, true));
  if (!pop || !fitness || !best) return set_error(DEOCT_ERR_INVALID, "NULL state");
  if (generation < 1) return set_error(DEOCT_ERR_INVALID, "generation must be >= 1");
  DEBuffers b;
  DEOCT_TRY(de_buffers(ctx, ds, params, &b));
  deoct_params p = *params;
  p.gens = generation;  // the trial kernel accepts g <= G
  DEArgs a = de_args(ds, &p, n_sub, stream_id, b, pop, fitness, best, nullptr, 0, ctx->d_status);
  DEOCT_TRY(de_launch_step(ctx, a, generation, DE_TRIAL, s));
  DEOCT_TRY(eval_single(ctx, ds, sample_idx, n_sub, b.nodes, b.counts, p.pop, p.depth, s));
  return de_launch_step(ctx, a, generation, DE_SELECT, s);
  API_END
}

int deoct_fit_subtree(deoct_ctx* ctx, const deoct_dataset* ds, const int32_t* sample_idx,
                      int64_t n_sub, const deoct_params* params, uint64_t stream_id,
                      const float* seeds, int32_t S, uint16_t* a_out, uint32_t* theta_out,
                      double* fitness_out, float* pop_out, void* stream) {
  API_BEGIN
  CTX_CHECK(ctx);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DEOCT_TRY(validate_dataset(ds));
  DEOCT_TRY(validate_subset(ds, sample_idx, n_sub));
  DEOCT_TRY(validate_params(params, true));
  if (!a_out || !theta_out || !fitness_out) return set_error(DEOCT_ERR_INVALID, "NULL host output");
  if (S < 0 || S > params->pop || (S > 0 && !seeds)) return set_error(DEOCT_ERR_INVALID, "bad seeds");
  const size_t P = (size_t)params->pop, B = ((size_t)1 << params->depth) - 1;
  float* pop = pop_out;
  if (!pop) DEOCT_TRY(scratch_get(ctx, SL_POP, P * 2 * B * sizeof(float), (void**)&pop));
  double* fit = nullptr;
  int32_t* best = nullptr;
  DEOCT_TRY(scratch_get(ctx, SL_FIT, P * sizeof(double), (void**)&fit));
  DEOCT_TRY(scratch_get(ctx, SL_BEST, 64, (void**)&best));
  DEOCT_TRY(run_deoct(ctx, ds, sample_idx, n_sub, params, stream_id, seeds, S, pop, fit, best, s));
  // decoded best tree -> host
  unsigned char* dres = nullptr;
  const size_t res_bytes = 8 + B * 2 + B * 4 + 16;
  DEOCT_TRY(scratch_get(ctx, SL_MISC, res_bytes + 64, (void**)&dres));
  double* d_fit = reinterpret_cast<double*>(dres);
  uint32_t* d_th = reinterpret_cast<uint32_t*>(dres + 8);
  uint16_t* d_a = reinterpret_cast<uint16_t*>(dres + 8 + B * 4);
  DEOCT_TRY(launch_best_extract(ctx, pop, fit, best, params->depth, ds->F, ds->n_unique, d_a, d_th,
                                d_fit, s));
  unsigned char* h = nullptr;
  DEOCT_TRY(pinned_get(ctx, res_bytes, (void**)&h));
  DEOCT_CUDA_TRY(cudaMemcpyAsync(h, dres, res_bytes, cudaMemcpyDeviceToHost, s));
  DEOCT_TRY(check_status(ctx, s));
  memcpy(fitness_out, h, 8);
  memcpy(theta_out, h + 8, B * 4);
  memcpy(a_out, h + 8 + B * 4, B * 2);
  return DEOCT_OK;
  API_END
}

int deoct_fit_moving_horizon(deoct_ctx* ctx, const deoct_dataset* ds, const deoct_params* params,
                             uint16_t* a_out, uint32_t* theta_out, uint8_t* leaf_class_out,
                             int32_t* kind_out, double* node_fit_out, void* stream) {
  API_BEGIN
  CTX_CHECK(ctx);
  DEOCT_TRY(validate_dataset(ds));
  DEOCT_TRY(validate_params(params, false));
  if (params->horizon < 1) return set_error(DEOCT_ERR_INVALID, "horizon must be >= 1");
  const bool needs_de = params->horizon >= 2 && params->depth >= 2;
  if (needs_de && (params->pop < kMinPop || params->pop > kMaxPop))
    return set_error(DEOCT_ERR_INVALID, "population %d outside %d..%d", params->pop, kMinPop, kMaxPop);
  if (!a_out || !theta_out || !leaf_class_out) return set_error(DEOCT_ERR_INVALID, "NULL host output");
  return mh_run(ctx, ds, params, a_out, theta_out, leaf_class_out, kind_out, node_fit_out,
                static_cast<cudaStream_t>(stream));
  API_END
}

int deoct_depth1_search(deoct_ctx* ctx, const deoct_dataset* ds, const int32_t* sample_idx,
                        int64_t n_sub, int32_t n_min, double alpha, uint16_t* a_out,
                        uint32_t* theta_out, double* fitness_out, void* stream) {
  API_BEGIN
  CTX_CHECK(ctx);
  DEOCT_TRY(validate_dataset(ds));
  DEOCT_TRY(validate_subset(ds, sample_idx, n_sub));
  if (n_min < 0) return set_error(DEOCT_ERR_INVALID, "n_min < 0");
  if (!(alpha == alpha)) return set_error(DEOCT_ERR_INVALID, "alpha is NaN");
  if (!a_out || !theta_out || !fitness_out) return set_error(DEOCT_ERR_INVALID, "NULL host output");
  return depth1_run(ctx, ds, sample_idx, n_sub, n_min, alpha, a_out, theta_out, fitness_out,
                    static_cast<cudaStream_t>(stream));
  API_END
}

}  // extern "C"
