// engine.cu -- continuous batching of moving-horizon level solves across jobs
// (the serving form: several tree-fitting jobs resident at once, their DE work
// interleaved in shared launches).
//
// A job's moving-horizon driver (Algorithm 2, batched level form) prepares the
// DEOCT problems of a level on its own stream -- compacted node segments, the
// initial population S^1, its evaluation and the first trial vectors -- and then
// hands the problems, now in steady state, to the engine attached to its
// context and waits.  The engine thread keeps the active problems of all jobs in
// groups: problems that share the rank width, the subtree depth, the DE
// constants and the size class of their level (total samples, by powers of 4),
// so that a small job does not tick at the pace of a large one.  One tick of a
// group is one evaluator launch over every problem's trials and one DE-step
// launch (Eq. selection, best, next trials of Algorithm 4).  Each group has its
// own stream and replays its captured tick as long as its set of problems does
// not change; the GPU overlaps the groups' streams.  Each problem keeps its own
// data, Philox key (seed, node id) and device-side generation counter, so
// problems join at any tick and leave after exactly their G generations: a
// job's result is the same alone and in any mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>

#include "internal.cuh"

namespace deoct {

namespace {

// Replays enqueued per round of a group, and rounds a group keeps in flight:
// small enough that a joining job waits little, large enough to keep the GPU fed.
constexpr int kReplaysPerRound = 4;
constexpr int kRoundsInFlight = 2;
// Pinned host memory for the uploads of a group's new set of problems (reused
// in a circle once the copies that read it have run) and for the status word
// copied back after every round (one slot per round, in a circle).
constexpr size_t kStagingBytes = size_t(8) << 20;
constexpr int kStatusSlots = 4096;

struct Event {
  cudaEvent_t ev = nullptr;
  Event() { cudaEventCreateWithFlags(&ev, cudaEventDisableTiming); }
  ~Event() {
    if (ev) cudaEventDestroy(ev);
  }
  Event(const Event&) = delete;
  Event& operator=(const Event&) = delete;
};

}  // namespace

struct EngineGroupKey {
  int W, Dt, P, n_min, dither, size_class;
  float M, CR;
  double alpha;
  bool operator<(const EngineGroupKey& o) const {
    return std::tie(W, Dt, P, n_min, dither, size_class, M, CR, alpha) <
           std::tie(o.W, o.Dt, o.P, o.n_min, o.dither, o.size_class, o.M, o.CR, o.alpha);
  }
};

// One level solve of one job: its problems in steady state (generation 1's
// trials built and their counts zeroed), G generations to go.
struct EngineSub {
  EngineGroupKey key;
  int G = 0, remaining = 0;
  const void* owner = nullptr;
  std::vector<DEProb> dp;
  std::vector<EvalProb> ep;
  std::shared_ptr<Event> done_ev;
  const int* status = nullptr;  // pinned copy of the device status word at done_ev
  bool done = false;
  int rc = DEOCT_OK;
  std::string err;
};

namespace {

// One group of the active set: its problems, stream, captured tick and device
// arrays.
struct Group {
  std::vector<EngineSub*> subs;
  cudaStream_t stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool dirty = true;
  std::deque<std::shared_ptr<Event>> inflight;
  uint64_t per_replay_launches = 0, per_replay_evals = 0;
  int owners = 0, probs = 0;
  DEProb* dp = nullptr;
  EvalProb* ep = nullptr;
  EvalJob* jobs = nullptr;
  size_t cap_dp = 0, cap_ep = 0, cap_jobs = 0;
};

}  // namespace
}  // namespace deoct

struct deoct_engine {
  int device = 0;
  deoct_ctx* ctx = nullptr;  // the engine's own context: status word, counters, capture stream
  std::thread thr;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::deque<deoct::EngineSub*> pending;
  std::map<deoct::EngineGroupKey, deoct::Group> groups;
  std::vector<deoct::EngineSub*> finishing;
  // pinned staging ring: [begin, end) regions still read by queued copies
  char* ring = nullptr;
  size_t ring_head = 0;
  std::deque<std::tuple<size_t, size_t, std::shared_ptr<deoct::Event>>> ring_live;
  int* status_ring = nullptr;
  uint64_t rounds = 0;
  deoct_engine_stats st;
};

namespace deoct {

namespace {

// A region of the pinned staging ring, waiting for the copies that still read
// the bytes it reuses.
int ring_alloc(deoct_engine* e, size_t bytes, char** out) {
  bytes = (bytes + 255) & ~size_t(255);
  if (bytes > kStagingBytes) return set_error(DEOCT_ERR_INVALID, "engine upload of %zu bytes", bytes);
  if (e->ring_head + bytes > kStagingBytes) e->ring_head = 0;
  const size_t lo = e->ring_head, hi = lo + bytes;
  while (!e->ring_live.empty()) {
    auto& f = e->ring_live.front();
    const bool overlap = std::get<0>(f) < hi && lo < std::get<1>(f);
    if (!overlap && cudaEventQuery(std::get<2>(f)->ev) != cudaSuccess) {
      cudaGetLastError();
      break;
    }
    if (overlap) DEOCT_CUDA_TRY(cudaEventSynchronize(std::get<2>(f)->ev));
    e->ring_live.pop_front();
  }
  *out = e->ring + lo;
  e->ring_head = hi;
  return DEOCT_OK;
}

// Stream-ordered upload of a host array into a device array grown on demand.
template <typename T>
int engine_upload(deoct_engine* e, cudaStream_t s, const std::vector<T>& h, T** d, size_t* cap) {
  const size_t bytes = sizeof(T) * std::max<size_t>(1, h.size());
  if (*cap < bytes) {
    if (*d) DEOCT_CUDA_TRY(cudaFree(*d));  // synchronises: no queued replay reads it
    *d = nullptr;
    *cap = 0;
    const size_t want = bytes + bytes / 2;
    DEOCT_CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(d), want));
    *cap = want;
  }
  if (h.empty()) return DEOCT_OK;
  char* pin = nullptr;
  DEOCT_TRY(ring_alloc(e, sizeof(T) * h.size(), &pin));
  memcpy(pin, h.data(), sizeof(T) * h.size());
  DEOCT_CUDA_TRY(cudaMemcpyAsync(*d, pin, sizeof(T) * h.size(), cudaMemcpyHostToDevice, s));
  auto ev = std::make_shared<Event>();
  DEOCT_CUDA_TRY(cudaEventRecord(ev->ev, s));
  const size_t lo = (size_t)(pin - e->ring);
  e->ring_live.push_back(std::make_tuple(lo, lo + ((sizeof(T) * h.size() + 255) & ~size_t(255)), ev));
  return DEOCT_OK;
}

// Upload the arrays of group g's problems and capture its tick (evaluator + DE
// step) as a graph.
int rebuild(deoct_engine* e, const EngineGroupKey& k, Group& g) {
  if (g.exec) {
    cudaGraphExecDestroy(g.exec);  // its queued launches still run
    g.exec = nullptr;
  }
  std::vector<DEProb> dp;
  std::vector<EvalProb> ep;
  std::vector<const void*> owners;
  for (EngineSub* s : g.subs) {
    dp.insert(dp.end(), s->dp.begin(), s->dp.end());
    ep.insert(ep.end(), s->ep.begin(), s->ep.end());
    if (std::find(owners.begin(), owners.end(), s->owner) == owners.end()) owners.push_back(s->owner);
  }
  const int M = (int)dp.size();
  g.owners = (int)owners.size();
  g.probs = M;
  int Fmax = 1, Kmax = 1;
  int64_t nsum = 0, mx = 0;
  std::vector<int64_t> counts(M);
  for (int m = 0; m < M; ++m) {
    Fmax = std::max(Fmax, ep[m].F);
    Kmax = std::max(Kmax, ep[m].K);
    counts[m] = ep[m].count;
    nsum += counts[m];
    mx = std::max(mx, counts[m]);
  }
  deoct_ctx* c = e->ctx;
  const EvalConfig cfg = eval_choose_config(c, k.W, k.Dt, Fmax, Kmax, k.P, std::max<int64_t>(1, nsum), M);
  std::vector<EvalJob> jobs;
  int64_t total = 0;
  eval_build_jobs(counts, std::vector<int>(M, k.P), cfg.S, cfg.TG, &jobs, &total);
  DEOCT_TRY(engine_upload(e, g.stream, dp, &g.dp, &g.cap_dp));
  DEOCT_TRY(engine_upload(e, g.stream, ep, &g.ep, &g.cap_ep));
  DEOCT_TRY(engine_upload(e, g.stream, jobs, &g.jobs, &g.cap_jobs));
  EvalPlan plan;
  plan.d_probs = g.ep;
  plan.d_jobs = g.jobs;
  plan.njobs = (int)jobs.size();
  plan.total_tiles = total;
  plan.Fmax = Fmax;
  plan.Kmax = Kmax;
  plan.Pmax = k.P;
  plan.max_count = mx;
  bool one_array = M > 0;  // one TMA tensor map when every problem reads one rank array
  for (int m = 1; m < M; ++m)
    one_array = one_array && ep[m].ranks == ep[0].ranks && ep[m].ld == ep[0].ld && ep[m].ncols == ep[0].ncols;
  if (one_array) {
    plan.shared_ranks = ep[0].ranks;
    plan.shared_ld = ep[0].ld;
    plan.shared_ncols = ep[0].ncols;
  }
  DEArgs a;
  memset(&a, 0, sizeof(a));
  a.probs = g.dp;
  a.nprob = M;
  a.P = k.P;
  a.depth = k.Dt;
  a.M = k.M;
  a.CR = k.CR;
  a.alpha = k.alpha;
  a.n_min = k.n_min;
  a.dither = k.dither;
  a.Kmax = Kmax;
  a.status = c->d_status;
  if (!c->cap_stream) DEOCT_CUDA_TRY(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  const uint64_t l0 = c->launches, v0 = c->eval_launches;
  cudaGraph_t graph = nullptr;
  DEOCT_CUDA_TRY(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = eval_launch(c, k.W, k.Dt, plan, cfg, c->cap_stream);
  if (rc == DEOCT_OK) rc = de_launch_step(c, a, 0, DE_SELECT | DE_TRIAL | DE_GEN_DEVICE, c->cap_stream);
  cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &graph);
  g.per_replay_launches = c->launches - l0;
  g.per_replay_evals = c->eval_launches - v0;
  c->launches = l0;
  c->eval_launches = v0;
  if (rc != DEOCT_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (ce != cudaSuccess) return set_error(DEOCT_ERR_CUDA, "engine graph capture failed: %s", cudaGetErrorString(ce));
  ce = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) {
    g.exec = nullptr;
    return set_error(DEOCT_ERR_CUDA, "engine graph instantiate failed: %s", cudaGetErrorString(ce));
  }
  g.dirty = false;
  return DEOCT_OK;
}

void finish(deoct_engine* e, EngineSub* s, int rc, const std::string& err) {
  std::lock_guard<std::mutex> lk(e->mu);
  s->rc = rc;
  s->err = err;
  s->done = true;
  if (rc == DEOCT_OK) e->st.completed += 1;
  e->cv.notify_all();
}

// Subs whose last replay has completed: check the status word copied at their
// event, then wake their jobs.
void reap(deoct_engine* e) {
  for (size_t i = 0; i < e->finishing.size();) {
    EngineSub* s = e->finishing[i];
    const cudaError_t q = cudaEventQuery(s->done_ev->ev);
    if (q == cudaErrorNotReady) {
      cudaGetLastError();
      ++i;
      continue;
    }
    e->finishing.erase(e->finishing.begin() + i);
    if (q != cudaSuccess) {
      finish(e, s, DEOCT_ERR_CUDA, std::string("engine: ") + cudaGetErrorString(q));
      continue;
    }
    const int st = *s->status;
    if (st & ST_TIMEOUT) finish(e, s, DEOCT_ERR_TIMEOUT, "engine: a bounded device wait expired");
    else if (st) finish(e, s, DEOCT_ERR_INVALID, "engine: device status 0x" + std::to_string(st));
    else finish(e, s, DEOCT_OK, "");
  }
}

void fail_group(deoct_engine* e, Group& g, int rc, const char* what) {
  std::vector<EngineSub*> subs;
  subs.swap(g.subs);
  g.dirty = true;
  for (EngineSub* s : subs) finish(e, s, rc, what);
}

// One round of group g if it has room in flight: k replays of its tick, the
// status word copied back, an event; subs that have done their generations
// move to `finishing`.  Returns whether it launched.
bool run_round(deoct_engine* e, const EngineGroupKey& k, Group& g) {
  while (!g.inflight.empty() && cudaEventQuery(g.inflight.front()->ev) == cudaSuccess) g.inflight.pop_front();
  cudaGetLastError();
  if (g.subs.empty() || (int)g.inflight.size() >= kRoundsInFlight) return false;
  if (g.dirty) {
    const int rc = rebuild(e, k, g);
    if (rc != DEOCT_OK) {
      fail_group(e, g, rc, "engine: building the shared launches failed");
      return false;
    }
  }
  int n = kReplaysPerRound;
  for (EngineSub* s : g.subs) n = std::min(n, s->remaining);
  cudaError_t ce = cudaSuccess;
  for (int i = 0; i < n && ce == cudaSuccess; ++i) ce = cudaGraphLaunch(g.exec, g.stream);
  auto ev = std::make_shared<Event>();
  int* status = e->status_ring + (e->rounds++ % kStatusSlots);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(status, e->ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, g.stream);
  if (ce == cudaSuccess) ce = cudaEventRecord(ev->ev, g.stream);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    fail_group(e, g, DEOCT_ERR_CUDA, "engine: launching the shared replays failed");
    return false;
  }
  g.inflight.push_back(ev);
  {
    std::lock_guard<std::mutex> lk(e->mu);
    e->st.ticks += (uint64_t)n;
    e->st.launches += (uint64_t)n * g.per_replay_launches;
    e->st.eval_launches += (uint64_t)n * g.per_replay_evals;
    if (g.owners > 1) e->st.shared_launches += (uint64_t)n * g.per_replay_launches;
    e->st.max_jobs_per_launch = std::max<uint64_t>(e->st.max_jobs_per_launch, (uint64_t)g.owners);
    e->st.max_problems_per_launch = std::max<uint64_t>(e->st.max_problems_per_launch, (uint64_t)g.probs);
  }
  for (size_t i = 0; i < g.subs.size();) {
    EngineSub* s = g.subs[i];
    s->remaining -= n;
    if (s->remaining <= 0) {
      s->done_ev = ev;
      s->status = status;
      e->finishing.push_back(s);
      g.subs.erase(g.subs.begin() + i);
      g.dirty = true;
    } else {
      ++i;
    }
  }
  return true;
}

void engine_loop(deoct_engine* e) {
  cudaSetDevice(e->device);
  for (;;) {
    std::vector<EngineSub*> joins;
    {
      std::unique_lock<std::mutex> lk(e->mu);
      bool busy = !e->finishing.empty();
      for (auto& kv : e->groups) busy = busy || !kv.second.subs.empty();
      if (busy) {
        // work in flight: wake for new submissions, else poll the rounds soon
        if (e->pending.empty()) e->cv.wait_for(lk, std::chrono::microseconds(20));
      } else {
        e->cv.wait(lk, [&] { return e->stop || !e->pending.empty(); });
        if (e->stop && e->pending.empty()) break;
      }
      joins.assign(e->pending.begin(), e->pending.end());
      e->pending.clear();
    }
    for (EngineSub* s : joins) {
      s->remaining = s->G;
      if (s->G <= 0) {
        finish(e, s, DEOCT_OK, "");
        continue;
      }
      Group& g = e->groups[s->key];
      if (!g.stream && cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        g.stream = nullptr;
        finish(e, s, DEOCT_ERR_CUDA, "engine: stream creation failed");
        continue;
      }
      g.subs.push_back(s);
      g.dirty = true;
    }
    for (auto& kv : e->groups) run_round(e, kv.first, kv.second);
    reap(e);
  }
  for (auto& kv : e->groups) {
    Group& g = kv.second;
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    if (g.stream) cudaStreamSynchronize(g.stream);
    g.inflight.clear();
  }
  e->ring_live.clear();
}

int size_class(const std::vector<EvalProb>& ep) {
  int64_t total = 0;
  for (const EvalProb& p : ep) total += p.count;
  int c = 0;
  for (int64_t t = total >> 12; t > 0; t >>= 2) ++c;  // 4096 samples, then by powers of 4
  return c;
}

}  // namespace

// Called by a job's batched level solve (mh.cu): run G generations of the
// problems `dp` / `ep` (already in steady state) in the engine's shared
// launches; returns once their last generation has completed on the device.
int engine_generations(deoct_engine* e, const void* owner, int W, int Dt, const DEArgs& a, int G,
                       const std::vector<DEProb>& dp, const std::vector<EvalProb>& ep) {
  EngineSub s;
  s.key = EngineGroupKey{W, Dt, a.P, a.n_min, a.dither, size_class(ep), a.M, a.CR, a.alpha};
  s.G = G;
  s.owner = owner;
  s.dp = dp;
  s.ep = ep;
  {
    std::unique_lock<std::mutex> lk(e->mu);
    if (e->stop) return set_error(DEOCT_ERR_INVALID, "the engine is shutting down");
    e->st.submissions += 1;
    e->pending.push_back(&s);
    e->cv.notify_all();
    e->cv.wait(lk, [&] { return s.done; });
  }
  if (s.rc != DEOCT_OK) return set_error(s.rc, "%s", s.err.c_str());
  return DEOCT_OK;
}

}  // namespace deoct

using namespace deoct;

extern "C" {

int deoct_engine_create(deoct_engine** out, int device) {
  clear_error();
  try {
    if (!out) return set_error(DEOCT_ERR_INVALID, "out is NULL");
    *out = nullptr;
    deoct_ctx* c = nullptr;
    int rc = deoct_create(&c, device);
    if (rc != DEOCT_OK) return rc;
    deoct_engine* e = new deoct_engine();
    e->device = device;
    e->ctx = c;
    memset(&e->st, 0, sizeof(e->st));
    cudaError_t ce = cudaMallocHost(reinterpret_cast<void**>(&e->ring), kStagingBytes);
    if (ce == cudaSuccess) ce = cudaMallocHost(reinterpret_cast<void**>(&e->status_ring), sizeof(int) * kStatusSlots);
    if (ce != cudaSuccess) {
      if (e->ring) cudaFreeHost(e->ring);
      deoct_destroy(c);
      delete e;
      return set_error(DEOCT_ERR_CUDA, "engine set-up: %s", cudaGetErrorString(ce));
    }
    e->thr = std::thread(engine_loop, e);
    *out = e;
    return DEOCT_OK;
  } catch (...) {
    return set_error(DEOCT_ERR_INVALID, "internal exception");
  }
}

int deoct_engine_destroy(deoct_engine* e) {
  clear_error();
  if (!e) return DEOCT_OK;
  {
    std::lock_guard<std::mutex> lk(e->mu);
    e->stop = true;
    e->cv.notify_all();
  }
  if (e->thr.joinable()) e->thr.join();
  cudaSetDevice(e->device);
  for (auto& kv : e->groups) {
    Group& g = kv.second;
    if (g.dp) cudaFree(g.dp);
    if (g.ep) cudaFree(g.ep);
    if (g.jobs) cudaFree(g.jobs);
    if (g.stream) cudaStreamDestroy(g.stream);
  }
  if (e->ring) cudaFreeHost(e->ring);
  if (e->status_ring) cudaFreeHost(e->status_ring);
  deoct_destroy(e->ctx);
  delete e;
  return DEOCT_OK;
}

int deoct_engine_attach(deoct_ctx* ctx, deoct_engine* e) {
  clear_error();
  if (!ctx) return set_error(DEOCT_ERR_INVALID, "context is NULL");
  if (e && e->device != ctx->device)
    return set_error(DEOCT_ERR_INVALID, "engine on device %d, context on device %d", e->device, ctx->device);
  ctx->engine = e;
  return DEOCT_OK;
}

int deoct_engine_get_stats(deoct_engine* e, deoct_engine_stats* out) {
  clear_error();
  if (!e || !out) return set_error(DEOCT_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(e->mu);
  *out = e->st;
  return DEOCT_OK;
}

}  // extern "C"
