// noalloc.cu -- deoct_eval_population_noalloc: the population evaluator without
// any device allocation.
//
// Some callers cannot allocate device memory: a host framework that owns all
// device memory through its own pool and forbids other allocators, or code that
// must not take the implicit device synchronisation that cudaMalloc/cudaFree
// can cause.  This entry point needs no context and allocates nothing: its
// scratch (the packed trees, the class counts when the caller passes no counts
// buffer, and a status word) lives in one file-scope __device__ array of fixed
// size that every GPU loading this library keeps until the process exits.
//
// Host code must not pass the array's name to a kernel: on the host it names a
// host-side stand-in, not device memory.  The device address is obtained once
// per device with cudaGetSymbolAddress, with that device current, during the
// first call made on that device.
#include <mutex>

#include "internal.cuh"

namespace deoct {
namespace {

constexpr size_t kNoAllocScratchBytes = DEOCT_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// status word at offset 0, packed trees at 256, then (optionally) counts
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mutex;
unsigned char* g_scratch_dev[kMaxDevices] = {nullptr};

// Device address of the scratch array on `device` (the current device).
int scratch_address(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices)
    return set_error(DEOCT_ERR_INVALID, "device %d outside 0..%d", device, kMaxDevices - 1);
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_dev[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return set_error(DEOCT_ERR_CUDA, "cudaGetSymbolAddress of the evaluator scratch failed: %s",
                       cudaGetErrorString(e));
    g_scratch_dev[device] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_dev[device];
  return DEOCT_OK;
}

}  // namespace
}  // namespace deoct

using namespace deoct;

extern "C" DEOCT_API int deoct_eval_population_noalloc(const deoct_dataset* ds,
                                                       const int32_t* sample_idx, int64_t n_sub,
                                                       const uint16_t* a, const uint32_t* theta,
                                                       int32_t P, int32_t depth,
                                                       uint32_t* counts_out, uint32_t* errors_out,
                                                       void* stream) {
  clear_error();
  try {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DEOCT_TRY(validate_dataset(ds));
    if (sample_idx == nullptr && n_sub != ds->n)
      return set_error(DEOCT_ERR_INVALID, "without sample_idx n_sub must equal n");
    if (n_sub < 0 || n_sub > kMaxN) return set_error(DEOCT_ERR_INVALID, "n_sub out of range");
    if (!a || !theta) return set_error(DEOCT_ERR_INVALID, "NULL tree arrays");
    if (P < 1 || P > kMaxPop * 64) return set_error(DEOCT_ERR_INVALID, "P = %d out of range", P);
    if (depth < 1 || depth > kMaxDepth) return set_error(DEOCT_ERR_INVALID, "depth out of range");
    const size_t B = ((size_t)1 << depth) - 1, L = (size_t)1 << depth;
    const size_t nodes_bytes = (size_t)P * B * 4;
    const size_t counts_bytes = (size_t)P * L * ds->K * 4;
    const size_t need = 256 + ((nodes_bytes + 255) & ~size_t(255)) + (counts_out ? 0 : counts_bytes);
    if (need > kNoAllocScratchBytes)
      return set_error(DEOCT_ERR_INVALID,
                       "deoct_eval_population_noalloc needs %zu bytes of scratch, more than its fixed "
                       "%zu (pass counts_out, or use fewer or shallower trees)",
                       need, kNoAllocScratchBytes);

    // a context on the stack: device properties only, nothing allocated
    deoct_ctx ctx;
    DEOCT_CUDA_TRY(cudaGetDevice(&ctx.device));
    DEOCT_CUDA_TRY(cudaDeviceGetAttribute(&ctx.num_sms, cudaDevAttrMultiProcessorCount, ctx.device));
    DEOCT_CUDA_TRY(cudaDeviceGetAttribute(&ctx.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                          ctx.device));
    DEOCT_CUDA_TRY(cudaDeviceGetAttribute(&ctx.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor,
                                          ctx.device));
    unsigned char* base = nullptr;
    DEOCT_TRY(scratch_address(ctx.device, &base));
    ctx.d_status = reinterpret_cast<int*>(base);
    uint32_t* nodes = reinterpret_cast<uint32_t*>(base + 256);
    uint32_t* counts = counts_out;
    if (!counts) counts = reinterpret_cast<uint32_t*>(base + 256 + ((nodes_bytes + 255) & ~size_t(255)));

    // the array keeps the previous call's contents: clear what must start at zero
    DEOCT_CUDA_TRY(cudaMemsetAsync(ctx.d_status, 0, sizeof(int), s));
    DEOCT_CUDA_TRY(cudaMemsetAsync(counts, 0, counts_bytes, s));
    DEOCT_TRY(launch_pack_nodes(&ctx, a, theta, (int64_t)P * B, ds->F, nodes, s));
    if (n_sub > 0) {
      EvalConfig cfg = eval_choose_config(&ctx, ds->rank_bytes, depth, ds->F, ds->K, P, n_sub, 1);
      EvalPlan plan = single_eval_plan(ds, sample_idx, n_sub, nodes, counts, P, cfg);
      DEOCT_TRY(eval_launch(&ctx, ds->rank_bytes, depth, plan, cfg, s));
    }
    // no later sync call can report the status word: a set bit (a tree naming a feature
    // > F, a sample index out of range, an expired bounded wait) turns every error count
    // into kErrorsInvalid, read on the device
    if (errors_out)
      DEOCT_TRY(launch_errors(&ctx, counts, P, (int)L, ds->K, n_sub, errors_out, s, ctx.d_status));
    return DEOCT_OK;
  } catch (...) {
    return set_error(DEOCT_ERR_INVALID, "internal exception");
  }
}
