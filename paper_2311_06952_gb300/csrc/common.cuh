// common.cuh -- shared internals of libdeoct (context, errors, PTX helpers, Philox).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <array>
#include <string>
#include <vector>

#include "../../include/deoct.h"

namespace deoct {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
int set_error(int code, const char* fmt, ...);
void clear_error();

#define DEOCT_CUDA_TRY(expr)                                                          \
  do {                                                                                \
    cudaError_t _e = (expr);                                                          \
    if (_e != cudaSuccess)                                                            \
      return ::deoct::set_error(DEOCT_ERR_CUDA, "%s failed: %s (%s:%d)", #expr,       \
                                cudaGetErrorString(_e), __FILE__, __LINE__);          \
  } while (0)

#define DEOCT_TRY(expr)            \
  do {                             \
    int _rc = (expr);              \
    if (_rc != DEOCT_OK) return _rc; \
  } while (0)

// device status word bits (ctx->d_status); read and cleared by sync calls
enum : int {
  ST_TIMEOUT = 1,      // a bounded mbarrier / flag wait ran out
  ST_BAD_NODE = 2,     // a decoded tree named a feature > F
  ST_NAN = 4,          // NaN feature value in the encoder input
  ST_BAD_INDEX = 8,    // sample index out of range
};

// ---------------------------------------------------------------------------
// limits
// ---------------------------------------------------------------------------
constexpr int kMaxDepth = 10;
constexpr int kMaxF = 256;
constexpr int kMaxK = 255;
constexpr int64_t kMaxN = int64_t(1) << 24;
constexpr int kMinPop = 4;
constexpr int kMaxPop = 4096;
constexpr uint32_t kThetaMask = 0x00FFFFFFu;
// error count written when a device status bit says the class counts are not to be
// trusted (no true count reaches it: n <= 2^24)
constexpr uint32_t kErrorsInvalid = 0xFFFFFFFFu;

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct Scratch {
  void* ptr = nullptr;
  size_t bytes = 0;
};

enum ScratchSlot : int {
  SL_POP_TRIAL = 0, SL_FIT_TRIAL, SL_NODES, SL_COUNTS, SL_BEST, SL_FIT, SL_POP, SL_GEN,
  SL_EVAL_PROBS, SL_EVAL_JOBS, SL_DE_PROBS, SL_PACKED,
  SL_ENC_K0, SL_ENC_K1, SL_ENC_V0, SL_ENC_V1, SL_ENC_HIST, SL_ENC_TOT, SL_ENC_TILE,
  SL_MH_NODEOF, SL_MH_STATS, SL_MH_IDX, SL_MH_RANKS, SL_MH_LABELS, SL_MH_SEG, SL_MH_CURSOR,
  SL_MH_D1KEYS, SL_MH_D1VALS, SL_MH_D1K1, SL_MH_D1V1, SL_MH_D1BEST, SL_MH_POP, SL_MH_FIT,
  SL_MH_BEST, SL_MH_HOSTBUF, SL_D1_RESULT, SL_MISC,
  SL_MH_RANKS2, SL_MH_LABELS2, SL_MH_IDX2, SL_MH_POS2, SL_MH_SUB, SL_MH_SUBHIST, SL_MH_SEEDS,
  SL_DE_PART,
  SL_EVAL_ACC,  // zero at rest: ticket word, then the counts of one fused evaluation
  SL_COUNT
};

struct deoct_ctx_impl;

}  // namespace deoct

struct deoct_ctx {
  int device = 0;
  int num_sms = 0;
  int max_smem_optin = 0;
  int smem_per_sm = 0;
  cudaStream_t cap_stream = nullptr;  // private stream used only to capture CUDA graphs
  int* d_status = nullptr;  // device status word (bits ST_*)
  deoct::Scratch scratch[deoct::SL_COUNT];
  // pinned host staging for small read-backs
  void* h_pinned = nullptr;
  size_t h_pinned_bytes = 0;
  // statistics
  uint64_t launches = 0;
  uint64_t eval_launches = 0;
  int timing = 0;
  std::vector<cudaEvent_t> ev_pairs;  // start/stop pairs of timed evaluator launches
  double eval_ms = 0.0;
  uint64_t eval_timed = 0;
  // evaluator shapes picked by the autotuner, keyed by workload class
  std::vector<std::pair<uint64_t, std::array<int, 4>>> tuned;  // S, TG, warps, stream
  // evaluator launch shape forced by deoct_set_eval_config (0 = automatic)
  int force_S = 0, force_TG = 0, force_warps = 0, force_grid = 0;
  int force_stream = 0;  // deoct_set_eval_streaming: streaming kernel for every ballot launch
  uint64_t scratch_limit = 0;  // deoct_set_scratch_limit: cap of the scratch held (0: none)
  // shared engine that runs the generations of this context's batched level
  // solves together with other contexts' (deoct_engine_attach; nullable)
  deoct_engine* engine = nullptr;
};

namespace deoct {

// grow-only device scratch; contents are not preserved on growth
int scratch_get(deoct_ctx* ctx, int slot, size_t bytes, void** out);
// pinned host buffer for read-backs (grow-only)
int pinned_get(deoct_ctx* ctx, size_t bytes, void** out);
// read, clear and translate the device status word (sync on `stream`)
int check_status(deoct_ctx* ctx, cudaStream_t stream);
// launch accounting
inline void count_launch(deoct_ctx* ctx, int n = 1) { ctx->launches += (uint64_t)n; }
int check_launch(const char* what);
int validate_dataset(const deoct_dataset* ds);

// Set a kernel's dynamic shared-memory limit to the largest value the device
// allows for it (opt-in maximum minus the kernel's static shared memory).  The
// attribute is per kernel and shared by every host thread, so it is always set
// to this same value and never to one launch's size.
template <typename Kern>
inline int set_max_dynamic_smem(deoct_ctx* ctx, Kern kern) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             ctx->max_smem_optin - (int)fa.sharedSizeBytes);
  if (e != cudaSuccess)
    return set_error(DEOCT_ERR_CUDA, "setting the shared-memory limit failed: %s", cudaGetErrorString(e));
  return DEOCT_OK;
}

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// try_wait with a suspend-time hint: the thread sleeps in hardware until the
// phase completes or about `ns` nanoseconds pass, instead of issuing polls.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}
// Bounded wait: at most `tries` hinted tries of up to 1 us each, then records
// ST_TIMEOUT and returns false.
__device__ __forceinline__ bool mbar_wait_tries(uint64_t* bar, uint32_t parity, uint32_t tries,
                                                int* status) {
  for (uint32_t it = 0; it < tries; ++it)
    if (mbar_try_wait_sleep(bar, parity, 1000u)) return true;
  atomicOr(status, ST_TIMEOUT);
  return false;
}
// The library's waits: 2^20 tries (order of a second).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* status) {
  return mbar_wait_tries(bar, parity, 1u << 20, status);
}
// 1-D TMA bulk copy global -> shared, completion counted on `bar` in bytes.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// 2-D tiled TMA copy global -> shared of the box at element coordinates (x, y)
// of the tensor map `tmap` (a __grid_constant__ kernel parameter); the box
// lands densely, row-major; columns past the tensor's width read as zero.
// x * element size must be a multiple of 16 bytes; dst 128-byte aligned.
__device__ __forceinline__ void bulk_tensor_2d_g2s(void* dst, const void* tmap, int x, int y,
                                                   uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): published multipliers and
// Weyl key increments, ten rounds, key bumped between rounds.
struct U64x4 {
  uint64_t x[4];
};
__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                               uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t lo0 = M0 * c0, hi0 = __umul64hi(M0, c0);
    uint64_t lo1 = M1 * c2, hi1 = __umul64hi(M1, c2);
    uint64_t y0 = hi1 ^ c1 ^ k0, y1 = lo1, y2 = hi0 ^ c3 ^ k1, y3 = lo0;
    c0 = y0;
    c1 = y1;
    c2 = y2;
    c3 = y3;
  }
  U64x4 r;
  r.x[0] = c0;
  r.x[1] = c1;
  r.x[2] = c2;
  r.x[3] = c3;
  return r;
}
__device__ __forceinline__ uint32_t draw_from_block(const U64x4& b, uint32_t s) {
  uint64_t w = b.x[(s & 7u) >> 1];
  return (s & 1u) ? (uint32_t)(w >> 32) : (uint32_t)w;
}
// uniform float in [0,1): top 24 bits times 2^-24 (exact)
__device__ __forceinline__ float u01(uint32_t x) {
  return __fmul_rn(__uint2float_rn(x >> 8), 5.9604644775390625e-08f);
}
__device__ __forceinline__ uint32_t below(uint32_t x, uint32_t m) {
  return (uint32_t)(((uint64_t)x * (uint64_t)m) >> 32);
}
// largest float below a positive bound
__device__ __forceinline__ float below_bound(float ub) {
  return __int_as_float(__float_as_int(ub) - 1);
}

// Pack one decoded node for the evaluator: (feature p = a-1) << 24 | theta.
// a = 0 packs to 0 (feature 0, theta 0): "rank < 0" never holds, so the sample
// goes right, as the forced b_t = 0 of Section 2 requires.
__device__ __forceinline__ uint32_t pack_node(int a, uint32_t theta) {
  return a == 0 ? 0u : ((uint32_t)(a - 1) << 24) | (theta & kThetaMask);
}

// floor(bhat * N) clamped to [0, N - 1], for N = n_p + 1 <= 2^24 + 1, in
// integers.  A finite bhat in [0, 1) is m 2^-s with a 24-bit significand m and
// s >= 24, so bhat N = m N 2^-s exactly (m N < 2^49) and its floor is
// (m N) >> s; negative values (and -0) give 0, values >= 1 and +inf give N - 1,
// NaN gives 0.  The same value as floor of the exact double product, clamped,
// without FP64 arithmetic (a slow pipe on this GPU).
__device__ __forceinline__ uint32_t floor_times(float bhat, uint32_t N) {
  const uint32_t b = __float_as_uint(bhat);
  if (b >> 31) return 0u;                                   // negative, -0
  if (b >= 0x7F800000u) return b == 0x7F800000u ? N - 1 : 0u;  // +inf, NaN
  if (b >= 0x3F800000u) return N - 1;                       // >= 1
  const uint32_t E = b >> 23;                               // biased exponent, <= 126
  const uint64_t m = (uint64_t)((b & 0x7FFFFFu) | (E ? 0x800000u : 0u));
  const uint32_t sh = E ? 150u - E : 149u;                  // bhat = m 2^-sh, sh >= 24
  return sh >= 64u ? 0u : (uint32_t)((m * N) >> sh);
}

// Decode one gene pair (Eq. aenc / Eq. benc in rank form): a = floor(ahat)
// clamped to {0..F}; theta = min(floor(bhat (n_p + 1)), n_p - 1).
__device__ __forceinline__ void decode_gene_pair(float ahat, float bhat, int F,
                                                 const uint32_t* __restrict__ n_unique, int* a_out,
                                                 uint32_t* theta_out) {
  int a = (int)floorf(ahat);
  a = a < 0 ? 0 : (a > F ? F : a);
  if (a == 0) {
    *a_out = 0;
    *theta_out = 0;
    return;
  }
  const uint32_t np = n_unique[a - 1];
  const uint32_t raw = floor_times(bhat, np + 1u);  // in 0..n_p
  *a_out = a;
  *theta_out = raw > np - 1 ? np - 1 : raw;
}

}  // namespace deoct
