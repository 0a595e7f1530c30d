// encode.cu -- rank encoder (the threshold sets of Section 3.1 as dense ranks).
//
// For every feature p the samples' float32 values are sorted (segmented LSD
// radix sort on order-preserving key bits, sample index as payload); a sample's
// rank is the number of distinct values before it in sorted order, i.e. an
// exclusive scan of "value differs from its predecessor" flags, scattered back
// to the sample's column.  n_p is the number of flags.  -0.0 is folded into
// +0.0 before sorting; NaN is reported.
#include "internal.cuh"

namespace deoct {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;  // keys per tile
constexpr int kTransSamples = 32;

__device__ __forceinline__ uint32_t orderable(float v) {
  if (v == 0.0f) v = 0.0f;  // -0.0 and +0.0 are one value
  uint32_t b = __float_as_uint(v);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float from_orderable(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// block-wide exclusive scan of one value per thread (blockDim.x == kThreads)
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* warp_tot,
                                                         uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = x;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, off);
    if (lane >= off) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kThreads / 32 ? warp_tot[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, off);
      if (lane >= off) wi += y;
    }
    if (lane < kThreads / 32) warp_tot[lane] = wi - w;
    if (lane == kThreads / 32 - 1 && total) *total = wi;
  }
  __syncthreads();
  uint32_t r = warp_tot[warp] + incl - x;
  __syncthreads();
  return r;
}

// X [n][F] -> keys [F][n] (orderable bits), vals [F][n] (sample index)
__global__ void keys_kernel(const float* __restrict__ X, int64_t n, int F, uint32_t* __restrict__ keys,
                            uint32_t* __restrict__ vals, int* status) {
  extern __shared__ float xs[];  // [kTransSamples][F + 1]
  const int64_t i0 = (int64_t)blockIdx.x * kTransSamples;
  const int64_t left = n - i0;
  const int ns = left < kTransSamples ? (int)left : kTransSamples;
  for (int e = threadIdx.x; e < ns * F; e += blockDim.x) {
    int l = e / F, f = e - l * F;
    float v = X[i0 * F + e];
    if (isnan(v)) atomicOr(status, ST_NAN);
    xs[l * (F + 1) + f] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kTransSamples * F; e += blockDim.x) {
    int f = e / kTransSamples, l = e - f * kTransSamples;
    if (l < ns) {
      keys[(int64_t)f * n + i0 + l] = orderable(xs[l * (F + 1) + f]);
      vals[(int64_t)f * n + i0 + l] = (uint32_t)(i0 + l);
    }
  }
}

// per-tile digit histogram: H[f][digit][tile]
__global__ void __launch_bounds__(kThreads) rs_hist_kernel(const uint32_t* __restrict__ keys, int64_t n,
                                                          int shift, int ntiles,
                                                          uint32_t* __restrict__ H) {
  __shared__ uint32_t h[256];
  const int f = blockIdx.y, tile = blockIdx.x;
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t* k = keys + (int64_t)f * n;
  const int64_t base = (int64_t)tile * kTile;
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    int64_t j = base + it * kThreads + threadIdx.x;
    if (j < n) atomicAdd(&h[(k[j] >> shift) & 255u], 1u);
  }
  __syncthreads();
  H[((int64_t)f * 256 + threadIdx.x) * ntiles + tile] = h[threadIdx.x];
}

// exclusive scan of each (segment, digit) column over tiles; totals per digit
__global__ void __launch_bounds__(kThreads) rs_colscan_kernel(uint32_t* __restrict__ H, int ntiles,
                                                             uint32_t* __restrict__ tot) {
  __shared__ uint32_t wt[kThreads / 32];
  __shared__ uint32_t chunk_total;
  const int d = blockIdx.x, f = blockIdx.y;
  uint32_t* col = H + ((int64_t)f * 256 + d) * ntiles;
  uint32_t carry = 0;
  for (int c0 = 0; c0 < ntiles; c0 += kThreads) {
    int j = c0 + threadIdx.x;
    uint32_t x = j < ntiles ? col[j] : 0u;
    uint32_t ex = block_exclusive_scan(x, wt, &chunk_total);
    if (j < ntiles) col[j] = carry + ex;
    carry += chunk_total;
    __syncthreads();
  }
  if (threadIdx.x == 0) tot[f * 256 + d] = carry;
}

// stable scatter of one tile by digit
__global__ void __launch_bounds__(kThreads) rs_scatter_kernel(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, int64_t n, int shift, int ntiles, const uint32_t* __restrict__ H,
    const uint32_t* __restrict__ tot) {
  __shared__ uint32_t base[256];
  __shared__ uint32_t wcnt[kThreads / 32][256];
  __shared__ uint32_t woff[kThreads / 32][256];
  __shared__ uint32_t wt[kThreads / 32];
  const int f = blockIdx.y, tile = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // digit base of this tile = exclusive scan over digits of the totals + tile prefix
  {
    uint32_t t = tot[f * 256 + threadIdx.x];
    uint32_t ex = block_exclusive_scan(t, wt, nullptr);
    base[threadIdx.x] = ex + H[((int64_t)f * 256 + threadIdx.x) * ntiles + tile];
  }
  for (int w = 0; w < kThreads / 32; ++w) wcnt[w][threadIdx.x] = 0;
  uint32_t run = 0;  // thread t: keys of digit t already placed in this tile
  __syncthreads();
  const uint32_t* k = kin + (int64_t)f * n;
  const uint32_t* v = vin + (int64_t)f * n;
  uint32_t* ko = kout + (int64_t)f * n;
  uint32_t* vo = vout + (int64_t)f * n;
  const int64_t tbase = (int64_t)tile * kTile;
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (int it = 0; it < kItems; ++it) {
    const int64_t j = tbase + it * kThreads + threadIdx.x;
    const bool valid = j < n;
    uint32_t key = 0, val = 0, d = 256;
    if (valid) {
      key = k[j];
      val = v[j];
      d = (key >> shift) & 255u;
    }
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
    const uint32_t wrank = __popc(peers & lt_mask);
    if (valid && (__ffs(peers) - 1) == lane) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t acc = run;
#pragma unroll
      for (int w = 0; w < kThreads / 32; ++w) {
        uint32_t c = wcnt[w][threadIdx.x];
        woff[w][threadIdx.x] = acc;
        wcnt[w][threadIdx.x] = 0;
        acc += c;
      }
      run = acc;
    }
    __syncthreads();
    if (valid) {
      uint32_t pos = base[d] + woff[warp][d] + wrank;
      ko[pos] = key;
      vo[pos] = val;
    }
  }
}

// number of "new value" flags per tile of sorted keys
__global__ void __launch_bounds__(kThreads) rank_count_kernel(const uint32_t* __restrict__ keys,
                                                             int64_t n, int ntiles,
                                                             uint32_t* __restrict__ C) {
  __shared__ uint32_t wt[kThreads / 32];
  __shared__ uint32_t total;
  const int f = blockIdx.y, tile = blockIdx.x;
  const uint32_t* k = keys + (int64_t)f * n;
  const int64_t j0 = (int64_t)tile * kTile + (int64_t)threadIdx.x * kItems;
  uint32_t cnt = 0;
  for (int e = 0; e < kItems; ++e) {
    int64_t j = j0 + e;
    if (j < n) cnt += (j == 0 || k[j] != k[j - 1]) ? 1u : 0u;
  }
  block_exclusive_scan(cnt, wt, &total);
  if (threadIdx.x == 0) C[(int64_t)f * ntiles + tile] = total;
}

// exclusive scan of tile flag counts per feature; n_unique = total
__global__ void __launch_bounds__(kThreads) rank_scan_kernel(uint32_t* __restrict__ C, int ntiles,
                                                            uint32_t* __restrict__ n_unique) {
  __shared__ uint32_t wt[kThreads / 32];
  __shared__ uint32_t chunk_total;
  const int f = blockIdx.x;
  uint32_t* c = C + (int64_t)f * ntiles;
  uint32_t carry = 0;
  for (int c0 = 0; c0 < ntiles; c0 += kThreads) {
    int j = c0 + threadIdx.x;
    uint32_t x = j < ntiles ? c[j] : 0u;
    uint32_t ex = block_exclusive_scan(x, wt, &chunk_total);
    if (j < ntiles) c[j] = carry + ex;
    carry += chunk_total;
    __syncthreads();
  }
  if (threadIdx.x == 0) n_unique[f] = carry;
}

template <typename RT>
__global__ void __launch_bounds__(kThreads) rank_scatter_kernel(
    const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals, int64_t n, int ntiles,
    const uint32_t* __restrict__ C, RT* __restrict__ ranks, int64_t ld, float* __restrict__ uniq) {
  __shared__ uint32_t wt[kThreads / 32];
  const int f = blockIdx.y, tile = blockIdx.x;
  const uint32_t* k = keys + (int64_t)f * n;
  const uint32_t* v = vals + (int64_t)f * n;
  const int64_t j0 = (int64_t)tile * kTile + (int64_t)threadIdx.x * kItems;
  uint32_t flags[kItems];
  uint32_t cnt = 0;
#pragma unroll
  for (int e = 0; e < kItems; ++e) {
    int64_t j = j0 + e;
    flags[e] = (j < n && (j == 0 || k[j] != k[j - 1])) ? 1u : 0u;
    cnt += flags[e];
  }
  uint32_t ex = block_exclusive_scan(cnt, wt, nullptr);
  uint32_t r = C[(int64_t)f * ntiles + tile] + ex;
  RT* out = ranks + (int64_t)f * ld;
#pragma unroll
  for (int e = 0; e < kItems; ++e) {
    int64_t j = j0 + e;
    r += flags[e];
    if (j < n) {
      out[v[j]] = (RT)(r - 1u);
      if (uniq && flags[e]) uniq[(int64_t)f * ld + (r - 1u)] = from_orderable(k[j]);
    }
  }
}

}  // namespace

int radix_sort_segments(deoct_ctx* ctx, uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1,
                        int64_t n, int F, int bits, uint32_t** keys_out, uint32_t** vals_out,
                        cudaStream_t s) {
  const int ntiles = (int)((n + kTile - 1) / kTile);
  uint32_t *H = nullptr, *tot = nullptr;
  DEOCT_TRY(scratch_get(ctx, SL_ENC_HIST, sizeof(uint32_t) * (size_t)F * 256 * ntiles, (void**)&H));
  DEOCT_TRY(scratch_get(ctx, SL_ENC_TOT, sizeof(uint32_t) * (size_t)F * 256, (void**)&tot));
  uint32_t *ki = k0, *vi = v0, *ko = k1, *vo = v1;
  for (int shift = 0; shift < bits; shift += 8) {
    dim3 g(ntiles, F);
    rs_hist_kernel<<<g, kThreads, 0, s>>>(ki, n, shift, ntiles, H);
    rs_colscan_kernel<<<dim3(256, F), kThreads, 0, s>>>(H, ntiles, tot);
    rs_scatter_kernel<<<g, kThreads, 0, s>>>(ki, vi, ko, vo, n, shift, ntiles, H, tot);
    count_launch(ctx, 3);
    DEOCT_TRY(check_launch("radix pass"));
    uint32_t* t;
    t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
  }
  *keys_out = ki;
  *vals_out = vi;
  return DEOCT_OK;
}

int encode_run(deoct_ctx* ctx, const float* X, int64_t n, int F, int W, void* ranks_out,
               int64_t ld, uint32_t* n_unique_out, float* unique_out, cudaStream_t s, int* W_used) {
  const size_t elems = (size_t)n * F;
  uint32_t *k0, *k1, *v0, *v1, *C;
  DEOCT_TRY(scratch_get(ctx, SL_ENC_K0, elems * 4, (void**)&k0));
  DEOCT_TRY(scratch_get(ctx, SL_ENC_K1, elems * 4, (void**)&k1));
  DEOCT_TRY(scratch_get(ctx, SL_ENC_V0, elems * 4, (void**)&v0));
  DEOCT_TRY(scratch_get(ctx, SL_ENC_V1, elems * 4, (void**)&v1));
  const int ntiles = (int)((n + kTile - 1) / kTile);
  DEOCT_TRY(scratch_get(ctx, SL_ENC_TILE, sizeof(uint32_t) * (size_t)F * ntiles, (void**)&C));

  const size_t tsm = sizeof(float) * kTransSamples * (F + 1);
  keys_kernel<<<(unsigned)((n + kTransSamples - 1) / kTransSamples), kThreads, tsm, s>>>(
      X, n, F, k0, v0, ctx->d_status);
  count_launch(ctx);
  DEOCT_TRY(check_launch("keys_kernel"));
  uint32_t *ks, *vs;
  DEOCT_TRY(radix_sort_segments(ctx, k0, v0, k1, v1, n, F, 32, &ks, &vs, s));
  dim3 g(ntiles, F);
  rank_count_kernel<<<g, kThreads, 0, s>>>(ks, n, ntiles, C);
  rank_scan_kernel<<<F, kThreads, 0, s>>>(C, ntiles, n_unique_out);
  if (W == 0) {
    // automatic width: n_p is known once the flags are scanned, before any rank is written
    DEOCT_TRY(check_launch("rank count / scan kernels"));
    uint32_t* h = nullptr;
    DEOCT_TRY(pinned_get(ctx, sizeof(uint32_t) * F, (void**)&h));
    DEOCT_CUDA_TRY(cudaMemcpyAsync(h, n_unique_out, sizeof(uint32_t) * F, cudaMemcpyDeviceToHost, s));
    DEOCT_CUDA_TRY(cudaStreamSynchronize(s));
    uint32_t mx = 0;
    for (int f = 0; f < F; ++f) mx = h[f] > mx ? h[f] : mx;
    W = mx <= 65536u ? 2 : 4;
  }
  if (W_used) *W_used = W;
  if (W == 2)
    rank_scatter_kernel<uint16_t><<<g, kThreads, 0, s>>>(ks, vs, n, ntiles, C,
                                                        static_cast<uint16_t*>(ranks_out), ld,
                                                        unique_out);
  else
    rank_scatter_kernel<uint32_t><<<g, kThreads, 0, s>>>(ks, vs, n, ntiles, C,
                                                        static_cast<uint32_t*>(ranks_out), ld,
                                                        unique_out);
  count_launch(ctx, 3);
  return check_launch("rank kernels");
}

}  // namespace deoct
