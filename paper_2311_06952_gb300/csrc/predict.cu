// predict.cu -- a fitted tree applied to raw feature values (unseen samples).
//
// A rank threshold theta of feature p is the threshold set entry beta_{p,
// theta+1} of Section 3.1 in raw units: the midpoint of the theta-th and
// (theta+1)-th smallest distinct training values (1-based), computed in double
// (exact for float32 inputs); theta = 0 is beta_{p,1} = 0 after min-max
// scaling, i.e. the smallest training value.  On training samples "x < b"
// then routes exactly like "rank < theta".
#include <algorithm>

#include "internal.cuh"

namespace deoct {
namespace {

__global__ void split_values_kernel(const float* __restrict__ unique, int64_t ld,
                                    const uint16_t* __restrict__ a, const uint32_t* __restrict__ theta,
                                    int B, double* __restrict__ b_out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B) return;
  const int av = a[t];
  if (av == 0) {
    b_out[t] = 0.0;  // unused: a_t = 0 sends every sample right
    return;
  }
  const float* u = unique + (int64_t)(av - 1) * ld;
  const uint32_t th = theta[t];
  b_out[t] = th == 0 ? (double)u[0] : __dmul_rn(__dadd_rn((double)u[th - 1], (double)u[th]), 0.5);
}

__global__ void predict_kernel(const float* __restrict__ X, int64_t m, int F,
                               const uint16_t* __restrict__ a, const double* __restrict__ b, int depth,
                               const uint8_t* __restrict__ leaf_class, const uint8_t* __restrict__ y,
                               uint8_t* __restrict__ pred, unsigned long long* __restrict__ correct) {
  extern __shared__ unsigned char sm[];
  const int B = (1 << depth) - 1, L = 1 << depth;
  double* bs = reinterpret_cast<double*>(sm);
  uint16_t* as = reinterpret_cast<uint16_t*>(bs + B);
  uint8_t* cs = reinterpret_cast<uint8_t*>(as + B);
  for (int t = threadIdx.x; t < B; t += blockDim.x) {
    bs[t] = b[t];
    as[t] = a[t];
  }
  for (int l = threadIdx.x; l < L; l += blockDim.x) cs[l] = leaf_class[l];
  __syncthreads();
  unsigned long long ok = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    int t = 1;
    while (t <= B) {
      const int p = as[t - 1];
      const bool left = p != 0 && p <= F && (double)X[i * F + (p - 1)] < bs[t - 1];
      t = left ? 2 * t : 2 * t + 1;
    }
    const uint8_t c = cs[t - L];
    if (pred) pred[i] = c;
    if (y) ok += (y[i] == c) ? 1ull : 0ull;
  }
  if (correct) {
    for (int off = 16; off > 0; off >>= 1) ok += __shfl_down_sync(0xFFFFFFFFu, ok, off);
    if ((threadIdx.x & 31) == 0 && ok) atomicAdd(correct, ok);
  }
}

}  // namespace

int launch_split_values(deoct_ctx* ctx, const float* unique, int64_t ld, const uint16_t* a,
                        const uint32_t* theta, int B, double* b_out, cudaStream_t s) {
  split_values_kernel<<<(B + 127) / 128, 128, 0, s>>>(unique, ld, a, theta, B, b_out);
  count_launch(ctx);
  return check_launch("split_values_kernel");
}

int launch_predict(deoct_ctx* ctx, const float* X, int64_t m, int F, const uint16_t* a,
                   const double* b, int depth, const uint8_t* leaf_class, const uint8_t* y,
                   uint8_t* pred_out, unsigned long long* correct_out, cudaStream_t s) {
  if (correct_out) DEOCT_CUDA_TRY(cudaMemsetAsync(correct_out, 0, sizeof(unsigned long long), s));
  if (m == 0) return DEOCT_OK;
  const int B = (1 << depth) - 1, L = 1 << depth;
  const size_t smem = (size_t)B * 8 + (size_t)B * 2 + (size_t)L;
  DEOCT_TRY(set_max_dynamic_smem(ctx, predict_kernel));
  const int grid = (int)std::min<int64_t>((m + 255) / 256, (int64_t)ctx->num_sms * 8);
  predict_kernel<<<grid, 256, smem, s>>>(X, m, F, a, b, depth, leaf_class, y, pred_out, correct_out);
  count_launch(ctx);
  return check_launch("predict_kernel");
}

}  // namespace deoct
