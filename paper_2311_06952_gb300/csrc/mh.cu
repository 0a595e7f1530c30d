// mh.cu -- moving-horizon DEOCT (Algorithm 2) and the exhaustive depth-1 search.
#include "internal.cuh"

using namespace deoct;

extern "C" {

int deoct_depth1_search(deoct_ctx* ctx, const deoct_dataset* ds, const int32_t* sample_idx,
                        int64_t n_sub, int32_t n_min, double alpha, uint16_t* a_out,
                        uint32_t* theta_out, double* fitness_out, void* stream) {
  (void)ctx; (void)ds; (void)sample_idx; (void)n_sub; (void)n_min; (void)alpha; (void)a_out;
  (void)theta_out; (void)fitness_out; (void)stream;
  return set_error(DEOCT_ERR_INVALID, "deoct_depth1_search: not available in this build");
}

int deoct_fit_moving_horizon(deoct_ctx* ctx, const deoct_dataset* ds, const deoct_params* params,
                             uint16_t* a_out, uint32_t* theta_out, uint8_t* leaf_class_out,
                             int32_t* kind_out, double* node_fit_out, void* stream) {
  (void)ctx; (void)ds; (void)params; (void)a_out; (void)theta_out; (void)leaf_class_out;
  (void)kind_out; (void)node_fit_out; (void)stream;
  return set_error(DEOCT_ERR_INVALID, "deoct_fit_moving_horizon: not available in this build");
}

}  // extern "C"
