// lj_morse_lbfgs_mixed.cu -- lbfgs_minimize_batched kernels for the Morse pair
// potential, mixed-precision path (FP32 tier, then FP64).
#include "lj_lbfgs.cuh"

namespace ljh {

cudaError_t lbfgs_plan_morse_mixed(int max_n, int m, int64_t n_cand, int device, int team,
                                  Plan* out, bool hist_global) {
  return ljlb::plan_impl<true, LJ_POT_MORSE>(max_n, m, n_cand, device, team, out, hist_global);
}

cudaError_t lbfgs_launch_morse_mixed(const LbfgsArgs& a, const Plan& plan, cudaStream_t s) {
  return ljlb::launch_impl<true, LJ_POT_MORSE>(a, plan, s);
}

}  // namespace ljh
