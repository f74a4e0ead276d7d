// lj_morse_lbfgs_fp64.cu -- lbfgs_minimize_batched kernels for the Morse pair
// potential, FP64 path.
#include "lj_lbfgs.cuh"

namespace ljh {

cudaError_t lbfgs_plan_morse_fp64(int max_n, int m, int64_t n_cand, int device, int team,
                                  Plan* out, bool hist_global) {
  return ljlb::plan_impl<false, LJ_POT_MORSE>(max_n, m, n_cand, device, team, out, hist_global);
}

cudaError_t lbfgs_launch_morse_fp64(const LbfgsArgs& a, const Plan& plan, cudaStream_t s) {
  return ljlb::launch_impl<false, LJ_POT_MORSE>(a, plan, s);
}

}  // namespace ljh
