// lj_morse_bh_mixed.cu -- bh_step_batched kernels for the Morse pair potential,
// mixed-precision path (FP32 tier, then FP64).
#include "lj_bh.cuh"

namespace ljh {

cudaError_t bh_plan_morse_mixed(int n_atoms, int m, int n_walkers, int K, int team, Plan* out,
                               bool hist_global) {
  return ljbh::plan_impl<true, LJ_POT_MORSE>(n_atoms, m, n_walkers, K, team, out, hist_global);
}

cudaError_t bh_launch_morse_mixed(const BhArgs& a, const Plan& plan, cudaStream_t s) {
  return ljbh::launch_impl<true, LJ_POT_MORSE>(a, plan, s);
}

}  // namespace ljh
