// lj_morse_bh_fp64.cu -- bh_step_batched kernels for the Morse pair potential,
// FP64 path.
#include "lj_bh.cuh"

namespace ljh {

cudaError_t bh_plan_morse_fp64(int n_atoms, int m, int n_walkers, int K, int team, Plan* out,
                               bool hist_global) {
  return ljbh::plan_impl<false, LJ_POT_MORSE>(n_atoms, m, n_walkers, K, team, out, hist_global);
}

cudaError_t bh_launch_morse_fp64(const BhArgs& a, const Plan& plan, cudaStream_t s) {
  return ljbh::launch_impl<false, LJ_POT_MORSE>(a, plan, s);
}

}  // namespace ljh
