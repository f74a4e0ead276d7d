// lj_bh_fp64.cu -- bh_step_batched kernels, FP64 path.
#include "lj_bh.cuh"

namespace ljh {

cudaError_t bh_plan_fp64(int n_atoms, int m, int n_walkers, int K, int team, Plan* out,
                          bool hist_global) {
  return ljbh::plan_impl<false>(n_atoms, m, n_walkers, K, team, out, hist_global);
}

cudaError_t bh_launch_fp64(const BhArgs& a, const Plan& plan, cudaStream_t s) {
  return ljbh::launch_impl<false>(a, plan, s);
}

}  // namespace ljh
