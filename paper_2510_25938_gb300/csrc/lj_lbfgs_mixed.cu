// lj_lbfgs_mixed.cu -- lbfgs_minimize_batched kernels, mixed-precision path.
#include "lj_lbfgs.cuh"

namespace ljh {

cudaError_t lbfgs_plan_mixed(int max_n, int m, int64_t n_cand, int device, int team, Plan* out,
                             bool hist_global) {
  return ljlb::plan_impl<true>(max_n, m, n_cand, device, team, out, hist_global);
}

cudaError_t lbfgs_launch_mixed(const LbfgsArgs& a, const Plan& plan, cudaStream_t s) {
  return ljlb::launch_impl<true>(a, plan, s);
}

}  // namespace ljh
