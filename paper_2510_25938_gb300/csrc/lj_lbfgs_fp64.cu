// lj_lbfgs_fp64.cu -- lbfgs_minimize_batched kernels, FP64 path.
#include "lj_lbfgs.cuh"

namespace ljh {

cudaError_t lbfgs_plan_fp64(int max_n, int m, int64_t n_cand, int device, int team, Plan* out) {
  return ljlb::plan_impl<false>(max_n, m, n_cand, device, team, out);
}

cudaError_t lbfgs_launch_fp64(const LbfgsArgs& a, const Plan& plan, cudaStream_t s) {
  return ljlb::launch_impl<false>(a, plan, s);
}

}  // namespace ljh
