// lj_lbfgs_fp64.cu -- lbfgs_minimize_batched kernels, FP64 path.
#include "lj_lbfgs.cuh"

namespace ljlb {

// Sort candidate indices into size buckets: bucket b takes the candidates
// with bound[b-1] < n <= bound[b] (the last bucket also takes anything
// larger, which the minimiser reports as LJ_CAND_BAD_INPUT).  List order
// within a bucket is arbitrary; every candidate is minimised by one team
// whichever list position it gets, so results do not depend on it.
__global__ void bucketize_kernel(const int64_t* __restrict__ off, long long n_cand, int nb,
                                 ljh::Buckets bk, unsigned* __restrict__ counts,
                                 int* __restrict__ lists) {
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n_cand;
       c += (long long)gridDim.x * blockDim.x) {
    const long long n = off[c + 1] - off[c];
    int b = 0;
    while (b < nb - 1 && n > bk.bound[b]) ++b;
    const unsigned q = atomicAdd(&counts[b], 1u);
    lists[(long long)b * n_cand + q] = (int)c;
  }
}

// Synthetic starts for the autotuner: coordinate q of candidate c uniform
// in [0, side), draw q of a Philox stream of its own (tag 5, counter (q, c)).
__global__ void tune_starts_kernel(double* __restrict__ x, long long n_cand, int n3, double side,
                                   unsigned long long seed) {
  const long long total = n_cand * n3;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long c = i / n3;
    const int q = (int)(i - c * n3);
    x[i] = side * ljd::stream_u01(seed, 5u, (uint32_t)q, (uint32_t)c, 0u, 0u);
  }
}

}  // namespace ljlb

namespace ljh {

cudaError_t tune_starts_launch(double* x, int64_t n_cand, int n, double side, uint64_t seed,
                               cudaStream_t s) {
  const long long total = n_cand * 3 * n;
  const long long blocks = (total + 255) / 256;
  ljlb::tune_starts_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(
      x, n_cand, 3 * n, side, seed);
  return cudaGetLastError();
}

cudaError_t lbfgs_plan_fp64(int max_n, int m, int64_t n_cand, int device, int team, Plan* out,
                            bool hist_global) {
  return ljlb::plan_impl<false>(max_n, m, n_cand, device, team, out, hist_global);
}

cudaError_t lbfgs_launch_fp64(const LbfgsArgs& a, const Plan& plan, cudaStream_t s) {
  return ljlb::launch_impl<false>(a, plan, s);
}

cudaError_t bucketize_launch(const int64_t* off, int64_t n_cand, int nb, const Buckets& bk,
                             unsigned* counts, int* lists, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(unsigned) * kMaxBuckets, s);
  if (e != cudaSuccess) return e;
  const long long blocks = (n_cand + 255) / 256;
  ljlb::bucketize_kernel<<<(unsigned)(blocks < 1024 ? blocks : 1024), 256, 0, s>>>(
      off, n_cand, nb, bk, counts, lists);
  return cudaGetLastError();
}

}  // namespace ljh
