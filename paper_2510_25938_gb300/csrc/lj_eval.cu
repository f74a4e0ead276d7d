// lj_eval.cu -- batched Eq. (1) energy + gradient (lj_energy_grad_batched).
//
// One team per candidate (a warp for N <= 64), teams stride over the batch.
// The candidate's coordinates are loaded from HBM once, staged in shared
// memory, and every thread sums the pair terms of its own atoms (one-sided
// form: deterministic, no atomics).
#include "lj_internal.h"
#include "lj_minimize.cuh"
#include "lj_teams.cuh"

namespace {

using namespace ljd;

template <int T, int A, typename X, typename IO>
__global__ void __launch_bounds__(cta_threads_for(T)) eval_kernel(ljh::EvalArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int TPC = cta_threads_for(T) / T;
  const int team = threadIdx.x / T;
  Team<T> tm;
  tm.rank = threadIdx.x % T;
  tm.bar = team + 1;
  void* pos;
  long long* word;
  void* hbuf;
  carve_team<T>(smem + team * team_smem_bytes<T>(a.max_n, false), a.max_n, false, pos, hbuf,
                tm.red, word);
  MinParams p{};
  p.eps = a.eps;
  p.sigma = a.sigma;
  const IO* __restrict__ xin = static_cast<const IO*>(a.x);
  IO* __restrict__ gout = static_cast<IO*>(a.grad);
  for (long long c = (long long)blockIdx.x * TPC + team; c < a.n_cand;
       c += (long long)gridDim.x * TPC) {
    long long a0;
    int n;
    if (a.uniform_n > 0) {
      a0 = c * a.uniform_n;
      n = a.uniform_n;
    } else {
      a0 = a.off[c];
      n = (int)(a.off[c + 1] - a0);
    }
    if (n > a.max_n || n < 0) {
      if (tm.rank == 0) a.energy[c] = __longlong_as_double(0x7ff8000000000000LL);
      continue;
    }
    X x[A][3], g[A][3];
#pragma unroll
    for (int s = 0; s < A; ++s) {
      const int i = tm.rank + s * T;
#pragma unroll
      for (int k = 0; k < 3; ++k) x[s][k] = i < n ? (X)xin[3 * (a0 + i) + k] : (X)0;
    }
    typename Tr<X>::F E;
    typename Tr<X>::S dummy;
    evaluate<T, A, X, X>(tm, n, x, g, pos, nullptr, p, nullptr, E, dummy);
    if (gout) {
#pragma unroll
      for (int s = 0; s < A; ++s) {
        const int i = tm.rank + s * T;
        if (i < n) {
#pragma unroll
          for (int k = 0; k < 3; ++k) gout[3 * (a0 + i) + k] = (IO)g[s][k];
        }
      }
    }
    if (tm.rank == 0) a.energy[c] = fto_double(E);
  }
}

template <int T, int A, typename X, typename IO>
cudaError_t launch_one(const ljh::EvalArgs& a, cudaStream_t s) {
  constexpr int threads = cta_threads_for(T);
  constexpr int TPC = threads / T;
  const size_t smem = TPC * team_smem_bytes<T>(a.max_n, false);
  auto k = eval_kernel<T, A, X, IO>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long need = (a.n_cand + TPC - 1) / TPC;
  long long grid = (long long)per_sm * sms;
  if (need < grid) grid = need;
  k<<<(unsigned)grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

namespace ljh {

cudaError_t eval_launch(const EvalArgs& a, cudaStream_t s) {
  return dispatch_team(a.max_n, [&](auto TT, auto AA) -> cudaError_t {
    constexpr int T = decltype(TT)::value;
    constexpr int A = decltype(AA)::value;
    const bool fp64 = a.prec == LJ_PREC_FP64;
    if (a.xtype == LJ_F32) {
      return fp64 ? launch_one<T, A, double, float>(a, s) : launch_one<T, A, float, float>(a, s);
    }
    return fp64 ? launch_one<T, A, double, double>(a, s) : launch_one<T, A, float, double>(a, s);
  });
}

}  // namespace ljh
