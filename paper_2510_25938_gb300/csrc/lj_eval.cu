// lj_eval.cu -- lj_energy_grad_batched: batched Eq. (1) energy + gradient.
//
// Uniform batches (2..512 atoms): flat layout, one thread per atom, several
// whole candidates per 512-thread CTA.  Uneven batches: one team per
// candidate (a warp for N <= 64), teams stride over the batch.  Either way
// a candidate's coordinates are read from HBM once, staged in shared memory,
// and every thread sums the pair terms of its own atom(s) (one-sided form:
// deterministic, no atomics).
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
  void* hist;
  carve_team<T>(smem + team * team_smem_bytes<T>(a.max_n, false), a.max_n, false, 0, pos, hbuf,
                hist, tm.red, word);
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
    evaluate<T, A, Prec<X, X, X, 0>>(tm, n, x, g, pos, nullptr, p, nullptr, E, dummy);
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

// Flat layout for uniform batches: one thread per atom, C = floor(512 / N)
// whole candidates per 512-thread CTA (several CTAs per SM overlap each
// other's barriers), candidates' positions staged in shared memory, each
// thread summing the pair terms of its own atom over its candidate
// (one-sided, no atomics), per-candidate energies summed by a fixed-order
// shared-memory tree (log2 N steps).
constexpr int kFlatThreads = 512;

__host__ __device__ constexpr int pow2_ceil(int n) {
  int p = 1;
  while (p < n) p <<= 1;
  return p;
}

template <typename X, typename IO>
__global__ void __launch_bounds__(kFlatThreads) eval_flat_kernel(ljh::EvalArgs a, int C) {
  extern __shared__ __align__(16) unsigned char smem[];
  using P = typename PosOf<X>::type;
  using F = typename Tr<X>::F;
  const int n = a.uniform_n;
  P* pos = reinterpret_cast<P*>(smem);
  F* esum = reinterpret_cast<F*>(smem + align16((size_t)C * n * sizeof(P)));
  const int tid = threadIdx.x;
  const int lc = tid / n;              // candidate within the CTA
  const int i = tid - lc * n;          // atom within the candidate
  const bool active = lc < C;
  const X sig2 = (X)(a.sigma * a.sigma);
  const X gscale = (X)(24.0 * a.eps / (a.sigma * a.sigma));
  const IO* __restrict__ xin = static_cast<const IO*>(a.x);
  IO* __restrict__ gout = static_cast<IO*>(a.grad);
  const int top = pow2_ceil(n) >> 1;
  for (long long c0 = (long long)blockIdx.x * C; c0 < a.n_cand; c0 += (long long)gridDim.x * C) {
    const long long c = c0 + lc;
    const bool live = active && c < a.n_cand;
    const long long a0 = c * n;
    X px = 0, py = 0, pz = 0;
    if (live) {
      px = (X)xin[3 * (a0 + i)];
      py = (X)xin[3 * (a0 + i) + 1];
      pz = (X)xin[3 * (a0 + i) + 2];
      P q;
      q.x = px; q.y = py; q.z = pz; q.w = (X)0;
      pos[lc * n + i] = q;
    }
    __syncthreads();
    if (live) {
      X ax, ay, az;
      F e;
      if constexpr (sizeof(X) == 4) {
        e = ff{0.f, 0.f};
        pair_row_f32(n, i, px, py, pz, pos + lc * n, sig2, ax, ay, az, e);
      } else {
        dd ed{0.0, 0.0};
        pair_row_f64(n, i, px, py, pz, pos + lc * n, sig2, ax, ay, az, ed);
        e = ed.hi + ed.lo;
      }
      if (gout) {
        gout[3 * (a0 + i)] = (IO)(-gscale * ax);
        gout[3 * (a0 + i) + 1] = (IO)(-gscale * ay);
        gout[3 * (a0 + i) + 2] = (IO)(-gscale * az);
      }
      esum[lc * n + i] = e;
    }
    // fixed-order tree over each candidate's n per-atom energies
    for (int stride = top; stride > 0; stride >>= 1) {
      __syncthreads();
      if (live && i < stride && i + stride < n) {
        F* ep = esum + lc * n;
        if constexpr (sizeof(X) == 4) {
          ep[i] = ff_add(ep[i], ep[i + stride]);
        } else {
          ep[i] = ep[i] + ep[i + stride];
        }
      }
    }
    __syncthreads();
    if (live && i == 0) a.energy[c] = fto_double(esum[lc * n]) * (2.0 * a.eps);
  }
}

template <typename X, typename IO>
cudaError_t launch_flat(const ljh::EvalArgs& a, cudaStream_t s) {
  using P = typename PosOf<X>::type;
  const int n = a.uniform_n;
  const int C = kFlatThreads / n;
  const size_t smem = align16((size_t)C * n * sizeof(P)) +
                      (size_t)C * n * sizeof(typename Tr<X>::F);
  auto k = eval_flat_kernel<X, IO>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kFlatThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long need = (a.n_cand + C - 1) / C;
  long long grid = (long long)per_sm * sms;
  if (need < grid) grid = need;
  k<<<(unsigned)grid, kFlatThreads, smem, s>>>(a, C);
  return cudaGetLastError();
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
  // uniform batches of 2..512 atoms: flat thread-per-atom layout
  if (a.uniform_n >= 2 && a.uniform_n <= kFlatThreads) {
    const bool fp64 = a.prec == LJ_PREC_FP64;
    if (a.xtype == LJ_F32) return fp64 ? launch_flat<double, float>(a, s) : launch_flat<float, float>(a, s);
    return fp64 ? launch_flat<double, double>(a, s) : launch_flat<float, double>(a, s);
  }
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
