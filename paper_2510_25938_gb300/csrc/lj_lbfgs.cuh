// lj_lbfgs.cuh -- lbfgs_minimize_batched: a persistent kernel in which every
// team takes candidates from a device work queue (one atomic counter) and
// runs the whole L-BFGS loop on chip -- direction, line search, convergence
// test -- with no host round trip per iteration.  Candidates converge after
// different iteration counts; the queue keeps every team busy until the
// batch is drained.
#pragma once
#include "lj_internal.h"
#include "lj_minimize.cuh"
#include "lj_teams.cuh"

namespace ljlb {

using namespace ljd;

__device__ __forceinline__ MinParams to_dev(const ljh::MinParamsH& h) {
  MinParams p;
  p.m = h.m; p.max_iter = h.max_iter; p.max_ls = h.max_ls;
  p.gtol = h.gtol; p.c1 = h.c1; p.c2 = h.c2; p.alpha_max = h.alpha_max;
  p.switch_gtol = h.switch_gtol; p.deadline = h.deadline; p.k = h.k;
  p.f32_resolution = h.f32_resolution; p.df_resolution = h.df_resolution;
  p.tiled = 0;
  return p;
}

// Register budget: teams for more than 256 atoms (which carry the tiled
// double-float evaluation) are allowed all registers of one CTA per SM; the
// others are left to the compiler's own occupancy choice.
// POT: pair potential (LJ_POT_LJ, Eq. (1); LJ_POT_MORSE).
template <int T, int A, bool MIXED, int POT = LJ_POT_LJ>
__global__ void __launch_bounds__(cta_threads_for(T), T * A > 256 ? 1 : 0)
    lbfgs_kernel(ljh::LbfgsArgs a) {
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
  const size_t hb = a.hist_on_chip ? a.hist_slot_bytes : 0;
  carve_team<T>(smem + team * team_smem_bytes<T>(a.max_n, true, hb), a.max_n, true, hb, pos,
                hbuf, hist, tm.red, word);
  MinParams p = to_dev(a.p);
  // hbuf: pair buffer up to 64 atoms, tile accumulators above 256.  With
  // one-sided rows chosen above 256 atoms there is no pair buffer to use: the
  // buffer holds 24 bytes per atom, not per pair, so it is withdrawn and every
  // tier evaluates in one-sided rows
  p.tiled = a.max_n > kTileMinN && !a.p.df_one_sided;
  if (a.max_n > kTileMinN && a.p.df_one_sided) hbuf = nullptr;
  const long long slot = (long long)blockIdx.x * TPC + team;
  if (!a.hist_on_chip) hist = static_cast<unsigned char*>(a.hist) + slot * a.hist_slot_bytes;

  for (;;) {
    long long c;
    if constexpr (T == 32) {
      unsigned long long v = 0;
      if (tm.rank == 0) v = atomicAdd(a.queue, 1ULL);
      c = (long long)__shfl_sync(kFull, v, 0);
    } else {
      if (tm.rank == 0) *word = (long long)atomicAdd(a.queue, 1ULL);
      tm.sync();
      c = *word;
      tm.sync();
    }
    if (a.list) {                         // bucketed launch: this bucket's candidates
      if (c >= (long long)*a.list_count) break;
      c = a.list[c];
    } else if (c >= a.n_cand) {
      break;
    }
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
      if (tm.rank == 0) {
        a.energy[c] = __longlong_as_double(0x7ff8000000000000LL);
        if (a.status) a.status[c] = ST_BAD_INPUT;
        if (a.iters) a.iters[c] = 0;
        if (a.nevals) a.nevals[c] = 0;
      }
      continue;
    }
    double x64[A][3];
#pragma unroll
    for (int s = 0; s < A; ++s) {
      const int i = tm.rank + s * T;
#pragma unroll
      for (int k = 0; k < 3; ++k) x64[s][k] = i < n ? a.x[3 * (a0 + i) + k] : 0.0;
    }
    MinResult r;
    minimise<T, A, MIXED, POT>(tm, n, x64, p, hist, pos, hbuf, r);
#pragma unroll
    for (int s = 0; s < A; ++s) {
      const int i = tm.rank + s * T;
      if (i < n) {
#pragma unroll
        for (int k = 0; k < 3; ++k) a.x[3 * (a0 + i) + k] = x64[s][k];
      }
    }
    if (tm.rank == 0) {
      a.energy[c] = r.E;
      if (a.status) a.status[c] = r.status;
      if (a.iters) a.iters[c] = r.iters;
      if (a.nevals) a.nevals[c] = r.evals32 + r.evals64 + r.evals_df;
      if (a.stats) {
        const unsigned long long np = (unsigned long long)n * (unsigned long long)(n > 0 ? n - 1 : 0) / 2;
        atomicAdd(&a.stats->evals32, (unsigned long long)r.evals32);
        atomicAdd(&a.stats->evals64, (unsigned long long)r.evals64);
        atomicAdd(&a.stats->evals_df, (unsigned long long)r.evals_df);
        atomicAdd(&a.stats->iters32, (unsigned long long)r.iters32);
        atomicAdd(&a.stats->iters64, (unsigned long long)r.iters64);
        atomicAdd(&a.stats->pairs32, np * (unsigned long long)r.evals32);
        atomicAdd(&a.stats->pairs64, np * (unsigned long long)r.evals64);
        atomicAdd(&a.stats->pairs_df, np * (unsigned long long)r.evals_df);
        atomicAdd(&a.stats->vec_elems32, (unsigned long long)r.vec32);
        atomicAdd(&a.stats->vec_elems64, (unsigned long long)r.vec64);
        atomicAdd(&a.stats->converged, r.status == ST_CONVERGED ? 1ULL : 0ULL);
        atomicAdd(&a.stats->minimisations, 1ULL);
        atomicAdd(&a.stats->cycles32, (unsigned long long)r.cyc32);
        atomicAdd(&a.stats->cycles_df, (unsigned long long)r.cycdf);
        atomicAdd(&a.stats->cycles64, (unsigned long long)r.cyc64);
        atomicAdd(&a.stats->cycles_direction, (unsigned long long)r.cycdir);
        atomicAdd(&a.stats->cycles_linesearch, (unsigned long long)r.cycls);
      }
    }
  }
}

template <int T, int A, bool MIXED, int POT>
cudaError_t plan_one(int max_n, int m, int64_t n_cand, int device, ljh::Plan* out,
                     bool hist_global) {
  constexpr int threads = cta_threads_for(T);
  constexpr int TPC = threads / T;
  const size_t hist_bytes = align16(2 * (size_t)m * A * 3 * T * (MIXED ? sizeof(float) : sizeof(double)));
  const bool on_chip =
      !hist_global && TPC * team_smem_bytes<T>(max_n, true, hist_bytes) <= kSmemBudget;
  const size_t smem = TPC * team_smem_bytes<T>(max_n, true, on_chip ? hist_bytes : 0);
  auto k = lbfgs_kernel<T, A, MIXED, POT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long need = (n_cand + TPC - 1) / TPC;
  long long grid = (long long)per_sm * sms;
  if (need < grid) grid = need;
  if (grid < 1) grid = 1;
  out->team = T;
  out->teams_per_cta = TPC;
  out->grid = (int)grid;
  out->smem = smem;
  out->slots = on_chip ? 0 : grid * TPC;
  out->slot_bytes = hist_bytes;
  out->hist_on_chip = on_chip ? 1 : 0;
  return cudaSuccess;
}

}  // namespace ljlb

namespace ljlb {

// Team size: the default by cluster size, or the team chosen with
// LJ_OPT_LBFGS_TEAM (32 / 64 / 128 threads) for clusters of up to 64 atoms.
template <class F>
cudaError_t dispatch_lb(int max_n, int team, F&& f) {
  // team = 0: the default shape for max_n; otherwise `team` threads per
  // candidate with A = ceil(max_n / team) atoms per thread when A <= 2 (a
  // team too small for max_n falls back to the default)
  using std::integral_constant;
  switch (team) {
    case 32:
      if (max_n <= 32) return f(integral_constant<int, 32>{}, integral_constant<int, 1>{});
      if (max_n <= 64) return f(integral_constant<int, 32>{}, integral_constant<int, 2>{});
      break;
    case 64:
      if (max_n <= 64) return f(integral_constant<int, 64>{}, integral_constant<int, 1>{});
      if (max_n <= 128) return f(integral_constant<int, 64>{}, integral_constant<int, 2>{});
      break;
    case 128:
      if (max_n <= 128) return f(integral_constant<int, 128>{}, integral_constant<int, 1>{});
      if (max_n <= 256) return f(integral_constant<int, 128>{}, integral_constant<int, 2>{});
      break;
    case 256:
      if (max_n <= 256) return f(integral_constant<int, 256>{}, integral_constant<int, 1>{});
      if (max_n <= 512) return f(integral_constant<int, 256>{}, integral_constant<int, 2>{});
      break;
    case 512:
      if (max_n <= 512) return f(integral_constant<int, 512>{}, integral_constant<int, 1>{});
      if (max_n <= 1024) return f(integral_constant<int, 512>{}, integral_constant<int, 2>{});
      break;
    default:
      // measured on GB300 (uneven cube starts, mixed and FP64 alike): one atom
      // per thread beats two up to 128 atoms
      if (max_n > 32 && max_n <= 64)
        return f(integral_constant<int, 64>{}, integral_constant<int, 1>{});
      if (max_n > 64 && max_n <= 128)
        return f(integral_constant<int, 128>{}, integral_constant<int, 1>{});
      break;
  }
  return dispatch_team(max_n, f);
}

template <bool MIXED, int POT = LJ_POT_LJ>
cudaError_t plan_impl(int max_n, int m, int64_t n_cand, int device, int team, ljh::Plan* out,
                      bool hist_global) {
  return dispatch_lb(max_n, team, [&](auto TT, auto AA) -> cudaError_t {
    return plan_one<decltype(TT)::value, decltype(AA)::value, MIXED, POT>(max_n, m, n_cand, device,
                                                                          out, hist_global);
  });
}

template <bool MIXED, int POT = LJ_POT_LJ>
cudaError_t launch_impl(const ljh::LbfgsArgs& a, const ljh::Plan& plan, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  return dispatch_lb(a.max_n, plan.team, [&](auto TT, auto AA) -> cudaError_t {
    constexpr int T = decltype(TT)::value;
    constexpr int A = decltype(AA)::value;
    lbfgs_kernel<T, A, MIXED, POT><<<plan.grid, cta_threads_for(T), plan.smem, s>>>(a);
    return cudaGetLastError();
  });
}

}  // namespace ljlb

