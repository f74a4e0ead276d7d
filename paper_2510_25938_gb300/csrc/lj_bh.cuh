// lj_bh.cuh -- bh_step_batched: whole Basin Hopping steps in one launch.
//
// One CTA per walker; its K teams (one per candidate) run, for each step
// (arXiv 2510.25938, Methodology, "Algorithm Overview"):
//   1. perturbation: x_k = x_cur + step * (2u - 1) for every coordinate, u from
//      Philox stream 1 at counter (coordinate, k, s, w) -- each team perturbs
//      the atoms it owns, straight into registers;
//   2. local minimisation of the K candidates in parallel (lj_minimize.cuh);
//   3. selection: the lowest finite FP64 energy (ties: lowest k);
//   4. Metropolis: accept if dE <= 0 or u < exp(-dE / kT), u from stream 2;
//   5. adaptation: after every step s with (s+1) % interval == 0 the window
//      acceptance rate moves the step size (up if above target, else down).
// Layout: one thread-block cluster per walker and one CTA (one team) per
// candidate (K <= 16), so the W*K candidates spread over every SM.  Each CTA
// keeps a replica of the walker state (x_cur, x_best, scalars) in shared
// memory for all n_steps; after the minimisations the CTAs read each other's
// energies and the winner's coordinates through distributed shared memory,
// and every CTA takes the same (deterministic) decision.
#pragma once
#include <cooperative_groups.h>

#include "lj_internal.h"
#include "lj_minimize.cuh"
#include "lj_teams.cuh"

namespace cg = cooperative_groups;

namespace ljbh {

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

struct BhShared {          // walker scalars, owned by thread 0 between barriers
  double e_cur, e_best, step;
  int win, nacc;
  int acc, kbest, better;
};

template <int T>
__host__ __device__ constexpr size_t bhc_head_bytes(int n_atoms) {
  return align16(sizeof(BhShared)) + 16 + 3 * align16((size_t)3 * n_atoms * sizeof(double));
}

// Teams of up to 64 threads ask for 3 CTAs per SM, which leaves ptxas the
// full 255 registers (no spills); its default stopped at 168 with spills.
// Measured on LJ38, 64 walkers x K = 8: 23.9 against 25.9 ms per 10-step
// launch.  At 255 registers 4 CTAs of 64 threads fit on an SM (608 on 152
// SMs, more than the 512 CTAs of that workload).
// POT: pair potential (LJ_POT_LJ, Eq. (1); LJ_POT_MORSE).
template <int T, int A, bool MIXED, int POT = LJ_POT_LJ>
__global__ void __launch_bounds__(T, T <= 64 ? 3 : 0) bh_cluster_kernel(ljh::BhArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cl = cg::this_cluster();
  const int n = a.n_atoms;
  const int K = a.K;
  const int k = (int)cl.block_rank();
  const int w = blockIdx.x / K;
  Team<T> tm;
  tm.rank = threadIdx.x;
  tm.bar = 1;
  unsigned char* sp = smem;
  BhShared* sh = reinterpret_cast<BhShared*>(sp);
  sp += align16(sizeof(BhShared));
  double* my_e = reinterpret_cast<double*>(sp);       // this candidate's energy
  sp += 16;
  double* xmine = reinterpret_cast<double*>(sp);      // this candidate's minimum
  sp += align16((size_t)3 * n * sizeof(double));
  double* xcur = reinterpret_cast<double*>(sp);
  sp += align16((size_t)3 * n * sizeof(double));
  double* xbest = reinterpret_cast<double*>(sp);
  sp += align16((size_t)3 * n * sizeof(double));
  void* pos;
  void* hbuf;
  void* hist;
  long long* word;
  carve_team<T>(sp, n, true, a.hist_on_chip ? a.hist_slot_bytes : 0, pos, hbuf, hist, tm.red,
                word);
  MinParams p = to_dev(a.p);
  // hbuf: pair buffer up to 64 atoms, tile accumulators above 256; with
  // one-sided rows chosen above 256 atoms it holds no pairs and is withdrawn
  p.tiled = n > kTileMinN && !a.p.df_one_sided;
  if (n > kTileMinN && a.p.df_one_sided) hbuf = nullptr;
  if (!a.hist_on_chip)
    hist = static_cast<unsigned char*>(a.hist) + ((size_t)w * K + k) * a.hist_slot_bytes;
  const uint32_t wg = (uint32_t)(a.walker0 + w);
  const int n3 = 3 * n;

  for (int q = threadIdx.x; q < n3; q += blockDim.x) {
    xcur[q] = a.x_cur[(size_t)w * n3 + q];
    xbest[q] = a.x_best[(size_t)w * n3 + q];
  }
  if (threadIdx.x == 0) {
    sh->e_cur = a.e_cur[w];
    sh->e_best = a.e_best[w];
    sh->step = a.stepsize[w];
    sh->win = a.win_accept[w];
    sh->nacc = a.n_accept[w];
  }
  __syncthreads();

  for (int it = 0; it < a.n_steps; ++it) {
    const long long s64 = a.step0 + it;
    const uint32_t s = (uint32_t)s64;
    const double step = sh->step;
    double x64[A][3];
#pragma unroll
    for (int sl = 0; sl < A; ++sl) {
      const int i = tm.rank + sl * T;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (i < n) {
          const int qd = 3 * i + c;
          const double u = stream_u01(a.seed, 1u, (uint32_t)qd, (uint32_t)k, s, wg);
          const double delta = __dmul_rn(step, __dsub_rn(__dmul_rn(2.0, u), 1.0));
          x64[sl][c] = __dadd_rn(xcur[qd], delta);
        } else {
          x64[sl][c] = 0.0;
        }
      }
    }
    MinResult r;
    minimise<T, A, MIXED, POT>(tm, n, x64, p, hist, pos, hbuf, r);
#pragma unroll
    for (int sl = 0; sl < A; ++sl) {
      const int i = tm.rank + sl * T;
      if (i < n) {
#pragma unroll
        for (int c = 0; c < 3; ++c) xmine[3 * i + c] = x64[sl][c];
      }
    }
    if (tm.rank == 0) {
      *my_e = r.E;
      const size_t tix = ((size_t)it * a.n_walkers + w) * K + k;
      if (a.tr.trial_e) a.tr.trial_e[tix] = r.E;
      if (a.tr.trial_status) a.tr.trial_status[tix] = r.status;
      if (a.tr.trial_iters) a.tr.trial_iters[tix] = r.iters;
      if (a.stats) {
        const unsigned long long np = (unsigned long long)n * (unsigned long long)(n - 1) / 2;
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
    cl.sync();   // every candidate's energy and minimum are visible cluster-wide
    if (threadIdx.x == 0) {
      int kb = -1;
      double eb = 0.0;
      for (int kk = 0; kk < K; ++kk) {
        const double e = *cl.map_shared_rank(my_e, kk);
        if (isfinite(e) && (kb < 0 || e < eb)) { kb = kk; eb = e; }
      }
      int acc = 0, better = 0, tie = 0;
      double e_sel = __longlong_as_double(0x7ff0000000000000LL);
      if (kb >= 0) {
        e_sel = eb;
        const double u = stream_u01(a.seed, 2u, 0u, 0u, s, wg);
        const double de = e_sel - sh->e_cur;
        const double thr = de > 0.0 ? exp(-de / a.kT) : 1.0;
        acc = (de <= 0.0) || (u < thr);
        // a decision within rounding of its threshold (see LJ_NEAR_TIE)
        tie = fabs(de) <= LJ_NEAR_TIE || (de > 0.0 && fabs(u - thr) <= LJ_NEAR_TIE * thr);
      }
      if (k == 0) {
        const size_t tw = (size_t)it * a.n_walkers + w;
        if (a.tr.best_trial_e) a.tr.best_trial_e[tw] = e_sel;
        if (a.tr.accepted) a.tr.accepted[tw] = (uint8_t)acc;
        if (a.tr.stepsize) a.tr.stepsize[tw] = step;
        if (a.tr.near_tie) a.tr.near_tie[tw] = (uint8_t)tie;
      }
      if (acc) {
        sh->e_cur = e_sel;
        sh->nacc += 1;
        sh->win += 1;
        if (sh->e_cur < sh->e_best) {
          sh->e_best = sh->e_cur;
          better = 1;
        }
      }
      if ((s64 + 1) % a.interval == 0) {
        const double rate = (double)sh->win / (double)a.interval;
        sh->step = rate > a.target_rate ? step / a.factor : step * a.factor;
        sh->win = 0;
      }
      sh->acc = acc;
      sh->kbest = kb;
      sh->better = better;
    }
    __syncthreads();
    if (sh->acc) {
      const double* xw = cl.map_shared_rank(xmine, sh->kbest);
      for (int q = threadIdx.x; q < n3; q += blockDim.x) {
        const double v = xw[q];
        xcur[q] = v;
        if (sh->better) xbest[q] = v;
      }
    }
    cl.sync();   // nobody overwrites its energy / minimum while others read them
  }
  if (k == 0) {
    for (int q = threadIdx.x; q < n3; q += blockDim.x) {
      a.x_cur[(size_t)w * n3 + q] = xcur[q];
      a.x_best[(size_t)w * n3 + q] = xbest[q];
    }
    if (threadIdx.x == 0) {
      a.e_cur[w] = sh->e_cur;
      a.e_best[w] = sh->e_best;
      a.stepsize[w] = sh->step;
      a.win_accept[w] = sh->win;
      a.n_accept[w] = sh->nacc;
    }
  }
}

template <int T, int A, bool MIXED, int POT>
cudaError_t plan_one(int n_atoms, int m, int n_walkers, int K, ljh::Plan* out, bool hist_global) {
  out->slot_bytes = align16(2 * (size_t)m * A * 3 * T * (MIXED ? sizeof(float) : sizeof(double)));
  out->team = T;
  if (K <= LJ_MAX_K) {                // one cluster of K CTAs per walker
    const bool on_chip = !hist_global && bhc_head_bytes<T>(n_atoms) +
                                             team_smem_bytes<T>(n_atoms, true, out->slot_bytes) <=
                                         kSmemBudget;
    out->hist_on_chip = on_chip ? 1 : 0;
    out->slots = on_chip ? 0 : (int64_t)n_walkers * K;
    const size_t smem = bhc_head_bytes<T>(n_atoms) +
                        team_smem_bytes<T>(n_atoms, true, on_chip ? out->slot_bytes : 0);
    auto k = bh_cluster_kernel<T, A, MIXED, POT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (K > 8) {
      e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    out->teams_per_cta = 1;
    out->grid = n_walkers * K;
    out->smem = smem;
    out->cluster = K;
    return cudaSuccess;
  }
  return cudaErrorNotSupported;
}

template <int T, int A, bool MIXED, int POT>
cudaError_t launch_cluster(const ljh::BhArgs& a, const ljh::Plan& plan, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)plan.grid, 1, 1);
  cfg.blockDim = dim3(T, 1, 1);
  cfg.dynamicSmemBytes = plan.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)plan.cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  // the hardware's load-balancing placement of a cluster's CTAs: on LJ38,
  // 64 walkers x K = 8, 47.2 against 48.1 ms per 25-step launch for the
  // default placement and for spreading a cluster's CTAs over SMs
  attr[1].id = cudaLaunchAttributeClusterSchedulingPolicyPreference;
  attr[1].val.clusterSchedulingPolicyPreference = cudaClusterSchedulingPolicyLoadBalancing;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, bh_cluster_kernel<T, A, MIXED, POT>, a);
}

}  // namespace ljbh

namespace ljbh {

// Team size for one candidate: the default by cluster size (64 threads for
// 33..64 atoms), or the team chosen with LJ_OPT_BH_TEAM (32 / 64 / 128
// threads) for clusters of up to 64 atoms.
template <class F>
cudaError_t dispatch_bh(int n, int team, F&& f) {
  using std::integral_constant;
  // measured on GB300 (LJ38, 64 walkers x K=8): 64 threads per candidate beat
  // 32 (one warp, two atoms per thread) and 128 (fewer clusters resident)
  if (team == 0 && n > 32 && n <= 64) team = 64;
  if (n <= 64 && team == 64) return f(integral_constant<int, 64>{}, integral_constant<int, 1>{});
  if (n <= 64 && team == 128) return f(integral_constant<int, 128>{}, integral_constant<int, 1>{});
  if (n <= 32) return f(integral_constant<int, 32>{}, integral_constant<int, 1>{});
  if (n <= 64) return f(integral_constant<int, 32>{}, integral_constant<int, 2>{});
  if (n <= 128) return f(integral_constant<int, 64>{}, integral_constant<int, 2>{});
  if (n <= 256) return f(integral_constant<int, 128>{}, integral_constant<int, 2>{});
  return cudaErrorNotSupported;
}

template <bool MIXED, int POT = LJ_POT_LJ>
cudaError_t plan_impl(int n_atoms, int m, int n_walkers, int K, int team, ljh::Plan* out,
                      bool hist_global) {
  return dispatch_bh(n_atoms, team, [&](auto TT, auto AA) -> cudaError_t {
    return plan_one<decltype(TT)::value, decltype(AA)::value, MIXED, POT>(n_atoms, m, n_walkers, K,
                                                                          out, hist_global);
  });
}

template <bool MIXED, int POT = LJ_POT_LJ>
cudaError_t launch_impl(const ljh::BhArgs& a, const ljh::Plan& plan, cudaStream_t s) {
  return dispatch_bh(a.n_atoms, plan.team, [&](auto TT, auto AA) -> cudaError_t {
    cudaError_t e =
        launch_cluster<decltype(TT)::value, decltype(AA)::value, MIXED, POT>(a, plan, s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  });
}

}  // namespace ljbh
