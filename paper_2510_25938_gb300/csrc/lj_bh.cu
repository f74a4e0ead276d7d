// lj_bh.cu -- bh_step_batched: whole Basin Hopping steps in one launch.
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
// The walker's x_cur and x_best live in shared memory for all n_steps; the
// winning team copies its registers into x_cur on acceptance.
#include "lj_internal.h"
#include "lj_minimize.cuh"
#include "lj_teams.cuh"

namespace {

using namespace ljd;

__device__ __forceinline__ MinParams to_dev(const ljh::MinParamsH& h) {
  MinParams p;
  p.m = h.m; p.max_iter = h.max_iter; p.max_ls = h.max_ls;
  p.gtol = h.gtol; p.c1 = h.c1; p.c2 = h.c2; p.alpha_max = h.alpha_max;
  p.switch_gtol = h.switch_gtol; p.deadline = h.deadline; p.eps = h.eps; p.sigma = h.sigma;
  return p;
}

struct BhShared {          // walker scalars, owned by thread 0 between barriers
  double e_cur, e_best, step;
  int win, nacc;
  int acc, kbest, better;
};

template <int T>
__host__ __device__ constexpr size_t bh_head_bytes(int n_atoms, int K) {
  return align16(sizeof(BhShared)) + align16((size_t)K * sizeof(double)) +
         2 * align16((size_t)3 * n_atoms * sizeof(double));
}

template <int T, int A, bool MIXED>
__global__ void __launch_bounds__(256) bh_kernel(ljh::BhArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = a.n_atoms;
  const int K = a.K;
  const int w = blockIdx.x;
  const int k = threadIdx.x / T;
  Team<T> tm;
  tm.rank = threadIdx.x % T;
  tm.bar = k + 1;
  unsigned char* sp = smem;
  BhShared* sh = reinterpret_cast<BhShared*>(sp);
  sp += align16(sizeof(BhShared));
  double* ek = reinterpret_cast<double*>(sp);
  sp += align16((size_t)K * sizeof(double));
  double* xcur = reinterpret_cast<double*>(sp);
  sp += align16((size_t)3 * n * sizeof(double));
  double* xbest = reinterpret_cast<double*>(sp);
  sp += align16((size_t)3 * n * sizeof(double));
  void* pos;
  long long* word;
  carve_team<T>(sp + k * team_smem_bytes<T>(n), n, pos, tm.red, word);
  const MinParams p = to_dev(a.p);
  void* hist = static_cast<unsigned char*>(a.hist) + ((size_t)w * K + k) * a.hist_slot_bytes;
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
    // 1. perturbation of the atoms this thread owns
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
    // 2. local minimisation
    MinResult r;
    minimise<T, A, MIXED>(tm, n, x64, p, hist, pos, r);
    if (tm.rank == 0) {
      ek[k] = r.E;
      const size_t tix = ((size_t)it * a.n_walkers + w) * K + k;
      if (a.tr.trial_e) a.tr.trial_e[tix] = r.E;
      if (a.tr.trial_status) a.tr.trial_status[tix] = r.status;
      if (a.tr.trial_iters) a.tr.trial_iters[tix] = r.iters;
      if (a.stats) {
        const unsigned long long np = (unsigned long long)n * (unsigned long long)(n - 1) / 2;
        atomicAdd(&a.stats->evals32, (unsigned long long)r.evals32);
        atomicAdd(&a.stats->evals64, (unsigned long long)r.evals64);
        atomicAdd(&a.stats->iters32, (unsigned long long)r.iters32);
        atomicAdd(&a.stats->iters64, (unsigned long long)r.iters64);
        atomicAdd(&a.stats->pairs32, np * (unsigned long long)r.evals32);
        atomicAdd(&a.stats->pairs64, np * (unsigned long long)r.evals64);
        atomicAdd(&a.stats->vec_elems32, (unsigned long long)r.vec32);
        atomicAdd(&a.stats->vec_elems64, (unsigned long long)r.vec64);
        atomicAdd(&a.stats->converged, r.status == ST_CONVERGED ? 1ULL : 0ULL);
        atomicAdd(&a.stats->minimisations, 1ULL);
      }
    }
    __syncthreads();
    // 3-5. selection, Metropolis, adaptation (one thread)
    if (threadIdx.x == 0) {
      int kb = -1;
      for (int kk = 0; kk < K; ++kk) {
        const double e = ek[kk];
        if (isfinite(e) && (kb < 0 || e < ek[kb])) kb = kk;
      }
      int acc = 0, better = 0;
      double e_sel = __longlong_as_double(0x7ff0000000000000LL);
      if (kb >= 0) {
        e_sel = ek[kb];
        const double u = stream_u01(a.seed, 2u, 0u, 0u, s, wg);
        const double de = e_sel - sh->e_cur;
        acc = (de <= 0.0) || (u < exp(-de / a.kT));
      }
      const size_t tw = (size_t)it * a.n_walkers + w;
      if (a.tr.best_trial_e) a.tr.best_trial_e[tw] = e_sel;
      if (a.tr.accepted) a.tr.accepted[tw] = (uint8_t)acc;
      if (a.tr.stepsize) a.tr.stepsize[tw] = step;
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
    if (sh->acc && k == sh->kbest) {
#pragma unroll
      for (int sl = 0; sl < A; ++sl) {
        const int i = tm.rank + sl * T;
        if (i < n) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            xcur[3 * i + c] = x64[sl][c];
            if (sh->better) xbest[3 * i + c] = x64[sl][c];
          }
        }
      }
    }
    __syncthreads();
  }
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

template <int T, int A, bool MIXED>
cudaError_t plan_one(int n_atoms, int m, int n_walkers, int K, ljh::Plan* out) {
  if (K * T > 256) return cudaErrorNotSupported;
  const size_t smem = bh_head_bytes<T>(n_atoms, K) + (size_t)K * team_smem_bytes<T>(n_atoms);
  auto k = bh_kernel<T, A, MIXED>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  out->team = T;
  out->teams_per_cta = K;
  out->grid = n_walkers;
  out->smem = smem;
  out->slots = (int64_t)n_walkers * K;
  out->slot_bytes = align16(2 * (size_t)m * A * 3 * T * (MIXED ? sizeof(float) : sizeof(double)));
  return cudaSuccess;
}

}  // namespace

namespace ljh {

// Basin Hopping keeps a walker's K teams in one CTA, so it supports the team
// sizes up to 256 atoms per cluster.
template <class F>
static cudaError_t dispatch_bh(int n, F&& f) {
  if (n > 256) return cudaErrorNotSupported;
  return dispatch_team(n, f);
}

cudaError_t bh_plan(int n_atoms, int m, int mixed, int n_walkers, int K, Plan* out) {
  return dispatch_bh(n_atoms, [&](auto TT, auto AA) -> cudaError_t {
    constexpr int T = decltype(TT)::value;
    constexpr int A = decltype(AA)::value;
    return mixed ? plan_one<T, A, true>(n_atoms, m, n_walkers, K, out)
                 : plan_one<T, A, false>(n_atoms, m, n_walkers, K, out);
  });
}

cudaError_t bh_launch(const BhArgs& a, const Plan& plan, cudaStream_t s) {
  return dispatch_bh(a.n_atoms, [&](auto TT, auto AA) -> cudaError_t {
    constexpr int T = decltype(TT)::value;
    constexpr int A = decltype(AA)::value;
    const int threads = a.K * T;
    if (a.mixed) {
      bh_kernel<T, A, true><<<plan.grid, threads, plan.smem, s>>>(a);
    } else {
      bh_kernel<T, A, false><<<plan.grid, threads, plan.smem, s>>>(a);
    }
    return cudaGetLastError();
  });
}

}  // namespace ljh
