// lj_internal.h -- host-side interface between the C-ABI layer (lj_api.cu)
// and the kernel translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/lj_bh.h"
#include "lj_consts.h"

namespace ljd { struct MinParams; }

namespace ljh {

struct MinParamsH {     // mirror of ljd::MinParams (plain data)
  int m, max_iter, max_ls;
  double gtol, c1, c2, alpha_max, switch_gtol;
  long long deadline;
  LjConsts k;             // pair-potential constants (Eq. (1) or Morse)
  double f32_resolution, df_resolution;   // handover thresholds, relative to |E|
  int df_one_sided = 0;   // double-float evaluations in one-sided rows even where
                          // the team could use tiles (clusters above 256 atoms)
};

struct EvalArgs {
  int64_t n_cand;
  int uniform_n;
  const int64_t* off;
  int max_n;
  int xtype;            // LJ_F32 / LJ_F64
  int prec;             // LJ_PREC_*
  const void* x;
  double* energy;
  void* grad;
  LjConsts k;           // pair-potential constants (Eq. (1) or Morse)
};

struct LbfgsArgs {
  int64_t n_cand;
  int uniform_n;
  const int64_t* off;
  int max_n;
  MinParamsH p;
  int mixed;
  double* x;
  double* energy;
  int32_t* status;
  int32_t* iters;
  int32_t* nevals;
  lj_stats* stats;
  unsigned long long* queue;   // zeroed before the launch
  void* hist;
  size_t hist_slot_bytes;
  int hist_on_chip;            // history in shared memory (hist unused)
  const int* list = nullptr;   // bucketed launch: candidate indices of this bucket
  const unsigned* list_count = nullptr;   // ... and their number (device)
};

// size classes of a bucketed uneven batch (upper atom count per bucket)
constexpr int kMaxBuckets = 6;
struct Buckets {
  int bound[kMaxBuckets];
};

struct BhArgs {
  int n_walkers, n_atoms;
  double *x_cur, *e_cur, *x_best, *e_best, *stepsize;
  int32_t *win_accept, *n_accept;
  int K;
  double kT, target_rate, factor;
  int interval;
  unsigned long long seed;
  long long step0;
  int n_steps;
  long long walker0;
  MinParamsH p;
  int mixed;
  lj_bh_trace tr;
  lj_stats* stats;
  void* hist;
  size_t hist_slot_bytes;
  int hist_on_chip;            // history in shared memory (hist unused)
};

struct Plan {
  int team;          // threads per team
  int teams_per_cta;
  int grid;          // CTAs
  size_t smem;       // dynamic shared memory per CTA
  int64_t slots;     // history slots the launch needs
  size_t slot_bytes; // bytes per history slot
  int cluster = 1;   // CTAs per thread-block cluster (Basin Hopping: K)
  int hist_on_chip = 0;   // L-BFGS history in shared memory
};

// largest atom count this build supports
constexpr int kMaxAtoms = LJ_MAX_ATOMS;

cudaError_t eval_launch(const EvalArgs& a, cudaStream_t s);
// team: threads per candidate requested for clusters of up to 64 atoms
// (32, 64 or 128); any other value picks the default for the cluster size.
// hist_global: keep the L-BFGS history in global memory even where it would
// fit in shared memory (a tuning choice; results do not change)
cudaError_t lbfgs_plan_fp64(int max_n, int m, int64_t n_cand, int device, int team, Plan* out,
                            bool hist_global = false);
cudaError_t lbfgs_plan_mixed(int max_n, int m, int64_t n_cand, int device, int team, Plan* out,
                             bool hist_global = false);
cudaError_t lbfgs_launch_fp64(const LbfgsArgs& a, const Plan& plan, cudaStream_t s);
cudaError_t lbfgs_launch_mixed(const LbfgsArgs& a, const Plan& plan, cudaStream_t s);
// sort candidates of an uneven batch into size buckets (device, no sync)
cudaError_t bucketize_launch(const int64_t* off, int64_t n_cand, int nb, const Buckets& bk,
                             unsigned* counts, int* lists, cudaStream_t s);
// autotuner inputs: n_cand uniform cube starts of n atoms, side `side` (device)
cudaError_t tune_starts_launch(double* x, int64_t n_cand, int n, double side, uint64_t seed,
                               cudaStream_t s);
cudaError_t bh_plan_fp64(int n_atoms, int m, int n_walkers, int K, int team, Plan* out,
                         bool hist_global = false);
cudaError_t bh_plan_mixed(int n_atoms, int m, int n_walkers, int K, int team, Plan* out,
                          bool hist_global = false);
cudaError_t bh_launch_fp64(const BhArgs& a, const Plan& plan, cudaStream_t s);
cudaError_t bh_launch_mixed(const BhArgs& a, const Plan& plan, cudaStream_t s);

// the same kernels on the Morse pair potential (lj_morse_*.cu)
cudaError_t lbfgs_plan_morse_fp64(int max_n, int m, int64_t n_cand, int device, int team,
                                  Plan* out, bool hist_global);
cudaError_t lbfgs_plan_morse_mixed(int max_n, int m, int64_t n_cand, int device, int team,
                                   Plan* out, bool hist_global);
cudaError_t lbfgs_launch_morse_fp64(const LbfgsArgs& a, const Plan& plan, cudaStream_t s);
cudaError_t lbfgs_launch_morse_mixed(const LbfgsArgs& a, const Plan& plan, cudaStream_t s);
cudaError_t bh_plan_morse_fp64(int n_atoms, int m, int n_walkers, int K, int team, Plan* out,
                               bool hist_global);
cudaError_t bh_plan_morse_mixed(int n_atoms, int m, int n_walkers, int K, int team, Plan* out,
                                bool hist_global);
cudaError_t bh_launch_morse_fp64(const BhArgs& a, const Plan& plan, cudaStream_t s);
cudaError_t bh_launch_morse_mixed(const BhArgs& a, const Plan& plan, cudaStream_t s);

// plan / launch by precision and pair potential
inline cudaError_t lbfgs_plan(bool mixed, int pot, int max_n, int m, int64_t n_cand, int device,
                              int team, Plan* out, bool hist_global = false) {
  if (pot == LJ_POT_MORSE)
    return mixed ? lbfgs_plan_morse_mixed(max_n, m, n_cand, device, team, out, hist_global)
                 : lbfgs_plan_morse_fp64(max_n, m, n_cand, device, team, out, hist_global);
  return mixed ? lbfgs_plan_mixed(max_n, m, n_cand, device, team, out, hist_global)
               : lbfgs_plan_fp64(max_n, m, n_cand, device, team, out, hist_global);
}
inline cudaError_t lbfgs_launch(const LbfgsArgs& a, const Plan& plan, cudaStream_t s) {
  if (a.p.k.pot == LJ_POT_MORSE)
    return a.mixed ? lbfgs_launch_morse_mixed(a, plan, s) : lbfgs_launch_morse_fp64(a, plan, s);
  return a.mixed ? lbfgs_launch_mixed(a, plan, s) : lbfgs_launch_fp64(a, plan, s);
}
inline cudaError_t bh_plan(bool mixed, int pot, int n_atoms, int m, int n_walkers, int K,
                           int team, Plan* out, bool hist_global = false) {
  if (pot == LJ_POT_MORSE)
    return mixed ? bh_plan_morse_mixed(n_atoms, m, n_walkers, K, team, out, hist_global)
                 : bh_plan_morse_fp64(n_atoms, m, n_walkers, K, team, out, hist_global);
  return mixed ? bh_plan_mixed(n_atoms, m, n_walkers, K, team, out, hist_global)
               : bh_plan_fp64(n_atoms, m, n_walkers, K, team, out, hist_global);
}
inline cudaError_t bh_launch(const BhArgs& a, const Plan& plan, cudaStream_t s) {
  if (a.p.k.pot == LJ_POT_MORSE)
    return a.mixed ? bh_launch_morse_mixed(a, plan, s) : bh_launch_morse_fp64(a, plan, s);
  return a.mixed ? bh_launch_mixed(a, plan, s) : bh_launch_fp64(a, plan, s);
}

}  // namespace ljh
