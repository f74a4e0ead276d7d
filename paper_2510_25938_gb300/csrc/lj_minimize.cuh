// lj_minimize.cuh -- one team minimises one LJ cluster with L-BFGS.
//
// Method (arXiv 2510.25938, Methodology, "Algorithm Overview" step 2 and
// "Implementation Notes": L-BFGS-B from scipy, no bounds), read as:
//   direction   two-loop recursion, H0 = (s^T y / y^T y) I of the newest pair
//               (Nocedal & Wright Alg. 7.4); steepest descent when the
//               history is empty or the direction is not a descent direction;
//   first trial alpha = min(1, 1/||d||_2) with an empty history, else 1;
//   line search strong Wolfe, c1 = 1e-3, c2 = 0.9, bracketing with doubling
//               (N&W Alg. 3.5) and zoom with safeguarded cubic interpolation
//               (N&W Alg. 3.6, eq. 3.59); a non-finite energy fails the
//               sufficient-decrease test; after max_ls evaluations the best
//               sufficient-decrease point is taken if it strictly lowers E;
//               on failure one retry along -g with an empty history;
//   curvature   the pair (s, y) is stored only if s^T y > eps_mach y^T y;
//   stopping    ||g||_inf < gtol after each accepted step (and at the start).
//
// Precision (GB300: FP64 issues ~1/62 of FP32, the FP64 reciprocal less):
//   FP64 path   every operation in FP64.
//   MIXED path  phase 1: coordinates, gradient, directions and history in
//               FP32, energy as float-float, line-search scalars in FP32, no
//               FP64 instruction at all; it ends when ||g32||_inf <
//               switch_gtol, when the predicted decrease falls below the FP32
//               energy resolution, or when its line search fails.
//               phase 2 (polish): coordinates and pair terms in double-float
//               arithmetic (FP32 pipes, ~1e-14 relative), gradient FP32
//               (only its relative precision is used there), energies
//               float-float, line-search scalars FP32: no FP64 instruction.
//               It hands over once the predicted decrease falls below the
//               double-float energy resolution (~32 * 2^-48 |E|).
//               phase 3: FP64 coordinates, gradient, energy and pair terms
//               for the last iterations (FP32 directions and scalars); the
//               convergence test and the returned energy are always FP64.
#pragma once
#include <type_traits>

#include "lj_device.cuh"
#include "lj_consts.h"
#include "../../include/lj_bh.h"

namespace ljd {

struct MinParams {
  int m, max_iter, max_ls;
  double gtol, c1, c2, alpha_max, switch_gtol;
  long long deadline;
  ljh::LjConsts k;         // pair-potential constants (host-derived)
  int tiled;               // hbuf holds tile accumulators (teams for > 64 atoms), not pairs
  double f32_resolution;   // FP32 phase hands over below this predicted decrease / |E|
  double df_resolution;    // double-float polish hands over below this / |E|
};

struct MinResult {
  double E;
  int status;
  int iters;
  int evals32, evals64, evals_df, iters32, iters64;
  long long vec32, vec64;   // sum over iterations of (history used) * 3N
  long long cyc32, cycdf, cyc64;   // SM clock cycles spent in each tier
  long long cycdir, cycls;          // ... in direction computations and line searches
};

enum : int { PH_CONVERGED = 0, PH_MAXITER = 1, PH_LSFAIL = 2, PH_SWITCH = 3, PH_TIMEOUT = 4 };

// FP32-tier iterations after which gradient-only FP32 steps hand over: a
// safety net for a switch_gtol below the FP32 gradient noise (~3e-5 eps/sigma
// on LJ clusters); normal minimisations stay far below it
constexpr int kFP32GradIters = 2000;

// Precision policy of an L-BFGS tier.
//   XP positions (float, double, or ff = double-float), XG gradient, V search
//   directions and history, PM pair arithmetic (0: XP's own, 1: double-float).
//   S line-search scalars: FP64 only on the all-FP64 path.  F energies: FP64
//   when positions are FP64, float-float otherwise (FP32 pipes only).
template <typename XP_, typename XG_, typename V_, int PM_, int POT_ = LJ_POT_LJ>
struct Prec {
  using XP = XP_;
  using XG = XG_;
  using V = V_;
  static constexpr int PM = PM_;
  static constexpr int POT = POT_;   // pair potential: LJ_POT_LJ or LJ_POT_MORSE
  using S = std::conditional_t<sizeof(V_) == 8, double, float>;
  using F = std::conditional_t<std::is_same<XP_, double>::value, double, ff>;
};
using PrecF32 = Prec<float, float, float, 0>;      // mixed: FP32 tier
using PrecDF = Prec<ff, float, float, 1>;          // mixed: double-float tier
using PrecF64m = Prec<double, double, float, 0>;   // mixed: FP64 tier
using PrecF64 = Prec<double, double, double, 0>;   // FP64 path

// Eval-only helper: scalars of a plain single-precision evaluation.
template <typename X> struct Tr;
template <> struct Tr<float> { using S = float; using F = ff; };
template <> struct Tr<double> { using S = double; using F = double; };

// trial position x + a d and step xt - x for each position type
__device__ __forceinline__ float pos_step(float x, float a, float d) { return x + a * d; }
template <typename SA, typename VD>
__device__ __forceinline__ double pos_step(double x, SA a, VD d) {
  return x + (double)a * (double)d;
}
__device__ __forceinline__ ff pos_step(ff x, float a, float d) {
  return df_add(x, df_two_prod(a, d));
}
template <typename V> __device__ __forceinline__ V pos_diff(float xt, float x) { return (V)(xt - x); }
template <typename V> __device__ __forceinline__ V pos_diff(double xt, double x) { return (V)(xt - x); }
template <typename V> __device__ __forceinline__ V pos_diff(ff xt, ff x) {
  const ff d = df_sub(xt, x);
  return (V)(d.hi + d.lo);
}

template <typename V> __device__ __forceinline__ V eps_mach();
template <> __device__ __forceinline__ float eps_mach<float>() { return 1.1920928955078125e-7f; }
template <> __device__ __forceinline__ double eps_mach<double>() { return 2.220446049250313e-16; }

__device__ __forceinline__ float S_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double S_sqrt(double x) { return sqrt(x); }

// history element (slot, atom slot a, component c) of this thread
template <int T, int A>
__device__ __forceinline__ int hidx(int slot, int a, int c, int rank) {
  return ((slot * A + a) * 3 + c) * T + rank;
}

// ---------------------------------------------------------------------------
// Energy and gradient at x (owned atoms), and dphi = g . d when d != nullptr.
// ---------------------------------------------------------------------------
// PM = 0: pair terms in X precision; PM = 1 (X = double only): pair terms in
// double-float arithmetic on coordinates scaled by 1/sigma.
// hbuf: the team's half-pair buffer (24 bytes per pair) or nullptr; used for
// FP64 / double-float evaluations, which then compute each pair once.
// ---------------------------------------------------------------------------
// Morse pair potential (Morse 1929, cluster form), the pair-potential
// extension of the method: V(r) = eps e (e - 2), e = exp(rho (1 - r / re)),
// re in the sigma slot.  One-sided rows: every thread sums, for each atom it
// owns, the terms of all other atoms (deterministic, no shared pair buffer);
// E = (eps / 2) sum_i sum_{j != i} e (e - 2), and
// g_i = -(2 eps rho / re) sum_{j != i} e (e - 1) (x_i - x_j) / r.
// FP32 (first tier of the mixed path; compensated energy), double-float
// (evaluate_morse_df, the polish tier) and FP64.  FP64 teams with
// a half-pair buffer (clusters of up to 64 atoms) take each pair once, as
// for Eq. (1): pair p's vector e (e - 1) (x_i - x_j) / r goes to the buffer,
// then every (atom, component) row is summed, +v over j > i, -v over j < i.
// Coincident atoms give E = +inf (and a non-finite gradient), as for Eq. (1).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pair_term_morse_f64(const PosD& a, const PosD& b, double rho,
                                                    double rr, double& vx, double& vy,
                                                    double& vz, double& e) {
  const double dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
  const double r = sqrt(r2);
  const double ex = exp(fma(-rr, r, rho));
  e = r2 > 0.0 ? ex * (ex - 2.0) : __longlong_as_double(0x7ff0000000000000LL);
  const double c = ex * (ex - 1.0) / r;
  vx = c * dx; vy = c * dy; vz = c * dz;
}

// Double-float Morse evaluation (the mixed path's polish tier): positions
// scaled by 1/re, pair terms by pair_term_morse_df (double-float exponential
// and square root); each pair once through the half-pair buffer for clusters
// of up to 64 atoms, one-sided rows above.
template <int T, int A, typename P>
__device__ __forceinline__ void evaluate_morse_df(const Team<T>& tm, int n,
                                                  const typename P::XP (&x)[A][3],
                                                  typename P::XG (&g)[A][3], void* posv,
                                                  void* hbuf, const MinParams& p,
                                                  const typename P::V (*d)[3],
                                                  typename P::F& E, typename P::S& dphi) {
  using V = typename P::V;
  using S = typename P::S;
  PosDF* pos = static_cast<PosDF*>(posv);
  tm.sync();  // previous readers of pos are done
#pragma unroll
  for (int a = 0; a < A; ++a) {
    const int i = tm.rank + a * T;
    if (i < n) {
      ff qx = x[a][0], qy = x[a][1], qz = x[a][2];
      if (p.k.sigma != 1.0) {
        const ff is{p.k.is_hi, p.k.is_lo};
        qx = df_mul(qx, is); qy = df_mul(qy, is); qz = df_mul(qz, is);
      }
      pos[i] = PosDF{qx.hi, qy.hi, qz.hi, 0.f, qx.lo, qy.lo, qz.lo, 0.f};
    }
  }
  tm.sync();
  const ff rho{p.k.rho_f, p.k.rho_lo};
  const float gs = p.k.m_g_f;
  V dp = (V)0;
  ff e{0.f, 0.f};
  if (hbuf != nullptr && !p.tiled) {
    const int np = n_pairs(n);
    ff* vb = static_cast<ff*>(hbuf);
    float* gsum = static_cast<float*>(posv);
    int i1, j1, i2, j2;
    pair_start(n, tm.rank, i1, j1);
    i2 = i1; j2 = j1;
    pair_advance(n, T, i2, j2);
    for (int q = tm.rank; q < np; q += 2 * T) {
      const bool two = q + T < np;
      const int ib = two ? i2 : 0, jb = two ? j2 : 1;
      ff ax, ay, az, ae, bx, by, bz, be;
      pair_term_morse_df(pos[i1], pos[j1], rho, ax, ay, az, ae);
      pair_term_morse_df(pos[ib], pos[jb], rho, bx, by, bz, be);
      vb[q] = ax; vb[np + q] = ay; vb[2 * np + q] = az;
      df_acc(e, ae);
      if (two) {
        vb[q + T] = bx; vb[np + q + T] = by; vb[2 * np + q + T] = bz;
        df_acc(e, be);
      }
      pair_advance(n, 2 * T, i1, j1);
      pair_advance(n, 2 * T, i2, j2);
    }
    tm.sync();
    for (int q3 = tm.rank; q3 < 3 * n; q3 += T) {
      const int ii = q3 / 3;
      const ff* vc = vb + (q3 - 3 * ii) * np;
      const int ri = row_base(n, ii);       // all lanes walk j together
      int rj = -1;
      ff sacc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
      for (int j0 = 0; j0 < n; j0 += 4) {
        ff v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = j0 + u;
          const int qq = j < ii ? rj + ii : ri + j;
          v[u] = ff{0.f, 0.f};
          if (j < n && j != ii) v[u] = vc[qq];
          if (j < ii) v[u] = ff{-v[u].hi, -v[u].lo};
          rj += n - j - 2;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) df_acc(sacc[u], v[u]);
      }
      const ff sum = df_add(df_add(sacc[0], sacc[1]), df_add(sacc[2], sacc[3]));
      gsum[q3] = -gs * (sum.hi + sum.lo);
    }
    tm.sync();
#pragma unroll
    for (int a = 0; a < A; ++a) {
      const int ii = tm.rank + a * T;
      if (ii < n) {
        g[a][0] = gsum[3 * ii]; g[a][1] = gsum[3 * ii + 1]; g[a][2] = gsum[3 * ii + 2];
      } else {
        g[a][0] = 0.f; g[a][1] = 0.f; g[a][2] = 0.f;
      }
      if (d) dp += (V)g[a][0] * d[a][0] + (V)g[a][1] * d[a][1] + (V)g[a][2] * d[a][2];
    }
    E = ff_scale(team_sum_ff<T>(tm, e), p.k.eps_f);
  } else {
#pragma unroll
    for (int a = 0; a < A; ++a) {
      const int i = tm.rank + a * T;
      if (i < n) {
        const PosDF pi = pos[i];
        ff ax{0.f, 0.f}, ay{0.f, 0.f}, az{0.f, 0.f};
        for (int j = 0; j < n; ++j) {
          ff vx, vy, vz, ep;
          pair_term_morse_df(pi, pos[j], rho, vx, vy, vz, ep);
          if (j != i) {
            df_acc(ax, vx); df_acc(ay, vy); df_acc(az, vz);
            df_acc(e, ep);
          }
        }
        g[a][0] = -gs * (ax.hi + ax.lo);
        g[a][1] = -gs * (ay.hi + ay.lo);
        g[a][2] = -gs * (az.hi + az.lo);
      } else {
        g[a][0] = 0.f; g[a][1] = 0.f; g[a][2] = 0.f;
      }
      if (d) dp += (V)g[a][0] * d[a][0] + (V)g[a][1] * d[a][1] + (V)g[a][2] * d[a][2];
    }
    E = ff_scale(team_sum_ff<T>(tm, e), p.k.m_half_f);
  }
  if (d) dphi = (S)team_sum1<T, V>(tm, dp);
}

template <int T, int A, typename P>
__device__ __forceinline__ void evaluate_morse(const Team<T>& tm, int n,
                                               const typename P::XP (&x)[A][3],
                                               typename P::XG (&g)[A][3], void* posv,
                                               void* hbuf, const MinParams& p,
                                               const typename P::V (*d)[3],
                                               typename P::F& E, typename P::S& dphi) {
  using X = typename P::XP;
  using V = typename P::V;
  using S = typename P::S;
  if constexpr (P::PM == 1) {
    evaluate_morse_df<T, A, P>(tm, n, x, g, posv, hbuf, p, d, E, dphi);
    return;
  } else {
  using Q = typename PosOf<X>::type;
  tm.sync();  // previous readers of pos are done
#pragma unroll
  for (int a = 0; a < A; ++a) {
    const int i = tm.rank + a * T;
    if (i < n) {
      if constexpr (sizeof(X) == 4) {
        stage_f32x2(static_cast<PosF2*>(posv), n, i, x[a][0], x[a][1], x[a][2]);   // packed
      } else {
        Q q;
        q.x = x[a][0]; q.y = x[a][1]; q.z = x[a][2]; q.w = (X)0;
        static_cast<Q*>(posv)[i] = q;
      }
    }
  }
  tm.sync();
  V dp = (V)0;
  if constexpr (sizeof(X) == 4) {
    // packed rows: two pair terms per instruction, as for Eq. (1)
    const PosF2* pos = static_cast<const PosF2*>(posv);
    const float gsc = p.k.m_g_f;
    ff e{0.f, 0.f};
#pragma unroll
    for (int a = 0; a < A; ++a) {
      const int i = tm.rank + a * T;
      if (i < n) {
        float bx, by, bz;
        ff ea{0.f, 0.f};
        morse_row_f32x2(n, i, x[a][0], x[a][1], x[a][2], pos, p.k.rho_f, p.k.rho_re_f, bx, by,
                        bz, ea);
        g[a][0] = gsc * bx; g[a][1] = gsc * by; g[a][2] = gsc * bz;
        e = ff_add(e, ea);
      } else {
        g[a][0] = 0.f; g[a][1] = 0.f; g[a][2] = 0.f;
      }
      if (d) dp += (V)g[a][0] * d[a][0] + (V)g[a][1] * d[a][1] + (V)g[a][2] * d[a][2];
    }
    if constexpr (std::is_same<V, float>::value) {
      if (d) {                  // energy and g.d in one team reduction
        team_sum_ff_f<T>(tm, e, dp);
        E = ff_scale(e, p.k.m_half_f);
        dphi = (S)dp;
        return;
      }
    }
    E = ff_scale(team_sum_ff<T>(tm, e), p.k.m_half_f);
  } else if (hbuf != nullptr && !p.tiled) {
    // ---- half-pair FP64 evaluation (pair phase, then row sums) -------------
    const int np = n_pairs(n);
    const PosD* pos = static_cast<const PosD*>(posv);
    double* vb = static_cast<double*>(hbuf);
    double* gsum = static_cast<double*>(posv);
    const double rho = p.k.rho, rr = p.k.rho_re;
    int i1, j1, i2, j2;
    pair_start(n, tm.rank, i1, j1);
    i2 = i1; j2 = j1;
    pair_advance(n, T, i2, j2);
    dd e{0.0, 0.0};
    for (int q = tm.rank; q < np; q += 2 * T) {
      const bool two = q + T < np;
      const int ib = two ? i2 : 0, jb = two ? j2 : 1;
      double ax, ay, az, ae, bx, by, bz, be;
      pair_term_morse_f64(pos[i1], pos[j1], rho, rr, ax, ay, az, ae);
      pair_term_morse_f64(pos[ib], pos[jb], rho, rr, bx, by, bz, be);
      vb[q] = ax; vb[np + q] = ay; vb[2 * np + q] = az;
      double eb = ae;
      if (two) {
        vb[q + T] = bx; vb[np + q + T] = by; vb[2 * np + q + T] = bz;
        eb += be;
      }
      const dd t = dd_two_sum(e.hi, eb);    // compensated energy sum
      e.hi = t.hi;
      e.lo = __dadd_rn(e.lo, t.lo);
      pair_advance(n, 2 * T, i1, j1);
      pair_advance(n, 2 * T, i2, j2);
    }
    tm.sync();
    const double gs = p.k.m_g;
    for (int q3 = tm.rank; q3 < 3 * n; q3 += T) {
      const int ii = q3 / 3;
      const double* vc = vb + (q3 - 3 * ii) * np;
      const int ri = row_base(n, ii);       // all lanes walk j together
      int rj = -1;
      double sacc[4] = {0.0, 0.0, 0.0, 0.0};
      for (int j0 = 0; j0 < n; j0 += 4) {
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = j0 + u;
          const int qq = j < ii ? rj + ii : ri + j;
          v[u] = 0.0;
          if (j < n && j != ii) v[u] = vc[qq];
          if (j < ii) v[u] = -v[u];
          rj += n - j - 2;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) sacc[u] += v[u];
      }
      gsum[q3] = -gs * ((sacc[0] + sacc[1]) + (sacc[2] + sacc[3]));
    }
    tm.sync();
#pragma unroll
    for (int a = 0; a < A; ++a) {
      const int ii = tm.rank + a * T;
      if (ii < n) {
        g[a][0] = gsum[3 * ii]; g[a][1] = gsum[3 * ii + 1]; g[a][2] = gsum[3 * ii + 2];
      } else {
        g[a][0] = 0.0; g[a][1] = 0.0; g[a][2] = 0.0;
      }
      if (d) dp += (V)g[a][0] * d[a][0] + (V)g[a][1] * d[a][1] + (V)g[a][2] * d[a][2];
    }
    E = team_sum_dd<T>(tm, e) * p.k.eps;
  } else {
    const Q* pos = static_cast<const Q*>(posv);
    const double rho = p.k.rho, rr = p.k.rho_re, gsc = p.k.m_g;
    const double kInf = __longlong_as_double(0x7ff0000000000000LL);
    dd e{0.0, 0.0};
#pragma unroll
    for (int a = 0; a < A; ++a) {
      const int i = tm.rank + a * T;
      if (i < n) {
        const double xi = x[a][0], yi = x[a][1], zi = x[a][2];
        double ax = 0.0, ay = 0.0, az = 0.0;
        double eb = 0.0;
        for (int j = 0; j < n; ++j) {
          const Q q = pos[j];
          const double dx = xi - q.x, dy = yi - q.y, dz = zi - q.z;
          const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
          const double r = sqrt(r2);
          const double ex = exp(fma(-rr, r, rho));
          double term = ex * (ex - 2.0);
          double c = ex * (ex - 1.0) / r;
          if (j == i) {
            term = 0.0;
            c = 0.0;
          } else if (!(r2 > 0.0)) {
            term = kInf;
          }
          const dd t = dd_two_sum(eb, term);      // compensated row energy
          eb = t.hi;
          e.lo = __dadd_rn(e.lo, t.lo);
          ax = fma(c, dx, ax);
          ay = fma(c, dy, ay);
          az = fma(c, dz, az);
        }
        const dd t = dd_two_sum(e.hi, eb);
        e.hi = t.hi;
        e.lo = __dadd_rn(e.lo, t.lo);
        g[a][0] = -gsc * ax; g[a][1] = -gsc * ay; g[a][2] = -gsc * az;
      } else {
        g[a][0] = 0.0; g[a][1] = 0.0; g[a][2] = 0.0;
      }
      if (d) dp += (V)g[a][0] * d[a][0] + (V)g[a][1] * d[a][1] + (V)g[a][2] * d[a][2];
    }
    E = team_sum_dd<T>(tm, e) * p.k.m_half;
  }
  if (d) dphi = (S)team_sum1<T, V>(tm, dp);
  }
}

template <int T, int A, typename P>
__device__ __forceinline__ void evaluate(const Team<T>& tm, int n,
                                         const typename P::XP (&x)[A][3],
                                         typename P::XG (&g)[A][3], void* posv, void* hbuf,
                                         const MinParams& p, const typename P::V (*d)[3],
                                         typename P::F& E, typename P::S& dphi) {
  using X = typename P::XP;
  using XG = typename P::XG;
  using V = typename P::V;
  using S = typename P::S;
  constexpr int PM = P::PM;
  if constexpr (P::POT != LJ_POT_LJ) {
    evaluate_morse<T, A, P>(tm, n, x, g, posv, hbuf, p, d, E, dphi);
    return;
  }
  tm.sync();  // previous readers of pos are done
#pragma unroll
  for (int a = 0; a < A; ++a) {
    const int i = tm.rank + a * T;
    if (i < n) {
      if constexpr (PM == 1) {
        // double-float positions, scaled by 1/sigma (exact for sigma = 1)
        ff qx = x[a][0], qy = x[a][1], qz = x[a][2];
        if (p.k.sigma != 1.0) {
          const ff is{p.k.is_hi, p.k.is_lo};
          qx = df_mul(qx, is); qy = df_mul(qy, is); qz = df_mul(qz, is);
        }
        static_cast<PosDF*>(posv)[i] = PosDF{qx.hi, qy.hi, qz.hi, 0.f, qx.lo, qy.lo, qz.lo, 0.f};
      } else if constexpr (sizeof(X) == 4) {
        stage_f32x2(static_cast<PosF2*>(posv), n, i, x[a][0], x[a][1], x[a][2]);   // packed
      } else {
        typename PosOf<X>::type q;
        q.x = x[a][0]; q.y = x[a][1]; q.z = x[a][2]; q.w = (X)0;
        static_cast<typename PosOf<X>::type*>(posv)[i] = q;
      }
    }
  }
  tm.sync();
  V dp = (V)0;
  if constexpr (PM == 1 || std::is_same<X, double>::value) {
    ff e_df{0.f, 0.f};          // PM == 1: this thread's pair energies
    if (hbuf != nullptr && !p.tiled) {
      // ---- half-pair evaluation ---------------------------------------------
      // pair phase: thread `rank` takes pairs rank, rank + T, ...; two pairs
      // per iteration (the second one clamped to a valid pair and discarded
      // past the end) keep two independent dependency chains in flight.
      // sum phase: one (atom, component) row sum per thread, written over the
      // position buffer (no longer needed), then read back by the owners.
      const int np = n_pairs(n);
      int i1, j1, i2, j2;
      pair_start(n, tm.rank, i1, j1);
      i2 = i1; j2 = j1;
      pair_advance(n, T, i2, j2);
      XG* gsum = static_cast<XG*>(posv);
      if constexpr (PM == 1) {
        const PosDF* pos = static_cast<const PosDF*>(posv);
        ff* vb = static_cast<ff*>(hbuf);
        ff e{0.f, 0.f};
        for (int q = tm.rank; q < np; q += 2 * T) {
          const bool two = q + T < np;
          const int ib = two ? i2 : 0, jb = two ? j2 : 1;
          ff ax, ay, az, ae, bx, by, bz, be;
          pair_term_df(pos[i1], pos[j1], ax, ay, az, ae);
          pair_term_df(pos[ib], pos[jb], bx, by, bz, be);
          vb[q] = ax; vb[np + q] = ay; vb[2 * np + q] = az;
          // cascaded TwoSum (Ogita, Rump and Oishi 2005, Sum2): the high
          // word's chain is one add; every rounding error and low word goes
          // to e.lo
          ff t = ff_two_sum(e.hi, ae.hi);
          e.hi = t.hi;
          e.lo = __fadd_rn(e.lo, __fadd_rn(t.lo, ae.lo));
          if (two) {
            vb[q + T] = bx; vb[np + q + T] = by; vb[2 * np + q + T] = bz;
            t = ff_two_sum(e.hi, be.hi);
            e.hi = t.hi;
            e.lo = __fadd_rn(e.lo, __fadd_rn(t.lo, be.lo));
          }
          pair_advance(n, 2 * T, i1, j1);
          pair_advance(n, 2 * T, i2, j2);
        }
        tm.sync();
        const float gs = p.k.gs_f;
        for (int q3 = tm.rank; q3 < 3 * n; q3 += T) {
          const int ii = q3 / 3;
          const ff* vc = vb + (q3 - 3 * ii) * np;
          // All lanes walk j = 0 .. n-1 together (no divergence), four
          // independent cascaded-TwoSum sums (Sum2, as for the energy),
          // loads issued a block of four ahead of the adds.
          const int ri = row_base(n, ii);
          int rj = -1;                          // row_base(n, j)
          ff s[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
          for (int j0 = 0; j0 < n; j0 += 4) {
            ff v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int j = j0 + u;
              const int q = j < ii ? rj + ii : ri + j;
              v[u] = ff{0.f, 0.f};
              if (j < n && j != ii) v[u] = vc[q];
              if (j < ii) v[u] = ff{-v[u].hi, -v[u].lo};   // -v over j < i
              rj += n - j - 2;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const ff t = ff_two_sum(s[u].hi, v[u].hi);
              s[u].hi = t.hi;
              s[u].lo = __fadd_rn(s[u].lo, __fadd_rn(t.lo, v[u].lo));
            }
          }
          const ff sum = df_add(df_add(s[0], s[1]), df_add(s[2], s[3]));
          gsum[q3] = -gs * (sum.hi + sum.lo);
        }
        tm.sync();
        e_df = e;               // reduced below, together with g.d
      } else {
        const PosD* pos = static_cast<const PosD*>(posv);
        double* vb = static_cast<double*>(hbuf);
        const double sig2 = p.k.sig2;
        dd e{0.0, 0.0};
        for (int q = tm.rank; q < np; q += 2 * T) {
          const bool two = q + T < np;
          const int ib = two ? i2 : 0, jb = two ? j2 : 1;
          double ax, ay, az, ae, bx, by, bz, be;
          pair_term_f64(pos[i1], pos[j1], sig2, ax, ay, az, ae);
          pair_term_f64(pos[ib], pos[jb], sig2, bx, by, bz, be);
          vb[q] = ax; vb[np + q] = ay; vb[2 * np + q] = az;
          double eb = ae;
          if (two) {
            vb[q + T] = bx; vb[np + q + T] = by; vb[2 * np + q + T] = bz;
            eb += be;
          }
          const dd t = dd_two_sum(e.hi, eb);    // compensated energy sum
          e.hi = t.hi;
          e.lo = __dadd_rn(e.lo, t.lo);
          pair_advance(n, 2 * T, i1, j1);
          pair_advance(n, 2 * T, i2, j2);
        }
        tm.sync();
        const double gs = p.k.gscale;
        for (int q3 = tm.rank; q3 < 3 * n; q3 += T) {
          const int ii = q3 / 3;
          const double* vc = vb + (q3 - 3 * ii) * np;
          const int ri = row_base(n, ii);       // same walk as the df sums
          int rj = -1;
          double s[4] = {0.0, 0.0, 0.0, 0.0};
          for (int j0 = 0; j0 < n; j0 += 4) {
            double v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int j = j0 + u;
              const int q = j < ii ? rj + ii : ri + j;
              v[u] = 0.0;
              if (j < n && j != ii) v[u] = vc[q];
              if (j < ii) v[u] = -v[u];
              rj += n - j - 2;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) s[u] += v[u];
          }
          gsum[q3] = -gs * ((s[0] + s[1]) + (s[2] + s[3]));
        }
        tm.sync();
        E = team_sum_dd<T>(tm, e) * p.k.e4;
      }
#pragma unroll
      for (int a = 0; a < A; ++a) {
        const int ii = tm.rank + a * T;
        if (ii < n) {
          g[a][0] = gsum[3 * ii]; g[a][1] = gsum[3 * ii + 1]; g[a][2] = gsum[3 * ii + 2];
        } else {
          g[a][0] = 0.0; g[a][1] = 0.0; g[a][2] = 0.0;
        }
        if (d) dp += (V)g[a][0] * d[a][0] + (V)g[a][1] * d[a][1] + (V)g[a][2] * d[a][2];
      }
      if constexpr (PM == 1) {
        // float-float team sum (FP32 pipes): its ~2^-47 relative error is far
        // below the double-float handover resolution; g.d in the same pass
        if constexpr (std::is_same<V, float>::value) {
          if (d) {
            team_sum_ff_f<T>(tm, e_df, dp);
            E = ff_scale(e_df, p.k.e4_f);
            dphi = (S)dp;
            return;
          }
        }
        E = ff_scale(team_sum_ff<T>(tm, e_df), p.k.e4_f);
      }
      if (d) dphi = (S)team_sum1<T, V>(tm, dp);
      return;
    }
  }
  if constexpr (PM == 1) {
    const PosDF* pos = static_cast<const PosDF*>(posv);
    const float gs = p.k.gs_f;
    ff e{0.f, 0.f};
    // ---- tiled half-pair evaluation (teams for more than 256 atoms; compiled
    // only for team shapes that can hold them) ------------------------------
    if constexpr (T * A > 256) {
    if (hbuf != nullptr && p.tiled) {
      ff* acc = static_cast<ff*>(hbuf);
      df_tile_eval<T>(tm, n, pos, acc, e);
#pragma unroll
      for (int a = 0; a < A; ++a) {
        const int i = tm.rank + a * T;
        if (i < n) {
          const ff sx = acc[i], sy = acc[n + i], sz = acc[2 * n + i];
          g[a][0] = -gs * (sx.hi + sx.lo);
          g[a][1] = -gs * (sy.hi + sy.lo);
          g[a][2] = -gs * (sz.hi + sz.lo);
        } else {
          g[a][0] = (XG)0; g[a][1] = (XG)0; g[a][2] = (XG)0;
        }
        if (d) dp += (V)g[a][0] * d[a][0] + (V)g[a][1] * d[a][1] + (V)g[a][2] * d[a][2];
      }
      if constexpr (std::is_same<V, float>::value) {
        if (d) {
          team_sum_ff_f<T>(tm, e, dp);
          E = ff_scale(e, p.k.e4_f);
          dphi = (S)dp;
          return;
        }
      }
      E = ff_scale(team_sum_ff<T>(tm, e), p.k.e4_f);
      if (d) dphi = (S)team_sum1<T, V>(tm, dp);
      return;
    }
    }
#pragma unroll
    for (int a = 0; a < A; ++a) {
      const int i = tm.rank + a * T;
      if (i < n) {
        const PosDF q = pos[i];
        ff ax, ay, az, ea{0.f, 0.f};
        pair_row_df(n, i, ff{q.xh, q.xl}, ff{q.yh, q.yl}, ff{q.zh, q.zl}, pos, ax, ay, az, ea);
        g[a][0] = -gs * (ax.hi + ax.lo);
        g[a][1] = -gs * (ay.hi + ay.lo);
        g[a][2] = -gs * (az.hi + az.lo);
        e = df_add(e, ea);
      } else {
        g[a][0] = (XG)0; g[a][1] = (XG)0; g[a][2] = (XG)0;
      }
      if (d) dp += (V)g[a][0] * d[a][0] + (V)g[a][1] * d[a][1] + (V)g[a][2] * d[a][2];
    }
    E = ff_scale(team_sum_ff<T>(tm, e), p.k.e2_f);
  } else if constexpr (sizeof(X) == 4) {
    const PosF2* pos = static_cast<const PosF2*>(posv);
    const float gs = p.k.gscale_f;
    const bool unit = p.k.sigma == 1.0;
    ff e{0.f, 0.f};
#pragma unroll
    for (int a = 0; a < A; ++a) {
      const int i = tm.rank + a * T;
      if (i < n) {
        float bx, by, bz;
        ff ea{0.f, 0.f};
        if (unit)
          pair_row_f32x2<false>(n, i, x[a][0], x[a][1], x[a][2], pos, 1.f, bx, by, bz, ea);
        else
          pair_row_f32x2<true>(n, i, x[a][0], x[a][1], x[a][2], pos, p.k.sig2_f, bx, by, bz, ea);
        g[a][0] = gs * bx; g[a][1] = gs * by; g[a][2] = gs * bz;
        e = ff_add(e, ea);
      } else {
        g[a][0] = 0.f; g[a][1] = 0.f; g[a][2] = 0.f;
      }
      if (d) dp += (V)g[a][0] * d[a][0] + (V)g[a][1] * d[a][1] + (V)g[a][2] * d[a][2];
    }
    if constexpr (std::is_same<V, float>::value) {
      if (d) {                  // energy and g.d in one team reduction
        team_sum_ff_f<T>(tm, e, dp);
        E = ff_scale(e, p.k.e2_f);
        dphi = (S)dp;
        return;
      }
    }
    ff et = team_sum_ff<T>(tm, e);
    E = ff_scale(et, p.k.e2_f);
  } else {
    const PosD* pos = static_cast<const PosD*>(posv);
    dd e{0.0, 0.0};
    // ---- tiled FP64 evaluation (teams for more than 256 atoms) -------------
    if constexpr (T * A > 256) {
    if (hbuf != nullptr && p.tiled) {
      double* acc = static_cast<double*>(hbuf);
      d_tile_eval<T>(tm, n, pos, p.k.sig2, acc, e);
#pragma unroll
      for (int a = 0; a < A; ++a) {
        const int i = tm.rank + a * T;
        if (i < n) {
          g[a][0] = -p.k.gscale * acc[i];
          g[a][1] = -p.k.gscale * acc[n + i];
          g[a][2] = -p.k.gscale * acc[2 * n + i];
        } else {
          g[a][0] = 0.0; g[a][1] = 0.0; g[a][2] = 0.0;
        }
        if (d) dp += (V)g[a][0] * d[a][0] + (V)g[a][1] * d[a][1] + (V)g[a][2] * d[a][2];
      }
      E = team_sum_dd<T>(tm, e) * p.k.e4;
      if (d) dphi = (S)team_sum1<T, V>(tm, dp);
      return;
    }
    }
#pragma unroll
    for (int a = 0; a < A; ++a) {
      const int i = tm.rank + a * T;
      if (i < n) {
        double ax, ay, az;
        pair_row_f64(n, i, x[a][0], x[a][1], x[a][2], pos, p.k.sig2, ax, ay, az, e);
        g[a][0] = -p.k.gscale * ax; g[a][1] = -p.k.gscale * ay; g[a][2] = -p.k.gscale * az;
      } else {
        g[a][0] = 0.0; g[a][1] = 0.0; g[a][2] = 0.0;
      }
      if (d) dp += (V)g[a][0] * d[a][0] + (V)g[a][1] * d[a][1] + (V)g[a][2] * d[a][2];
    }
    E = team_sum_dd<T>(tm, e) * p.k.e2;
  }
  if (d) dphi = (S)team_sum1<T, V>(tm, dp);
}

template <int T, int A, typename X>
__device__ __forceinline__ X grad_max(const Team<T>& tm, const X (&g)[A][3]) {
  X m = (X)0;
#pragma unroll
  for (int a = 0; a < A; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) m = fmax(m, abs_nan_inf(g[a][c]));
  X v[1] = {m};
  team_max<T, 1, X>(tm, v);
  return v[0];
}

// Sufficient decrease f(a) <= f(0) + c1 a phi'(0).  FP64-valued energies use
// exactly that expression (the right side rounded to FP64, as the oracle does:
// near the FP64 floor a threshold below half an ulp of f(0) then asks only
// f(a) <= f(0)); float-float energies compare the exact difference.
__device__ __forceinline__ bool armijo_ok(double fa, double f0, double t) {
  return isfinite(fa) && fa <= f0 + t;
}
__device__ __forceinline__ bool armijo_ok(ff fa, ff f0, float t) {
  return fisfinite(fa) && fdiff(fa, f0) <= t;
}

// safeguarded cubic interpolation (N&W eq. 3.59), kept 10% inside the bracket
template <typename S, typename F>
__device__ __forceinline__ S cubic_step(S a, F fa, S ga, S b, F fb, S gb) {
  const S lo = a < b ? a : b;
  const S hi = a < b ? b : a;
  const S w = hi - lo;
  const S mid = (S)0.5 * (a + b);
  if (!(fisfinite(fa) && fisfinite(fb) && isfinite(ga) && isfinite(gb))) return mid;
  const S d1 = ga + gb - (S)3 * ((S)fdiff(fa, fb) / (a - b));
  const S disc = d1 * d1 - ga * gb;
  if (!(disc >= (S)0)) return mid;
  S d2 = S_sqrt(disc);
  if (b - a < (S)0) d2 = -d2;
  const S den = gb - ga + (S)2 * d2;
  if (den == (S)0) return mid;
  S t = b - (b - a) * ((gb + d2 - d1) / den);
  if (!isfinite(t)) return mid;
  const S tlo = lo + (S)0.1 * w;
  const S thi = hi - (S)0.1 * w;
  if (t < tlo) t = tlo;
  if (t > thi) t = thi;
  return t;
}

// ---------------------------------------------------------------------------
// Two-loop recursion by the team's first warp (teams of 1 to 4 warps; float
// history staged through the idle position buffer, FP64 history through the
// idle half-pair buffer).  The recursion is a chain of 2 cnt + 1 dependent inner products;
// done by the whole team, each one crosses warps through shared memory and a
// barrier.  Instead every thread stages its gradient in `xb` (the idle
// position buffer, 12 A T + 4 bytes), warp 0 runs the recursion over all T
// ranks' entries (lane l covers ranks l, l + 32, ...: the history is
// addressable by rank) with shuffle-only reductions, and stages d and
// g.d back: two team barriers per direction instead of 2 cnt + 1.
//
// Pairs are taken two at a time, so that one two-value reduction serves two
// steps of each loop.  With q the vector before pair t (first loop, newest
// first) the next pair's product follows from this one's:
//   s_{t-1}.(q - alpha_t y_t) = s_{t-1}.q - alpha_t (s_{t-1}.y_t),
// and in the second loop (oldest first), with r before pair t,
//   y_{t+1}.(r + c_t s_t) = y_{t+1}.r + c_t (s_t.y_{t+1}),  c_t = alpha_t - beta_t.
// s_{t-1}.y_t -- the previous pair's s against this pair's y -- is reduced
// when pair t is stored (`sup`).  The same quantities as the one-at-a-time
// recursion (Algorithm 7.4 of Nocedal & Wright), half as many dependent
// reductions.
// ---------------------------------------------------------------------------
template <typename V>
__device__ __forceinline__ V warp_sum(V v) {   // xor butterfly: every lane gets the sum
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

template <typename V>
__device__ __forceinline__ void warp_sum2(V& v0, V& v1) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v0 += __shfl_xor_sync(kFull, v0, o);
    v1 += __shfl_xor_sync(kFull, v1, o);
  }
}

template <int T, int A, typename XG, typename V>
__device__ __forceinline__ V lead_two_loop(const Team<T>& tm, int m, int cnt, int head,
                                           const V* __restrict__ Sh, const V* __restrict__ Yh,
                                           const V (&rho)[LJ_MAX_M], const V (&gmv)[LJ_MAX_M],
                                           const V (&sup)[LJ_MAX_M], const XG (&g)[A][3],
                                           V* xb, V (&d)[A][3]) {
  constexpr int W = T / 32;
#pragma unroll
  for (int a = 0; a < A; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) xb[(a * 3 + c) * T + tm.rank] = (V)g[a][c];
  tm.sync();
  if (tm.rank < 32) {
    const int lane = tm.rank;
    auto slot_of = [&](int t) { const int sl = head + t; return sl >= m ? sl - m : sl; };
    V q[W][A][3], gl[W][A][3];
    V alpha[LJ_MAX_M];
#pragma unroll
    for (int w = 0; w < W; ++w)
#pragma unroll
      for (int a = 0; a < A; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          gl[w][a][c] = xb[(a * 3 + c) * T + lane + 32 * w];
          q[w][a][c] = gl[w][a][c];
        }
    // ---- first loop, newest first --------------------------------------------
    int t = cnt - 1;
    for (; t >= 1; t -= 2) {
      const int s0 = slot_of(t), s1 = slot_of(t - 1);
      V sv0[W][A][3], yv0[W][A][3], sv1[W][A][3], yv1[W][A][3];
#pragma unroll
      for (int w = 0; w < W; ++w)
#pragma unroll
        for (int a = 0; a < A; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            sv0[w][a][c] = Sh[hidx<T, A>(s0, a, c, lane + 32 * w)];
            yv0[w][a][c] = Yh[hidx<T, A>(s0, a, c, lane + 32 * w)];
            sv1[w][a][c] = Sh[hidx<T, A>(s1, a, c, lane + 32 * w)];
            yv1[w][a][c] = Yh[hidx<T, A>(s1, a, c, lane + 32 * w)];
          }
      const V r0 = rho[s0], r1 = rho[s1], u01 = sup[s0];
      V p0 = (V)0, p1 = (V)0;
#pragma unroll
      for (int w = 0; w < W; ++w)
#pragma unroll
        for (int a = 0; a < A; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            p0 += sv0[w][a][c] * q[w][a][c];
            p1 += sv1[w][a][c] * q[w][a][c];
          }
      warp_sum2(p0, p1);
      const V a0 = r0 * p0;
      const V a1 = r1 * (p1 - a0 * u01);
      alpha[t] = a0;
      alpha[t - 1] = a1;
#pragma unroll
      for (int w = 0; w < W; ++w)
#pragma unroll
        for (int a = 0; a < A; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            q[w][a][c] -= a0 * yv0[w][a][c];
            q[w][a][c] -= a1 * yv1[w][a][c];
          }
    }
    if (t == 0) {
      const int s0 = slot_of(0);
      V sv0[W][A][3], yv0[W][A][3];
#pragma unroll
      for (int w = 0; w < W; ++w)
#pragma unroll
        for (int a = 0; a < A; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            sv0[w][a][c] = Sh[hidx<T, A>(s0, a, c, lane + 32 * w)];
            yv0[w][a][c] = Yh[hidx<T, A>(s0, a, c, lane + 32 * w)];
          }
      V part = (V)0;
#pragma unroll
      for (int w = 0; w < W; ++w)
#pragma unroll
        for (int a = 0; a < A; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) part += sv0[w][a][c] * q[w][a][c];
      const V a0 = rho[s0] * warp_sum(part);
      alpha[0] = a0;
#pragma unroll
      for (int w = 0; w < W; ++w)
#pragma unroll
        for (int a = 0; a < A; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) q[w][a][c] -= a0 * yv0[w][a][c];
    }
    const V gam = gmv[slot_of(cnt - 1)];
#pragma unroll
    for (int w = 0; w < W; ++w)
#pragma unroll
      for (int a = 0; a < A; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) q[w][a][c] *= gam;
    // ---- second loop, oldest first ---------------------------------------------
    t = 0;
    for (; t + 1 < cnt; t += 2) {
      const int s0 = slot_of(t), s1 = slot_of(t + 1);
      V sv0[W][A][3], yv0[W][A][3], sv1[W][A][3], yv1[W][A][3];
#pragma unroll
      for (int w = 0; w < W; ++w)
#pragma unroll
        for (int a = 0; a < A; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            sv0[w][a][c] = Sh[hidx<T, A>(s0, a, c, lane + 32 * w)];
            yv0[w][a][c] = Yh[hidx<T, A>(s0, a, c, lane + 32 * w)];
            sv1[w][a][c] = Sh[hidx<T, A>(s1, a, c, lane + 32 * w)];
            yv1[w][a][c] = Yh[hidx<T, A>(s1, a, c, lane + 32 * w)];
          }
      const V r0 = rho[s0], r1 = rho[s1], u01 = sup[s1];
      const V al0 = alpha[t], al1 = alpha[t + 1];
      V p0 = (V)0, p1 = (V)0;
#pragma unroll
      for (int w = 0; w < W; ++w)
#pragma unroll
        for (int a = 0; a < A; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            p0 += yv0[w][a][c] * q[w][a][c];
            p1 += yv1[w][a][c] * q[w][a][c];
          }
      warp_sum2(p0, p1);
      const V c0 = al0 - r0 * p0;
      const V c1 = al1 - r1 * (p1 + c0 * u01);
#pragma unroll
      for (int w = 0; w < W; ++w)
#pragma unroll
        for (int a = 0; a < A; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            q[w][a][c] += c0 * sv0[w][a][c];
            q[w][a][c] += c1 * sv1[w][a][c];
          }
    }
    if (t < cnt) {
      const int s0 = slot_of(t);
      V sv0[W][A][3], yv0[W][A][3];
#pragma unroll
      for (int w = 0; w < W; ++w)
#pragma unroll
        for (int a = 0; a < A; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            sv0[w][a][c] = Sh[hidx<T, A>(s0, a, c, lane + 32 * w)];
            yv0[w][a][c] = Yh[hidx<T, A>(s0, a, c, lane + 32 * w)];
          }
      V part = (V)0;
#pragma unroll
      for (int w = 0; w < W; ++w)
#pragma unroll
        for (int a = 0; a < A; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) part += yv0[w][a][c] * q[w][a][c];
      const V c0 = alpha[t] - rho[s0] * warp_sum(part);
#pragma unroll
      for (int w = 0; w < W; ++w)
#pragma unroll
        for (int a = 0; a < A; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) q[w][a][c] += c0 * sv0[w][a][c];
    }
    V part = (V)0;
#pragma unroll
    for (int w = 0; w < W; ++w)
#pragma unroll
      for (int a = 0; a < A; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          xb[(a * 3 + c) * T + lane + 32 * w] = -q[w][a][c];
          part += gl[w][a][c] * -q[w][a][c];
        }
    const V dphi = warp_sum(part);
    if (lane == 0) xb[A * 3 * T] = dphi;
  }
  tm.sync();
#pragma unroll
  for (int a = 0; a < A; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) d[a][c] = xb[(a * 3 + c) * T + tm.rank];
  return xb[A * 3 * T];
}

// ---------------------------------------------------------------------------
// One L-BFGS phase: iterate from (x, g, f) until a stop condition.
// X: coordinates/gradient precision, V: direction/history precision,
// PM: pair arithmetic (0 native X, 1 double-float).
// MODE 0 (FP64, final): stops on ||g||_inf < gtol (CONVERGED) or a failed
//   line search (LSFAIL).
// MODE 1 (mixed, FP32 phase): hands over (SWITCH) once ||g||_inf <
//   switch_gtol or when a line search fails; never converges.  Once the
//   predicted decrease -alpha phi'(0) is below f32_resolution |E| (default 4
//   FP32 ulps) its line searches accept steps on the gradient alone.
// MODE 2 (mixed, double-float polish): CONVERGED on ||g||_inf < gtol (to be
//   confirmed in FP64); once the predicted decrease is below df_resolution
//   |E| (default 32 * 2^-48) its line searches accept steps on the gradient
//   alone (approximate Wolfe conditions); hands over to FP64 when a line
//   search fails.
// In MODE 1, gradient-only steps past kFP32GradIters tier iterations also
// hand over (a switch_gtol below the FP32 gradient noise).
// ---------------------------------------------------------------------------
template <int T, int A, typename P, int MODE>
__device__ __forceinline__ int run_phase(const Team<T>& tm, int n, typename P::XP (&x)[A][3],
                         typename P::XG (&g)[A][3], typename P::F& f,
                         typename P::V* __restrict__ Sh, typename P::V* __restrict__ Yh,
                         typename P::V (&rho)[LJ_MAX_M], typename P::V (&gmv)[LJ_MAX_M],
                         typename P::V (&sup)[LJ_MAX_M], int& cnt,
                         int& head, int& iters,
                         int& evals, int& phase_iters, long long& vec, void* pos,
                         void* hbuf, const MinParams& p, long long t0, long long (&cyc)[2]) {
  using X = typename P::XP;
  using XG = typename P::XG;
  using V = typename P::V;
  using S = typename P::S;
  using F = typename P::F;
  const int m = p.m;
  const S c1 = (S)p.c1, c2 = (S)p.c2, amax = (S)p.alpha_max;
  const S resolution = (S)(MODE == 1 ? p.f32_resolution : p.df_resolution);
  const XG stop_gtol = MODE == 1 ? (XG)p.switch_gtol : (XG)p.gtol;
  V alpha[LJ_MAX_M];
  V d[A][3];
  bool gmode = false;   // MODE 1, 2: energy below resolution, gradient-only line search
  X xt[A][3];
  XG gt[A][3];
  while (iters < p.max_iter) {
    // ---- search direction -------------------------------------------------
    long long tc = clock64();
    S dphi0 = (S)1;
    bool led = false;
    if constexpr (T <= 128) {
      // staging buffer for the lead warp: the idle position buffer (32 n
      // bytes) for float history, the idle half-pair buffer (24 bytes per
      // pair) for double history
      V* xb = nullptr;
      if constexpr (std::is_same<V, float>::value) {
        if (12 * A * T + 4 <= 32 * n) xb = static_cast<V*>(pos);
      } else {
        if (hbuf != nullptr && !p.tiled && 24 * A * T + 8 <= 24 * n_pairs(n))
          xb = static_cast<V*>(hbuf);
      }
      if (cnt > 0 && xb != nullptr) {
        dphi0 = (S)lead_two_loop<T, A, XG, V>(tm, m, cnt, head, Sh, Yh, rho, gmv, sup, g, xb, d);
        vec += (long long)cnt * 3 * n;
        led = true;
      }
    }
    if (cnt > 0 && !led) {
      V q[A][3];
#pragma unroll
      for (int a = 0; a < A; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) q[a][c] = (V)g[a][c];
      // two-loop recursion; each step prefetches the next pair's vectors and
      // 1/s.y before its own team reduction, so loads overlap the reduction
      auto slot_of = [&](int t) { const int sl = head + t; return sl >= m ? sl - m : sl; };
      V sc[A][3], yc[A][3], sn[A][3], yn[A][3];
      {
        const int sl = slot_of(cnt - 1);
#pragma unroll
        for (int a = 0; a < A; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            sc[a][c] = Sh[hidx<T, A>(sl, a, c, tm.rank)];
            yc[a][c] = Yh[hidx<T, A>(sl, a, c, tm.rank)];
          }
      }
      V rho_c = rho[slot_of(cnt - 1)];
      for (int t = cnt - 1; t >= 0; --t) {
        const int nsl = slot_of(t > 0 ? t - 1 : 0);
#pragma unroll
        for (int a = 0; a < A; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            sn[a][c] = Sh[hidx<T, A>(nsl, a, c, tm.rank)];
            yn[a][c] = Yh[hidx<T, A>(nsl, a, c, tm.rank)];
          }
        const V rho_n = rho[nsl];
        V part = (V)0;
#pragma unroll
        for (int a = 0; a < A; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) part += sc[a][c] * q[a][c];
        const V al = rho_c * team_sum1<T, V>(tm, part);
        alpha[t] = al;
#pragma unroll
        for (int a = 0; a < A; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            q[a][c] -= al * yc[a][c];
            sc[a][c] = sn[a][c];
            yc[a][c] = yn[a][c];
          }
        rho_c = rho_n;
      }
      const int newest = slot_of(cnt - 1);
      const V gam = gmv[newest];
#pragma unroll
      for (int a = 0; a < A; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) q[a][c] *= gam;
      // (sc, yc) now hold the oldest pair, the first one of the second loop
      rho_c = rho[slot_of(0)];
      for (int t = 0; t < cnt; ++t) {
        const int nsl = slot_of(t + 1 < cnt ? t + 1 : t);
#pragma unroll
        for (int a = 0; a < A; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            sn[a][c] = Sh[hidx<T, A>(nsl, a, c, tm.rank)];
            yn[a][c] = Yh[hidx<T, A>(nsl, a, c, tm.rank)];
          }
        const V rho_n = rho[nsl];
        V part = (V)0;
#pragma unroll
        for (int a = 0; a < A; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) part += yc[a][c] * q[a][c];
        const V coef = alpha[t] - rho_c * team_sum1<T, V>(tm, part);
#pragma unroll
        for (int a = 0; a < A; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            q[a][c] += coef * sc[a][c];
            sc[a][c] = sn[a][c];
            yc[a][c] = yn[a][c];
          }
        rho_c = rho_n;
      }
      V part = (V)0;
#pragma unroll
      for (int a = 0; a < A; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          d[a][c] = -q[a][c];
          part += (V)g[a][c] * d[a][c];
        }
      dphi0 = (S)team_sum1<T, V>(tm, part);
      vec += (long long)cnt * 3 * n;
    }
    if (!(dphi0 < (S)0)) {  // empty history or not a descent direction
      cnt = 0;
      head = 0;
      V part = (V)0;
#pragma unroll
      for (int a = 0; a < A; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          d[a][c] = -(V)g[a][c];
          part += d[a][c] * d[a][c];
        }
      dphi0 = -(S)team_sum1<T, V>(tm, part);
    }
    bool ok = false;
    F ft;
    {
      const long long t1 = clock64();
      cyc[0] += t1 - tc;
      tc = t1;
    }
    for (int attempt = 0; attempt < 2 && !ok; ++attempt) {
      if (attempt == 1) {
        if (cnt == 0) break;  // already steepest descent: no retry
        cnt = 0;
        head = 0;
        V part = (V)0;
#pragma unroll
        for (int a = 0; a < A; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            d[a][c] = -(V)g[a][c];
            part += d[a][c] * d[a][c];
          }
        dphi0 = -(S)team_sum1<T, V>(tm, part);
      }
      S a1 = (S)1;
      if (cnt == 0) {
        a1 = (S)1 / S_sqrt(-dphi0);
        if (a1 > (S)1) a1 = (S)1;
      }
      if constexpr (MODE == 1 || MODE == 2) {
        // predicted decrease below this tier's energy resolution: from here
        // on, steps are accepted on the gradient instead (the FP32 gradient
        // is trusted down to switch_gtol, the double-float one to ~1e-11)
        if (-dphi0 * a1 < resolution * fabsf(f.hi)) gmode = true;
      }
      // ---- strong-Wolfe line search ----------------------------------------
      int ev = 0;
      S a_prev = (S)0, dp_prev = dphi0;
      F f_prev = f;
      S a = a1;
      bool have_best = false;
      S best_a = (S)0, last_a = (S)-1;
      F best_f = f;
      S lo = 0, hi = 0, dp_lo = 0, dp_hi = 0;
      F f_lo = f, f_hi = f;
      S dp;
      bool done = false, zoom = false;
      auto trial = [&](S al, F& fo, S& dpo) {
#pragma unroll
        for (int aa = 0; aa < A; ++aa)
#pragma unroll
          for (int c = 0; c < 3; ++c) xt[aa][c] = pos_step(x[aa][c], al, d[aa][c]);
        evaluate<T, A, P>(tm, n, xt, gt, pos, hbuf, p, d, fo, dpo);
        ++ev;
        last_a = al;
      };
      bool gsearch = false;
      if constexpr (MODE == 1 || MODE == 2) {
      if (gmode) {
        gsearch = true;
        // ---- gradient-only search (approximate Wolfe conditions, Hager and
        // Zhang 2005): accept |phi'(a)| <= c2 |phi'(0)| with the energy no
        // more than the resolution above f(0) (which, for a near-quadratic
        // phi, also implies the Armijo decrease); bracket on the sign of
        // phi' and interpolate by secant steps on phi'.
        const S tol_f = (S)2 * resolution * fabsf(f.hi);
        S glo = (S)0, ghi = (S)-1, dlo = dphi0, dhi = (S)0;
        bool hi_slope = false;
        while (ev < p.max_ls) {
          F fa;
          trial(a, fa, dp);
          const bool eok = fisfinite(fa) && isfinite(dp) && (S)fdiff(fa, f) <= tol_f;
          if (!eok || dp > -c2 * dphi0) {          // too long
            ghi = a; dhi = dp; hi_slope = eok;
          } else if (dp < c2 * dphi0) {            // too short
            glo = a; dlo = dp;
          } else {
            ft = fa; done = true;
            break;
          }
          if (ghi < (S)0) {
            a = (S)2 * a;
            if (a > amax) a = amax;
          } else {
            const S w = ghi - glo;
            S t = (hi_slope && dhi > dlo) ? glo - dlo * w / (dhi - dlo) : glo + (S)0.5 * w;
            const S tlo = glo + (S)0.1 * w, thi = ghi - (S)0.1 * w;
            if (!(t >= tlo)) t = tlo;
            if (!(t <= thi)) t = thi;
            a = t;
          }
        }
      }
      }
      if (!gsearch) {
      for (int i = 1; !done && !zoom; ++i) {
        if (ev >= p.max_ls) break;
        F fa;
        trial(a, fa, dp);
        const bool armijo = armijo_ok(fa, f, c1 * a * dphi0);
        if (armijo && (!have_best || (S)fdiff(fa, best_f) < (S)0)) {
          have_best = true; best_f = fa; best_a = a;
        }
        if (!armijo || (i > 1 && (S)fdiff(fa, f_prev) >= (S)0)) {
          lo = a_prev; f_lo = f_prev; dp_lo = dp_prev;
          hi = a; f_hi = fa; dp_hi = dp;
          zoom = true;
        } else if (fabs(dp) <= -c2 * dphi0) {
          ft = fa; done = true;
        } else if (dp >= (S)0) {
          lo = a; f_lo = fa; dp_lo = dp;
          hi = a_prev; f_hi = f_prev; dp_hi = dp_prev;
          zoom = true;
        } else {
          a_prev = a; f_prev = fa; dp_prev = dp;
          a = (S)2 * a;
          if (a > amax) a = amax;
        }
      }
      while (zoom && !done) {
        if (ev >= p.max_ls) break;
        const S aj = cubic_step<S, F>(lo, f_lo, dp_lo, hi, f_hi, dp_hi);
        F fa;
        trial(aj, fa, dp);
        const bool armijo = armijo_ok(fa, f, c1 * aj * dphi0);
        if (armijo && (!have_best || (S)fdiff(fa, best_f) < (S)0)) {
          have_best = true; best_f = fa; best_a = aj;
        }
        if (!armijo || (S)fdiff(fa, f_lo) >= (S)0) {
          hi = aj; f_hi = fa; dp_hi = dp;
        } else {
          if (fabs(dp) <= -c2 * dphi0) {
            ft = fa; done = true;
          } else {
            if (dp * (hi - lo) >= (S)0) {
              hi = lo; f_hi = f_lo; dp_hi = dp_lo;
            }
            lo = aj; f_lo = fa; dp_lo = dp;
          }
        }
      }
      if (!done && have_best && (S)fdiff(best_f, f) < (S)0) {
        if (last_a != best_a) {
          F fa;
          trial(best_a, fa, dp);
          ft = fa;
        } else {
          ft = best_f;
        }
        done = true;
      }
      }
      evals += ev;
      ok = done;
    }
    cyc[1] += clock64() - tc;
    if (!ok) return MODE == 0 ? PH_LSFAIL : PH_SWITCH;

    // ---- curvature pair, then move ------------------------------------------
    V sv[A][3], yv[A][3];
    // s.y, y.y and s_prev.y (the newest stored pair's s against the new y:
    // the superdiagonal entry the blocked two-loop recursion uses)
    V pr[3] = {(V)0, (V)0, (V)0};
    const int prev = cnt > 0 ? (head + cnt - 1 >= m ? head + cnt - 1 - m : head + cnt - 1) : -1;
#pragma unroll
    for (int a = 0; a < A; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        sv[a][c] = pos_diff<V>(xt[a][c], x[a][c]);
        yv[a][c] = (V)(gt[a][c] - g[a][c]);
        pr[0] += sv[a][c] * yv[a][c];
        pr[1] += yv[a][c] * yv[a][c];
        if (prev >= 0) pr[2] += Sh[hidx<T, A>(prev, a, c, tm.rank)] * yv[a][c];
      }
    // stopping-test values of the new point (||g||_inf, deadline), reduced
    // in the same pass as the curvature pair's s.y and y.y
    XG mv[2];
    mv[0] = (XG)0;
#pragma unroll
    for (int a = 0; a < A; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) mv[0] = fmax(mv[0], abs_nan_inf(gt[a][c]));
    mv[1] = (p.deadline > 0 && (clock64() - t0) > p.deadline) ? (XG)1 : (XG)0;
    team_sums_max2<T, V, XG>(tm, pr, mv);
    if (pr[0] > eps_mach<V>() * pr[1]) {
      int slot;
      if (cnt < m) {
        slot = head + cnt;
        if (slot >= m) slot -= m;
        ++cnt;
      } else {
        slot = head;
        head = head + 1 == m ? 0 : head + 1;
      }
#pragma unroll
      for (int a = 0; a < A; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          Sh[hidx<T, A>(slot, a, c, tm.rank)] = sv[a][c];
          Yh[hidx<T, A>(slot, a, c, tm.rank)] = yv[a][c];
        }
      rho[slot] = (V)1 / pr[0];      // rho = 1 / s.y and the scaling s.y / y.y, formed
      gmv[slot] = pr[0] / pr[1];     // once here instead of in every recursion step
      sup[slot] = pr[2];             // s_prev . y (undefined for the oldest pair: unused)
    }
#pragma unroll
    for (int a = 0; a < A; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        x[a][c] = xt[a][c];
        g[a][c] = gt[a][c];
      }
    f = ft;
    ++iters;
    ++phase_iters;
    // ---- stopping tests (values reduced above) -----------------------------
    if (mv[0] < stop_gtol) return MODE == 1 ? PH_SWITCH : PH_CONVERGED;
    if (mv[1] > (XG)0) return PH_TIMEOUT;
    if constexpr (MODE == 1) {
      // a switch_gtol below the FP32 gradient noise would keep gradient-only
      // FP32 steps iterating on noise: past kFP32GradIters iterations of the
      // tier the double-float tier takes over
      if (gmode && phase_iters >= kFP32GradIters) return PH_SWITCH;
    }
  }
  return PH_MAXITER;
}

// ---------------------------------------------------------------------------
// Minimise the cluster whose owned coordinates are in x64 (in place).
// hist: this team's history slot (2 m A 3 T values of the phase's V type).
// pos:  this team's shared position buffer (n entries of 32 bytes).
// hbuf: this team's half-pair buffer (24 n(n-1)/2 bytes) or nullptr.
// MIXED: FP32 phase, then polish iterations whose evaluations run in
// double-float arithmetic; convergence is confirmed, and the returned energy
// computed, by a true FP64 evaluation (if FP64 disagrees, polishing goes on).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int status_of(int code) {
  return code == PH_CONVERGED ? ST_CONVERGED
       : code == PH_LSFAIL   ? ST_LS_FAIL
       : code == PH_TIMEOUT  ? ST_TIMEOUT : ST_MAXITER;
}

template <int T, int A, bool MIXED, int POT = LJ_POT_LJ>
__device__ __forceinline__ void minimise(const Team<T>& tm, int n, double (&x64)[A][3], const MinParams& p,
                         void* hist, void* pos, void* hbuf, MinResult& r) {
  using P32 = Prec<float, float, float, 0, POT>;       // mixed: FP32 tier
  using PDF = Prec<ff, float, float, 1, POT>;          // mixed: double-float tier
  using P64m = Prec<double, double, float, 0, POT>;    // mixed: FP64 tier
  using P64 = Prec<double, double, double, 0, POT>;    // FP64 path
  r.E = 0.0; r.status = ST_CONVERGED; r.iters = 0;
  r.evals32 = 0; r.evals64 = 0; r.evals_df = 0; r.iters32 = 0; r.iters64 = 0;
  r.vec32 = 0; r.vec64 = 0;
  r.cyc32 = 0; r.cycdf = 0; r.cyc64 = 0; r.cycdir = 0; r.cycls = 0;
  long long cyc[2] = {0, 0};
  if (n <= 1) return;
  const long long t0 = clock64();
  long long tmark = t0;
  auto lap = [&](long long& acc) {
    const long long t = clock64();
    acc += t - tmark;
    tmark = t;
    r.cycdir = cyc[0];
    r.cycls = cyc[1];
  };
  int cnt = 0, head = 0, iters = 0;
  const size_t hstride = (size_t)p.m * A * 3 * T;
  const double kInf = __longlong_as_double(0x7ff0000000000000LL);
  if constexpr (!MIXED) {
    double g[A][3];
    double f, dummy;
    evaluate<T, A, P64>(tm, n, x64, g, pos, hbuf, p, nullptr, f, dummy);
    r.evals64 = 1;
    const double gm = grad_max<T, A, double>(tm, g);
    if (!isfinite(f) || !(gm < kInf)) {
      r.E = f; r.status = ST_NONFINITE; lap(r.cyc64); return;
    }
    if (gm < p.gtol) { r.E = f; lap(r.cyc64); return; }
    double rho[LJ_MAX_M], gmv[LJ_MAX_M], sup[LJ_MAX_M];
    double* Sh = (double*)hist;
    const int code = run_phase<T, A, P64, 0>(tm, n, x64, g, f, Sh, Sh + hstride, rho, gmv, sup, cnt,
                                                 head, iters, r.evals64, r.iters64, r.vec64, pos,
                                                 hbuf, p, t0, cyc);
    r.E = f;
    r.iters = iters;
    r.status = status_of(code);
    lap(r.cyc64);
  } else {
    float* Sh = (float*)hist;
    float* Yh = Sh + hstride;
    float rho[LJ_MAX_M], gmv[LJ_MAX_M], sup[LJ_MAX_M];
    int code = PH_SWITCH;
    float dummy32;
    // ---- tier 1: FP32 -------------------------------------------------------
    float x32[A][3];
    bool moved32 = false;
    {
      float g32[A][3];
#pragma unroll
      for (int a = 0; a < A; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) x32[a][c] = (float)x64[a][c];
      ff f32;
      evaluate<T, A, P32>(tm, n, x32, g32, pos, nullptr, p, nullptr, f32, dummy32);
      r.evals32 = 1;
      const float gm = grad_max<T, A, float>(tm, g32);
      if (fisfinite(f32) && gm < __int_as_float(0x7f800000) && !(gm < (float)p.switch_gtol)) {
        code = run_phase<T, A, P32, 1>(tm, n, x32, g32, f32, Sh, Yh, rho, gmv, sup, cnt, head,
                                           iters, r.evals32, r.iters32, r.vec32, pos, nullptr, p,
                                           t0, cyc);
        moved32 = r.iters32 > 0;
      }
    }
    lap(r.cyc32);
    int status = -1;
    bool need_fp64 = false;
    if (code == PH_MAXITER || code == PH_TIMEOUT) {
      status = status_of(code);
      if (moved32) {
#pragma unroll
        for (int a = 0; a < A; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) x64[a][c] = (double)x32[a][c];
      }
    } else {
      // ---- tier 2: double-float positions and pair terms, FP32 elsewhere -----
      ff xdf[A][3];
      float gdf[A][3];
#pragma unroll
      for (int a = 0; a < A; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          xdf[a][c] = moved32 ? ff{x32[a][c], 0.f} : df_from_double(x64[a][c]);
      ff fdf;
      evaluate<T, A, PDF>(tm, n, xdf, gdf, pos, hbuf, p, nullptr, fdf, dummy32);
      r.evals_df += 1;
      float gm = grad_max<T, A, float>(tm, gdf);
      if (!fisfinite(fdf) || !(gm < __int_as_float(0x7f800000))) need_fp64 = true;
      while (status < 0 && !need_fp64) {
        if (gm < (float)p.gtol) {
          need_fp64 = true;               // confirm (and finish) in FP64
          break;
        }
        code = run_phase<T, A, PDF, 2>(tm, n, xdf, gdf, fdf, Sh, Yh, rho, gmv, sup, cnt, head, iters,
                                          r.evals_df, r.iters64, r.vec64, pos, hbuf, p, t0, cyc);
        if (code == PH_CONVERGED) {
          gm = 0.f;
        } else if (code == PH_SWITCH) {
          need_fp64 = true;
        } else {
          status = status_of(code);
        }
      }
#pragma unroll
      for (int a = 0; a < A; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) x64[a][c] = (double)xdf[a][c].hi + (double)xdf[a][c].lo;
    }
    lap(r.cycdf);
    double g[A][3];
    double f, dummy;
    if (need_fp64) {
      // ---- tier 3: FP64 -------------------------------------------------------
      evaluate<T, A, P64m>(tm, n, x64, g, pos, hbuf, p, nullptr, f, dummy32);
      r.evals64 += 1;
      const double gm = grad_max<T, A, double>(tm, g);
      if (!isfinite(f) || !(gm < kInf)) {
        r.E = f; r.iters = iters; r.status = ST_NONFINITE; lap(r.cyc64); return;
      }
      if (gm < p.gtol) {
        r.E = f; r.iters = iters; r.status = ST_CONVERGED; lap(r.cyc64); return;
      }
      code = run_phase<T, A, P64m, 0>(tm, n, x64, g, f, Sh, Yh, rho, gmv, sup, cnt, head, iters,
                                          r.evals64, r.iters64, r.vec64, pos, hbuf, p, t0, cyc);
      r.E = f;
      r.iters = iters;
      r.status = status_of(code);
      lap(r.cyc64);
      return;
    }
    // final energy (and the non-finite test) in FP64
    evaluate<T, A, P64>(tm, n, x64, g, pos, hbuf, p, nullptr, f, dummy);
    r.evals64 += 1;
    const double gm = grad_max<T, A, double>(tm, g);
    r.E = f;
    r.iters = iters;
    if (!isfinite(f) || !(gm < kInf)) {
      r.status = ST_NONFINITE;
    } else if (gm < p.gtol) {
      r.status = ST_CONVERGED;
    } else {
      r.status = status;
    }
    lap(r.cyc64);
  }
}

}  // namespace ljd
