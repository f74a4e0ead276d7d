/*
 * lj_oracle.c -- FP64 CPU oracle for batched Lennard-Jones Basin Hopping.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and
 * bench.py's cpu_baseline / reference leg may load this library.  The product
 * path (the CUDA library under paper_2510_25938_gb300/) never links, loads or
 * calls it, and shares no code, header or constant with it.
 *
 * It is deliberately plain and slow: serial double loops, textbook L-BFGS
 * two-loop recursion, textbook strong-Wolfe line search, no blocking, no fusion.
 * Build with -O2 -ffp-contract=off (no FMA contraction, no fast-math) so that
 * every product and sum is rounded separately on x86-64 and aarch64 alike.
 *
 * What it follows (paper: "Revisiting and Accelerating the Basin Hopping
 * Algorithm for Lennard-Jones Clusters", arXiv 2510.25938):
 *   - LJ energy: Methodology, "Lennard-Jones Potential", Eq. (1); the gradient
 *     is the analytic derivative of Eq. (1) (the paper never writes it).
 *   - Morse energy (Morse 1929, cluster form): the pair-potential extension
 *     the Conclusions point to ("empirical force fields"); pinned in
 *     tests/test_oracle_morse.py by its depth, zero crossing, harmonic
 *     constant, closed-form small clusters, the icosahedral breathing
 *     minimum, finite differences, invariants and the scaling law.
 *   - Local minimiser: Methodology, "Algorithm Overview" step 2 and
 *     "Implementation Notes" (L-BFGS-B from scipy, unbounded).  Read here as
 *     L-BFGS with the two-loop recursion (Nocedal & Wright, Numerical
 *     Optimization, 2nd ed., Alg. 7.4), strong-Wolfe line search (N&W
 *     Alg. 3.5 + 3.6, cubic interpolation eq. 3.59), gradient-infinity-norm
 *     stopping rule.
 *   - Perturbation, selection, Metropolis, adaptation: Methodology,
 *     "Algorithm Overview" steps 1, 3, 4, 5; Results (direction of the
 *     step-size adaptation).
 *   - Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
 *     random numbers: as easy as 1, 2, 3", SC'11), written from that
 *     definition.
 *
 * Parity pins (tests/test_oracle_pins.py): closed-form dimer / trimer /
 * tetramer / scaled-icosahedron minima, central finite differences,
 * translation / rotation / permutation invariance, epsilon/sigma scaling law,
 * brute force on 2-4 atoms, quadratic and Rosenbrock minimisers, two-loop vs
 * explicit BFGS inverse-Hessian recursion, cubic interpolation on cubics,
 * Philox known-answer vectors, Metropolis / adaptation properties, and a
 * black-box cross-check against scipy's L-BFGS-B.  The line search is pinned
 * in tests/test_oracle_linesearch.py: one-dimensional lines whose correct
 * trial sequence follows from N&W Alg. 3.5/3.6 by hand (doubling, exact
 * zoom on quadratics, strong versus weak curvature, alpha_max, non-finite
 * trials, the exhausted-budget rule), zoom's bracket invariants checked on
 * every trial of quartic, Rosenbrock and LJ lines, and both strong-Wolfe
 * conditions on every step a minimisation accepts.
 */
#include <math.h>
#include <float.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <sched.h>

#include "lj_oracle.h"

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the 4x32 S-box; round   */
/* multipliers and the Weyl key schedule are those of the published family.  */
/* ------------------------------------------------------------------------- */
static uint32_t orc_mulhilo32(uint32_t a, uint32_t b, uint32_t* lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *lo = (uint32_t)p;
    return (uint32_t)(p >> 32);
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {                 /* key bump between rounds */
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t lo0, lo1;
        uint32_t hi0 = orc_mulhilo32(0xD2511F53u, c0, &lo0);
        uint32_t hi1 = orc_mulhilo32(0xCD9E8D57u, c2, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 53-bit uniform in [0,1) from two 32-bit words: 27 high bits of a, 26 high
 * bits of b.  Exact in binary64. */
double orc_u01(uint32_t a, uint32_t b)
{
    double hi = (double)(a >> 5);
    double lo = (double)(b >> 6);
    return (hi * 67108864.0 + lo) * (1.0 / 9007199254740992.0);
}

/* Uniform number `draw` of Philox stream `tag` at counter (k, s, w):
 * block = draw / 2, first or second half of the block by draw parity. */
double orc_stream_uniform(uint64_t seed, uint32_t tag, uint32_t draw,
                          uint32_t k, uint32_t s, uint32_t w)
{
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) ^ tag };
    uint32_t ctr[4] = { draw >> 1, k, s, w };
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    if ((draw & 1u) == 0u) return orc_u01(r[0], r[1]);
    return orc_u01(r[2], r[3]);
}

/* ------------------------------------------------------------------------- */
/* Eq. (1): E = 4 eps sum_{i<j} [(sigma/r)^12 - (sigma/r)^6], and its         */
/* analytic gradient.  x is the flattened 3N coordinate vector              */
/* (Methodology, "Initial Structures and Input").                           */
/* ------------------------------------------------------------------------- */
double orc_lj_energy_grad(int64_t n_atoms, const double* x, double* g,
                          double eps, double sigma)
{
    double energy = 0.0, comp = 0.0;
    double sig2 = sigma * sigma;
    if (g) {
        for (int64_t c = 0; c < 3 * n_atoms; ++c) g[c] = 0.0;
    }
    for (int64_t i = 0; i < n_atoms; ++i) {
        for (int64_t j = i + 1; j < n_atoms; ++j) {
            double dx = x[3 * i + 0] - x[3 * j + 0];
            double dy = x[3 * i + 1] - x[3 * j + 1];
            double dz = x[3 * i + 2] - x[3 * j + 2];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0) {
                /* coincident atoms: Eq. (1) is infinite there */
                if (g) {
                    for (int64_t c = 0; c < 3 * n_atoms; ++c) g[c] = NAN;
                }
                return INFINITY;
            }
            double s2 = sig2 / r2;
            double s6 = s2 * s2 * s2;
            double s12 = s6 * s6;
            /* Neumaier-compensated sum: near a minimum of LJ38 (|E| ~ 170)
             * the rounding noise of a plain running sum (~1e-13) is as large
             * as the decreases the sufficient-decrease test has to resolve at
             * ||g||_inf ~ 1e-6 */
            double term = 4.0 * eps * (s12 - s6);
            double t = energy + term;
            if (fabs(energy) >= fabs(term)) comp += (energy - t) + term;
            else comp += (term - t) + energy;
            energy = t;
            if (g) {
                /* dphi/dr * (1/r) = -24 eps (2 s12 - s6) / r^2 */
                double c = 24.0 * eps * (2.0 * s12 - s6) / r2;
                g[3 * i + 0] -= c * dx;
                g[3 * i + 1] -= c * dy;
                g[3 * i + 2] -= c * dz;
                g[3 * j + 0] += c * dx;
                g[3 * j + 1] += c * dy;
                g[3 * j + 2] += c * dz;
            }
        }
    }
    return energy + comp;
}

/* ------------------------------------------------------------------------- */
/* Morse pair potential (P. M. Morse, Phys. Rev. 34, 57 (1929)) in the form   */
/* used for atomic clusters: V(r) = eps e^{rho(1 - r/re)} (e^{rho(1 - r/re)}  */
/* - 2), depth eps at r = re, range set by rho.  It is an empirical pair      */
/* potential of the kind the paper's Conclusions name as the next use of the  */
/* method: the minimiser and Basin Hopping run on it unchanged.  Gradient:    */
/* dV/dr = -(2 eps rho / re) e (e - 1), e = e^{rho(1 - r/re)}, and            */
/* dE/dx_i = sum_j (dV/dr)(r_ij) (x_i - x_j) / r_ij.                          */
/* ------------------------------------------------------------------------- */
double orc_morse_energy_grad(int64_t n_atoms, const double* x, double* g,
                             double eps, double re, double rho)
{
    double energy = 0.0, comp = 0.0;
    if (g) {
        for (int64_t c = 0; c < 3 * n_atoms; ++c) g[c] = 0.0;
    }
    for (int64_t i = 0; i < n_atoms; ++i) {
        for (int64_t j = i + 1; j < n_atoms; ++j) {
            double dx = x[3 * i + 0] - x[3 * j + 0];
            double dy = x[3 * i + 1] - x[3 * j + 1];
            double dz = x[3 * i + 2] - x[3 * j + 2];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0) {
                /* coincident atoms: V is finite there but its gradient has no
                 * direction; treated as an invalid configuration, as for LJ */
                if (g) {
                    for (int64_t c = 0; c < 3 * n_atoms; ++c) g[c] = NAN;
                }
                return INFINITY;
            }
            double r = sqrt(r2);
            double e = exp(rho * (1.0 - r / re));
            double term = eps * e * (e - 2.0);
            double t = energy + term;          /* Neumaier-compensated sum */
            if (fabs(energy) >= fabs(term)) comp += (energy - t) + term;
            else comp += (term - t) + energy;
            energy = t;
            if (g) {
                double c = -2.0 * eps * rho / re * e * (e - 1.0) / r;   /* (dV/dr) / r */
                g[3 * i + 0] += c * dx;
                g[3 * i + 1] += c * dy;
                g[3 * i + 2] += c * dz;
                g[3 * j + 0] -= c * dx;
                g[3 * j + 1] -= c * dy;
                g[3 * j + 2] -= c * dz;
            }
        }
    }
    return energy + comp;
}

/* ------------------------------------------------------------------------- */
/* Objectives the minimiser can run on (LJ is the method, Morse its pair-   */
/* potential extension; the quadratic, Rosenbrock and one-dimensional        */
/* polynomial functions exist only to pin the minimiser).                   */
/* ------------------------------------------------------------------------- */
static double orc_objective_eval(const orc_objective* o, const double* x, double* g)
{
    int64_t n = o->n;
    if (o->kind == ORC_OBJ_LJ) {
        return orc_lj_energy_grad(n / 3, x, g, o->eps, o->sigma);
    }
    if (o->kind == ORC_OBJ_MORSE) {
        return orc_morse_energy_grad(n / 3, x, g, o->eps, o->sigma, o->rho);
    }
    if (o->kind == ORC_OBJ_QUADRATIC) {
        /* f = 1/2 x^T A x - b^T x, g = A x - b (A symmetric, row-major) */
        double f = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double ax = 0.0;
            for (int64_t j = 0; j < n; ++j) ax += o->A[i * n + j] * x[j];
            g[i] = ax - o->b[i];
            f += 0.5 * x[i] * ax - o->b[i] * x[i];
        }
        return f;
    }
    if (o->kind == ORC_OBJ_POLY1D) {
        /* one variable: f = c0 + c1 x + c2 x^2 + c3 x^3 + c4 x^4 (b = c),
         * non-finite beyond x > A[0] when A is given */
        const double* c = o->b;
        double t = x[0];
        if (o->A && t > o->A[0]) {
            g[0] = NAN;
            return INFINITY;
        }
        g[0] = c[1] + t * (2.0 * c[2] + t * (3.0 * c[3] + t * 4.0 * c[4]));
        return c[0] + t * (c[1] + t * (c[2] + t * (c[3] + t * c[4])));
    }
    /* extended Rosenbrock: sum over pairs (x_{2i}, x_{2i+1}) */
    double f = 0.0;
    for (int64_t i = 0; i < n; ++i) g[i] = 0.0;
    for (int64_t i = 0; i + 1 < n; i += 2) {
        double a = x[i], b = x[i + 1];
        double t = b - a * a;
        double u = 1.0 - a;
        f += 100.0 * t * t + u * u;
        g[i] += -400.0 * a * t - 2.0 * u;
        g[i + 1] += 200.0 * t;
    }
    return f;
}

static double orc_dot(int64_t n, const double* a, const double* b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

static double orc_norm_inf(int64_t n, const double* a)
{
    double m = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double v = fabs(a[i]);
        if (!(v <= m)) m = v;          /* propagates NaN */
    }
    return m;
}

/* ------------------------------------------------------------------------- */
/* L-BFGS direction by the two-loop recursion (N&W Alg. 7.4) with            */
/* H0 = gamma I, gamma = s^T y / y^T y of the newest pair (N&W eq. 7.20).     */
/* History S, Y hold `cnt` pairs, oldest first.  d = -H g.                  */
/* ------------------------------------------------------------------------- */
void orc_lbfgs_direction(int64_t n, int32_t cnt, const double* S, const double* Y,
                         const double* g, double* d, double* alpha_work)
{
    for (int64_t i = 0; i < n; ++i) d[i] = g[i];            /* q = g */
    for (int32_t t = cnt - 1; t >= 0; --t) {
        const double* s = S + (int64_t)t * n;
        const double* y = Y + (int64_t)t * n;
        double rho = 1.0 / orc_dot(n, s, y);
        double a = rho * orc_dot(n, s, d);
        alpha_work[t] = a;
        for (int64_t i = 0; i < n; ++i) d[i] -= a * y[i];
    }
    double gamma = 1.0;
    if (cnt > 0) {
        const double* s = S + (int64_t)(cnt - 1) * n;
        const double* y = Y + (int64_t)(cnt - 1) * n;
        gamma = orc_dot(n, s, y) / orc_dot(n, y, y);
    }
    for (int64_t i = 0; i < n; ++i) d[i] *= gamma;           /* r = H0 q */
    for (int32_t t = 0; t < cnt; ++t) {
        const double* s = S + (int64_t)t * n;
        const double* y = Y + (int64_t)t * n;
        double rho = 1.0 / orc_dot(n, s, y);
        double b = rho * orc_dot(n, y, d);
        double coef = alpha_work[t] - b;
        for (int64_t i = 0; i < n; ++i) d[i] += coef * s[i];
    }
    for (int64_t i = 0; i < n; ++i) d[i] = -d[i];
}

/* ------------------------------------------------------------------------- */
/* Safeguarded cubic interpolation between (a, fa, ga) and (b, fb, gb),       */
/* N&W eq. (3.59).  The result is kept in [lo + 0.1 w, hi - 0.1 w] of the     */
/* bracket; a non-finite input or an empty discriminant gives the midpoint.  */
/* ------------------------------------------------------------------------- */
double orc_cubic_interpolate(double a, double fa, double ga, double b, double fb, double gb)
{
    double lo = a < b ? a : b;
    double hi = a < b ? b : a;
    double w = hi - lo;
    double mid = 0.5 * (a + b);
    if (!(isfinite(fa) && isfinite(fb) && isfinite(ga) && isfinite(gb))) return mid;
    double d1 = ga + gb - 3.0 * (fa - fb) / (a - b);
    double disc = d1 * d1 - ga * gb;
    if (!(disc >= 0.0)) return mid;
    double d2 = sqrt(disc);
    if (b - a < 0.0) d2 = -d2;
    double den = gb - ga + 2.0 * d2;
    if (den == 0.0) return mid;
    double t = b - (b - a) * ((gb + d2 - d1) / den);
    if (!isfinite(t)) return mid;
    double tlo = lo + 0.1 * w;
    double thi = hi - 0.1 * w;
    if (t < tlo) t = tlo;
    if (t > thi) t = thi;
    return t;
}

/* phi(alpha) = f(x + alpha d), phi'(alpha) = g(x + alpha d)^T d */
static double orc_phi(const orc_objective* o, int64_t n, const double* x, const double* d,
                      double alpha, double* xt, double* gt, double* dphi)
{
    for (int64_t i = 0; i < n; ++i) xt[i] = x[i] + alpha * d[i];
    double f = orc_objective_eval(o, xt, gt);
    *dphi = orc_dot(n, gt, d);
    return f;
}

/* ------------------------------------------------------------------------- */
/* Strong-Wolfe line search, N&W Alg. 3.5 (bracketing, alpha_{i+1} =          */
/* min(2 alpha_i, alpha_max)) and Alg. 3.6 (zoom).  A non-finite phi counts   */
/* as failing the sufficient-decrease test.  After max_ls evaluations the     */
/* best point that satisfied sufficient decrease is taken, if there is one.   */
/* On return 1, xt/gt/f_out hold the accepted point.                          */
/* ------------------------------------------------------------------------- */
/* Optional record of one line search: every trial (alpha, phi, phi') in the
 * order evaluated, and how it ended.  Only tests read it. */
static void orc_log_trial(orc_ls_log* log, double a, double f, double dp)
{
    if (!log) return;
    if (log->n_trial < ORC_LS_LOG_MAX) {
        log->trial[log->n_trial][0] = a;
        log->trial[log->n_trial][1] = f;
        log->trial[log->n_trial][2] = dp;
    }
    log->n_trial++;
}

static int orc_wolfe_search(const orc_objective* o, int64_t n, const double* x, double f0,
                            const double* d, double dphi0, double alpha1,
                            const orc_lbfgs_params* p, double* xt, double* gt,
                            double* f_out, double* alpha_out, int32_t* nevals,
                            orc_ls_log* log)
{
    const double c1 = p->c1, c2 = p->c2;
    int evals = 0;
    double a_prev = 0.0, f_prev = f0, dp_prev = dphi0;
    double a = alpha1;
    double best_a = -1.0, best_f = INFINITY;
    double lo = 0, f_lo = 0, dp_lo = 0, hi = 0, f_hi = 0, dp_hi = 0;
    double last_a = -1.0;
    double f, dp;
    if (log) { log->n_trial = 0; log->exit = ORC_LS_FAILED; log->f0 = f0; log->dphi0 = dphi0; }

    for (int i = 1;; ++i) {
        if (evals >= p->max_ls) goto exhausted;
        f = orc_phi(o, n, x, d, a, xt, gt, &dp);
        ++evals;
        orc_log_trial(log, a, f, dp);
        last_a = a;
        int armijo = isfinite(f) && (f <= f0 + c1 * a * dphi0);
        if (armijo && f < best_f) { best_f = f; best_a = a; }
        if (!armijo || (i > 1 && f >= f_prev)) {
            lo = a_prev; f_lo = f_prev; dp_lo = dp_prev;
            hi = a; f_hi = f; dp_hi = dp;
            break;
        }
        if (fabs(dp) <= -c2 * dphi0) {
            *f_out = f; *alpha_out = a; *nevals += evals;
            if (log) log->exit = ORC_LS_WOLFE;
            return 1;
        }
        if (dp >= 0.0) {
            lo = a; f_lo = f; dp_lo = dp;
            hi = a_prev; f_hi = f_prev; dp_hi = dp_prev;
            break;
        }
        a_prev = a; f_prev = f; dp_prev = dp;
        a = 2.0 * a;
        if (a > p->alpha_max) a = p->alpha_max;
    }
    for (;;) {                                   /* zoom(lo, hi) */
        if (evals >= p->max_ls) goto exhausted;
        double aj = orc_cubic_interpolate(lo, f_lo, dp_lo, hi, f_hi, dp_hi);
        f = orc_phi(o, n, x, d, aj, xt, gt, &dp);
        ++evals;
        orc_log_trial(log, aj, f, dp);
        last_a = aj;
        int armijo = isfinite(f) && (f <= f0 + c1 * aj * dphi0);
        if (armijo && f < best_f) { best_f = f; best_a = aj; }
        if (!armijo || f >= f_lo) {
            hi = aj; f_hi = f; dp_hi = dp;
        } else {
            if (fabs(dp) <= -c2 * dphi0) {
                *f_out = f; *alpha_out = aj; *nevals += evals;
                if (log) log->exit = ORC_LS_WOLFE;
                return 1;
            }
            if (dp * (hi - lo) >= 0.0) {
                hi = lo; f_hi = f_lo; dp_hi = dp_lo;
            }
            lo = aj; f_lo = f; dp_lo = dp;
        }
    }
exhausted:
    /* the best sufficient-decrease point is taken only if it strictly lowers
     * f; a point that merely ties f0 (the test's c1 alpha phi'(0) term lost
     * below one ulp of f0) would make no progress */
    if (best_a > 0.0 && best_f < f0) {
        if (last_a != best_a) {
            f = orc_phi(o, n, x, d, best_a, xt, gt, &dp);
            ++evals;
        } else {
            f = best_f;
        }
        *f_out = f; *alpha_out = best_a; *nevals += evals;
        if (log) log->exit = ORC_LS_FALLBACK;
        return 1;
    }
    *nevals += evals;
    return 0;
}

/* One line search from x along d with first trial alpha1, for tests: phi(0)
 * and phi'(0) are evaluated here, then the search above runs with `log`.
 * work must hold 3 n doubles.  Returns 1 when a step was accepted. */
int32_t orc_line_search(const orc_objective* o, const double* x, const double* d,
                        double alpha1, const orc_lbfgs_params* p, double* alpha_out,
                        double* f_out, orc_ls_log* log, double* work)
{
    const int64_t n = o->n;
    double* g0 = work;
    double* xt = g0 + n;
    double* gt = xt + n;
    double f0 = orc_objective_eval(o, x, g0);
    double dphi0 = orc_dot(n, g0, d);
    int32_t ne = 0;
    *alpha_out = 0.0;
    *f_out = f0;
    return orc_wolfe_search(o, n, x, f0, d, dphi0, alpha1, p, xt, gt, f_out, alpha_out, &ne,
                            log);
}

/* ------------------------------------------------------------------------- */
/* L-BFGS minimiser (Algorithm Overview step 2 read as unbounded L-BFGS).     */
/* work must hold (4 + 2m) n + m doubles.                                     */
/* ------------------------------------------------------------------------- */
static int32_t orc_lbfgs_run(const orc_objective* o, double* x, const orc_lbfgs_params* p,
                             double* f_out, int32_t* iters_out, int32_t* nevals_out,
                             double* work, orc_step_log* slog, int32_t max_steps);

int32_t orc_lbfgs_minimize(const orc_objective* o, double* x, const orc_lbfgs_params* p,
                           double* f_out, int32_t* iters_out, int32_t* nevals_out,
                           double* work)
{
    return orc_lbfgs_run(o, x, p, f_out, iters_out, nevals_out, work, NULL, 0);
}

/* The same minimisation, recording every accepted step in slog[0..max_steps)
 * (tests only).  *n_steps receives the number of accepted steps. */
int32_t orc_lbfgs_minimize_log(const orc_objective* o, double* x, const orc_lbfgs_params* p,
                               double* f_out, int32_t* iters_out, int32_t* nevals_out,
                               double* work, orc_step_log* slog, int32_t max_steps)
{
    return orc_lbfgs_run(o, x, p, f_out, iters_out, nevals_out, work, slog, max_steps);
}

static int32_t orc_lbfgs_run(const orc_objective* o, double* x, const orc_lbfgs_params* p,
                             double* f_out, int32_t* iters_out, int32_t* nevals_out,
                             double* work, orc_step_log* slog, int32_t max_steps)
{
    const int64_t n = o->n;
    const int32_t m = p->m;
    double* g = work;
    double* d = g + n;
    double* xt = d + n;
    double* gt = xt + n;
    double* S = gt + n;                 /* m rows, oldest first */
    double* Y = S + (int64_t)m * n;
    double* alpha = Y + (int64_t)m * n;
    int32_t cnt = 0, iters = 0, nevals = 0;
    int32_t status = ORC_MAXITER;

    double f = orc_objective_eval(o, x, g);
    nevals = 1;
    if (!isfinite(f) || !(orc_norm_inf(n, g) < INFINITY)) {
        status = ORC_NONFINITE;
        goto done;
    }
    if (orc_norm_inf(n, g) < p->gtol) {
        status = ORC_CONVERGED;
        goto done;
    }
    while (iters < p->max_iter) {
        double dphi0;
        if (cnt > 0) {
            orc_lbfgs_direction(n, cnt, S, Y, g, d, alpha);
            dphi0 = orc_dot(n, g, d);
        } else {
            dphi0 = 1.0;                   /* forces the steepest-descent branch */
        }
        if (!(dphi0 < 0.0)) {              /* not a descent direction: restart */
            cnt = 0;
            for (int64_t i = 0; i < n; ++i) d[i] = -g[i];
            dphi0 = -orc_dot(n, g, g);
        }
        double a1 = 1.0;
        if (cnt == 0) {
            double dn = sqrt(orc_dot(n, d, d));
            a1 = 1.0 / dn;
            if (a1 > 1.0) a1 = 1.0;
        }
        double ft, at;
        orc_ls_log ls;
        orc_ls_log* lsp = slog ? &ls : NULL;
        int retried = 0;
        int ok = orc_wolfe_search(o, n, x, f, d, dphi0, a1, p, xt, gt, &ft, &at, &nevals, lsp);
        if (!ok && cnt > 0) {              /* one retry along -g with no history */
            cnt = 0;
            for (int64_t i = 0; i < n; ++i) d[i] = -g[i];
            dphi0 = -orc_dot(n, g, g);
            double dn = sqrt(-dphi0);
            a1 = 1.0 / dn;
            if (a1 > 1.0) a1 = 1.0;
            retried = 1;
            ok = orc_wolfe_search(o, n, x, f, d, dphi0, a1, p, xt, gt, &ft, &at, &nevals, lsp);
        }
        if (!ok) {
            status = ORC_LINESEARCH_FAIL;
            break;
        }
        if (slog && iters < max_steps) {
            orc_step_log* r = &slog[iters];
            r->alpha = at;
            r->f0 = f;
            r->f = ft;
            r->dphi0 = dphi0;
            r->dphi = orc_dot(n, gt, d);
            r->exit = ls.exit;
            r->retried = retried;
            r->n_trial = ls.n_trial;
        }
        /* new curvature pair s = x_{k+1} - x_k, y = g_{k+1} - g_k; it is
         * stored only if s^T y > eps_mach y^T y (curvature guard) */
        double sy = 0.0, yy = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double si = xt[i] - x[i];
            double yi = gt[i] - g[i];
            sy += si * yi;
            yy += yi * yi;
        }
        if (sy > DBL_EPSILON * yy) {
            if (cnt == m) {                /* drop the oldest pair */
                memmove(S, S + n, sizeof(double) * (size_t)(n * (m - 1)));
                memmove(Y, Y + n, sizeof(double) * (size_t)(n * (m - 1)));
                --cnt;
            }
            double* s_new = S + (int64_t)cnt * n;
            double* y_new = Y + (int64_t)cnt * n;
            for (int64_t i = 0; i < n; ++i) {
                s_new[i] = xt[i] - x[i];
                y_new[i] = gt[i] - g[i];
            }
            ++cnt;
        }
        for (int64_t i = 0; i < n; ++i) { x[i] = xt[i]; g[i] = gt[i]; }
        f = ft;
        ++iters;
        if (orc_norm_inf(n, g) < p->gtol) {
            status = ORC_CONVERGED;
            break;
        }
    }
done:
    *f_out = f;
    *iters_out = iters;
    *nevals_out = nevals;
    return status;
}

/* ------------------------------------------------------------------------- */
/* Basin Hopping pieces (Methodology, "Algorithm Overview").                  */
/* ------------------------------------------------------------------------- */

/* Step 1: random displacement of every atom inside a cube of side
 * 2 * stepsize: each coordinate moves by step * (2u - 1), u ~ U[0,1) from
 * Philox stream 1 at counter (draw = coordinate index, k, s, w). */
void orc_perturb(int64_t n_coords, const double* x, double step, uint64_t seed,
                 uint32_t k, uint32_t s, uint32_t w, double* out)
{
    for (int64_t c = 0; c < n_coords; ++c) {
        double u = orc_stream_uniform(seed, 1u, (uint32_t)c, k, s, w);
        double delta = step * (2.0 * u - 1.0);
        out[c] = x[c] + delta;
    }
}

/* Step 4: accept if the energy does not rise, else with probability
 * exp(-dE / kT).  Returns 1 for accept. */
int32_t orc_metropolis(double e_cur, double e_new, double kT, double u)
{
    double de = e_new - e_cur;
    if (de <= 0.0) return 1;
    return u < exp(-de / kT) ? 1 : 0;
}

/* Step 5 (and Results, first paragraph): after each window of `interval`
 * steps, a window acceptance rate above target grows the step (step / factor),
 * otherwise the step shrinks (step * factor). */
double orc_adapt_step(double step, int32_t win_accept, int32_t interval,
                      double target_rate, double factor)
{
    double rate = (double)win_accept / (double)interval;
    if (rate > target_rate) return step / factor;
    return step * factor;
}

int32_t orc_num_threads(void)
{
    cpu_set_t set;
    CPU_ZERO(&set);
    if (sched_getaffinity(0, sizeof(set), &set) == 0) {
        int c = CPU_COUNT(&set);
        if (c > 0) return c;
    }
    return 1;
}

/* A tiny work queue: threads take item indices from a shared counter. */
typedef struct {
    int64_t n_items;
    int64_t next;
    pthread_mutex_t lock;
    void (*fn)(void* ctx, int64_t item, double* work);
    void* ctx;
    size_t work_doubles;
} orc_queue;

static void* orc_worker(void* arg)
{
    orc_queue* q = (orc_queue*)arg;
    double* work = (double*)malloc(sizeof(double) * (q->work_doubles ? q->work_doubles : 1));
    for (;;) {
        pthread_mutex_lock(&q->lock);
        int64_t it = q->next++;
        pthread_mutex_unlock(&q->lock);
        if (it >= q->n_items) break;
        q->fn(q->ctx, it, work);
    }
    free(work);
    return NULL;
}

static void orc_parallel_for(int64_t n_items, int32_t n_threads, size_t work_doubles,
                             void (*fn)(void*, int64_t, double*), void* ctx)
{
    if (n_items <= 0) return;
    if (n_threads <= 0) n_threads = orc_num_threads();
    if (n_threads > n_items) n_threads = (int32_t)n_items;
    orc_queue q;
    q.n_items = n_items;
    q.next = 0;
    pthread_mutex_init(&q.lock, NULL);
    q.fn = fn;
    q.ctx = ctx;
    q.work_doubles = work_doubles;
    if (n_threads == 1) {
        orc_worker(&q);
    } else {
        pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)n_threads);
        for (int32_t t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, orc_worker, &q);
        for (int32_t t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
        free(th);
    }
    pthread_mutex_destroy(&q.lock);
}

typedef struct {
    int32_t uniform_n;
    const int64_t* atom_off;
    const double* x_in;
    double* x;
    double* energy;
    double* grad;
    int32_t kind;            /* ORC_OBJ_LJ or ORC_OBJ_MORSE */
    double eps, sigma, rho;
    const orc_lbfgs_params* p;
    int32_t* status;
    int32_t* iters;
    int32_t* nevals;
} orc_batch_ctx;

static void orc_cand_range(const orc_batch_ctx* b, int64_t c, int64_t* a0, int64_t* na)
{
    if (b->uniform_n > 0) {
        *a0 = c * b->uniform_n;
        *na = b->uniform_n;
    } else {
        *a0 = b->atom_off[c];
        *na = b->atom_off[c + 1] - b->atom_off[c];
    }
}

static void orc_eval_item(void* vctx, int64_t c, double* work)
{
    (void)work;
    orc_batch_ctx* b = (orc_batch_ctx*)vctx;
    int64_t a0, na;
    orc_cand_range(b, c, &a0, &na);
    double* gc = b->grad ? b->grad + 3 * a0 : NULL;
    if (b->kind == ORC_OBJ_MORSE)
        b->energy[c] = orc_morse_energy_grad(na, b->x_in + 3 * a0, gc, b->eps, b->sigma, b->rho);
    else
        b->energy[c] = orc_lj_energy_grad(na, b->x_in + 3 * a0, gc, b->eps, b->sigma);
}

void orc_eval_batch_pot(int64_t n_cand, int32_t uniform_n, const int64_t* atom_off,
                        const double* x, double* energy, double* grad, int32_t kind,
                        double eps, double sigma, double rho, int32_t n_threads)
{
    orc_batch_ctx b;
    memset(&b, 0, sizeof(b));
    b.uniform_n = uniform_n;
    b.atom_off = atom_off;
    b.x_in = x;
    b.energy = energy;
    b.grad = grad;
    b.kind = kind;
    b.eps = eps;
    b.sigma = sigma;
    b.rho = rho;
    orc_parallel_for(n_cand, n_threads, 0, orc_eval_item, &b);
}

void orc_eval_batch(int64_t n_cand, int32_t uniform_n, const int64_t* atom_off,
                    const double* x, double* energy, double* grad,
                    double eps, double sigma, int32_t n_threads)
{
    orc_eval_batch_pot(n_cand, uniform_n, atom_off, x, energy, grad, ORC_OBJ_LJ, eps, sigma,
                       0.0, n_threads);
}

static int64_t orc_max_atoms(int64_t n_cand, int32_t uniform_n, const int64_t* atom_off)
{
    if (uniform_n > 0) return uniform_n;
    int64_t mx = 0;
    for (int64_t c = 0; c < n_cand; ++c) {
        int64_t na = atom_off[c + 1] - atom_off[c];
        if (na > mx) mx = na;
    }
    return mx;
}

static void orc_lbfgs_item(void* vctx, int64_t c, double* work)
{
    orc_batch_ctx* b = (orc_batch_ctx*)vctx;
    int64_t a0, na;
    orc_cand_range(b, c, &a0, &na);
    orc_objective o;
    memset(&o, 0, sizeof(o));
    o.kind = b->kind;
    o.n = 3 * na;
    o.eps = b->eps;
    o.sigma = b->sigma;
    o.rho = b->rho;
    double f;
    int32_t it, ne;
    int32_t st = orc_lbfgs_minimize(&o, b->x + 3 * a0, b->p, &f, &it, &ne, work);
    b->energy[c] = f;
    if (b->status) b->status[c] = st;
    if (b->iters) b->iters[c] = it;
    if (b->nevals) b->nevals[c] = ne;
}

void orc_lbfgs_batch(int64_t n_cand, int32_t uniform_n, const int64_t* atom_off,
                     double* x, const orc_lbfgs_params* p, double eps, double sigma,
                     double* energy, int32_t* status, int32_t* iters, int32_t* nevals,
                     int32_t n_threads)
{
    orc_lbfgs_batch_pot(n_cand, uniform_n, atom_off, x, p, ORC_OBJ_LJ, eps, sigma, 0.0,
                        energy, status, iters, nevals, n_threads);
}

void orc_lbfgs_batch_pot(int64_t n_cand, int32_t uniform_n, const int64_t* atom_off,
                         double* x, const orc_lbfgs_params* p, int32_t kind, double eps,
                         double sigma, double rho, double* energy, int32_t* status,
                         int32_t* iters, int32_t* nevals, int32_t n_threads)
{
    orc_batch_ctx b;
    memset(&b, 0, sizeof(b));
    b.uniform_n = uniform_n;
    b.atom_off = atom_off;
    b.x = x;
    b.energy = energy;
    b.kind = kind;
    b.eps = eps;
    b.sigma = sigma;
    b.rho = rho;
    b.p = p;
    b.status = status;
    b.iters = iters;
    b.nevals = nevals;
    int64_t n = 3 * orc_max_atoms(n_cand, uniform_n, atom_off);
    size_t work = (size_t)((4 + 2 * (int64_t)p->m) * n + p->m + 1);
    orc_parallel_for(n_cand, n_threads, work, orc_lbfgs_item, &b);
}

typedef struct {
    int32_t n_atoms;
    int64_t n_walkers;
    double* x_cur;
    double* e_cur;
    double* x_best;
    double* e_best;
    double* stepsize;
    int32_t* win_accept;
    int32_t* n_accept;
    const orc_bh_params* bp;
    double* trace_trial_e;
    int32_t* trace_trial_status;
    double* trace_best_e;
    uint8_t* trace_accepted;
    double* trace_step;
} orc_bh_ctx;

/* One walker for n_steps steps (Algorithm Overview, steps 1-5).  The K
 * candidates are minimised one after another here; their independence is
 * what the parallel implementation exploits. */
static void orc_bh_item(void* vctx, int64_t wi, double* work)
{
    orc_bh_ctx* b = (orc_bh_ctx*)vctx;
    const orc_bh_params* bp = b->bp;
    const int64_t n = 3 * (int64_t)b->n_atoms;
    const int32_t K = bp->K;
    double* xc = b->x_cur + wi * n;
    double* xb = b->x_best + wi * n;
    double* cand = work;                               /* K x n */
    double* ek = cand + (int64_t)K * n;                /* K */
    double* mwork = ek + K;
    const uint32_t w = (uint32_t)(bp->walker0 + wi);
    orc_objective o;
    memset(&o, 0, sizeof(o));
    o.kind = bp->potential == ORC_OBJ_MORSE ? ORC_OBJ_MORSE : ORC_OBJ_LJ;
    o.n = n;
    o.eps = bp->eps;
    o.sigma = bp->sigma;
    o.rho = bp->rho;

    for (int32_t i = 0; i < bp->n_steps; ++i) {
        const int64_t s64 = bp->step0 + i;
        const uint32_t s = (uint32_t)s64;
        const double step = b->stepsize[wi];
        int32_t kbest = -1;
        for (int32_t k = 0; k < K; ++k) {
            double* xk = cand + (int64_t)k * n;
            orc_perturb(n, xc, step, bp->seed, (uint32_t)k, s, w, xk);
            double f;
            int32_t it, ne;
            int32_t st = orc_lbfgs_minimize(&o, xk, &bp->min, &f, &it, &ne, mwork);
            ek[k] = f;
            int64_t tix = ((int64_t)i * b->n_walkers + wi) * K + k;
            if (b->trace_trial_e) b->trace_trial_e[tix] = f;
            if (b->trace_trial_status) b->trace_trial_status[tix] = st;
            /* Step 3: the lowest finite energy wins; ties keep the lower k */
            if (isfinite(f) && (kbest < 0 || f < ek[kbest])) kbest = k;
        }
        int32_t acc = 0;
        double e_sel = INFINITY;
        if (kbest >= 0) {
            e_sel = ek[kbest];
            double u = orc_stream_uniform(bp->seed, 2u, 0u, 0u, s, w);
            acc = orc_metropolis(b->e_cur[wi], e_sel, bp->kT, u);
        }
        int64_t tw = (int64_t)i * b->n_walkers + wi;
        if (b->trace_best_e) b->trace_best_e[tw] = e_sel;
        if (b->trace_accepted) b->trace_accepted[tw] = (uint8_t)acc;
        if (b->trace_step) b->trace_step[tw] = step;
        if (acc) {
            memcpy(xc, cand + (int64_t)kbest * n, sizeof(double) * (size_t)n);
            b->e_cur[wi] = e_sel;
            b->n_accept[wi] += 1;
            b->win_accept[wi] += 1;
            if (b->e_cur[wi] < b->e_best[wi]) {
                b->e_best[wi] = b->e_cur[wi];
                memcpy(xb, xc, sizeof(double) * (size_t)n);
            }
        }
        if ((s64 + 1) % bp->interval == 0) {
            b->stepsize[wi] = orc_adapt_step(step, b->win_accept[wi], bp->interval,
                                             bp->target_rate, bp->factor);
            b->win_accept[wi] = 0;
        }
    }
}

void orc_bh_run(int64_t n_walkers, int32_t n_atoms, double* x_cur, double* e_cur,
                double* x_best, double* e_best, double* stepsize, int32_t* win_accept,
                int32_t* n_accept, const orc_bh_params* bp,
                double* trace_trial_e, int32_t* trace_trial_status,
                double* trace_best_e, uint8_t* trace_accepted, double* trace_step,
                int32_t n_threads)
{
    orc_bh_ctx b;
    b.n_atoms = n_atoms;
    b.n_walkers = n_walkers;
    b.x_cur = x_cur;
    b.e_cur = e_cur;
    b.x_best = x_best;
    b.e_best = e_best;
    b.stepsize = stepsize;
    b.win_accept = win_accept;
    b.n_accept = n_accept;
    b.bp = bp;
    b.trace_trial_e = trace_trial_e;
    b.trace_trial_status = trace_trial_status;
    b.trace_best_e = trace_best_e;
    b.trace_accepted = trace_accepted;
    b.trace_step = trace_step;
    int64_t n = 3 * (int64_t)n_atoms;
    size_t work = (size_t)((int64_t)bp->K * n + bp->K + (4 + 2 * (int64_t)bp->min.m) * n
                           + bp->min.m + 1);
    orc_parallel_for(n_walkers, n_threads, work, orc_bh_item, &b);
}
