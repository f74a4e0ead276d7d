/*
 * lj_oracle.h -- declarations of the FP64 CPU oracle (TEST INFRASTRUCTURE ONLY;
 * see lj_oracle.c).  Nothing outside oracle/, tests/, __graft_entry__.smoke()
 * and bench.py's CPU baseline leg includes or loads this.
 */
#ifndef LJ_ORACLE_H
#define LJ_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* per-candidate outcome of a local minimisation */
enum { ORC_CONVERGED = 0, ORC_MAXITER = 1, ORC_LINESEARCH_FAIL = 2, ORC_NONFINITE = 3,
       ORC_TIMEOUT = 4, ORC_BAD_INPUT = 5 };

enum { ORC_OBJ_LJ = 0, ORC_OBJ_QUADRATIC = 1, ORC_OBJ_ROSENBROCK = 2, ORC_OBJ_POLY1D = 3,
       ORC_OBJ_MORSE = 4 };

typedef struct {
    int32_t kind;          /* ORC_OBJ_* */
    int64_t n;             /* number of variables (3N for LJ) */
    const double* A;       /* quadratic: n x n symmetric, row-major;
                              POLY1D: NULL, or A[0] = bound above which f = +inf */
    const double* b;       /* quadratic: n; POLY1D: 5 coefficients c0..c4 */
    double eps, sigma;     /* LJ: eps, sigma; Morse: eps, re */
    double rho;            /* Morse range parameter */
} orc_objective;

typedef struct {
    int32_t m;             /* history length */
    double gtol;           /* stop when ||g||_inf < gtol */
    int32_t max_iter;
    int32_t max_ls;        /* evaluations per line search */
    double c1, c2;         /* strong-Wolfe constants */
    double alpha_max;
} orc_lbfgs_params;

typedef struct {
    int32_t K;             /* candidates per walker and step */
    double kT;             /* Metropolis temperature (energy units) */
    double target_rate;    /* adaptation target acceptance rate */
    int32_t interval;      /* adapt every `interval` steps */
    double factor;         /* step *= factor (rate <= target) or step /= factor */
    uint64_t seed;
    int64_t step0;         /* global index of the first step of this call */
    int32_t n_steps;
    int64_t walker0;       /* global index of walker 0 of this call */
    double eps, sigma;
    orc_lbfgs_params min;
    int32_t potential;     /* ORC_OBJ_LJ (0) or ORC_OBJ_MORSE (sigma = re) */
    double rho;            /* Morse range parameter */
} orc_bh_params;

/* record of one line search (tests only) */
#define ORC_LS_LOG_MAX 64
enum { ORC_LS_FAILED = 0, ORC_LS_WOLFE = 1, ORC_LS_FALLBACK = 2 };
typedef struct {
    double f0, dphi0;
    double trial[ORC_LS_LOG_MAX][3];   /* alpha, phi(alpha), phi'(alpha) */
    int32_t n_trial;
    int32_t exit;                      /* ORC_LS_* */
} orc_ls_log;

/* record of one accepted L-BFGS step (tests only) */
typedef struct {
    double alpha, f0, f, dphi0, dphi;
    int32_t exit;                      /* ORC_LS_WOLFE or ORC_LS_FALLBACK */
    int32_t retried;                   /* accepted on the retry along -g */
    int32_t n_trial;
    int32_t pad;
} orc_step_log;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_u01(uint32_t a, uint32_t b);
double orc_stream_uniform(uint64_t seed, uint32_t tag, uint32_t draw,
                          uint32_t k, uint32_t s, uint32_t w);

double orc_lj_energy_grad(int64_t n_atoms, const double* x, double* g,
                          double eps, double sigma);
double orc_morse_energy_grad(int64_t n_atoms, const double* x, double* g,
                             double eps, double re, double rho);
void orc_lbfgs_direction(int64_t n, int32_t cnt, const double* S, const double* Y,
                         const double* g, double* d, double* alpha_work);
double orc_cubic_interpolate(double a, double fa, double ga, double b, double fb, double gb);
int32_t orc_lbfgs_minimize(const orc_objective* o, double* x, const orc_lbfgs_params* p,
                           double* f_out, int32_t* iters_out, int32_t* nevals_out,
                           double* work);
int32_t orc_lbfgs_minimize_log(const orc_objective* o, double* x, const orc_lbfgs_params* p,
                               double* f_out, int32_t* iters_out, int32_t* nevals_out,
                               double* work, orc_step_log* slog, int32_t max_steps);
int32_t orc_line_search(const orc_objective* o, const double* x, const double* d,
                        double alpha1, const orc_lbfgs_params* p, double* alpha_out,
                        double* f_out, orc_ls_log* log, double* work);

/* perturbation of one candidate: out_c = x_c + step * (2 u_c - 1) */
void orc_perturb(int64_t n_coords, const double* x, double step, uint64_t seed,
                 uint32_t k, uint32_t s, uint32_t w, double* out);
int32_t orc_metropolis(double e_cur, double e_new, double kT, double u);
double orc_adapt_step(double step, int32_t win_accept, int32_t interval,
                      double target_rate, double factor);

/* batched drivers; n_threads <= 0 uses every core this process may run on */
int32_t orc_num_threads(void);
void orc_eval_batch(int64_t n_cand, int32_t uniform_n, const int64_t* atom_off,
                    const double* x, double* energy, double* grad,
                    double eps, double sigma, int32_t n_threads);
void orc_lbfgs_batch(int64_t n_cand, int32_t uniform_n, const int64_t* atom_off,
                     double* x, const orc_lbfgs_params* p, double eps, double sigma,
                     double* energy, int32_t* status, int32_t* iters, int32_t* nevals,
                     int32_t n_threads);
/* the same drivers for a chosen pair potential: kind ORC_OBJ_LJ or
 * ORC_OBJ_MORSE (sigma = re, rho its range) */
void orc_eval_batch_pot(int64_t n_cand, int32_t uniform_n, const int64_t* atom_off,
                        const double* x, double* energy, double* grad, int32_t kind,
                        double eps, double sigma, double rho, int32_t n_threads);
void orc_lbfgs_batch_pot(int64_t n_cand, int32_t uniform_n, const int64_t* atom_off,
                         double* x, const orc_lbfgs_params* p, int32_t kind, double eps,
                         double sigma, double rho, double* energy, int32_t* status,
                         int32_t* iters, int32_t* nevals, int32_t n_threads);
void orc_bh_run(int64_t n_walkers, int32_t n_atoms, double* x_cur, double* e_cur,
                double* x_best, double* e_best, double* stepsize, int32_t* win_accept,
                int32_t* n_accept, const orc_bh_params* bp,
                double* trace_trial_e, int32_t* trace_trial_status,
                double* trace_best_e, uint8_t* trace_accepted, double* trace_step,
                int32_t n_threads);

#ifdef __cplusplus
}
#endif
#endif
