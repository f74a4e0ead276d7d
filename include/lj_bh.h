/*
 * lj_bh.h -- C ABI of the GB300 (sm_103a) batched Lennard-Jones local
 * minimisation and Basin Hopping library (liblj_bh.so).
 *
 * Method: arXiv 2510.25938, "Revisiting and Accelerating the Basin Hopping
 * Algorithm for Lennard-Jones Clusters".  The three compute entry points are
 * the data-parallel hot path of that method:
 *
 *   lj_energy_grad_batched  -- Eq. (1) and its analytic gradient for a batch of
 *                              clusters (Methodology, "Lennard-Jones Potential").
 *   lbfgs_minimize_batched  -- local minimisation of many candidates at once
 *                              (Methodology, "Algorithm Overview" step 2,
 *                              "Parallel Evaluation of Candidates",
 *                              "Implementation Notes": L-BFGS-B, read as
 *                              unbounded L-BFGS, strong-Wolfe line search,
 *                              ||grad E||_inf stopping rule).
 *   bh_step_batched         -- whole Basin Hopping steps for many independent
 *                              walkers: perturbation, K parallel minimisations,
 *                              best-of-K selection, Metropolis test, step-size
 *                              adaptation ("Algorithm Overview" steps 1-5).
 *
 * Besides Eq. (1), every entry point runs on the Morse pair potential
 * (lj_potential), the kind of empirical force field the paper's Conclusions
 * name as the method's next use: the minimiser and Basin Hopping are the same.
 *
 * Conventions for every call:
 *   - Coordinates are packed xyz per atom, atoms of a candidate contiguous,
 *     candidates contiguous: the flattened 3N vector of the paper
 *     ("Initial Structures and Input").  Row-major, no padding.
 *   - Every d_* pointer is caller-owned DEVICE memory (e.g. torch tensors on
 *     the ctx's device).  The library never frees or reallocates it.
 *     Host-side structs (lj_batch, lj_*_params, lj_bh_state, lj_bh_trace)
 *     are read during the call only and may be reused immediately.
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL = legacy default stream).  The return value covers argument
 *     validation and launch errors only; per-candidate outcomes are written
 *     to device status arrays (lj_cand_status).
 *   - A ctx owns the workspace (L-BFGS history, work queue).  It is not
 *     thread-safe: use one ctx per host thread / stream.  Calls on one ctx
 *     that overlap on the GPU race on the workspace.
 *   - After lj_ctx_reserve, calls within the reserved sizes allocate nothing
 *     (safe inside CUDA-graph capture).  Without a reservation the ctx grows
 *     its workspace on demand with cudaMalloc (not capture-safe); a call
 *     beyond an explicit reservation returns LJ_ERR_NO_WORKSPACE.
 *   - n_cand == 0 returns LJ_OK without a launch.  A candidate with 0 or 1
 *     atoms has E = 0, gradient 0, status CONVERGED after 0 iterations.
 *   - Coincident atoms (r = 0) or overflow give a non-finite energy; the
 *     minimiser then reports LJ_CAND_NONFINITE for that candidate.
 */
#ifndef LJ_BH_H
#define LJ_BH_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lj_ctx lj_ctx;

typedef enum {
    LJ_OK = 0,
    LJ_ERR_INVALID_ARG = -1,   /* NULL pointer, negative size, bad enum, ... */
    LJ_ERR_CUDA = -2,          /* a CUDA runtime call or launch failed */
    LJ_ERR_NO_WORKSPACE = -3,  /* call exceeds lj_ctx_reserve sizes */
    LJ_ERR_UNSUPPORTED = -4    /* valid but outside this build's limits */
} lj_status;

typedef enum { LJ_F32 = 0, LJ_F64 = 1 } lj_dtype;

/* Pair potential of every energy the library computes.
 *   LJ_POT_LJ     Eq. (1): E = 4 eps sum_{i<j} [(sigma/r)^12 - (sigma/r)^6].
 *   LJ_POT_MORSE  Morse (Morse 1929, the form used for clusters):
 *                 E = eps sum_{i<j} e_ij (e_ij - 2), e_ij = exp(rho (1 - r_ij / re)),
 *                 with re passed in the sigma slot and 0 < rho <= 64 its range
 *                 (rho = 6 has the width of the LJ well; the bound keeps e^rho
 *                 inside FP32's range).  Coincident atoms give a non-finite
 *                 energy, as for Eq. (1).  The MIXED minimiser's three tiers are
 *                 those of Eq. (1); its double-float tier forms e^x with a
 *                 double-float exponential (argument reduction by ln 2 and a
 *                 Taylor polynomial, ~2^-42 relative). */
typedef enum { LJ_POT_LJ = 0, LJ_POT_MORSE = 1 } lj_potential;

typedef enum {
    LJ_PREC_FP64 = 0,   /* every operation in FP64 */
    LJ_PREC_FP32 = 1,   /* evaluation only: FP32 pair terms, compensated energy */
    LJ_PREC_MIXED = 2   /* minimisation: an FP32 phase, then a polish phase
                           that carries x, gradient and energy in FP64 with
                           pair terms in double-float arithmetic (FP32 pipes,
                           ~1e-14 relative) and FP32 search directions; the
                           convergence test and the returned energy come from
                           a true FP64 evaluation */
} lj_precision;

/* per-candidate outcome, written by the device */
typedef enum {
    LJ_CAND_CONVERGED = 0,       /* ||grad||_inf < gtol (FP64 gradient) */
    LJ_CAND_MAXITER = 1,
    LJ_CAND_LINESEARCH_FAIL = 2, /* no sufficient decrease, also along -grad */
    LJ_CAND_NONFINITE = 3,       /* non-finite energy or gradient at the start */
    LJ_CAND_TIMEOUT = 4,         /* deadline_cycles exceeded */
    LJ_CAND_BAD_INPUT = 5        /* candidate larger than batch.max_n */
} lj_cand_status;

/* Library limits of this build. */
#define LJ_MAX_ATOMS 1024        /* atoms per candidate */
#define LJ_MAX_M 32              /* L-BFGS history length */
#define LJ_MAX_K 16              /* candidates per walker and step */

typedef struct {
    int64_t n_cand;                /* number of candidates (>= 0) */
    int32_t uniform_n;             /* > 0: every candidate has uniform_n atoms */
    const int64_t* d_atom_offset;  /* uniform_n == 0: DEVICE int64[n_cand+1],
                                      exclusive scan of atom counts */
    int32_t max_n;                 /* uniform_n == 0: upper bound on atoms per
                                      candidate (<= LJ_MAX_ATOMS) */
} lj_batch;

typedef struct {
    int32_t m;               /* history length, 1..LJ_MAX_M (10 in the paper's setting) */
    double gtol;             /* stop when ||grad E||_inf < gtol (1e-6) */
    int32_t max_iter;        /* iteration cap (15000) */
    int32_t max_ls;          /* energy evaluations per line search (20) */
    double c1, c2;           /* strong-Wolfe constants (1e-3, 0.9) */
    double alpha_max;        /* largest trial step (1e10) */
    lj_precision prec;       /* LJ_PREC_FP64 or LJ_PREC_MIXED */
    double switch_gtol;      /* MIXED: FP32 phase ends once ||g32||_inf < switch_gtol;
                                0 = automatic: the value lj_ctx_autotune chose for the
                                candidate's size bucket, else 1e-3.  The best value is
                                workload-dependent (1e-4 for LJ38 Basin Hopping and for
                                500-1000 atom fcc fragments, 1e-3 for <= 150-atom cube
                                starts); it must sit above the FP32 gradient noise,
                                ~3e-5 eps/sigma on LJ clusters, and a value below that
                                costs up to 2000 FP32 iterations per minimisation) */
    int64_t deadline_cycles; /* > 0: a candidate still running after this many
                                SM clock cycles stops with LJ_CAND_TIMEOUT */
    double eps, sigma;       /* LJ parameters of Eq. (1) (1, 1); Morse: eps, re */
    int32_t potential;       /* lj_potential (LJ_POT_LJ = 0: Eq. (1)) */
    double rho;              /* LJ_POT_MORSE: range parameter (> 0); unused for LJ */
} lj_lbfgs_params;

typedef struct {
    int32_t K;               /* candidates per walker and step, 1..LJ_MAX_K */
    double kT;               /* Metropolis temperature in energy units */
    double target_rate;      /* acceptance rate the adaptation aims at (0.5) */
    int32_t interval;        /* adapt after every `interval` global steps (10) */
    double factor;           /* rate > target: step /= factor, else step *= factor */
    uint64_t seed;           /* Philox key */
    int64_t step0;           /* global index of the first step of this call */
    int32_t n_steps;         /* steps done by this call (>= 0) */
    int64_t walker0;         /* global index of walker 0 (for sharding) */
    lj_lbfgs_params min;     /* local minimiser */
} lj_bh_params;

/* Walker state, DEVICE arrays, updated in place.  All walkers share n_atoms. */
typedef struct {
    int32_t n_walkers;
    int32_t n_atoms;
    double* x_cur;     /* [W][3N] current (minimised) structure */
    double* e_cur;     /* [W] its FP64 energy */
    double* x_best;    /* [W][3N] lowest-energy accepted structure */
    double* e_best;    /* [W] */
    double* stepsize;  /* [W] perturbation half-width */
    int32_t* win_accept; /* [W] acceptances in the current adaptation window */
    int32_t* n_accept;   /* [W] total acceptances */
} lj_bh_state;

/* Optional per-step trace, DEVICE arrays; any pointer may be NULL. */
typedef struct {
    double* trial_e;        /* [n_steps][W][K] minimised candidate energies */
    int32_t* trial_status;  /* [n_steps][W][K] lj_cand_status */
    int32_t* trial_iters;   /* [n_steps][W][K] L-BFGS iterations */
    double* best_trial_e;   /* [n_steps][W] energy of the selected candidate */
    uint8_t* accepted;      /* [n_steps][W] Metropolis outcome */
    double* stepsize;       /* [n_steps][W] step size used in that step */
    uint8_t* near_tie;      /* [n_steps][W] 1 when the Metropolis decision sat within
                               LJ_NEAR_TIE of its threshold: |dE| <= LJ_NEAR_TIE (energy
                               units) or, for dE > 0, |u - exp(-dE/kT)| <= LJ_NEAR_TIE *
                               exp(-dE/kT).  Another FP64 implementation (other summation
                               order, another exp) may decide such a step the other way */
} lj_bh_trace;

/* Near-tie margin of the Metropolis test: far above the ~1e-12 by which two
 * FP64 evaluations of the same minimum differ, far below what one trial move
 * changes. */
#define LJ_NEAR_TIE 1e-9

/* Device-side work counters, accumulated (atomically) by a call; the caller
 * zeroes them.  Used for flop accounting and throughput. */
typedef struct {
    unsigned long long evals32;     /* FP32 energy+gradient evaluations */
    unsigned long long evals64;     /* FP64 energy+gradient evaluations */
    unsigned long long evals_df;    /* double-float evaluations (mixed polish) */
    unsigned long long iters32;     /* L-BFGS iterations in the FP32 phase */
    unsigned long long iters64;     /* L-BFGS iterations in FP64 / polish */
    unsigned long long pairs32;     /* unordered atom pairs evaluated in FP32 */
    unsigned long long pairs64;     /* unordered atom pairs evaluated in FP64 */
    unsigned long long pairs_df;    /* unordered atom pairs evaluated in double-float */
    unsigned long long vec_elems32; /* sum over iterations of m_used * 3N (FP32 vectors) */
    unsigned long long vec_elems64; /* same for FP64 vectors */
    unsigned long long converged;   /* candidates with LJ_CAND_CONVERGED */
    unsigned long long minimisations; /* candidates minimised */
    unsigned long long cycles32;    /* SM clock cycles in FP32 iterations (summed over candidates) */
    unsigned long long cycles_df;   /* ... in double-float polish iterations */
    unsigned long long cycles64;    /* ... in FP64 iterations and FP64 evaluations */
    unsigned long long cycles_direction;  /* ... of which in L-BFGS direction computations */
    unsigned long long cycles_linesearch; /* ... of which in line searches (with their evaluations) */
} lj_stats;

/* Tuning options of a context. */
typedef enum {
    LJ_OPT_BH_TEAM = 1,      /* threads per candidate in bh_step_batched for
                                clusters of <= 64 atoms: 0 (automatic), 32, 64, 128 */
    LJ_OPT_LBFGS_TEAM = 2,   /* threads per candidate in lbfgs_minimize_batched, all
                                sizes: 0 (automatic or autotuned), 32, 64, 128, 256,
                                512; a size too small for a bucket (more than two
                                atoms per thread) falls back to the default there */
    LJ_OPT_F32_HANDOVER = 3, /* MIXED: below this many FP32 ulps of |E| of predicted
                                decrease -alpha phi'(0), the FP32 phase accepts
                                steps on the gradient alone (1..4096; 0 = default 4) */
    LJ_OPT_DF_HANDOVER = 4,  /* MIXED: below this many 2^-48 |E| of predicted
                                decrease, the double-float polish accepts steps on
                                the gradient alone (1..65536; 0 = default 32) */
    LJ_OPT_HISTORY = 5,      /* L-BFGS history placement, both minimising calls:
                                0 (automatic: the autotuned choice, else shared memory
                                when a CTA's shared memory stays within ~100 KB),
                                1 global memory always, 2 automatic ignoring the
                                autotuner.  Results do not depend on it */
    LJ_OPT_DF_EVAL = 6       /* MIXED double-float evaluations of clusters above 256
                                atoms: 0 (automatic: the autotuned choice, else 32 x 32
                                tiles taking each pair once), 1 one-sided rows (each
                                pair from both atoms), 2 tiles */
} lj_option;

const char* lj_status_string(lj_status s);

/* Create a context on CUDA device `device`.  *out receives the handle. */
lj_status lj_ctx_create(lj_ctx** out, int device);
/* Destroy a context and free its workspace (synchronises its device). */
lj_status lj_ctx_destroy(lj_ctx* ctx);
/* Reserve workspace for calls with up to max_cand candidates (or walkers x K
 * for bh_step_batched) of up to max_n atoms and history length max_m.  After
 * a reservation no call allocates. */
lj_status lj_ctx_reserve(lj_ctx* ctx, int64_t max_cand, int32_t max_n, int32_t max_m);
/* Set a tuning option (lj_option); affects later calls on this ctx only. */
lj_status lj_ctx_set_option(lj_ctx* ctx, lj_option opt, int64_t value);
/* Human-readable description of the last error on this ctx ("" if none). */
const char* lj_ctx_last_error(const lj_ctx* ctx);

/*
 * Eq. (1) energy (FP64 result) and gradient for every candidate of `batch`.
 *   prec   LJ_PREC_FP32 (or MIXED): FP32 pair terms with compensated energy
 *          accumulation; LJ_PREC_FP64: every operation in FP64.
 *   xtype  dtype of d_x and d_grad (LJ_F32 or LJ_F64).
 *   d_x    [total_atoms*3] coordinates.
 *   d_energy [n_cand] FP64 energies.
 *   d_grad [total_atoms*3] gradient dE/dx in xtype, or NULL for energy only.
 *   eps, sigma  Eq. (1) parameters (> 0).
 */
lj_status lj_energy_grad_batched(lj_ctx* ctx, const lj_batch* batch, lj_precision prec,
                                 lj_dtype xtype, const void* d_x, double* d_energy,
                                 void* d_grad, double eps, double sigma, void* stream);

/*
 * lj_energy_grad_batched for a chosen pair potential: potential LJ_POT_LJ
 * gives exactly lj_energy_grad_batched (eps, sigma; rho unused);
 * LJ_POT_MORSE evaluates E = eps sum_{i<j} e (e - 2), e = exp(rho (1 - r/re)),
 * with re = sigma, and its gradient dE/dx_i = -(2 eps rho / re) sum_{j != i}
 * e (e - 1) (x_i - x_j) / r_ij.  Morse clusters run one team per candidate
 * in one-sided rows, FP32 (FP32 exp and reciprocal square root,
 * compensated energy) or FP64.  Errors as lj_energy_grad_batched, plus
 * INVALID_ARG for an unknown potential or rho outside (0, 64] (Morse).
 */
lj_status lj_energy_grad_batched_pot(lj_ctx* ctx, const lj_batch* batch, lj_precision prec,
                                     lj_dtype xtype, const void* d_x, double* d_energy,
                                     void* d_grad, int32_t potential, double eps,
                                     double sigma, double rho, void* stream);

/*
 * Local minimisation of every candidate of `batch`, in place.
 *   d_x      [total_atoms*3] FP64 start coordinates in, minimised out.
 *   d_energy [n_cand] FP64 energy at the returned coordinates.
 *   d_status [n_cand] lj_cand_status (may be NULL).
 *   d_iters  [n_cand] L-BFGS iterations (may be NULL).
 *   d_nevals [n_cand] energy+gradient evaluations (may be NULL).
 *   d_stats  device lj_stats accumulated by this call (may be NULL).
 */
lj_status lbfgs_minimize_batched(lj_ctx* ctx, const lj_batch* batch, const lj_lbfgs_params* p,
                                 double* d_x, double* d_energy, int32_t* d_status,
                                 int32_t* d_iters, int32_t* d_nevals, lj_stats* d_stats,
                                 void* stream);

/*
 * p->n_steps Basin Hopping steps for every walker of `state`, in one launch.
 * Step s (global index step0 + i) of walker w (global walker0 + w):
 *   1. K candidates x_k = x_cur + step * (2u - 1) per coordinate, u from
 *      Philox4x32-10 stream 1 at counter (coordinate, k, s, w);
 *   2. each candidate minimised as in lbfgs_minimize_batched;
 *   3. k* = lowest finite energy (ties: lowest k);
 *   4. accept if E_k* <= E_cur or u < exp(-(E_k* - E_cur)/kT), u from stream 2;
 *   5. after step s with (s+1) % interval == 0: window rate > target_rate ->
 *      step /= factor, else step *= factor; window counter reset.
 * state must hold minimised structures with their energies (e.g. from
 * lbfgs_minimize_batched).  trace and d_stats may be NULL.
 */
lj_status bh_step_batched(lj_ctx* ctx, const lj_bh_state* state, const lj_bh_params* p,
                          const lj_bh_trace* trace, lj_stats* d_stats, void* stream);

/*
 * lj_ctx_autotune -- choose, per size bucket, the threads per candidate that
 * lbfgs_minimize_batched uses on this ctx and, for MIXED, the FP32 tier's
 * hand-over gradient.  (A tuning aid of this library, not part of the
 * paper's method.)
 *   Buckets: N <= 32, 64, 128, 256, 512, 1024 atoms (LJ_TUNE_BUCKETS), the
 *   same size classes an uneven batch is split into.  For every bucket up to
 *   the one holding max_n, each team size the bucket can take (32..512
 *   threads, one or two atoms per thread) minimises the same batch of
 *   synthetic cube starts (reduced density 0.3, three quarters of the
 *   bucket's upper size, history m, precision prec) twice; the second,
 *   timed run decides by converged minimisations per second.  For MIXED the
 *   same batch then runs with switch_gtol 1e-3, 3e-4 and 1e-4 on the chosen
 *   team, and the fastest is kept; then, where they are alternatives, the
 *   history in global memory instead of shared memory, and (MIXED, buckets
 *   above 256 atoms) one-sided double-float rows instead of tiles.  The
 *   whole entry can be read back with lj_ctx_get_tuning.
 *   out_team         [LJ_TUNE_BUCKETS] chosen team sizes, 0 beyond max_n's
 *                    bucket (may be NULL).
 *   out_switch_gtol  [LJ_TUNE_BUCKETS] chosen switch_gtol (MIXED), 0 beyond
 *                    max_n's bucket or for FP64 (may be NULL).
 * Later lbfgs_minimize_batched calls on this ctx use the chosen team sizes
 * unless LJ_OPT_LBFGS_TEAM is set (the option wins), and the chosen
 * switch_gtol wherever the call passes switch_gtol = 0.  A setup call: it allocates
 * and frees device memory, may enlarge the ctx workspace and synchronises
 * `stream` -- call it before lj_ctx_reserve and outside graph capture.  It
 * takes from well under a second (small max_n) to a few seconds (1024).
 * Errors: INVALID_ARG (max_n < 2, m outside 1..LJ_MAX_M, prec FP32),
 * UNSUPPORTED (max_n > LJ_MAX_ATOMS), CUDA.  On error the ctx keeps its
 * previous choices.
 */
#define LJ_TUNE_BUCKETS 6
#define LJ_TUNE_BH LJ_TUNE_BUCKETS   /* lj_ctx_get_tuning: the bh_step_batched entry */

/* One entry of a context's tuning table. */
typedef struct {
    int32_t team;            /* threads per candidate (0: default shape) */
    double switch_gtol;      /* MIXED FP32-tier hand-over gradient (0: library default) */
    int32_t history_global;  /* 1: L-BFGS history in global memory */
    int32_t df_one_sided;    /* 1: one-sided double-float rows instead of tiles */
    int32_t tuned;           /* 1 once an autotuning call has set this entry */
} lj_tuning;
lj_status lj_ctx_autotune(lj_ctx* ctx, int32_t max_n, int32_t m, lj_precision prec,
                          int32_t* out_team, double* out_switch_gtol, void* stream);

/*
 * lj_ctx_get_tuning -- the context's tuning entry for size bucket `bucket`
 * (0 .. LJ_TUNE_BUCKETS-1, lbfgs_minimize_batched) or LJ_TUNE_BH
 * (bh_step_batched).  Errors: INVALID_ARG (bucket out of range, NULL out).
 */
lj_status lj_ctx_get_tuning(const lj_ctx* ctx, int32_t bucket, lj_tuning* out);

/*
 * lj_ctx_autotune_bh -- tune bh_step_batched on the caller's own walkers.
 * (A tuning aid of this library, not part of the paper's method.)
 * Copies of `state` (left unchanged) run p->n_steps Basin Hopping steps
 * (p as given: K, kT, seed, ...; p->min.prec FP64 or MIXED) twice for each
 * choice -- the first run a warm-up, the second timed by converged
 * minimisations per second -- choosing in turn the threads per candidate
 * (32, 64 or 128 for clusters of up to 64 atoms; the default shape above),
 * for MIXED the FP32 tier's switch_gtol (1e-3, 3e-4, 1e-4), and the history
 * placement (shared memory when it fits, or global memory).  Later
 * bh_step_batched calls on this ctx use the chosen team and placement
 * unless LJ_OPT_BH_TEAM / LJ_OPT_HISTORY are set, and the chosen
 * switch_gtol wherever p->min.switch_gtol = 0.  *out receives the choice
 * (may be NULL).  A setup call like lj_ctx_autotune: it allocates device
 * memory, may grow the workspace and synchronises `stream`.
 * Errors: INVALID_ARG (as bh_step_batched; n_steps < 1), UNSUPPORTED, CUDA.
 */
lj_status lj_ctx_autotune_bh(lj_ctx* ctx, const lj_bh_state* state, const lj_bh_params* p,
                             lj_tuning* out, void* stream);

/*
 * lj_ctx_autotune_batch -- the same choice for one size bucket, measured on
 * the caller's own starts: a uniform batch (uniform_n >= 1) whose first
 * min(n_cand, max_sample) candidates of d_x (device, FP64, left unchanged)
 * are minimised on copies with each choice.  Sets the entries of the bucket
 * holding uniform_n; out_team / out_switch_gtol receive them (may be NULL).
 * Use it when the workload's starts differ from random cube starts (e.g.
 * perturbed lattice fragments).  Same setup-call rules and errors as
 * lj_ctx_autotune; INVALID_ARG also for an uneven batch or max_sample < 1.
 */
lj_status lj_ctx_autotune_batch(lj_ctx* ctx, const lj_batch* batch, const double* d_x, int32_t m,
                                lj_precision prec, int64_t max_sample, int32_t* out_team,
                                double* out_switch_gtol, void* stream);

/*
 * lbfgs_minimize_batched_noalloc -- the same minimisation as
 * lbfgs_minimize_batched, for callers that must not allocate device memory.
 * (Not part of the method: the paper has no counterpart; it only changes
 * where this library keeps its scratch memory.)
 *
 * Who needs it: applications whose memory manager has already taken the
 * device memory it is allowed and forbids further cudaMalloc/cudaFree (a
 * framework's caching allocator, a pool sized once at start-up), code that
 * runs where an allocation's implicit device synchronisation is not
 * acceptable, and latency-critical loops that cannot pay for an allocation.
 * It takes no lj_ctx (creating one allocates) and uses the default tuning
 * options.
 *
 * Scratch: a fixed array of LJ_NOALLOC_SCRATCH_BYTES in the library's
 * device-global memory holds the work-queue counters (256 bytes), the
 * size-bucket lists of an uneven batch (6 x 4 bytes per candidate) and any
 * L-BFGS history that does not fit in shared memory.  Every GPU that loads
 * the library holds this array until the process exits.
 * Limits: an uneven batch of more than
 * (LJ_NOALLOC_SCRATCH_BYTES - 256) / 24 = 699,040 candidates returns
 * LJ_ERR_NO_WORKSPACE.  When the off-chip history of all teams would not fit
 * in what is left, fewer teams are launched (each still drains the shared
 * work queue), so the batch takes longer but still runs; for large clusters
 * this caps the launch hard: a history slot holds 2 m x 3 x 1024 values for
 * clusters of 513..1024 atoms (4 bytes each for LJ_PREC_MIXED, 8 for
 * LJ_PREC_FP64), so with m = 20 about 34 (mixed) or 17 (FP64) teams run, on
 * a small part of the GPU.  A batch whose smallest launch (one CTA) would not
 * fit returns LJ_ERR_NO_WORKSPACE.
 *
 * Set-up: the first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it; make that
 * first call before any stream capture.  Later calls use the cached address.
 *
 * Calls share the array: the counter is cleared at the start of every call
 * and the previous call's contents are otherwise left in place.  Calls that
 * overlap on the GPU (other streams, other host threads) race on it; order
 * them on one stream.
 *
 * Arguments, results and errors are those of lbfgs_minimize_batched; the
 * call runs on the device that is current for the calling host thread.
 */
#define LJ_NOALLOC_SCRATCH_BYTES (16u << 20)
lj_status lbfgs_minimize_batched_noalloc(const lj_batch* batch, const lj_lbfgs_params* p,
                                         double* d_x, double* d_energy, int32_t* d_status,
                                         int32_t* d_iters, int32_t* d_nevals, lj_stats* d_stats,
                                         void* stream);

#ifdef __cplusplus
}
#endif
#endif
