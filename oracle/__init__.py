"""FP64 CPU oracle for batched Lennard-Jones Basin Hopping.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import this package.  The
product (``paper_2510_25938_gb300``) never imports it, and the two share no
code: the oracle is a separate plain-C library (``lj_oracle.c``) built with
``-O2 -ffp-contract=off`` and called here through ctypes.

Every function states the passage of arXiv 2510.25938 it follows:

* ``lj_energy_grad`` -- Methodology, "Lennard-Jones Potential", Eq. (1), and
  its analytic gradient.
* ``morse_energy_grad`` -- the Morse pair potential (Morse 1929, cluster
  form), the pair-potential extension the Conclusions point to; every batch
  driver, the minimiser and ``bh_run`` take it as ``potential=OBJ_MORSE``.
* ``lbfgs_minimize`` -- Methodology, "Algorithm Overview" step 2 and
  "Implementation Notes" (L-BFGS-B, read as unbounded L-BFGS with the
  two-loop recursion, a strong-Wolfe line search and the gradient inf-norm
  stopping rule).
* ``perturb`` / ``metropolis`` / ``adapt_step`` / ``bh_run`` -- "Algorithm
  Overview" steps 1, 3, 4 and 5; Results, first paragraph (direction of the
  adaptation).
* ``philox4x32_10`` -- the counter-based generator of Salmon et al. (SC'11),
  from its published definition.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblj_oracle.so")
_SRC = [os.path.join(_HERE, "lj_oracle.c"), os.path.join(_HERE, "lj_oracle.h")]

CONVERGED, MAXITER, LINESEARCH_FAIL, NONFINITE, TIMEOUT, BAD_INPUT = range(6)
OBJ_LJ, OBJ_QUADRATIC, OBJ_ROSENBROCK, OBJ_POLY1D, OBJ_MORSE = range(5)
LS_FAILED, LS_WOLFE, LS_FALLBACK = range(3)
LS_LOG_MAX = 64

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle library with gcc (plain C11, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest_src = max(os.path.getmtime(p) for p in _SRC)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest_src:
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
           "-D_GNU_SOURCE", "-Wall", "-fPIC", "-shared", "-pthread",
           "-o", tmp, _SRC[0], "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class LbfgsParams(C.Structure):
    _fields_ = [("m", C.c_int32), ("gtol", C.c_double), ("max_iter", C.c_int32),
                ("max_ls", C.c_int32), ("c1", C.c_double), ("c2", C.c_double),
                ("alpha_max", C.c_double)]


class Objective(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n", C.c_int64), ("A", C.c_void_p),
                ("b", C.c_void_p), ("eps", C.c_double), ("sigma", C.c_double),
                ("rho", C.c_double)]


class LsLog(C.Structure):
    _fields_ = [("f0", C.c_double), ("dphi0", C.c_double),
                ("trial", (C.c_double * 3) * LS_LOG_MAX), ("n_trial", C.c_int32),
                ("exit", C.c_int32)]


class StepLog(C.Structure):
    _fields_ = [("alpha", C.c_double), ("f0", C.c_double), ("f", C.c_double),
                ("dphi0", C.c_double), ("dphi", C.c_double), ("exit", C.c_int32),
                ("retried", C.c_int32), ("n_trial", C.c_int32), ("pad", C.c_int32)]


class BhParams(C.Structure):
    _fields_ = [("K", C.c_int32), ("kT", C.c_double), ("target_rate", C.c_double),
                ("interval", C.c_int32), ("factor", C.c_double), ("seed", C.c_uint64),
                ("step0", C.c_int64), ("n_steps", C.c_int32), ("walker0", C.c_int64),
                ("eps", C.c_double), ("sigma", C.c_double), ("min", LbfgsParams),
                ("potential", C.c_int32), ("rho", C.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            lib.orc_philox4x32_10.argtypes = [P, P, P]
            lib.orc_philox4x32_10.restype = None
            lib.orc_u01.argtypes = [C.c_uint32, C.c_uint32]
            lib.orc_u01.restype = C.c_double
            lib.orc_stream_uniform.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32,
                                               C.c_uint32, C.c_uint32, C.c_uint32]
            lib.orc_stream_uniform.restype = C.c_double
            lib.orc_lj_energy_grad.argtypes = [C.c_int64, P, P, C.c_double, C.c_double]
            lib.orc_lj_energy_grad.restype = C.c_double
            lib.orc_morse_energy_grad.argtypes = [C.c_int64, P, P, C.c_double, C.c_double,
                                                  C.c_double]
            lib.orc_morse_energy_grad.restype = C.c_double
            lib.orc_lbfgs_direction.argtypes = [C.c_int64, C.c_int32, P, P, P, P, P]
            lib.orc_lbfgs_direction.restype = None
            lib.orc_cubic_interpolate.argtypes = [C.c_double] * 6
            lib.orc_cubic_interpolate.restype = C.c_double
            lib.orc_lbfgs_minimize.argtypes = [C.POINTER(Objective), P,
                                               C.POINTER(LbfgsParams), P, P, P, P]
            lib.orc_lbfgs_minimize.restype = C.c_int32
            lib.orc_lbfgs_minimize_log.argtypes = [C.POINTER(Objective), P,
                                                   C.POINTER(LbfgsParams), P, P, P, P, P,
                                                   C.c_int32]
            lib.orc_lbfgs_minimize_log.restype = C.c_int32
            lib.orc_line_search.argtypes = [C.POINTER(Objective), P, P, C.c_double,
                                            C.POINTER(LbfgsParams), P, P,
                                            C.POINTER(LsLog), P]
            lib.orc_line_search.restype = C.c_int32
            lib.orc_perturb.argtypes = [C.c_int64, P, C.c_double, C.c_uint64,
                                        C.c_uint32, C.c_uint32, C.c_uint32, P]
            lib.orc_perturb.restype = None
            lib.orc_metropolis.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double]
            lib.orc_metropolis.restype = C.c_int32
            lib.orc_adapt_step.argtypes = [C.c_double, C.c_int32, C.c_int32,
                                           C.c_double, C.c_double]
            lib.orc_adapt_step.restype = C.c_double
            lib.orc_num_threads.argtypes = []
            lib.orc_num_threads.restype = C.c_int32
            lib.orc_eval_batch.argtypes = [C.c_int64, C.c_int32, P, P, P, P,
                                           C.c_double, C.c_double, C.c_int32]
            lib.orc_eval_batch.restype = None
            lib.orc_lbfgs_batch.argtypes = [C.c_int64, C.c_int32, P, P,
                                            C.POINTER(LbfgsParams), C.c_double, C.c_double,
                                            P, P, P, P, C.c_int32]
            lib.orc_lbfgs_batch.restype = None
            lib.orc_eval_batch_pot.argtypes = [C.c_int64, C.c_int32, P, P, P, P, C.c_int32,
                                               C.c_double, C.c_double, C.c_double, C.c_int32]
            lib.orc_eval_batch_pot.restype = None
            lib.orc_lbfgs_batch_pot.argtypes = [C.c_int64, C.c_int32, P, P,
                                                C.POINTER(LbfgsParams), C.c_int32, C.c_double,
                                                C.c_double, C.c_double, P, P, P, P, C.c_int32]
            lib.orc_lbfgs_batch_pot.restype = None
            lib.orc_bh_run.argtypes = [C.c_int64, C.c_int32, P, P, P, P, P, P, P,
                                       C.POINTER(BhParams), P, P, P, P, P, C.c_int32]
            lib.orc_bh_run.restype = None
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class MinParams:
    """L-BFGS settings.  m=10 and gtol=1e-6 on ||g||_inf are the workload's;
    c1=1e-3, c2=0.9, 20 evaluations per line search and alpha_max=1e10 are the
    reading of the unstated L-BFGS-B line search; max_iter=15000 is scipy's
    L-BFGS-B default iteration cap."""
    m: int = 10
    gtol: float = 1e-6
    max_iter: int = 15000
    max_ls: int = 20
    c1: float = 1e-3
    c2: float = 0.9
    alpha_max: float = 1e10

    def c(self) -> LbfgsParams:
        return LbfgsParams(self.m, self.gtol, self.max_iter, self.max_ls,
                           self.c1, self.c2, self.alpha_max)


def num_threads() -> int:
    return int(_load().orc_num_threads())


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block: 4 x uint32 counter, 2 x uint32 key -> 4 x uint32."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def u01(a: int, b: int) -> float:
    return float(_load().orc_u01(a, b))


def stream_uniform(seed: int, tag: int, draw: int, k: int, s: int, w: int) -> float:
    return float(_load().orc_stream_uniform(seed, tag, draw, k, s, w))


def lj_energy_grad(x, eps: float = 1.0, sigma: float = 1.0):
    """Eq. (1) and its gradient for one cluster; x is (N,3) or flat 3N."""
    x = _f64(x).reshape(-1)
    g = np.zeros_like(x)
    e = _load().orc_lj_energy_grad(x.size // 3, _ptr(x), _ptr(g), eps, sigma)
    return float(e), g


def morse_energy_grad(x, eps: float = 1.0, re: float = 1.0, rho: float = 6.0):
    """Morse energy eps sum_{i<j} e_ij (e_ij - 2), e_ij = exp(rho (1 - r_ij / re)),
    and its gradient for one cluster; x is (N,3) or flat 3N."""
    x = _f64(x).reshape(-1)
    g = np.zeros_like(x)
    e = _load().orc_morse_energy_grad(x.size // 3, _ptr(x), _ptr(g), eps, re, rho)
    return float(e), g


def lbfgs_direction(S, Y, g) -> np.ndarray:
    """Two-loop recursion: d = -H g for history rows S, Y (oldest first)."""
    S = _f64(S)
    Y = _f64(Y)
    g = _f64(g).reshape(-1)
    cnt = S.shape[0] if S.ndim == 2 else 0
    d = np.zeros_like(g)
    work = np.zeros(max(cnt, 1))
    _load().orc_lbfgs_direction(g.size, cnt, _ptr(S), _ptr(Y), _ptr(g), _ptr(d), _ptr(work))
    return d


def cubic_interpolate(a, fa, ga, b, fb, gb) -> float:
    return float(_load().orc_cubic_interpolate(a, fa, ga, b, fb, gb))


def minimize(x0, kind: int = OBJ_LJ, params: MinParams | None = None, A=None, b=None,
             eps: float = 1.0, sigma: float = 1.0, rho: float = 6.0):
    """Minimise one objective from x0 (OBJ_MORSE: eps, sigma = re, rho).
    Returns (x, f, status, iters, nevals)."""
    p = params or MinParams()
    x = _f64(x0).reshape(-1).copy()
    n = x.size
    Aa = _f64(A) if A is not None else None
    ba = _f64(b) if b is not None else None
    obj = Objective(kind, n, _ptr(Aa), _ptr(ba), eps, sigma, rho)
    work = np.zeros((4 + 2 * p.m) * n + p.m + 1)
    f = C.c_double()
    it = C.c_int32()
    ne = C.c_int32()
    pc = p.c()
    st = _load().orc_lbfgs_minimize(C.byref(obj), _ptr(x), C.byref(pc), C.byref(f),
                                    C.byref(it), C.byref(ne), _ptr(work))
    return x, float(f.value), int(st), int(it.value), int(ne.value)


def minimize_log(x0, kind: int = OBJ_LJ, params: MinParams | None = None, A=None, b=None,
                 eps: float = 1.0, sigma: float = 1.0, max_steps: int = 20000,
                 rho: float = 6.0):
    """minimize() that also returns a record of every accepted step: a
    structured array with alpha, f0, f, dphi0, dphi (phi'(alpha) along the
    step's direction), exit (LS_WOLFE / LS_FALLBACK), retried, n_trial."""
    p = params or MinParams()
    x = _f64(x0).reshape(-1).copy()
    n = x.size
    Aa = _f64(A) if A is not None else None
    ba = _f64(b) if b is not None else None
    obj = Objective(kind, n, _ptr(Aa), _ptr(ba), eps, sigma, rho)
    work = np.zeros((4 + 2 * p.m) * n + p.m + 1)
    logs = (StepLog * max_steps)()
    f = C.c_double()
    it = C.c_int32()
    ne = C.c_int32()
    pc = p.c()
    st = _load().orc_lbfgs_minimize_log(C.byref(obj), _ptr(x), C.byref(pc), C.byref(f),
                                        C.byref(it), C.byref(ne), _ptr(work), logs, max_steps)
    n_steps = min(int(it.value), max_steps)
    rec = [{k: getattr(logs[i], k) for k, _ in StepLog._fields_ if k != "pad"}
           for i in range(n_steps)]
    return x, float(f.value), int(st), int(it.value), int(ne.value), rec


def line_search(x, d, alpha1: float, kind: int = OBJ_POLY1D, params: MinParams | None = None,
                A=None, b=None, eps: float = 1.0, sigma: float = 1.0, rho: float = 6.0):
    """One strong-Wolfe line search of the oracle from x along d with first
    trial alpha1.  Returns a dict: ok, alpha, f (accepted point), f0, dphi0,
    trials (k x 3 array of alpha, phi, phi' in evaluation order; a final
    re-evaluation of an earlier trial after an exhausted budget included)
    and exit (LS_WOLFE, LS_FALLBACK or LS_FAILED)."""
    p = params or MinParams()
    x = _f64(x).reshape(-1)
    d = _f64(d).reshape(-1)
    n = x.size
    Aa = _f64(A) if A is not None else None
    ba = _f64(b) if b is not None else None
    obj = Objective(kind, n, _ptr(Aa), _ptr(ba), eps, sigma, rho)
    work = np.zeros(3 * n)
    log = LsLog()
    a = C.c_double()
    f = C.c_double()
    pc = p.c()
    ok = _load().orc_line_search(C.byref(obj), _ptr(x), _ptr(d), alpha1, C.byref(pc),
                                 C.byref(a), C.byref(f), C.byref(log), _ptr(work))
    k = min(log.n_trial, LS_LOG_MAX)
    trials = np.array([[log.trial[i][j] for j in range(3)] for i in range(k)]).reshape(-1, 3)
    return {"ok": bool(ok), "alpha": float(a.value), "f": float(f.value), "f0": log.f0,
            "dphi0": log.dphi0, "trials": trials, "exit": int(log.exit)}


def _layout(n_cand, uniform_n, atom_off):
    if uniform_n and uniform_n > 0:
        return int(uniform_n), None
    off = np.ascontiguousarray(atom_off, dtype=np.int64)
    assert off.size == n_cand + 1
    return 0, off


def eval_batch(x, n_cand: int, uniform_n: int = 0, atom_off=None, eps=1.0, sigma=1.0,
               grad: bool = True, n_threads: int = 0, potential: int = OBJ_LJ,
               rho: float = 6.0):
    """Energy (and gradient) of a batch of clusters with packed xyz coordinates
    (potential OBJ_LJ, or OBJ_MORSE with sigma = re and range rho)."""
    un, off = _layout(n_cand, uniform_n, atom_off)
    x = _f64(x).reshape(-1)
    e = np.zeros(n_cand)
    g = np.zeros_like(x) if grad else None
    _load().orc_eval_batch_pot(n_cand, un, _ptr(off), _ptr(x), _ptr(e), _ptr(g), potential,
                               eps, sigma, rho, n_threads)
    return e, g


def lbfgs_batch(x, n_cand: int, uniform_n: int = 0, atom_off=None,
                params: MinParams | None = None, eps=1.0, sigma=1.0, n_threads: int = 0,
                potential: int = OBJ_LJ, rho: float = 6.0):
    """Minimise a batch of clusters (LJ, or Morse with potential=OBJ_MORSE)
    in place (a copy is returned)."""
    p = params or MinParams()
    un, off = _layout(n_cand, uniform_n, atom_off)
    x = _f64(x).reshape(-1).copy()
    e = np.zeros(n_cand)
    st = np.zeros(n_cand, dtype=np.int32)
    it = np.zeros(n_cand, dtype=np.int32)
    ne = np.zeros(n_cand, dtype=np.int32)
    pc = p.c()
    _load().orc_lbfgs_batch_pot(n_cand, un, _ptr(off), _ptr(x), C.byref(pc), potential, eps,
                                sigma, rho, _ptr(e), _ptr(st), _ptr(it), _ptr(ne), n_threads)
    return x, e, st, it, ne


def perturb(x, step: float, seed: int, k: int, s: int, w: int) -> np.ndarray:
    x = _f64(x).reshape(-1)
    out = np.zeros_like(x)
    _load().orc_perturb(x.size, _ptr(x), step, seed, k, s, w, _ptr(out))
    return out


def metropolis(e_cur: float, e_new: float, kT: float, u: float) -> bool:
    return bool(_load().orc_metropolis(e_cur, e_new, kT, u))


def adapt_step(step: float, win_accept: int, interval: int, target: float,
               factor: float) -> float:
    return float(_load().orc_adapt_step(step, win_accept, interval, target, factor))


@dataclass
class BhParamsPy:
    K: int = 1
    kT: float = 0.8
    target_rate: float = 0.5
    interval: int = 10
    factor: float = 0.9
    seed: int = 0
    step0: int = 0
    n_steps: int = 1
    walker0: int = 0
    eps: float = 1.0
    sigma: float = 1.0
    min: MinParams = None
    potential: int = OBJ_LJ     # or OBJ_MORSE (sigma = re)
    rho: float = 6.0

    def c(self) -> BhParams:
        mp = (self.min or MinParams()).c()
        return BhParams(self.K, self.kT, self.target_rate, self.interval, self.factor,
                        self.seed, self.step0, self.n_steps, self.walker0, self.eps,
                        self.sigma, mp, self.potential, self.rho)


def bh_run(state: dict, params: BhParamsPy, n_threads: int = 0, trace: bool = True):
    """Advance every walker of ``state`` by params.n_steps BH steps (in place).

    state: x_cur (W,3N), e_cur (W), x_best, e_best, stepsize (W),
    win_accept (W int32), n_accept (W int32).  Returns the trace dict."""
    x_cur = state["x_cur"]
    W = x_cur.shape[0]
    n_atoms = x_cur.shape[1] // 3
    for key, dt in (("x_cur", np.float64), ("e_cur", np.float64), ("x_best", np.float64),
                    ("e_best", np.float64), ("stepsize", np.float64),
                    ("win_accept", np.int32), ("n_accept", np.int32)):
        a = state[key]
        assert a.dtype == dt and a.flags.c_contiguous, key
    S, K = params.n_steps, params.K
    tr = None
    if trace:
        tr = {"trial_e": np.zeros((S, W, K)), "trial_status": np.zeros((S, W, K), np.int32),
              "best_trial_e": np.zeros((S, W)), "accepted": np.zeros((S, W), np.uint8),
              "stepsize": np.zeros((S, W))}
    bp = params.c()
    g = (lambda k: _ptr(tr[k]) if tr else None)
    _load().orc_bh_run(W, n_atoms, _ptr(state["x_cur"]), _ptr(state["e_cur"]),
                       _ptr(state["x_best"]), _ptr(state["e_best"]), _ptr(state["stepsize"]),
                       _ptr(state["win_accept"]), _ptr(state["n_accept"]), C.byref(bp),
                       g("trial_e"), g("trial_status"), g("best_trial_e"), g("accepted"),
                       g("stepsize"), n_threads)
    return tr
