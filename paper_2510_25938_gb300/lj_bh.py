"""Thin ctypes binding of liblj_bh.so (include/lj_bh.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of the library.  Tensors are torch CUDA tensors (PyTorch is used for
device memory and streams); their data pointers and the current CUDA stream
are passed straight to the C ABI.  If the library has not been built, every
call raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass, field

import torch

from . import build as _build

# ---- enums of include/lj_bh.h -------------------------------------------------
LJ_OK, LJ_ERR_INVALID_ARG, LJ_ERR_CUDA, LJ_ERR_NO_WORKSPACE, LJ_ERR_UNSUPPORTED = 0, -1, -2, -3, -4
LJ_F32, LJ_F64 = 0, 1
LJ_PREC_FP64, LJ_PREC_FP32, LJ_PREC_MIXED = 0, 1, 2
LJ_POT_LJ, LJ_POT_MORSE = 0, 1
(LJ_CAND_CONVERGED, LJ_CAND_MAXITER, LJ_CAND_LINESEARCH_FAIL, LJ_CAND_NONFINITE,
 LJ_CAND_TIMEOUT, LJ_CAND_BAD_INPUT) = range(6)
LJ_MAX_ATOMS, LJ_MAX_M, LJ_MAX_K = 1024, 32, 16
LJ_OPT_BH_TEAM, LJ_OPT_LBFGS_TEAM, LJ_OPT_F32_HANDOVER, LJ_OPT_DF_HANDOVER = 1, 2, 3, 4
LJ_OPT_HISTORY, LJ_OPT_DF_EVAL = 5, 6
LJ_TUNE_BUCKETS = 6
LJ_TUNE_BH = LJ_TUNE_BUCKETS
STATS_FIELDS = ("evals32", "evals64", "evals_df", "iters32", "iters64", "pairs32", "pairs64",
                "pairs_df", "vec_elems32", "vec_elems64", "converged", "minimisations",
                "cycles32", "cycles_df", "cycles64", "cycles_direction", "cycles_linesearch")


class LjError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class _Batch(C.Structure):
    _fields_ = [("n_cand", C.c_int64), ("uniform_n", C.c_int32),
                ("d_atom_offset", C.c_void_p), ("max_n", C.c_int32)]


class _Lbfgs(C.Structure):
    _fields_ = [("m", C.c_int32), ("gtol", C.c_double), ("max_iter", C.c_int32),
                ("max_ls", C.c_int32), ("c1", C.c_double), ("c2", C.c_double),
                ("alpha_max", C.c_double), ("prec", C.c_int), ("switch_gtol", C.c_double),
                ("deadline_cycles", C.c_int64), ("eps", C.c_double), ("sigma", C.c_double),
                ("potential", C.c_int32), ("rho", C.c_double)]


class _Bh(C.Structure):
    _fields_ = [("K", C.c_int32), ("kT", C.c_double), ("target_rate", C.c_double),
                ("interval", C.c_int32), ("factor", C.c_double), ("seed", C.c_uint64),
                ("step0", C.c_int64), ("n_steps", C.c_int32), ("walker0", C.c_int64),
                ("min", _Lbfgs)]


class _Tuning(C.Structure):
    _fields_ = [("team", C.c_int32), ("switch_gtol", C.c_double),
                ("history_global", C.c_int32), ("df_one_sided", C.c_int32),
                ("tuned", C.c_int32)]


class _State(C.Structure):
    _fields_ = [("n_walkers", C.c_int32), ("n_atoms", C.c_int32), ("x_cur", C.c_void_p),
                ("e_cur", C.c_void_p), ("x_best", C.c_void_p), ("e_best", C.c_void_p),
                ("stepsize", C.c_void_p), ("win_accept", C.c_void_p), ("n_accept", C.c_void_p)]


class _Trace(C.Structure):
    _fields_ = [("trial_e", C.c_void_p), ("trial_status", C.c_void_p),
                ("trial_iters", C.c_void_p), ("best_trial_e", C.c_void_p),
                ("accepted", C.c_void_p), ("stepsize", C.c_void_p),
                ("near_tie", C.c_void_p)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Load liblj_bh.so; raises if it is missing (build it with build.build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                raise RuntimeError(
                    f"CUDA library {_build.LIB} is not built; run "
                    "`python -m paper_2510_25938_gb300.build` (needs nvcc)")
            lib = C.CDLL(_build.LIB)
            P = C.c_void_p
            lib.lj_status_string.argtypes = [C.c_int]
            lib.lj_status_string.restype = C.c_char_p
            lib.lj_ctx_create.argtypes = [C.POINTER(C.c_void_p), C.c_int]
            lib.lj_ctx_create.restype = C.c_int
            lib.lj_ctx_destroy.argtypes = [P]
            lib.lj_ctx_destroy.restype = C.c_int
            lib.lj_ctx_reserve.argtypes = [P, C.c_int64, C.c_int32, C.c_int32]
            lib.lj_ctx_reserve.restype = C.c_int
            lib.lj_ctx_set_option.argtypes = [P, C.c_int, C.c_int64]
            lib.lj_ctx_set_option.restype = C.c_int
            lib.lj_ctx_last_error.argtypes = [P]
            lib.lj_ctx_last_error.restype = C.c_char_p
            lib.lj_energy_grad_batched.argtypes = [P, C.POINTER(_Batch), C.c_int, C.c_int, P, P,
                                                   P, C.c_double, C.c_double, P]
            lib.lj_energy_grad_batched.restype = C.c_int
            lib.lj_energy_grad_batched_pot.argtypes = [P, C.POINTER(_Batch), C.c_int, C.c_int,
                                                       P, P, P, C.c_int32, C.c_double,
                                                       C.c_double, C.c_double, P]
            lib.lj_energy_grad_batched_pot.restype = C.c_int
            lib.lbfgs_minimize_batched.argtypes = [P, C.POINTER(_Batch), C.POINTER(_Lbfgs), P, P,
                                                   P, P, P, P, P]
            lib.lbfgs_minimize_batched.restype = C.c_int
            lib.bh_step_batched.argtypes = [P, C.POINTER(_State), C.POINTER(_Bh),
                                            C.POINTER(_Trace), P, P]
            lib.bh_step_batched.restype = C.c_int
            lib.lbfgs_minimize_batched_noalloc.argtypes = [C.POINTER(_Batch), C.POINTER(_Lbfgs),
                                                           P, P, P, P, P, P, P]
            lib.lbfgs_minimize_batched_noalloc.restype = C.c_int
            lib.lj_ctx_autotune.argtypes = [P, C.c_int32, C.c_int32, C.c_int,
                                            C.POINTER(C.c_int32), C.POINTER(C.c_double), P]
            lib.lj_ctx_autotune.restype = C.c_int
            lib.lj_ctx_autotune_batch.argtypes = [P, C.POINTER(_Batch), P, C.c_int32, C.c_int,
                                                  C.c_int64, C.POINTER(C.c_int32),
                                                  C.POINTER(C.c_double), P]
            lib.lj_ctx_autotune_batch.restype = C.c_int
            lib.lj_ctx_get_tuning.argtypes = [P, C.c_int32, C.POINTER(_Tuning)]
            lib.lj_ctx_get_tuning.restype = C.c_int
            lib.lj_ctx_autotune_bh.argtypes = [P, C.POINTER(_State), C.POINTER(_Bh),
                                               C.POINTER(_Tuning), P]
            lib.lj_ctx_autotune_bh.restype = C.c_int
            _lib = lib
    return _lib


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tensor must be on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _check(ctx, st: int, what: str):
    if st != LJ_OK:
        lib = load()
        name = lib.lj_status_string(st).decode()
        msg = lib.lj_ctx_last_error(ctx.handle).decode() if ctx is not None else ""
        raise LjError(st, f"{what}: {name}: {msg}")


class Ctx:
    """A library context (workspace owner) on one CUDA device."""

    def __init__(self, device: int | None = None):
        lib = load()
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        h = C.c_void_p()
        st = lib.lj_ctx_create(C.byref(h), self.device)
        if st != LJ_OK:
            raise LjError(st, "lj_ctx_create")
        self.handle = h

    def reserve(self, max_cand: int, max_n: int, max_m: int):
        _check(self, load().lj_ctx_reserve(self.handle, max_cand, max_n, max_m), "lj_ctx_reserve")

    def set_option(self, opt: int, value: int):
        """lj_ctx_set_option: e.g. set_option(LJ_OPT_BH_TEAM, 64)."""
        _check(self, load().lj_ctx_set_option(self.handle, opt, value), "lj_ctx_set_option")

    def autotune(self, max_n: int, m: int = 10, prec: int = 2, stream=None) -> dict:
        """lj_ctx_autotune: {"team": [...], "switch_gtol": [...]}, one entry per
        LJ_TUNE_BUCKETS size bucket (0 beyond max_n's bucket)."""
        team = (C.c_int32 * LJ_TUNE_BUCKETS)()
        sg = (C.c_double * LJ_TUNE_BUCKETS)()
        _check(self, load().lj_ctx_autotune(self.handle, max_n, m, prec, team, sg,
                                            _stream(stream)), "lj_ctx_autotune")
        return {"team": list(team), "switch_gtol": list(sg)}

    def autotune_batch(self, x: torch.Tensor, n_cand: int, uniform_n: int, m: int = 10,
                       prec: int = 2, max_sample: int = 1024, stream=None) -> dict:
        """lj_ctx_autotune_batch on the caller's own uniform batch x (float64,
        left unchanged): {"team": t, "switch_gtol": s} of the bucket of uniform_n."""
        if x.dtype != torch.float64:
            raise ValueError("x must be float64")
        team = C.c_int32()
        sg = C.c_double()
        b = _Batch(n_cand, uniform_n, None, uniform_n)
        _check(self, load().lj_ctx_autotune_batch(self.handle, C.byref(b), _ptr(x), m, prec,
                                                  max_sample, C.byref(team), C.byref(sg),
                                                  _stream(stream)), "lj_ctx_autotune_batch")
        return {"team": team.value, "switch_gtol": sg.value}

    def tuning(self, bucket: int) -> dict:
        """lj_ctx_get_tuning: the tuning entry of a size bucket (0..5) or of
        bh_step_batched (LJ_TUNE_BH)."""
        t = _Tuning()
        _check(self, load().lj_ctx_get_tuning(self.handle, bucket, C.byref(t)), "lj_ctx_get_tuning")
        return {k: getattr(t, k) for k, _ in _Tuning._fields_}

    def autotune_bh(self, state: dict, params: "BhParams", stream=None) -> dict:
        """lj_ctx_autotune_bh on copies of the walker state (left unchanged):
        team, switch_gtol and history placement for bh_step_batched."""
        for k, dt in STATE_KEYS:
            if state[k].dtype != dt:
                raise ValueError(f"state[{k}] must be {dt}")
        W, n3 = state["x_cur"].shape
        s = _State(W, n3 // 3, *(_ptr(state[k]) for k, _ in STATE_KEYS))
        t = _Tuning()
        p = params.c()
        _check(self, load().lj_ctx_autotune_bh(self.handle, C.byref(s), C.byref(p), C.byref(t),
                                               _stream(stream)), "lj_ctx_autotune_bh")
        return {k: getattr(t, k) for k, _ in _Tuning._fields_}

    def close(self):
        if getattr(self, "handle", None):
            load().lj_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class LbfgsParams:
    """Local-minimiser settings (field meaning in include/lj_bh.h)."""
    m: int = 10
    gtol: float = 1e-6
    max_iter: int = 15000
    max_ls: int = 20
    c1: float = 1e-3
    c2: float = 0.9
    alpha_max: float = 1e10
    prec: int = LJ_PREC_MIXED
    switch_gtol: float = 0.0       # 0: automatic (autotuned per bucket, else 1e-3)
    deadline_cycles: int = 0
    eps: float = 1.0
    sigma: float = 1.0             # Morse: re
    potential: int = LJ_POT_LJ     # or LJ_POT_MORSE
    rho: float = 6.0               # Morse range (unused for LJ)

    def c(self) -> _Lbfgs:
        return _Lbfgs(self.m, self.gtol, self.max_iter, self.max_ls, self.c1, self.c2,
                      self.alpha_max, self.prec, self.switch_gtol, self.deadline_cycles,
                      self.eps, self.sigma, self.potential, self.rho)


@dataclass
class BhParams:
    """Basin Hopping settings (field meaning in include/lj_bh.h)."""
    K: int = 8
    kT: float = 0.8
    target_rate: float = 0.5
    interval: int = 10
    factor: float = 0.9
    seed: int = 0
    step0: int = 0
    n_steps: int = 1
    walker0: int = 0
    min: LbfgsParams = field(default_factory=LbfgsParams)

    def c(self) -> _Bh:
        return _Bh(self.K, self.kT, self.target_rate, self.interval, self.factor, self.seed,
                   self.step0, self.n_steps, self.walker0, self.min.c())


def _batch(n_cand, uniform_n, atom_offset, max_n) -> _Batch:
    if uniform_n and uniform_n > 0:
        return _Batch(int(n_cand), int(uniform_n), None, int(uniform_n))
    if atom_offset is None:
        raise ValueError("uneven batches need atom_offset (int64 CUDA tensor, n_cand+1)")
    if atom_offset.dtype != torch.int64:
        raise ValueError("atom_offset must be int64")
    return _Batch(int(n_cand), 0, _ptr(atom_offset), int(max_n))


def new_stats(device=None) -> torch.Tensor:
    """Zeroed device lj_stats (10 x uint64, held in an int64 tensor)."""
    return torch.zeros(len(STATS_FIELDS), dtype=torch.int64, device=device or "cuda")


def stats_dict(stats: torch.Tensor) -> dict:
    return dict(zip(STATS_FIELDS, (int(v) for v in stats.cpu().tolist())))


def lj_energy_grad_batched(ctx: Ctx, x: torch.Tensor, energy: torch.Tensor,
                           grad: torch.Tensor | None = None, *, n_cand: int, uniform_n: int = 0,
                           atom_offset: torch.Tensor | None = None, max_n: int = 0,
                           prec: int = LJ_PREC_FP64, eps: float = 1.0, sigma: float = 1.0,
                           potential: int = LJ_POT_LJ, rho: float = 6.0, stream=None):
    """Energies (float64 [n_cand]) and gradients (x's dtype) of a batch: Eq. (1),
    or the Morse potential with potential=LJ_POT_MORSE (sigma = re, range rho)."""
    if x.dtype not in (torch.float32, torch.float64):
        raise ValueError("x must be float32 or float64")
    if energy.dtype != torch.float64:
        raise ValueError("energy must be float64")
    if grad is not None and grad.dtype != x.dtype:
        raise ValueError("grad must have x's dtype")
    xt = LJ_F32 if x.dtype == torch.float32 else LJ_F64
    b = _batch(n_cand, uniform_n, atom_offset, max_n)
    if potential == LJ_POT_LJ:
        st = load().lj_energy_grad_batched(ctx.handle, C.byref(b), prec, xt, _ptr(x),
                                           _ptr(energy), _ptr(grad), eps, sigma, _stream(stream))
    else:
        st = load().lj_energy_grad_batched_pot(ctx.handle, C.byref(b), prec, xt, _ptr(x),
                                               _ptr(energy), _ptr(grad), potential, eps, sigma,
                                               rho, _stream(stream))
    _check(ctx, st, "lj_energy_grad_batched")


def lbfgs_minimize_batched(ctx: Ctx, x: torch.Tensor, energy: torch.Tensor,
                           status: torch.Tensor | None = None, iters: torch.Tensor | None = None,
                           nevals: torch.Tensor | None = None, stats: torch.Tensor | None = None,
                           *, n_cand: int, uniform_n: int = 0,
                           atom_offset: torch.Tensor | None = None, max_n: int = 0,
                           params: LbfgsParams | None = None, stream=None):
    """Minimise every candidate of the batch in place (x float64)."""
    if x.dtype != torch.float64 or energy.dtype != torch.float64:
        raise ValueError("x and energy must be float64")
    for t in (status, iters, nevals):
        if t is not None and t.dtype != torch.int32:
            raise ValueError("status / iters / nevals must be int32")
    p = (params or LbfgsParams()).c()
    b = _batch(n_cand, uniform_n, atom_offset, max_n)
    st = load().lbfgs_minimize_batched(ctx.handle, C.byref(b), C.byref(p), _ptr(x), _ptr(energy),
                                       _ptr(status), _ptr(iters), _ptr(nevals), _ptr(stats),
                                       _stream(stream))
    _check(ctx, st, "lbfgs_minimize_batched")


def lbfgs_minimize_batched_noalloc(x: torch.Tensor, energy: torch.Tensor,
                                   status: torch.Tensor | None = None,
                                   iters: torch.Tensor | None = None,
                                   nevals: torch.Tensor | None = None,
                                   stats: torch.Tensor | None = None, *, n_cand: int,
                                   uniform_n: int = 0, atom_offset: torch.Tensor | None = None,
                                   max_n: int = 0, params: LbfgsParams | None = None,
                                   stream=None):
    """lbfgs_minimize_batched without a context and without any device
    allocation (scratch in a fixed library array; see include/lj_bh.h).
    Runs on the current CUDA device."""
    if x.dtype != torch.float64 or energy.dtype != torch.float64:
        raise ValueError("x and energy must be float64")
    p = (params or LbfgsParams()).c()
    b = _batch(n_cand, uniform_n, atom_offset, max_n)
    st = load().lbfgs_minimize_batched_noalloc(C.byref(b), C.byref(p), _ptr(x), _ptr(energy),
                                               _ptr(status), _ptr(iters), _ptr(nevals),
                                               _ptr(stats), _stream(stream))
    if st != LJ_OK:
        raise LjError(st, "lbfgs_minimize_batched_noalloc: "
                          + load().lj_status_string(st).decode())


STATE_KEYS = (("x_cur", torch.float64), ("e_cur", torch.float64), ("x_best", torch.float64),
              ("e_best", torch.float64), ("stepsize", torch.float64),
              ("win_accept", torch.int32), ("n_accept", torch.int32))
TRACE_KEYS = (("trial_e", torch.float64), ("trial_status", torch.int32),
              ("trial_iters", torch.int32), ("best_trial_e", torch.float64),
              ("accepted", torch.uint8), ("stepsize", torch.float64),
              ("near_tie", torch.uint8))
LJ_NEAR_TIE = 1e-9


def bh_step_batched(ctx: Ctx, state: dict, params: BhParams, trace: dict | None = None,
                    stats: torch.Tensor | None = None, stream=None):
    """params.n_steps Basin Hopping steps of every walker, state updated in place.

    state: x_cur / x_best (W, 3N) float64, e_cur / e_best / stepsize (W,) float64,
    win_accept / n_accept (W,) int32.  trace (optional): trial_e / trial_status /
    trial_iters (n_steps, W, K), best_trial_e / accepted / stepsize / near_tie
    (n_steps, W)."""
    for k, dt in STATE_KEYS:
        if state[k].dtype != dt:
            raise ValueError(f"state[{k}] must be {dt}")
    W, n3 = state["x_cur"].shape
    s = _State(W, n3 // 3, *(_ptr(state[k]) for k, _ in STATE_KEYS))
    tr = _Trace()
    if trace:
        for k, dt in TRACE_KEYS:
            if trace.get(k) is not None and trace[k].dtype != dt:
                raise ValueError(f"trace[{k}] must be {dt}")
        tr = _Trace(*(_ptr(trace.get(k)) for k, _ in TRACE_KEYS))
    p = params.c()
    st = load().bh_step_batched(ctx.handle, C.byref(s), C.byref(p), C.byref(tr), _ptr(stats),
                                _stream(stream))
    _check(ctx, st, "bh_step_batched")


def new_trace(n_steps: int, n_walkers: int, K: int, device=None) -> dict:
    dev = device or "cuda"
    return {"trial_e": torch.empty((n_steps, n_walkers, K), dtype=torch.float64, device=dev),
            "trial_status": torch.empty((n_steps, n_walkers, K), dtype=torch.int32, device=dev),
            "trial_iters": torch.empty((n_steps, n_walkers, K), dtype=torch.int32, device=dev),
            "best_trial_e": torch.empty((n_steps, n_walkers), dtype=torch.float64, device=dev),
            "accepted": torch.empty((n_steps, n_walkers), dtype=torch.uint8, device=dev),
            "stepsize": torch.empty((n_steps, n_walkers), dtype=torch.float64, device=dev),
            "near_tie": torch.empty((n_steps, n_walkers), dtype=torch.uint8, device=dev)}
