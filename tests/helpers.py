"""Test-side property checks (independent of both the oracle and the CUDA path).

* fingerprint: sorted pair distances of a cluster -- invariant under
  translation, rotation, reflection and permutation; two minima are the same
  basin when their fingerprints agree to 1e-3 sigma (max abs difference).
* numpy_energy_grad: vectorised Eq. (1) energy and gradient, used only to
  check properties of returned minima (||g||_inf, E(x) consistency).
* grad_scale: the no-cancellation gradient scale ||(sum_j |c_ij d_ij|)_i||_2,
  the denominator that keeps relative gradient errors meaningful near minima.
* record: keeps the achieved figures of a parity test (printed, and appended
  to the file LJ_PARITY_REPORT names, if any).
"""
import json
import os

import numpy as np

SAME_BASIN_TOL = 1e-3


RECORDS = []     # every record() of this session, printed in the terminal summary


def record(tag, **metrics):
    """Print the achieved parity figures of a test and, when the environment
    variable LJ_PARITY_REPORT names a file, append them to it as one JSON
    line, so that a run keeps the numbers its assertions were checked on.
    The session's figures are also printed at its end (tests/conftest.py),
    where a quiet run keeps them."""
    clean = {k: (float(v) if isinstance(v, (np.floating, np.integer)) else v)
             for k, v in metrics.items()}
    RECORDS.append({"test": tag, **clean})
    print(f"[parity] {tag}: " + ", ".join(f"{k}={v}" for k, v in clean.items()))
    path = os.environ.get("LJ_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"test": tag, **clean}) + "\n")


def fingerprint(x):
    p = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    d = np.sqrt(((p[:, None, :] - p[None, :, :]) ** 2).sum(-1))
    return np.sort(d[np.triu_indices(len(p), 1)])


def same_basin(xa, xb, tol=SAME_BASIN_TOL):
    fa, fb = fingerprint(xa), fingerprint(xb)
    return fa.shape == fb.shape and (fa.size == 0 or np.abs(fa - fb).max() <= tol)


def _pair_terms(x, eps=1.0, sigma=1.0):
    p = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    n = len(p)
    d = p[:, None, :] - p[None, :, :]
    r2 = (d ** 2).sum(-1)
    np.fill_diagonal(r2, np.inf)
    s6 = (sigma * sigma / r2) ** 3
    c = 24.0 * eps * (2 * s6 * s6 - s6) / r2
    return p, n, d, s6, c


def numpy_energy_grad(x, eps=1.0, sigma=1.0):
    p, n, d, s6, c = _pair_terms(x, eps, sigma)
    e = 2.0 * eps * (s6 * s6 - s6).sum()
    g = -(c[:, :, None] * d).sum(1)
    return float(e), g.reshape(-1)


def grad_scale(x, eps=1.0, sigma=1.0):
    p, n, d, s6, c = _pair_terms(x, eps, sigma)
    return float(np.linalg.norm((np.abs(c)[:, :, None] * np.abs(d)).sum(1)))


def energy_scale(x, eps=1.0, sigma=1.0):
    """No-cancellation scale of Eq. (1): 4 eps sum_{i<j} (s12 + s6), the bound
    that a sum of rounded pair terms has its error measured against."""
    p, n, d, s6, c = _pair_terms(x, eps, sigma)
    return float(2.0 * eps * (s6 * s6 + s6).sum())


def grad_scale_terms(x, eps=1.0, sigma=1.0):
    """Term-wise no-cancellation scale of the gradient: the norm of
    sum_j 24 eps (2 s12 + s6) / r^2 |x_i - x_j|, which stays away from zero
    where a pair sits at the minimum of its term (2 s12 = s6)."""
    p, n, d, s6, c = _pair_terms(x, eps, sigma)
    r2 = (d ** 2).sum(-1)
    np.fill_diagonal(r2, np.inf)
    cn = 24.0 * eps * (2 * s6 * s6 + s6) / r2
    return float(np.linalg.norm((cn[:, :, None] * np.abs(d)).sum(1)))


def morse_bounds(x, eps=1.0, re=1.0, rho=6.0, u=2.0 ** -24):
    """Error bounds of a Morse evaluation whose pair terms carry relative
    rounding u: per pair the exponent x = rho (1 - r/re) is off by about
    7 rho (r/re) u (r from r^2 and a reciprocal square root) plus |x| u, the
    FP32 exponential adds 2 + 1.2 |x| ulp (CUDA's __expf bound), and the
    products a few u more, so the pair energy e (e - 2) is off by at most
    amp u e (e + 2) with amp = 8 + 5 |x| + 14 rho r / re, and the pair vector
    e (e - 1) d / r alike.  Returns (energy bound, per-coordinate gradient
    bounds), each twice the sum of those terms (no cancellation assumed)."""
    p = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    d = p[:, None, :] - p[None, :, :]
    r = np.sqrt((d ** 2).sum(-1))
    iu = np.triu_indices(len(p), 1)
    off = ~np.eye(len(p), dtype=bool)
    xx = rho * (1.0 - r / re)
    ex = np.exp(np.where(off, xx, 0.0))
    amp = 8.0 + 5.0 * np.abs(xx) + 14.0 * rho * r / re
    e_bound = 2.0 * u * eps * (amp * ex * (ex + 2.0))[iu].sum()
    rs = np.where(off, r, 1.0)
    c = np.where(off, amp * (2.0 * eps * rho / re) * ex * (ex + 1.0) / rs, 0.0)
    g_bound = 2.0 * u * (c[:, :, None] * np.abs(d)).sum(1)
    return float(e_bound), g_bound.reshape(-1)
