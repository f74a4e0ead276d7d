"""Pins of the oracle's line search (strong Wolfe; Nocedal & Wright,
Numerical Optimization, Alg. 3.5 bracketing + Alg. 3.6 zoom, with the
readings the oracle states: c1 = 1e-3, c2 = 0.9, doubling up to alpha_max,
cubic interpolation kept 10% inside the bracket, a non-finite trial counted
as failing sufficient decrease, and after an exhausted budget the best
sufficient-decrease point taken only if it strictly lowers f).

The paper runs scipy's L-BFGS-B and does not describe its line search, so
these pins come from the algorithm's own definition, not from the paper:

* one-dimensional lines whose correct trial sequence is derived by hand
  below (doubling, zoom exact on a quadratic, strong against weak curvature,
  alpha_max, non-finite trials, the exhausted-budget rules);
* zoom's invariants (N&W Sect. 3.5: the bracket [lo, hi] always holds the
  lowest sufficient-decrease point as lo, and hi lies on the side of lo that
  phi'(lo) descends toward, so every new trial falls strictly between them),
  checked on every trial of random quartic, Rosenbrock and LJ lines;
* both strong-Wolfe conditions on every step an LJ minimisation accepts.

A weak-Wolfe curvature test, a bracketing step that does not double, a wrong
swap rule in zoom, or a fallback that accepts f == f0 each fails one of them.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2510_25938_gb300 import inputs

C1, C2 = 1e-3, 0.9


def quad(lam, b):
    """phi(alpha) = lam/2 alpha^2 - b alpha along x = alpha (d = 1): minimiser
    alpha* = b / lam, phi'(0) = -b."""
    return [0.0, -b, lam / 2.0, 0.0, 0.0]


def search(coef, alpha1, bound=None, **kw):
    return O.line_search([0.0], [1.0], alpha1, kind=O.OBJ_POLY1D, b=coef,
                         A=None if bound is None else [bound], params=O.MinParams(**kw))


# ---------------------------------------------------------------------------
# hand-derived trial sequences
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("lam,b", [(2.0, 3.0), (0.37, 5.5), (40.0, 0.01)])
def test_bracketing_doubles_until_strong_curvature_holds(lam, b):
    # alpha1 = alpha*/100: phi'(alpha) = lam alpha - b < 0 with sufficient
    # decrease all the way, so Alg. 3.5 doubles alpha until
    # |phi'(alpha)| <= c2 b, i.e. the first k with lam alpha1 2^k >= (1 - c2) b
    astar = b / lam
    a1 = astar / 100.0
    k = math.ceil(math.log2((1.0 - C2) * b / (lam * a1)))
    r = search(quad(lam, b), a1)
    assert r["ok"] and r["exit"] == O.LS_WOLFE
    expect = [a1 * 2.0 ** i for i in range(k + 1)]
    assert r["trials"][:, 0].tolist() == expect          # exact: doubling is exact
    assert r["alpha"] == expect[-1]


@pytest.mark.parametrize("lam,b", [(2.0, 3.0), (0.37, 5.5)])
def test_overshoot_with_sufficient_decrease_is_strong_not_weak(lam, b):
    # alpha1 = 1.95 alpha*: sufficient decrease holds (it does up to
    # 2(1 - c1) alpha*), phi'(alpha1) = 0.95 b > 0: a weak-Wolfe test
    # (phi' >= c2 phi'(0)) would accept alpha1; the strong test rejects it,
    # phi' >= 0 turns the bracket to zoom(alpha1, 0), and the cubic
    # interpolant of a quadratic is the quadratic: one trial lands on alpha*
    astar = b / lam
    r = search(quad(lam, b), 1.95 * astar)
    assert r["ok"] and r["exit"] == O.LS_WOLFE
    assert r["trials"].shape[0] == 2
    assert r["trials"][0, 0] == 1.95 * astar
    assert abs(r["alpha"] - astar) <= 1e-14 * astar


@pytest.mark.parametrize("ratio", [2.5, 3.0, 8.0])
def test_overshoot_without_sufficient_decrease_zooms_from_zero(ratio):
    # alpha1 beyond 2(1 - c1) alpha*: no sufficient decrease, so zoom(0,
    # alpha1); the interpolant is exact, its minimiser alpha* lies inside
    # [0.1 w, 0.9 w] for these ratios, and phi'(alpha*) = 0 ends the search
    lam, b = 2.0, 3.0
    astar = b / lam
    r = search(quad(lam, b), ratio * astar)
    assert r["ok"] and r["exit"] == O.LS_WOLFE
    assert r["trials"].shape[0] == 2
    assert abs(r["alpha"] - astar) <= 1e-14 * astar


def test_safeguard_keeps_trial_ten_percent_inside_the_bracket():
    # alpha1 = 12 alpha*: the exact minimiser sits at 1/12 of the bracket
    # [0, alpha1], below 0.1 w, so the first zoom trial is clamped to
    # 0.1 alpha1 exactly
    lam, b = 2.0, 3.0
    astar = b / lam
    a1 = 12.0 * astar
    r = search(quad(lam, b), a1)
    assert r["trials"][1, 0] == pytest.approx(0.1 * a1, rel=1e-15)


def test_alpha_max_caps_the_bracketing_steps():
    lam, b = 2.0, 3.0
    a1 = (b / lam) / 100.0
    r = search(quad(lam, b), a1, alpha_max=3.0 * a1)
    t = r["trials"][:, 0]
    assert t[:3].tolist() == [a1, 2 * a1, 3 * a1]
    assert t.max() <= 3 * a1
    # the cap stops progress before the curvature condition can hold: the
    # budget runs out and the best sufficient-decrease point (alpha_max) is
    # taken because it lowers f
    assert r["ok"] and r["exit"] == O.LS_FALLBACK and r["alpha"] == 3 * a1


def test_non_finite_trials_count_as_too_long():
    # phi is +inf beyond 1.5, alpha* = 1: alpha1 = 8 fails, zoom(0, 8) has a
    # non-finite end so the trial is the midpoint: 4, 2 (both +inf), then 1 =
    # alpha*, where phi' = 0
    lam, b = 2.0, 2.0
    r = search(quad(lam, b), 8.0, bound=1.5)
    assert r["trials"][:, 0].tolist() == [8.0, 4.0, 2.0, 1.0]
    assert r["ok"] and r["exit"] == O.LS_WOLFE and r["alpha"] == 1.0


def test_exhausted_budget_takes_the_sufficient_decrease_point():
    lam, b = 2.0, 3.0
    a1 = (b / lam) / 100.0
    r = search(quad(lam, b), a1, max_ls=1)
    assert r["ok"] and r["exit"] == O.LS_FALLBACK and r["alpha"] == a1
    assert r["f"] < r["f0"]
    r = search(quad(lam, b), a1, max_ls=3)
    assert r["ok"] and r["exit"] == O.LS_FALLBACK and r["alpha"] == 4 * a1


def test_exhausted_budget_rejects_a_point_that_only_ties_f0():
    # phi = 1e16 - 1e-3 alpha: every trial rounds to f0 = 1e16, so the
    # sufficient-decrease inequality f <= f0 + c1 alpha phi'(0) holds only
    # because its right side rounds to f0 too.  Such a point makes no
    # progress; the search must fail instead of accepting it.
    r = search([1e16, -1e-3, 0.0, 0.0, 0.0], 1.0)
    assert not r["ok"] and r["exit"] == O.LS_FAILED


# ---------------------------------------------------------------------------
# zoom invariants on every trial of generic lines
# ---------------------------------------------------------------------------
def check_trace(r, alpha1, alpha_max=1e10, max_ls=20, c1=C1, c2=C2):
    """Check one line-search record against Alg. 3.5/3.6's invariants."""
    f0, dp0 = r["f0"], r["dphi0"]
    tr = r["trials"]
    assert dp0 < 0.0
    n = tr.shape[0]
    assert n >= 1
    n_search = min(n, max_ls)              # a final re-evaluation may follow

    def armijo(a, f):
        return np.isfinite(f) and f <= f0 + c1 * a * dp0

    def strong(dp):
        return abs(dp) <= -c2 * dp0

    # bracketing phase: trial i+1 = min(2 alpha_i, alpha_max) while trial i
    # has sufficient decrease, is lower than its predecessor, descends and
    # misses the curvature condition
    assert tr[0, 0] == alpha1
    i = 0
    while i + 1 < n_search:
        a, f, dp = tr[i]
        lower = i == 0 or f < tr[i - 1, 1]
        if armijo(a, f) and lower and dp < 0.0 and not strong(dp):
            assert tr[i + 1, 0] == min(2.0 * a, alpha_max)
            i += 1
        else:
            break
    first_zoom = i + 1
    # zoom phase: each trial lies in [lo + 0.1 w, hi - 0.1 w], lo the lowest
    # sufficient-decrease point so far (alpha = 0 counts; ties keep the
    # earlier), hi the nearest earlier point on the side phi'(lo) descends to
    pts = [(0.0, f0, dp0, True)] + [(a, f, dp, armijo(a, f)) for a, f, dp in tr[:first_zoom]]
    for j in range(first_zoom, n_search):
        best = None
        for p in pts:
            if p[3] and (best is None or p[1] < best[1]):
                best = p
        lo, dlo = best[0], best[2]
        assert dlo != 0.0
        if dlo < 0.0:
            hi = min(p[0] for p in pts if p[0] > lo)
        else:
            hi = max(p[0] for p in pts if p[0] < lo)
        w = abs(hi - lo)
        a_lo, a_hi = min(lo, hi) + 0.1 * w, max(lo, hi) - 0.1 * w
        slack = 4 * np.spacing(max(abs(lo), abs(hi)))
        assert a_lo - slack <= tr[j, 0] <= a_hi + slack, (j, tr[j, 0], lo, hi)
        a, f, dp = tr[j]
        pts.append((a, f, dp, armijo(a, f)))
    # how the search ended
    if r["exit"] == O.LS_WOLFE:
        a, f, dp = tr[n - 1]
        assert n <= max_ls and r["alpha"] == a and r["f"] == f
        assert armijo(a, f) and strong(dp)
        # the accepted trial is a new lowest point: strictly below phi(0) and
        # below every earlier sufficient-decrease trial (Alg. 3.5 stops on
        # phi(alpha_i) >= phi(alpha_{i-1}), Alg. 3.6 on phi(alpha_j) >= phi(lo))
        assert f < f0 and all(f < fp for ap, fp, _ in tr[:n - 1] if armijo(ap, fp))
    else:
        assert n_search == max_ls
        ok = [(f, a) for a, f, dp in tr[:n_search] if armijo(a, f)]
        if r["exit"] == O.LS_FALLBACK:
            fb, ab = min(ok)
            assert r["alpha"] == ab and fb < f0 and r["f"] == fb
        else:
            assert not ok or min(ok)[0] >= f0
            assert not r["ok"]


def random_quartic(rng):
    c4 = 10.0 ** rng.uniform(-2, 1)
    c3 = rng.normal() * c4 * 3
    c2 = rng.normal() * 4
    c1 = -(10.0 ** rng.uniform(-2, 1))
    return [rng.normal(), c1, c2, c3, c4]


@pytest.mark.parametrize("c1,c2", [(1e-3, 0.9), (0.3, 0.4), (0.45, 0.5), (1e-4, 0.1)])
def test_zoom_invariants_on_random_quartic_lines(c1, c2):
    # other (c1, c2) pairs than the minimiser's widen the band between
    # "lower than phi(0)" and "sufficient decrease" and tighten the
    # curvature test, so that zoom loops run long and visit every branch
    rng = np.random.default_rng(2510)
    counts = {O.LS_WOLFE: 0, O.LS_FALLBACK: 0, O.LS_FAILED: 0}
    n_zoom = 0
    for t in range(400):
        coef = random_quartic(rng)
        a1 = 10.0 ** rng.uniform(-3, 2)
        max_ls = int(rng.choice([2, 3, 5, 20]))
        r = search(coef, a1, max_ls=max_ls, c1=c1, c2=c2)
        check_trace(r, a1, max_ls=max_ls, c1=c1, c2=c2)
        counts[r["exit"]] += 1
        n_zoom += r["trials"].shape[0] > 2
    # the lines exercise every way out, and zoom loops of several trials
    assert counts[O.LS_WOLFE] > 100 and counts[O.LS_FALLBACK] > 10
    assert n_zoom > 50


def test_zoom_invariants_on_rosenbrock_lines():
    rng = np.random.default_rng(7)
    for t in range(100):
        x = rng.uniform(-2, 2, size=6)
        _, f, _, _, _ = O.minimize(x, kind=O.OBJ_ROSENBROCK, params=O.MinParams(max_iter=0))
        g = rosen_grad(x)
        d = -g + 0.3 * rng.normal(size=6) * np.abs(g)
        if d @ g >= 0:
            d = -g
        a1 = min(1.0, 1.0 / np.linalg.norm(d)) * 10.0 ** rng.uniform(-1, 1)
        r = O.line_search(x, d, a1, kind=O.OBJ_ROSENBROCK)
        check_trace(r, a1)


def rosen_grad(x):
    g = np.zeros_like(x)
    for i in range(0, x.size - 1, 2):
        a, b = x[i], x[i + 1]
        g[i] = -400 * a * (b - a * a) - 2 * (1 - a)
        g[i + 1] = 200 * (b - a * a)
    return g


@pytest.mark.parametrize("n_atoms", [13, 38])
def test_zoom_invariants_on_lj_lines(n_atoms):
    rng = np.random.default_rng(n_atoms)
    x0 = inputs.cube_starts(20, n_atoms, 3.2 if n_atoms == 38 else 2.0, 99)
    for c in range(20):
        # a line from a partly minimised structure (so that the gradient is
        # moderate), along -g with some noise, first trial min(1, 1/||d||)
        x, _, _, _, _ = O.minimize(x0[c], params=O.MinParams(max_iter=int(rng.integers(3, 40))))
        e, g = O.lj_energy_grad(x)
        d = -g * (1.0 + 0.2 * rng.normal(size=g.size))
        a1 = min(1.0, 1.0 / np.linalg.norm(d)) * 10.0 ** rng.uniform(-0.5, 1.5)
        r = O.line_search(x, d, a1, kind=O.OBJ_LJ)
        check_trace(r, a1)


# ---------------------------------------------------------------------------
# every accepted step of an LJ minimisation satisfies strong Wolfe
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n_atoms,side", [(13, 2.0), (38, 3.2)])
def test_minimisation_steps_satisfy_strong_wolfe(n_atoms, side):
    x0 = inputs.cube_starts(6, n_atoms, side, 1234)
    n_wolfe = n_all = 0
    for c in range(6):
        x, f, st, it, ne, rec = O.minimize_log(x0[c])
        assert st == O.CONVERGED and len(rec) == it
        for r in rec:
            n_all += 1
            armijo = r["f"] <= r["f0"] + C1 * r["alpha"] * r["dphi0"]
            assert r["dphi0"] < 0.0 and armijo, r
            if r["exit"] == O.LS_WOLFE:
                n_wolfe += 1
                assert abs(r["dphi"]) <= -C2 * r["dphi0"], r
            else:
                assert r["exit"] == O.LS_FALLBACK and r["f"] < r["f0"], r
        # the returned energy is the energy of the returned structure
        assert f == pytest.approx(O.lj_energy_grad(x)[0], rel=0, abs=1e-12)
    assert n_wolfe >= 0.9 * n_all
