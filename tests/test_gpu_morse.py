"""GPU parity of the Morse pair potential -- the pair-potential extension the
paper's Conclusions point to (V = eps e (e - 2), e = exp(rho (1 - r/re)), re in
the sigma slot) -- through the C ABI, against the oracle's Morse.

Tolerances: FP64 evaluations within 1e-10 relative in energy and gradient, as
for Eq. (1), or within the term-by-term rounding bound at FP64's unit where
that is larger (near-zero energies and gradient components near a minimum);
FP32 pair terms within the bounds of tests.helpers.morse_bounds (the rounding
of r, of the exponent and of CUDA's __expf, term by term, no cancellation);
minima reached in the same basin within 1e-10 relative (FP64) or 1e-6 absolute
(mixed); Basin Hopping trajectories compared step by step as for Eq. (1).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2510_25938_gb300 import inputs as I
from tests.helpers import morse_bounds, record, same_basin

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_REL = 1e-10
MIX_ABS_FINAL = 1e-6
GTOL = 1e-6
RHO = 6.0


@pytest.fixture(scope="module")
def lj():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_25938_gb300 import build
    build.build()
    from paper_2510_25938_gb300 import lj_bh
    return lj_bh


@pytest.fixture(scope="module")
def ctx(lj):
    c = lj.Ctx(0)
    yield c
    c.close()


def _cuda(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _gpu_eval(lj, ctx, x, off, prec, xdtype, eps=1.0, re=1.0, rho=RHO):
    n_cand = off.size - 1
    xd = _cuda(x, xdtype)
    e = torch.empty(n_cand, dtype=torch.float64, device="cuda")
    g = torch.empty_like(xd)
    lj.lj_energy_grad_batched(ctx, xd, e, g, n_cand=n_cand, atom_offset=_cuda(off, torch.int64),
                              max_n=int(np.diff(off).max()), prec=prec, eps=eps, sigma=re,
                              potential=lj.LJ_POT_MORSE, rho=rho)
    torch.cuda.synchronize()
    return e.cpu().numpy(), g.cpu().numpy().astype(np.float64)


def _eval_compare(lj, ctx, x, off, prec, xdtype, eps=1.0, re=1.0, rho=RHO):
    n_cand = off.size - 1
    # FP32 coordinates (given, or rounded by the FP32 path itself): the oracle
    # evaluates the same rounded coordinates, so that the bounds measure the
    # arithmetic and not the input rounding
    rounded = xdtype == torch.float32 or prec != lj.LJ_PREC_FP64
    xin = x.astype(np.float32).astype(np.float64) if rounded else x
    e_ref, g_ref = O.eval_batch(xin, n_cand, atom_off=off, eps=eps, sigma=re,
                                potential=O.OBJ_MORSE, rho=rho)
    e, g = _gpu_eval(lj, ctx, x if xdtype == torch.float64 else xin, off, prec, xdtype, eps, re,
                     rho)
    worst_e = worst_g = 0.0
    for c in range(n_cand):
        a0, a1 = 3 * off[c], 3 * off[c + 1]
        if a1 - a0 <= 3:
            assert e[c] == 0.0 and np.all(g[a0:a1] == 0)
            continue
        if prec == lj.LJ_PREC_FP64:
            # 1e-10 relative, or the rounding bound of the terms at FP64's unit
            eb, gb = morse_bounds(xin[a0:a1], eps, re, rho, u=2.0 ** -53)
            tol_e = max(FP64_REL * abs(e_ref[c]), eb)
            tol_g = np.maximum(FP64_REL * np.abs(g_ref[a0:a1]), gb) + 1e-300
        else:
            eb, gb = morse_bounds(xin[a0:a1], eps, re, rho)
            tol_e = eb
            tol_g = gb + 1e-300
        if xdtype == torch.float32:
            tol_g = tol_g + 2.0 ** -24 * np.abs(g_ref[a0:a1])    # gradient written in FP32
        de = abs(e[c] - e_ref[c])
        dg = np.abs(g[a0:a1] - g_ref[a0:a1])
        worst_e = max(worst_e, de / tol_e)
        worst_g = max(worst_g, float((dg / tol_g).max()))
        assert de <= tol_e, (c, a1 // 3 - a0 // 3, e[c], e_ref[c])
        assert np.all(dg <= tol_g), (c, int(np.argmax(dg / tol_g)))
    return worst_e, worst_g


RAGGED_SIZES = [0, 1, 2, 3, 13, 31, 32, 33, 38, 63, 64, 65, 100, 127, 128, 129, 150, 255, 256,
                257, 300, 511, 512, 513, 700]


@pytest.mark.parametrize("prec,xdt", [(0, torch.float64), (0, torch.float32), (1, torch.float32),
                                      (1, torch.float64)])
def test_morse_eval_ragged(lj, ctx, prec, xdt):
    x, off = I.uneven_cube_starts(RAGGED_SIZES, 0.3, 31 + prec)
    we, wg = _eval_compare(lj, ctx, x, off, prec, xdt)
    record(f"morse_eval_ragged_p{prec}_{str(xdt)[-7:]}", worst_E_over_tol=we, worst_g_over_tol=wg)


def _oracle_minima(n_cand, n, side, seed, rho=RHO):
    x0 = I.cube_starts(n_cand, n, side, seed)
    xm, em, st, _, _ = O.lbfgs_batch(x0, n_cand, uniform_n=n, potential=O.OBJ_MORSE, rho=rho)
    return x0, xm.reshape(n_cand, -1), em, st


@pytest.mark.parametrize("prec", [0, 1])
def test_morse_eval_jittered_minima_uniform(lj, ctx, prec):
    """256 clusters of 38 atoms near Morse minima (the regime a minimiser's
    evaluations live in), several tiles of teams and a ragged last CTA."""
    n, nc = 38, 257
    _, xm, _, _ = _oracle_minima(nc, n, 3.2, 2101)
    x = I.jitter(xm, 1e-3, 7).reshape(-1)
    off = np.arange(nc + 1) * n
    xdt = torch.float64 if prec == 0 else torch.float32
    we, wg = _eval_compare(lj, ctx, x, off, prec, xdt)
    record(f"morse_eval_minima_p{prec}", worst_E_over_tol=we, worst_g_over_tol=wg)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("eps,re,rho", [(0.7, 1.3, 10.0), (2.0, 0.9, 3.0), (1.0, 1.0, 14.0)])
def test_morse_eval_parameters(lj, ctx, prec, eps, re, rho):
    x, off = I.uneven_cube_starts([5, 13, 38, 80], 0.3, 41)
    x = x * re
    _eval_compare(lj, ctx, x, off, prec, torch.float64, eps, re, rho)


def test_morse_eval_degenerate(lj, ctx):
    # coincident atoms: non-finite energy, as for Eq. (1); one atom: zero
    x = np.array([[0, 0, 0], [1, 0, 0], [1, 0, 0], [3, 0, 0], [0, 0, 0.]]).reshape(-1)
    off = np.array([0, 3, 4, 5])
    for prec in (0, 1):
        e, g = _gpu_eval(lj, ctx, x, off, prec, torch.float64)
        assert not np.isfinite(e[0])
        assert e[1] == 0.0 and e[2] == 0.0 and np.all(g[9:] == 0.0)


def test_morse_invalid_arguments(lj, ctx):
    x = _cuda(np.zeros(6))
    e = torch.empty(1, dtype=torch.float64, device="cuda")
    for pot, rho in ((lj.LJ_POT_MORSE, 0.0), (lj.LJ_POT_MORSE, -1.0), (lj.LJ_POT_MORSE, math.inf),
                     (lj.LJ_POT_MORSE, 65.0),
                     (7, 6.0)):
        with pytest.raises(lj.LjError) as ei:
            lj.lj_energy_grad_batched(ctx, x, e, n_cand=1, uniform_n=2, potential=pot, rho=rho)
        assert ei.value.status == lj.LJ_ERR_INVALID_ARG
    with pytest.raises(lj.LjError):
        lj.lbfgs_minimize_batched(ctx, x, e, n_cand=1, uniform_n=2,
                                  params=lj.LbfgsParams(potential=lj.LJ_POT_MORSE, rho=0.0))


def _minimise(lj, ctx, x0, n, prec, rho=RHO):
    nc = x0.shape[0]
    xd = _cuda(x0.reshape(-1))
    e = torch.empty(nc, dtype=torch.float64, device="cuda")
    st = torch.empty(nc, dtype=torch.int32, device="cuda")
    lj.lbfgs_minimize_batched(ctx, xd, e, st, n_cand=nc, uniform_n=n,
                              params=lj.LbfgsParams(prec=prec, potential=lj.LJ_POT_MORSE, rho=rho))
    torch.cuda.synchronize()
    return xd.cpu().numpy().reshape(nc, -1), e.cpu().numpy(), st.cpu().numpy()


# floors just under the measured same-basin fractions
SAME_FLOOR = {(13, 0): 0.9, (38, 0): 0.8, (13, 2): 0.2, (38, 2): 0.0}


@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("n,side", [(13, 2.0), (38, 3.2)])
def test_morse_minimise_cube_starts(lj, ctx, prec, n, side):
    nc = 48
    x0, xo, eo, so = _oracle_minima(nc, n, side, 2200 + n)
    xg, eg, sg = _minimise(lj, ctx, x0, n, prec)
    n_same = n_both = 0
    max_de = 0.0
    for c in range(nc):
        e_chk, g_chk = O.morse_energy_grad(xg[c], 1.0, 1.0, RHO)
        assert abs(e_chk - eg[c]) <= 1e-9 * max(1.0, abs(eg[c])), c
        assert eg[c] <= O.morse_energy_grad(x0[c], 1.0, 1.0, RHO)[0] + 1e-12, c   # descent
        if sg[c] == O.CONVERGED:
            assert np.abs(g_chk).max() < GTOL * 1.01, c
        if sg[c] == O.CONVERGED and so[c] == O.CONVERGED:
            n_both += 1
            if same_basin(xg[c], xo[c]):
                n_same += 1
                de = abs(eg[c] - eo[c])
                max_de = max(max_de, de)
                tol = FP64_REL * abs(eo[c]) if prec == 0 else MIX_ABS_FINAL
                assert de <= tol, (c, eg[c], eo[c])
    conv = float((sg == O.CONVERGED).mean())
    frac = n_same / max(n_both, 1)
    record(f"morse_minimise_n{n}_p{prec}", same_basin_fraction=frac, both=n_both,
           max_abs_dE_same_basin=max_de, gpu_converged_fraction=conv,
           floor=SAME_FLOOR[(n, prec)])
    assert conv >= 0.95
    assert frac >= SAME_FLOOR[(n, prec)]


def _bh_start(W, n, side, seed, rho=RHO):
    _, xm, em, st = _oracle_minima(W, n, side, seed, rho)
    assert np.all(st == O.CONVERGED)
    return {"x_cur": xm.copy(), "e_cur": em.copy(), "x_best": xm.copy(), "e_best": em.copy(),
            "stepsize": np.full(W, 0.4), "win_accept": np.zeros(W, np.int32),
            "n_accept": np.zeros(W, np.int32)}


@pytest.mark.parametrize("prec,n,K,steps,floor", [(0, 13, 1, 30, 0.7), (2, 13, 1, 30, 0.2),
                                                  (0, 38, 8, 4, 0.5), (2, 38, 8, 4, 0.0)])
def test_morse_bh_matches_oracle(lj, ctx, prec, n, K, steps, floor):
    W, seed = 4, 2300 + n
    st = _bh_start(W, n, 2.0 if n == 13 else 3.2, seed)
    st0 = {k: v.copy() for k, v in st.items()}
    gs = {k: _cuda(st[k], dt) for k, dt in lj.STATE_KEYS}
    p = lj.BhParams(K=K, kT=0.8, seed=seed, n_steps=steps,
                    min=lj.LbfgsParams(prec=prec, potential=lj.LJ_POT_MORSE, rho=RHO))
    tr = lj.new_trace(steps, W, K)
    lj.bh_step_batched(ctx, gs, p, tr)
    torch.cuda.synchronize()
    trg = {k: v.cpu().numpy() for k, v in tr.items()}
    tro = O.bh_run(st, O.BhParamsPy(K=K, kT=0.8, seed=seed, n_steps=steps,
                                   potential=O.OBJ_MORSE, rho=RHO))
    strict = total = 0
    for w in range(W):
        for s in range(steps):
            total += 1
            eg, eo = trg["trial_e"][s, w], tro["trial_e"][s, w]
            tol = FP64_REL * np.abs(eo) if prec == 0 else MIX_ABS_FINAL
            if not np.all(np.abs(eg - eo) <= tol):
                break
            if trg["accepted"][s, w] != tro["accepted"][s, w]:
                assert trg["near_tie"][s, w] == 1, (w, s)
                break
            assert trg["stepsize"][s, w] == tro["stepsize"][s, w]
            strict += 1
        # the GPU trace is self-consistent: selection, Metropolis, adaptation
        e_cur, step, win = st0["e_cur"][w], st0["stepsize"][w], 0
        for s in range(steps):
            assert trg["stepsize"][s, w] == step
            te = trg["trial_e"][s, w]
            k = int(np.argmin(te))
            u = O.stream_uniform(seed, 2, 0, 0, s, w)
            de = te[k] - e_cur
            acc = de <= 0 or u < math.exp(-de / 0.8)
            assert bool(trg["accepted"][s, w]) == acc
            if acc:
                e_cur, win = te[k], win + 1
            if (s + 1) % 10 == 0:
                step = step / 0.9 if win / 10 > 0.5 else step * 0.9
                win = 0
        assert gs["e_cur"][w].item() == e_cur
        # the walker's best is a Morse minimum with that energy
        xb = gs["x_best"][w].cpu().numpy()
        eb, gb = O.morse_energy_grad(xb, 1.0, 1.0, RHO)
        assert abs(eb - gs["e_best"][w].item()) <= 1e-9 * abs(eb)
    frac = strict / total
    record(f"morse_bh_n{n}_k{K}_p{prec}", steps_matching=strict, steps=total, fraction=frac,
           floor=floor)
    assert frac >= floor


@pytest.mark.parametrize("prec", [0, 2])
def test_morse_minimise_uneven_batch(lj, ctx, prec):
    """An uneven Morse batch across the size buckets (one-sided rows, half-pair
    FP64 up to 64 atoms, the 257..300-atom teams above): every GPU minimum is a
    Morse minimum (FP64 gradient below gtol where converged, its energy), and
    candidates both sides minimise into the same basin agree in energy."""
    sizes = [5, 13, 31, 33, 38, 64, 65, 100, 150, 257, 300]
    x0, off = I.uneven_cube_starts(sizes, 0.3, 2400 + prec)
    n_cand = off.size - 1
    xd = _cuda(x0)
    e = torch.empty(n_cand, dtype=torch.float64, device="cuda")
    st = torch.empty(n_cand, dtype=torch.int32, device="cuda")
    lj.lbfgs_minimize_batched(ctx, xd, e, st, n_cand=n_cand, atom_offset=_cuda(off, torch.int64),
                              max_n=max(sizes),
                              params=lj.LbfgsParams(prec=prec, potential=lj.LJ_POT_MORSE, rho=RHO))
    torch.cuda.synchronize()
    xg, eg, sg = xd.cpu().numpy(), e.cpu().numpy(), st.cpu().numpy()
    xo, eo, so, _, _ = O.lbfgs_batch(x0, n_cand, atom_off=off, potential=O.OBJ_MORSE, rho=RHO)
    same = 0
    for c in range(n_cand):
        a0, a1 = 3 * off[c], 3 * off[c + 1]
        e_chk, g_chk = O.morse_energy_grad(xg[a0:a1], 1.0, 1.0, RHO)
        assert abs(e_chk - eg[c]) <= 1e-9 * max(1.0, abs(eg[c])), c
        if sg[c] == O.CONVERGED:
            assert np.abs(g_chk).max() < GTOL * 1.01, c
        if sg[c] == O.CONVERGED and so[c] == O.CONVERGED and same_basin(xg[a0:a1], xo[a0:a1]):
            same += 1
            tol = FP64_REL * abs(eo[c]) if prec == 0 else MIX_ABS_FINAL
            assert abs(eg[c] - eo[c]) <= tol, (c, eg[c], eo[c])
    record(f"morse_minimise_uneven_p{prec}", same_basin=same, candidates=n_cand,
           gpu_converged=int((sg == O.CONVERGED).sum()))
    assert (sg == O.CONVERGED).mean() >= 0.9


@pytest.mark.parametrize("prec", [0, 2])
def test_morse_minimise_eps_re(lj, ctx, prec):
    """Morse with eps = 0.7, re = 1.3, rho = 10: every GPU minimum is a
    minimum of that potential, same-basin energies agree with the oracle's,
    and the mixed path's polish stays in double-float (about one FP64
    evaluation per minimisation)."""
    n, nc, rho = 13, 24, 10.0
    x0 = I.cube_starts(nc, n, 2.0 * 1.3, 2500)
    xo, eo, so, _, _ = O.lbfgs_batch(x0, nc, uniform_n=n, eps=0.7, sigma=1.3,
                                     potential=O.OBJ_MORSE, rho=rho)
    xo = xo.reshape(nc, -1)
    xd = _cuda(x0.reshape(-1))
    e = torch.empty(nc, dtype=torch.float64, device="cuda")
    st = torch.empty(nc, dtype=torch.int32, device="cuda")
    stats = lj.new_stats()
    lj.lbfgs_minimize_batched(ctx, xd, e, st, None, None, stats, n_cand=nc, uniform_n=n,
                              params=lj.LbfgsParams(prec=prec, eps=0.7, sigma=1.3,
                                                    potential=lj.LJ_POT_MORSE, rho=rho))
    torch.cuda.synchronize()
    xg, eg, sg = xd.cpu().numpy().reshape(nc, -1), e.cpu().numpy(), st.cpu().numpy()
    same = 0
    for c in range(nc):
        e_chk, g_chk = O.morse_energy_grad(xg[c], 0.7, 1.3, rho)
        assert abs(e_chk - eg[c]) <= 1e-9 * max(1.0, abs(eg[c])), c
        if sg[c] == O.CONVERGED:
            assert np.abs(g_chk).max() < GTOL * 1.01, c
        if sg[c] == O.CONVERGED and so[c] == O.CONVERGED and same_basin(xg[c], xo[c]):
            same += 1
            tol = FP64_REL * abs(eo[c]) if prec == 0 else MIX_ABS_FINAL
            assert abs(eg[c] - eo[c]) <= tol, (c, eg[c], eo[c])
    sd = lj.stats_dict(stats)
    record(f"morse_minimise_eps_re_p{prec}", same_basin=same, candidates=nc,
           gpu_converged=int((sg == O.CONVERGED).sum()),
           fp64_evals_per_minimisation=sd["evals64"] / nc)
    assert (sg == O.CONVERGED).mean() >= 0.95
    if prec == 2:
        assert sd["evals64"] / nc < 3.0     # the FP64 path: ~100 per minimisation
