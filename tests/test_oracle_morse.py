"""Pins of the oracle's Morse pair potential (the pair-potential extension the
paper's Conclusions point to; Morse 1929 in the cluster form
V(r) = eps e^{rho(1 - r/re)} (e^{rho(1 - r/re)} - 2)).

Each check rests on a fact of the potential or of the geometry, not on the
formula retyped: the well depth -eps at re with zero force, the zero crossing
at re (1 - ln 2 / rho), the harmonic force constant 2 eps rho^2 / re^2 of a
Morse oscillator, the long-range limit, small clusters whose pairs all sit at
re, the octahedron's and icosahedron's distance multisets, the icosahedral
breathing minimum found by a one-dimensional search, central finite
differences, invariances, and the eps / re scaling law.
"""
import math

import numpy as np
import pytest

import oracle as O

RHOS = [3.0, 6.0, 10.0, 14.0]


def dimer(r):
    return np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])


@pytest.mark.parametrize("rho", RHOS)
@pytest.mark.parametrize("eps,re", [(1.0, 1.0), (0.7, 1.3), (2.5, 0.8)])
def test_dimer_well_depth_zero_crossing_and_force_constant(rho, eps, re):
    # depth -eps at re, no force there
    e, g = O.morse_energy_grad(dimer(re), eps, re, rho)
    assert e == pytest.approx(-eps, rel=1e-15)
    assert np.abs(g).max() < 1e-13 * eps / re
    # V = 0 where e^{rho(1 - r/re)} = 2; there dV/dr = -(2 eps rho/re) * 2 * 1
    r0 = re * (1.0 - math.log(2.0) / rho)
    e0, g0 = O.morse_energy_grad(dimer(r0), eps, re, rho)
    assert abs(e0) < 1e-14 * eps
    # dE/dx_1 = dV/dr (atom 1 sits at +r on the x axis); atom 0 gets the opposite
    assert g0[3] == pytest.approx(-4.0 * eps * rho / re, rel=1e-13)
    assert g0[0] == pytest.approx(4.0 * eps * rho / re, rel=1e-13)
    # harmonic constant of the well: V''(re) = 2 eps rho^2 / re^2
    h = 1e-5 * re
    gp = O.morse_energy_grad(dimer(re + h), eps, re, rho)[1][3]
    gm = O.morse_energy_grad(dimer(re - h), eps, re, rho)[1][3]
    k = (gp - gm) / (2 * h)
    assert k == pytest.approx(2 * eps * rho * rho / (re * re), rel=1e-6)
    # long range: the well is gone
    e_far, g_far = O.morse_energy_grad(dimer(60.0 * re), eps, re, rho)
    assert e_far <= 0.0 and abs(e_far) < 1e-60
    assert np.abs(g_far).max() < 1e-60


def test_dimer_energy_is_monotone_on_each_side_of_the_well():
    rs = np.linspace(0.5, 3.0, 401)
    es = np.array([O.morse_energy_grad(dimer(r), 1.0, 1.0, 6.0)[0] for r in rs])
    left = rs < 1.0
    assert np.all(np.diff(es[left]) < 0)
    assert np.all(np.diff(es[~left]) > 0)
    assert es.min() == pytest.approx(-1.0, abs=1e-3)


def regular_tetrahedron(a):
    v = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float)
    return v * a / (2 * math.sqrt(2))


@pytest.mark.parametrize("rho", RHOS)
def test_all_pairs_at_re_give_minus_pairs_eps_and_no_force(rho):
    # triangle and tetrahedron with side re: every pair at the well bottom
    tri = np.array([[0, 0, 0], [1, 0, 0], [0.5, math.sqrt(3) / 2, 0]], float) * 1.1
    e, g = O.morse_energy_grad(tri, 0.9, 1.1, rho)
    assert e == pytest.approx(-3 * 0.9, rel=1e-14)
    assert np.abs(g).max() < 1e-12
    tet = regular_tetrahedron(1.1)
    e, g = O.morse_energy_grad(tet, 0.9, 1.1, rho)
    assert e == pytest.approx(-6 * 0.9, rel=1e-14)
    assert np.abs(g).max() < 1e-12


def octahedron(a):
    s = a / math.sqrt(2)
    return np.array([[s, 0, 0], [-s, 0, 0], [0, s, 0], [0, -s, 0], [0, 0, s], [0, 0, -s]])


@pytest.mark.parametrize("rho", RHOS)
def test_octahedron_from_its_distance_multiset(rho):
    # 12 edges at a and 3 diagonals at a sqrt(2); the dimer supplies V(r)
    a = 1.05
    v = lambda r: O.morse_energy_grad(dimer(r), 1.0, 1.0, rho)[0]
    e, g = O.morse_energy_grad(octahedron(a), 1.0, 1.0, rho)
    assert e == pytest.approx(12 * v(a) + 3 * v(a * math.sqrt(2)), rel=1e-13)
    # every atom feels the same radial force (O_h), and the forces sum to zero
    gr = g.reshape(6, 3)
    radial = np.einsum("ij,ij->i", gr, octahedron(a)) / (a / math.sqrt(2))
    assert np.allclose(radial, radial[0], rtol=1e-12)
    assert np.abs(gr.sum(0)).max() < 1e-12


def icosahedron13(radius):
    phi = (1 + math.sqrt(5)) / 2
    v = []
    for s1 in (-1, 1):
        for s2 in (-1, 1):
            v += [(0, s1, s2 * phi), (s1, s2 * phi, 0), (s2 * phi, 0, s1)]
    v = np.array(v, float)
    v *= radius / np.linalg.norm(v[0])
    return np.vstack([np.zeros(3), v])


def test_icosahedron_distance_multiset_and_breathing_minimum():
    """The centred icosahedron of circumradius R has 12 centre-vertex pairs at
    R, 30 edges at a = 4R / sqrt(10 + 2 sqrt 5), 30 second neighbours at
    phi a and 6 antipodes at 2R.  Under I_h the breathing mode is the only
    symmetric degree of freedom, so the R minimising that sum is a stationary
    point of the full potential, and the oracle's minimiser started from a
    breathed copy has to land on its energy."""
    from scipy.optimize import minimize_scalar
    rho = 6.0
    phi = (1 + math.sqrt(5)) / 2
    v = lambda r: O.morse_energy_grad(dimer(r), 1.0, 1.0, rho)[0]
    k_edge = 4 / math.sqrt(10 + 2 * math.sqrt(5))

    def e_of_R(R):
        a = k_edge * R
        return 12 * v(R) + 30 * v(a) + 30 * v(phi * a) + 6 * v(2 * R)

    for R in (0.9, 1.0, 1.1):
        assert O.morse_energy_grad(icosahedron13(R), 1.0, 1.0, rho)[0] == pytest.approx(
            e_of_R(R), rel=1e-13)
    res = minimize_scalar(e_of_R, bracket=(0.85, 0.95, 1.1), tol=1e-12)
    R_star, e_star = res.x, res.fun
    e, g = O.morse_energy_grad(icosahedron13(R_star), 1.0, 1.0, rho)
    assert e == pytest.approx(e_star, rel=1e-13)
    assert np.abs(g).max() < 1e-6
    x, f, st, it, _ = O.minimize(icosahedron13(R_star * 1.03), kind=O.OBJ_MORSE, rho=rho)
    assert st == O.CONVERGED
    assert f == pytest.approx(e_star, abs=1e-9)
    d = np.linalg.norm(x.reshape(13, 3)[1:] - x.reshape(13, 3)[0], axis=1)
    assert np.ptp(d) < 1e-6


def rand_cluster(n, seed, dmin=0.8):
    rng = np.random.default_rng(seed)
    side = (n / 0.6) ** (1 / 3)
    pts = []
    while len(pts) < n:
        p = rng.uniform(0, side, 3)
        if all(np.linalg.norm(p - q) >= dmin for q in pts):
            pts.append(p)
    return np.array(pts)


@pytest.mark.parametrize("n,seed,rho", [(5, 1, 6.0), (13, 2, 3.0), (24, 3, 10.0), (38, 4, 6.0)])
def test_gradient_central_differences(n, seed, rho):
    x = rand_cluster(n, seed).reshape(-1)
    _, g = O.morse_energy_grad(x, 1.3, 1.1, rho)
    h = 1e-6
    rng = np.random.default_rng(seed)
    for c in rng.choice(x.size, size=min(12, x.size), replace=False):
        xp, xm = x.copy(), x.copy()
        xp[c] += h
        xm[c] -= h
        fd = (O.morse_energy_grad(xp, 1.3, 1.1, rho)[0] - O.morse_energy_grad(xm, 1.3, 1.1, rho)[0]) / (2 * h)
        assert fd == pytest.approx(g[c], abs=2e-7 * max(1.0, abs(g[c])))


def test_translation_rotation_permutation_invariance_and_zero_net_force():
    x = rand_cluster(17, 5)
    e0, g0 = O.morse_energy_grad(x, 1.0, 1.0, 6.0)
    assert np.abs(g0.reshape(-1, 3).sum(0)).max() < 1e-11
    e1, _ = O.morse_energy_grad(x + np.array([3.0, -7.0, 0.25]), 1.0, 1.0, 6.0)
    assert e1 == pytest.approx(e0, rel=1e-13)
    q, _ = np.linalg.qr(np.random.default_rng(6).normal(size=(3, 3)))
    e2, g2 = O.morse_energy_grad(x @ q.T, 1.0, 1.0, 6.0)
    assert e2 == pytest.approx(e0, rel=1e-13)
    assert np.allclose(g2.reshape(-1, 3), g0.reshape(-1, 3) @ q.T, atol=1e-11)
    perm = np.random.default_rng(7).permutation(17)
    e3, g3 = O.morse_energy_grad(x[perm], 1.0, 1.0, 6.0)
    assert e3 == pytest.approx(e0, rel=1e-13)
    assert np.allclose(g3.reshape(-1, 3), g0.reshape(-1, 3)[perm], atol=1e-12)


def test_eps_re_scaling_law():
    # E(x; eps, re, rho) = eps E(x / re; 1, 1, rho), g scales by eps / re
    x = rand_cluster(11, 8)
    e1, g1 = O.morse_energy_grad(x / 1.7, 1.0, 1.0, 6.0)
    e2, g2 = O.morse_energy_grad(x, 0.4, 1.7, 6.0)
    assert e2 == pytest.approx(0.4 * e1, rel=1e-13)
    assert np.allclose(g2, 0.4 / 1.7 * g1, rtol=1e-12, atol=1e-14)


def test_degenerate_sizes_and_coincident_atoms():
    e, g = O.morse_energy_grad(np.zeros((1, 3)), 1.0, 1.0, 6.0)
    assert e == 0.0 and np.all(g == 0.0)
    e, g = O.morse_energy_grad(np.zeros((0, 3)), 1.0, 1.0, 6.0)
    assert e == 0.0
    x = rand_cluster(4, 9)
    x[2] = x[1]
    e, g = O.morse_energy_grad(x, 1.0, 1.0, 6.0)
    assert e == math.inf and np.all(np.isnan(g))


def test_batch_drivers_and_minimiser_use_the_chosen_potential():
    xs = [rand_cluster(n, 10 + n) for n in (3, 7, 13)]
    off = np.cumsum([0] + [len(c) for c in xs])
    flat = np.concatenate([c.reshape(-1) for c in xs])
    e, g = O.eval_batch(flat, 3, 0, off, eps=0.8, sigma=1.2, potential=O.OBJ_MORSE, rho=4.0)
    for i, c in enumerate(xs):
        ei, gi = O.morse_energy_grad(c, 0.8, 1.2, 4.0)
        assert e[i] == ei
        assert np.array_equal(g[3 * off[i]:3 * off[i + 1]], gi)
    x, em, st, it, ne = O.lbfgs_batch(flat, 3, 0, off, eps=0.8, sigma=1.2,
                                      potential=O.OBJ_MORSE, rho=4.0)
    for i, c in enumerate(xs):
        xi, fi, sti, _, _ = O.minimize(c, kind=O.OBJ_MORSE, eps=0.8, sigma=1.2, rho=4.0)
        assert st[i] == sti == O.CONVERGED
        assert em[i] == fi
        assert np.array_equal(x[3 * off[i]:3 * off[i + 1]], xi)
        # a minimum of Morse, not of LJ: its own gradient vanishes there
        assert np.abs(O.morse_energy_grad(xi, 0.8, 1.2, 4.0)[1]).max() < 1e-6


def test_matches_scipy_lbfgsb_as_black_box():
    """scipy's L-BFGS-B on the oracle's own Morse energy lands on the same
    minimum energy from most starts (the two line searches differ, so a
    different basin now and then is allowed)."""
    from scipy.optimize import minimize
    same = 0
    for seed in range(8):
        x0 = rand_cluster(9, 100 + seed).reshape(-1)
        x, f, st, _, _ = O.minimize(x0, kind=O.OBJ_MORSE, rho=6.0)
        assert st == O.CONVERGED
        res = minimize(lambda z: O.morse_energy_grad(z, 1.0, 1.0, 6.0), x0, jac=True,
                       method="L-BFGS-B", options={"maxcor": 10, "gtol": 1e-9, "ftol": 1e-15})
        same += abs(res.fun - f) < 1e-7
    assert same >= 6


def test_bh_runs_on_morse_and_stays_self_consistent():
    n, W = 7, 2
    x0 = np.stack([rand_cluster(n, 40 + w).reshape(-1) for w in range(W)])
    xs, es = [], []
    for w in range(W):
        x, f, st, _, _ = O.minimize(x0[w], kind=O.OBJ_MORSE, rho=6.0)
        xs.append(x)
        es.append(f)
    state = {"x_cur": np.array(xs), "e_cur": np.array(es), "x_best": np.array(xs),
             "e_best": np.array(es), "stepsize": np.full(W, 0.4),
             "win_accept": np.zeros(W, np.int32), "n_accept": np.zeros(W, np.int32)}
    bp = O.BhParamsPy(K=3, kT=0.8, seed=11, n_steps=12, potential=O.OBJ_MORSE, rho=6.0)
    tr = O.bh_run(state, bp, n_threads=1)
    for w in range(W):
        # every recorded trial energy is a Morse energy of a minimum, the walker's
        # energy is that of its structure, and the best never rises
        e_cur, _ = O.morse_energy_grad(state["x_cur"][w], 1.0, 1.0, 6.0)
        assert e_cur == pytest.approx(state["e_cur"][w], abs=1e-12)
        e_lj, _ = O.lj_energy_grad(state["x_cur"][w])
        assert abs(e_lj - e_cur) > 1e-3
        assert state["e_best"][w] <= min(es[w], tr["best_trial_e"][:, w].min()) + 1e-12
        assert np.all(np.diff(np.minimum.accumulate(tr["best_trial_e"][:, w])) <= 0)
