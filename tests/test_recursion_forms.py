"""The rearranged two-loop recursion of the kernels' lead warp gives the
oracle's L-BFGS direction (Algorithm 7.4 of Nocedal & Wright).

The kernels take history pairs two at a time: one two-value reduction gives
s_t.q and s_{t-1}.q, and s_{t-1}.(q - alpha_t y_t) follows as
s_{t-1}.q - alpha_t (s_{t-1}.y_t), with s_{t-1}.y_t stored when pair t is
pushed; the second loop uses y_{t+1}.(r + c_t s_t) = y_{t+1}.r + c_t (s_t.y_{t+1}).
The function below restates that order of operations in numpy (FP64) over a
history kept in a ring of slots, and is checked against the oracle's textbook
recursion.  It tests the rearrangement, not the CUDA code.
"""
import numpy as np
import pytest

import oracle as O


def blocked_direction(S, Y, g, head, cnt, m, sup):
    slot = lambda t: (head + t) % m
    rho = {slot(t): 1.0 / (S[slot(t)] @ Y[slot(t)]) for t in range(cnt)}
    q = g.copy()
    alpha = np.zeros(cnt)
    t = cnt - 1
    while t >= 1:
        s0, s1 = slot(t), slot(t - 1)
        p0, p1 = S[s0] @ q, S[s1] @ q                       # one two-value reduction
        a0 = rho[s0] * p0
        a1 = rho[s1] * (p1 - a0 * sup[s0])
        q -= a0 * Y[s0] + a1 * Y[s1]
        alpha[t], alpha[t - 1] = a0, a1
        t -= 2
    if t == 0:
        s0 = slot(0)
        alpha[0] = rho[s0] * (S[s0] @ q)
        q -= alpha[0] * Y[s0]
    sn = slot(cnt - 1)
    q *= (S[sn] @ Y[sn]) / (Y[sn] @ Y[sn])
    t = 0
    while t + 1 < cnt:
        s0, s1 = slot(t), slot(t + 1)
        p0, p1 = Y[s0] @ q, Y[s1] @ q
        c0 = alpha[t] - rho[s0] * p0
        c1 = alpha[t + 1] - rho[s1] * (p1 + c0 * sup[s1])
        q += c0 * S[s0] + c1 * S[s1]
        t += 2
    if t < cnt:
        s0 = slot(t)
        q += (alpha[t] - rho[s0] * (Y[s0] @ q)) * S[s0]
    return -q


@pytest.mark.parametrize("m,pushes", [(10, 3), (10, 10), (10, 23), (7, 16), (1, 4), (2, 5)])
def test_blocked_recursion_matches_oracle(m, pushes):
    rng = np.random.default_rng(1000 * m + pushes)
    n = 57
    M = rng.standard_normal((n, n))
    H = M @ M.T / n + np.eye(n)                 # positive curvature: s.y > 0
    S = np.zeros((m, n))
    Y = np.zeros((m, n))
    sup = np.zeros(m)
    head = cnt = 0
    for _ in range(pushes):                     # ring of slots, oldest dropped when full
        s = rng.standard_normal(n)
        y = H @ s
        prev = (head + cnt - 1) % m if cnt > 0 else None
        sp = S[prev] @ y if prev is not None else 0.0   # before the new pair is written
        if cnt < m:
            sl = (head + cnt) % m
            cnt += 1
        else:
            sl = head
            head = (head + 1) % m
        S[sl], Y[sl], sup[sl] = s, y, sp
    g = rng.standard_normal(n)
    order = [(head + t) % m for t in range(cnt)]     # oldest first, as the oracle takes them
    d_ref = O.lbfgs_direction(S[order], Y[order], g)
    d = blocked_direction(S, Y, g, head, cnt, m, sup)
    assert np.abs(d - d_ref).max() <= 1e-12 * np.abs(d_ref).max()
