"""The rearranged two-loop recursion of the kernels' lead warp gives the
oracle's L-BFGS direction (Algorithm 7.4 of Nocedal & Wright).

The kernels take history pairs two at a time (B = 2: on GB300 larger blocks
measured no faster); the rearrangement holds for any block size B and is
checked here for B = 1..5.  One B-value reduction gives
s_{t-k}.q for k < B, and the products the textbook recursion forms after
q has already been updated follow from them:
  s_{t-k}.(q - sum_{l<k} alpha_{t-l} y_{t-l})
      = s_{t-k}.q - sum_{l<k} alpha_{t-l} (s_{t-k}.y_{t-l}),
and in the second loop, with r before pair t and c_i = alpha_i - beta_i,
  y_{t+k}.(r + sum_{l<k} c_{t+l} s_{t+l})
      = y_{t+k}.r + sum_{l<k} c_{t+l} (s_{t+l}.y_{t+k}).
The cross products s_i.y_j (j - B < i < j) are reduced when pair j is
pushed, against the pairs stored before it.  The function below restates
that order of operations in numpy (FP64) over a history kept in a ring of
slots, and is checked against the oracle's textbook recursion.  It tests the
rearrangement, not the CUDA code.
"""
import numpy as np
import pytest

import oracle as O


def blocked_direction(S, Y, g, head, cnt, m, sup, B):
    """sup[slot_j][lag - 1] = s_{j - lag} . y_j for the pair in slot_j."""
    slot = lambda t: (head + t) % m
    rho = {slot(t): 1.0 / (S[slot(t)] @ Y[slot(t)]) for t in range(cnt)}
    u = lambda i, j: sup[slot(j)][j - i - 1]             # s_i . y_j, i < j
    q = g.copy()
    alpha = np.zeros(cnt)
    t = cnt - 1
    while t >= 0:                                        # newest first
        nb = min(B, t + 1)
        p = [S[slot(t - k)] @ q for k in range(nb)]      # one nb-value reduction
        a = []
        for k in range(nb):
            v = p[k] - sum(a[l] * u(t - k, t - l) for l in range(k))
            a.append(rho[slot(t - k)] * v)
        for k in range(nb):
            q -= a[k] * Y[slot(t - k)]
            alpha[t - k] = a[k]
        t -= nb
    sn = slot(cnt - 1)
    q *= (S[sn] @ Y[sn]) / (Y[sn] @ Y[sn])
    t = 0
    while t < cnt:                                       # oldest first
        nb = min(B, cnt - t)
        p = [Y[slot(t + k)] @ q for k in range(nb)]
        c = []
        for k in range(nb):
            v = p[k] + sum(c[l] * u(t + l, t + k) for l in range(k))
            c.append(alpha[t + k] - rho[slot(t + k)] * v)
        for k in range(nb):
            q += c[k] * S[slot(t + k)]
        t += nb
    return -q


@pytest.mark.parametrize("B", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("m,pushes", [(10, 3), (10, 10), (10, 23), (7, 16), (1, 4), (2, 5),
                                      (3, 11)])
def test_blocked_recursion_matches_oracle(m, pushes, B):
    rng = np.random.default_rng(1000 * m + pushes)
    n = 57
    M = rng.standard_normal((n, n))
    H = M @ M.T / n + np.eye(n)                 # positive curvature: s.y > 0
    S = np.zeros((m, n))
    Y = np.zeros((m, n))
    L = max(B - 1, 1)
    sup = np.zeros((m, L))
    head = cnt = 0
    for _ in range(pushes):                     # ring of slots, oldest dropped when full
        s = rng.standard_normal(n)
        y = H @ s
        # products of the stored pairs' s with the new y, before it is written
        sp = [S[(head + cnt - lag) % m] @ y if cnt >= lag else 0.0 for lag in range(1, L + 1)]
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
    d = blocked_direction(S, Y, g, head, cnt, m, sup, B)
    assert np.abs(d - d_ref).max() <= 1e-12 * np.abs(d_ref).max()
