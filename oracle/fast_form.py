"""Alg. 2 of the paper as a fold of scans -- TEST INFRASTRUCTURE ONLY.

Written from the algorithm's description (Sec. 3, Theorem 1, and the scan /
fold operators of Appendix A), in float64 numpy on a precomputed matrix of
squared distances:

* a scan ``f\\(t0, x)`` returns t0 followed by the running applications of f
  (length N + 1); for a same-typed f, the first element is the initial value;
* a fold ``f/(t0, x)`` returns only the last running value;
* ``maxmin(a, (x1, x2)) = max(min(a, x1), x2)``;
* ``next(a, x)``: first a_{2..Q} <- min(a_{1..Q-1}, a_{2..Q}) elementwise, then
  the maxmin scan seeded with max(a_1, x_1) over the stacked columns
  (a_{2..Q} | x_{2..Q});
* the distance is element Q of the fold of ``next`` over rows 2..P, seeded
  with the max-scan of row 1.

The degenerate shapes follow from these definitions: with one row the fold
is empty and the result is the last element of the max-scan of row 1; with
one column the maxmin scan is empty and each row contributes max(a_1, x_1).
"""
from __future__ import annotations

import numpy as np


def scan(f, t0, xs):
    out = [t0]
    t = t0
    for x in xs:
        t = f(t, x)
        out.append(t)
    return out


def scan1(f, xs):
    xs = list(xs)
    return scan(f, xs[0], xs[1:])


def fold(f, t0, xs):
    t = t0
    for x in xs:
        t = f(t, x)
    return t


def maxmin(a, x):
    return max(min(a, x[0]), x[1])


def frechet_next(a, x):
    a = list(a)
    shifted = [min(a[j - 1], a[j]) for j in range(1, len(a))]
    pairs = list(zip(shifted, list(x[1:])))
    return scan(maxmin, max(a[0], x[0]), pairs)


def frechet_distance_sq(d2: np.ndarray) -> float:
    """Alg. 2 on a P x Q matrix of squared distances; returns delta^2."""
    rows = [list(map(float, r)) for r in np.asarray(d2, dtype=np.float64)]
    first = scan1(max, rows[0])
    return fold(frechet_next, first, rows[1:])[-1]


def d2_matrix(p, q) -> np.ndarray:
    p = np.asarray(p, np.float64)
    q = np.asarray(q, np.float64)
    if p.ndim == 1:
        p = p[:, None]
    if q.ndim == 1:
        q = q[:, None]
    diff = p[:, None, :] - q[None, :, :]
    out = np.zeros(diff.shape[:2])
    for k in range(diff.shape[2]):          # left-to-right, like the C oracle
        out = out + diff[:, :, k] * diff[:, :, k]
    return out
