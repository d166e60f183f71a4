"""Brute-force discrete Frechet distance -- TEST INFRASTRUCTURE ONLY.

Definition (paper, Sec. 2: two frogs hopping along the stones of p and q,
neither going back): a coupling is a sequence of index pairs from (1, 1) to
(n, m) in which each step advances i, j or both by one.  The discrete
Frechet distance is the minimum over all couplings of the longest leash
(largest ground distance) used along it.  This module enumerates every
coupling explicitly -- there are Delannoy(n-1, m-1) of them, 48,639 for
n = m = 8 -- so it shares no step with the dynamic program of Eq. 1 and can
pin it.  Squared distances, exact Python arithmetic on float64 / int.
"""
from __future__ import annotations

import numpy as np


def _d2_table(p, q):
    p = np.asarray(p)
    q = np.asarray(q)
    if p.ndim == 1:
        p = p[:, None]
    if q.ndim == 1:
        q = q[:, None]
    integer = p.dtype.kind in "iu" and q.dtype.kind in "iu"
    n, m = p.shape[0], q.shape[0]
    tab = [[0] * m for _ in range(n)]
    for i in range(n):
        for j in range(m):
            s = 0 if integer else 0.0
            for k in range(p.shape[1]):
                t = (int(p[i, k]) - int(q[j, k])) if integer else (float(p[i, k]) - float(q[j, k]))
                s += t * t
            tab[i][j] = s
    return tab


def couplings(n: int, m: int):
    """Yield every monotone coupling of (0..n-1) and (0..m-1) as a list of cells."""
    path = [(0, 0)]

    def rec(i, j):
        if i == n - 1 and j == m - 1:
            yield list(path)
            return
        for di, dj in ((1, 0), (0, 1), (1, 1)):
            a, b = i + di, j + dj
            if a < n and b < m:
                path.append((a, b))
                yield from rec(a, b)
                path.pop()

    yield from rec(0, 0)


def dfd2_bruteforce(p, q):
    """min over couplings of the max squared ground distance along the coupling."""
    tab = _d2_table(p, q)
    n, m = len(tab), len(tab[0])
    best = None
    for path in couplings(n, m):
        worst = max(tab[i][j] for i, j in path)
        if best is None or worst < best:
            best = worst
    return best


def count_couplings(n: int, m: int) -> int:
    return sum(1 for _ in couplings(n, m))
