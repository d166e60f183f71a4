"""Seeded synthetic inputs for the discrete Frechet distance (DFD) workloads.

This module draws curves and nothing else: it contains none of the DFD
arithmetic, so both the CPU oracle (``oracle/``) and the CUDA path may take
their inputs from it.  Every function is deterministic in its ``seed``.

Floating-point curves are generated in float64 and rounded once to float32;
integer curves are int32.  Curves are row-major ``[n, dim]`` arrays
(array-of-structures), batches are CSR packed: one ``[total_points, dim]``
array plus ``int64`` offsets of length ``n_curves + 1``.

Workloads (the paper's experiments use random walks only, Sec. 4):

* ``gaussian_walk_pair``  -- two independent Gaussian random walks (step
  sigma = 1), e.g. a 2000 x 1500 pair of 2-D curves.
* ``warped_long_pair``    -- one long 3-D random walk ``p`` and ``q = p o w +
  jitter`` with a random monotone time warp ``w``, e.g. n = m = 200,000.
* ``ragged_int_batch``    -- many pairs of int32 2-D curves with lengths drawn
  independently and uniformly, integer steps, clipped coordinates.
* ``ar1_curves``          -- curves whose coordinates follow an AR(1)
  process (a smoothed Gaussian process), for the all-pairs matrix.
* ``serving_pool`` / ``serving_requests`` -- a resident candidate pool and a
  Poisson stream of query-vs-k-candidates requests.
* ``paper_walks``         -- the paper's own generator (Sec. 4): steps drawn
  uniformly from {-1, 0, +1} in each of two dimensions.
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "gaussian_walk",
    "gaussian_walk_pair",
    "warped_long_pair",
    "ragged_int_batch",
    "ar1_curves",
    "serving_pool",
    "serving_requests",
    "paper_walks",
    "Batch",
    "Request",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def gaussian_walk(rng: np.random.Generator, n: int, dim: int, sigma: float = 1.0) -> np.ndarray:
    """float64 random walk starting at the origin with N(0, sigma^2 I) steps."""
    steps = rng.normal(0.0, sigma, size=(n, dim))
    steps[0, :] = 0.0
    return np.cumsum(steps, axis=0)


def gaussian_walk_pair(n: int = 2000, m: int = 1500, dim: int = 2, seed_p: int = 1, seed_q: int = 2):
    """Two independent Gaussian random walks (sigma = 1), rounded to float32."""
    p = gaussian_walk(_rng(seed_p), n, dim).astype(np.float32)
    q = gaussian_walk(_rng(seed_q), m, dim).astype(np.float32)
    return p, q


def warped_long_pair(n: int = 200_000, m: int = 200_000, dim: int = 3, seed: int = 3,
                     jitter_sigma: float = 0.5):
    """A long random walk p and a time-warped, jittered copy q.

    p: Gaussian random walk, sigma = 1.  The warp w maps the m samples of q
    onto [0, n-1]: cumulative sums of U[0.5, 1.5] increments rescaled to that
    interval (strictly increasing).  q_j = p(w_j) by linear interpolation plus
    N(0, jitter_sigma^2) noise per coordinate.
    """
    rng = _rng(seed)
    p64 = gaussian_walk(rng, n, dim)
    inc = rng.uniform(0.5, 1.5, size=m)
    c = np.cumsum(inc)
    if m > 1:
        w = (c - c[0]) / (c[-1] - c[0]) * (n - 1)
    else:
        w = np.zeros(1)
    lo = np.clip(np.floor(w).astype(np.int64), 0, n - 1)
    hi = np.minimum(lo + 1, n - 1)
    frac = (w - lo)[:, None]
    q64 = p64[lo] * (1.0 - frac) + p64[hi] * frac
    q64 += rng.normal(0.0, jitter_sigma, size=q64.shape)
    return p64.astype(np.float32), q64.astype(np.float32)


@dataclasses.dataclass
class Batch:
    """CSR-packed curves plus a list of (a, b) curve-id pairs."""
    points: np.ndarray   # [total_points, dim], float32 or int32
    offsets: np.ndarray  # [n_curves + 1], int64
    pairs: np.ndarray    # [n_pairs, 2], int32 (may be empty for matrix inputs)

    @property
    def n_curves(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def dim(self) -> int:
        return int(self.points.shape[1])

    def curve(self, i: int) -> np.ndarray:
        return self.points[self.offsets[i]:self.offsets[i + 1]]

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)

    def cells(self) -> int:
        """Sum over pairs of n_a * m_b (the logical DP cells)."""
        ln = self.lengths()
        if self.pairs.size == 0:
            return 0
        return int(np.sum(ln[self.pairs[:, 0]].astype(np.int64) * ln[self.pairs[:, 1]].astype(np.int64)))


def _offsets(lengths: np.ndarray) -> np.ndarray:
    off = np.zeros(lengths.shape[0] + 1, dtype=np.int64)
    np.cumsum(lengths, out=off[1:])
    return off


def _int_walks(rng, lengths, dim, step_lo, step_hi, bound):
    """int32 random walks from the origin with clip-and-continue at +-bound."""
    total = int(lengths.sum())
    steps = rng.integers(step_lo, step_hi + 1, size=(total, dim), dtype=np.int64)
    off = _offsets(lengths)
    steps[off[:-1], :] = 0
    pts = np.empty((total, dim), dtype=np.int64)
    # Vectorised cumulative sum per curve (segment ids), then exact
    # clip-and-continue for the curves whose unclipped walk leaves the box.
    seg = np.repeat(np.arange(lengths.shape[0]), lengths)
    cs = np.cumsum(steps, axis=0)
    base = np.zeros((lengths.shape[0], dim), dtype=np.int64)
    base[1:] = cs[off[1:-1] - 1]
    pts[:] = cs - base[seg]
    bad = np.unique(seg[np.any(np.abs(pts) > bound, axis=1)])
    for c in bad:
        x = np.zeros(dim, dtype=np.int64)
        for t in range(off[c], off[c + 1]):
            x = np.clip(x + steps[t], -bound, bound)
            pts[t] = x
    return pts.astype(np.int32), off


def ragged_int_batch(n_pairs: int = 65_536, len_lo: int = 16, len_hi: int = 512, dim: int = 2,
                     seed: int = 4, step: int = 64, bound: int = 1 << 20) -> Batch:
    """n_pairs disjoint pairs of int32 curves, lengths i.i.d. U{len_lo..len_hi}.

    Curve 2k is paired with curve 2k+1.  Coordinates are random walks from
    the origin with i.i.d. integer steps in [-step, step], clipped to
    [-bound, bound] after every step.
    """
    rng = _rng(seed)
    n_curves = 2 * n_pairs
    lengths = rng.integers(len_lo, len_hi + 1, size=n_curves, dtype=np.int64)
    pts, off = _int_walks(rng, lengths, dim, -step, step, bound)
    pairs = np.stack([np.arange(0, n_curves, 2), np.arange(1, n_curves, 2)], axis=1).astype(np.int32)
    return Batch(points=pts, offsets=off, pairs=pairs)


def ar1_curves(n_curves: int = 4096, len_lo: int = 64, len_hi: int = 256, dim: int = 16,
               phi: float = 0.95, seed: int = 5) -> Batch:
    """Curves whose coordinates are independent AR(1) processes per dimension.

    x_0 ~ N(0, 1), x_t = phi * x_{t-1} + sqrt(1 - phi^2) * eps_t (unit
    stationary variance).  No pair list: the all-pairs matrix uses i < j.
    """
    rng = _rng(seed)
    lengths = rng.integers(len_lo, len_hi + 1, size=n_curves, dtype=np.int64)
    tmax = int(lengths.max())
    x = np.empty((tmax, n_curves, dim), dtype=np.float64)
    x[0] = rng.normal(0.0, 1.0, size=(n_curves, dim))
    s = np.sqrt(1.0 - phi * phi)
    eps = rng.normal(0.0, 1.0, size=(tmax, n_curves, dim))
    for t in range(1, tmax):
        x[t] = phi * x[t - 1] + s * eps[t]
    off = _offsets(lengths)
    pts = np.empty((int(lengths.sum()), dim), dtype=np.float32)
    for c in range(n_curves):
        pts[off[c]:off[c + 1]] = x[:lengths[c], c, :]
    return Batch(points=pts, offsets=off, pairs=np.zeros((0, 2), dtype=np.int32))


def _lognormal_lengths(rng, size, median, sigma, lo, hi):
    ln = rng.lognormal(np.log(median), sigma, size=size)
    return np.clip(np.rint(ln), lo, hi).astype(np.int64)


def serving_pool(n_curves: int = 1 << 16, dim: int = 2, median: float = 256.0, sigma: float = 0.75,
                 len_lo: int = 32, len_hi: int = 4096, seed: int = 6) -> Batch:
    """Resident candidate pool: float32 Gaussian random walks, lognormal lengths."""
    rng = _rng(seed)
    lengths = _lognormal_lengths(rng, n_curves, median, sigma, len_lo, len_hi)
    total = int(lengths.sum())
    steps = rng.normal(0.0, 1.0, size=(total, dim))
    off = _offsets(lengths)
    steps[off[:-1], :] = 0.0
    seg = np.repeat(np.arange(n_curves), lengths)
    cs = np.cumsum(steps, axis=0)
    base = np.zeros((n_curves, dim))
    base[1:] = cs[off[1:-1] - 1]
    pts = (cs - base[seg]).astype(np.float32)
    return Batch(points=pts, offsets=off, pairs=np.zeros((0, 2), dtype=np.int32))


@dataclasses.dataclass
class Request:
    arrival_s: float          # scheduled arrival time (open loop)
    dim: int                  # 2 or 3
    query: np.ndarray         # [n, dim] float32
    cand_ids: np.ndarray      # [k] int64, ids into the pool of this dim


def serving_requests(n_requests: int, rate_per_s: float, pool_sizes: dict, k_lo: int = 1,
                     k_hi: int = 1024, median: float = 256.0, sigma: float = 0.75,
                     len_lo: int = 32, len_hi: int = 4096, seed: int = 7) -> list:
    """Open-loop Poisson request stream.

    Each request: dim in {2, 3} with probability 1/2, a float32 Gaussian
    random-walk query with lognormal length, and k ~ U{k_lo..k_hi}
    candidate ids drawn uniformly from the resident pool of that dim
    (``pool_sizes[dim]`` curves).
    """
    rng = _rng(seed)
    t = 0.0
    out = []
    for _ in range(n_requests):
        t += rng.exponential(1.0 / rate_per_s)
        dim = 2 if rng.random() < 0.5 else 3
        n = int(_lognormal_lengths(rng, 1, median, sigma, len_lo, len_hi)[0])
        k = int(rng.integers(k_lo, k_hi + 1))
        q = gaussian_walk(rng, n, dim).astype(np.float32)
        ids = rng.integers(0, pool_sizes[dim], size=k, dtype=np.int64)
        out.append(Request(arrival_s=t, dim=dim, query=q, cand_ids=ids))
    return out


def paper_walks(n_pairs: int, length: int, seed: int = 8) -> Batch:
    """The paper's generator (Sec. 4): 2-D walks, steps uniform in {-1,0,1}^2.

    Returns 2 * n_pairs float32 curves of equal length, paired (2k, 2k+1).
    """
    rng = _rng(seed)
    n_curves = 2 * n_pairs
    steps = rng.integers(-1, 2, size=(n_curves, length, 2)).astype(np.float64)
    steps[:, 0, :] = 0.0
    pts = np.cumsum(steps, axis=1).reshape(-1, 2).astype(np.float32)
    lengths = np.full(n_curves, length, dtype=np.int64)
    pairs = np.stack([np.arange(0, n_curves, 2), np.arange(1, n_curves, 2)], axis=1).astype(np.int32)
    return Batch(points=pts, offsets=_offsets(lengths), pairs=pairs)
