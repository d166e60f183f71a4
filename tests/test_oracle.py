"""Pins for the CPU oracle (no GPU).

The oracle is checked against facts that do not come from itself:
  * brute-force enumeration of all monotone couplings (the definition, Sec. 2);
  * closed forms (one-point curves, pure translation, identical curves);
  * the metric and invariance properties the paper states (Sec. 2 and the
    footnote of Sec. 4: symmetry, triangle inequality, Hausdorff lower bound,
    repeated points);
  * an independent decision search (threshold + reachability) on larger inputs.
Every oracle routine must agree exactly with the others on the same squared
distances, because the recurrence only selects among them.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import brute, fast_form

ALL_F = (oracle.dfd2_linear, oracle.dfd2_full, oracle.dfd2_memo, oracle.dfd2_decide)


def rand_int_curve(rng, n, dim, lo=-6, hi=6):
    return rng.integers(lo, hi + 1, size=(n, dim)).astype(np.int32)


def rand_f32_curve(rng, n, dim, scale=3.0):
    return (rng.normal(0, scale, size=(n, dim))).astype(np.float32)


# ------------------------------------------------------------ definition pins

@pytest.mark.parametrize("dtype", ["i32", "f32"])
def test_all_forms_equal_bruteforce_tiny(dtype):
    rng = np.random.default_rng(11)
    for trial in range(160):
        n = int(rng.integers(1, 7))
        m = int(rng.integers(1, 7))
        dim = int(rng.integers(1, 4))
        if dtype == "i32":
            p, q = rand_int_curve(rng, n, dim), rand_int_curve(rng, m, dim)
        else:
            p, q = rand_f32_curve(rng, n, dim), rand_f32_curve(rng, m, dim)
        ref = brute.dfd2_bruteforce(p, q)
        for f in ALL_F:
            assert f(p, q) == ref, (f.__name__, trial, n, m, dim)
        if dtype == "f32":
            assert fast_form.frechet_distance_sq(fast_form.d2_matrix(p, q)) == ref


def test_bruteforce_enumerates_delannoy_numbers():
    # Delannoy numbers D(a, b): lattice paths with steps E, N, NE.
    delannoy = {(0, 0): 1, (1, 1): 3, (2, 2): 13, (3, 3): 63, (2, 3): 25, (4, 4): 321}
    for (a, b), v in delannoy.items():
        assert brute.count_couplings(a + 1, b + 1) == v


def test_decide_matches_linear_medium():
    rng = np.random.default_rng(12)
    for _ in range(6):
        n, m = int(rng.integers(20, 160)), int(rng.integers(20, 160))
        p = np.cumsum(rng.integers(-5, 6, size=(n, 2)), axis=0).astype(np.int32)
        q = np.cumsum(rng.integers(-5, 6, size=(m, 2)), axis=0).astype(np.int32)
        assert oracle.dfd2_decide(p, q) == oracle.dfd2_linear(p, q) == oracle.dfd2_full(p, q)
        pf, qf = p.astype(np.float32) * 0.37, q.astype(np.float32) * 0.37
        assert oracle.dfd2_decide(pf, qf) == oracle.dfd2_linear(pf, qf)


def test_decide_matches_linear_2000():
    from paper_2404_05708_gb300 import workloads
    p, q = workloads.gaussian_walk_pair(600, 450)
    assert oracle.dfd2_decide(p, q) == oracle.dfd2_linear(p, q)


# ------------------------------------------------------------ closed forms

def test_one_point_curve_is_max_distance():
    rng = np.random.default_rng(13)
    for _ in range(30):
        m = int(rng.integers(1, 50))
        p = rand_int_curve(rng, 1, 3, -1000, 1000)
        q = rand_int_curve(rng, m, 3, -1000, 1000)
        d2 = [int(np.sum((p[0].astype(np.int64) - q[j]) ** 2)) for j in range(m)]
        assert oracle.dfd2_linear(p, q) == max(d2)
        assert oracle.dfd2_linear(q, p) == max(d2)
        assert oracle.dfd2_memo(q, p) == max(d2)


def test_translation_closed_form():
    rng = np.random.default_rng(14)
    for _ in range(20):
        n = int(rng.integers(1, 300))
        dim = int(rng.integers(1, 5))
        p = rand_int_curve(rng, n, dim, -10**6, 10**6)
        t = rng.integers(-1000, 1000, size=dim).astype(np.int32)
        q = (p + t).astype(np.int32)
        assert oracle.dfd2_linear(p, q) == int(np.sum(t.astype(np.int64) ** 2))
        # float32 with small integer coordinates: all arithmetic exact
        pf = rand_int_curve(rng, n, dim, -2000, 2000).astype(np.float32)
        assert oracle.dfd2_linear(pf, pf + t.astype(np.float32)) == float(np.sum(t.astype(np.float64) ** 2))


def test_identity_is_zero():
    from paper_2404_05708_gb300 import workloads
    p, _ = workloads.gaussian_walk_pair(300, 10)
    assert oracle.dfd2_linear(p, p) == 0.0
    assert oracle.dfd2_full(p, p) == 0.0


def test_hand_worked_example():
    # p = (0,0),(1,1),(2,0); q = (0,1),(2,1).  Squared distances
    #   row p1: 1, 5;  row p2: 1, 1;  row p3: 5, 1.
    # Coupling (1,1)->(2,1)->(3,2) uses 1, 1, 1, so delta^2 = 1; no coupling
    # can do better since every coupling starts at d^2_11 = 1.
    p = np.array([[0, 0], [1, 1], [2, 0]], np.int32)
    q = np.array([[0, 1], [2, 1]], np.int32)
    for f in ALL_F:
        assert f(p, q) == 1
    # With q reversed, q = (2,1),(0,1): every coupling starts at (p1, (2,1)) with
    # d^2 = 5 and ends at (p3, (0,1)) with d^2 = 5, and (1,1)->(2,1)->(2,2)->(3,2)
    # uses nothing larger, so delta^2 = 5.
    for f in ALL_F:
        assert f(p, q[::-1].copy()) == 5


# ------------------------------------------------------------ invariants

def test_symmetry_reversal_duplication():
    rng = np.random.default_rng(15)
    for _ in range(40):
        n, m = int(rng.integers(1, 60)), int(rng.integers(1, 60))
        p = rand_f32_curve(rng, n, 2)
        q = rand_f32_curve(rng, m, 2)
        base = oracle.dfd2_linear(p, q)
        assert oracle.dfd2_linear(q, p) == base
        assert oracle.dfd2_linear(p[::-1].copy(), q[::-1].copy()) == base
        k = int(rng.integers(0, n))
        pd = np.insert(p, k, p[k], axis=0)          # repeat one vertex (Sec. 4 footnote)
        assert oracle.dfd2_linear(pd, q) == base


def test_lower_bounds_and_triangle():
    rng = np.random.default_rng(16)
    for _ in range(40):
        n, m, r = (int(x) for x in rng.integers(1, 40, size=3))
        p, q, s = rand_f32_curve(rng, n, 3), rand_f32_curve(rng, m, 3), rand_f32_curve(rng, r, 3)
        dpq = oracle.dfd2_linear(p, q)
        end0 = float(np.sum((p[0].astype(np.float64) - q[0]) ** 2))
        end1 = float(np.sum((p[-1].astype(np.float64) - q[-1]) ** 2))
        assert dpq >= max(end0, end1) * (1 - 1e-15)
        assert dpq >= oracle.hausdorff2(p, q)
        a = math.sqrt(oracle.dfd2_linear(p, s))
        b = math.sqrt(dpq) + math.sqrt(oracle.dfd2_linear(q, s))
        assert a <= b + 1e-12


# ------------------------------------------------ discrete Hausdorff (Sec. 2)
# The Frechet distance is never below the Hausdorff distance of the two point
# sets (Sec. 2).  The oracle's Hausdorff routine is pinned here by closed
# forms that separate it from the Frechet distance and from its one-sided
# half, by the set properties it must have, and by a threshold search.

def _as(kind, pts):
    return np.array(pts, np.int32 if kind == "i32" else np.float32)


@pytest.mark.parametrize("kind", ["i32", "f32"])
def test_hausdorff_closed_forms(kind):
    # a curve and its reverse: the same point set, so Hausdorff 0, while a
    # coupling must pair (0,0) with (2,0) at an end, so delta^2 = 4
    p = _as(kind, [[0, 0], [1, 0], [2, 0]])
    q = p[::-1].copy()
    assert oracle.hausdorff2(p, q) == 0
    assert oracle.dfd2_linear(p, q) == 4
    # one point against a curve that also reaches a far point: the one-sided
    # distance from p is 0, the symmetric one is 5^2
    p1 = _as(kind, [[0, 0]])
    q1 = _as(kind, [[0, 0], [5, 0]])
    assert oracle.hausdorff2(p1, q1) == 25
    assert oracle.hausdorff2(q1, p1) == 25
    # both directions nonzero and different: p = {(0,0), (10,0)},
    # q = {(1,0), (2,0), (9,0)}; p -> q: max(1, 1) = 1; q -> p: max(1, 4, 1) = 4
    p2 = _as(kind, [[0, 0], [10, 0]])
    q2 = _as(kind, [[1, 0], [2, 0], [9, 0]])
    assert oracle.hausdorff2(p2, q2) == 4
    assert oracle.hausdorff2(q2, p2) == 4


@pytest.mark.parametrize("kind", ["i32", "f32"])
def test_hausdorff_one_point_curve_equals_frechet(kind):
    """For a one-point curve both distances are the largest distance from
    that point to the other curve (the fold over an empty sequence)."""
    rng = np.random.default_rng(17)
    for _ in range(30):
        m = int(rng.integers(1, 30))
        a = rand_int_curve(rng, 1, 2) if kind == "i32" else rand_f32_curve(rng, 1, 2)
        q = rand_int_curve(rng, m, 2) if kind == "i32" else rand_f32_curve(rng, m, 2)
        far = max(float(np.sum((a[0].astype(np.float64) - q[j]) ** 2)) for j in range(m))
        assert oracle.hausdorff2(a, q) == far
        assert oracle.hausdorff2(q, a) == far
        assert oracle.hausdorff2(a, q) == oracle.dfd2_linear(a, q)


@pytest.mark.parametrize("kind", ["i32", "f32"])
def test_hausdorff_is_a_set_distance(kind):
    """Hausdorff depends on the point sets only: symmetric, unchanged by any
    reordering or duplication of points, zero on equal sets, and equal to the
    smallest squared distance t at which every point of either curve has a
    point of the other within t (a threshold search, not the max-min loops)."""
    rng = np.random.default_rng(18)
    for _ in range(40):
        n, m = int(rng.integers(1, 25)), int(rng.integers(1, 25))
        mk = rand_int_curve if kind == "i32" else rand_f32_curve
        p, q = mk(rng, n, 3), mk(rng, m, 3)
        h = oracle.hausdorff2(p, q)
        assert oracle.hausdorff2(q, p) == h
        pp = p[rng.permutation(n)]
        qq = np.concatenate([q, q[rng.integers(0, m, size=3)]])[rng.permutation(m + 3)]
        assert oracle.hausdorff2(pp, qq) == h
        assert oracle.hausdorff2(p, pp) == 0
        d2 = ((p[:, None, :].astype(np.float64) - q[None, :, :].astype(np.float64)) ** 2).sum(-1)
        t = next(v for v in np.unique(d2) if (d2 <= v).any(1).all() and (d2 <= v).any(0).all())
        assert h == t
        assert oracle.dfd2_linear(p, q) >= h


def test_hausdorff_pins_catch_the_one_sided_mistake(tmp_path):
    """A Hausdorff that drops the second direction must fail a pin."""
    path = oracle.build(str(tmp_path / "mut6.so"), mutant=6, force=True)
    lib = oracle.load(path)
    p1 = np.array([[0, 0]], np.int32)
    q1 = np.array([[0, 0], [5, 0]], np.int32)
    assert oracle.hausdorff2(p1, q1, lib=lib) != 25
    assert oracle.hausdorff2(p1.astype(np.float32), q1.astype(np.float32), lib=lib) != 25


def test_int_extremes_no_overflow():
    # precondition: dim * (2 * max|c|)^2 < 2^63
    big = (1 << 29) - 1
    p = np.array([[big, -big], [-big, big]], np.int32)
    q = np.array([[-big, big]], np.int32)
    want = 2 * (2 * big) ** 2
    assert oracle.dfd2_linear(p, q) == want
    assert brute.dfd2_bruteforce(p, q) == want


# ------------------------------------------------------------ mirror & batch

def test_f32_mirror_exact_on_exact_inputs_and_close_otherwise():
    rng = np.random.default_rng(17)
    for _ in range(30):
        n, m = int(rng.integers(1, 40)), int(rng.integers(1, 40))
        p = rand_int_curve(rng, n, 3, -500, 500).astype(np.float32)
        q = rand_int_curve(rng, m, 3, -500, 500).astype(np.float32)
        assert float(oracle.dfd2_f32mirror(p, q)) == oracle.dfd2_linear(p, q)
        pf, qf = rand_f32_curve(rng, n, 3), rand_f32_curve(rng, m, 3)
        ref = oracle.dfd2_linear(pf, qf)
        got = float(oracle.dfd2_f32mirror(pf, qf))
        assert abs(got - ref) <= 6 * 2.0 ** -24 * ref


def _rows_dp(d):
    """All rows of Eq. 1 over a matrix of ground distances (plain loops)."""
    n, m = d.shape
    M = np.empty((n, m))
    for i in range(n):
        for j in range(m):
            if i == 0 and j == 0:
                M[i, j] = d[i, j]
                continue
            best = math.inf
            if i > 0:
                best = min(best, M[i - 1, j])
            if j > 0:
                best = min(best, M[i, j - 1])
            if i > 0 and j > 0:
                best = min(best, M[i - 1, j - 1])
            M[i, j] = max(best, d[i, j])
    return M


def test_meeting_in_the_middle_identity():
    """The two-front wavefront's combine: with F the last row of the DP over
    rows 0..n1-1 and B the last row of the DP over the remaining rows with
    both curves reversed (read back in forward column order), the oracle's
    delta^2 equals min_j max(F[j], min(B[j], B[j+1])) for every split."""
    rng = np.random.default_rng(17)
    for _ in range(60):
        n, m = int(rng.integers(2, 12)), int(rng.integers(1, 12))
        p, q = rand_int_curve(rng, n, 2), rand_int_curve(rng, m, 2)
        want = oracle.dfd2_linear(p, q)
        d = ((p[:, None, :].astype(np.int64) - q[None, :, :]) ** 2).sum(-1).astype(float)
        for n1 in range(1, n):
            F = _rows_dp(d[:n1])[-1]
            B = _rows_dp(d[n1:][::-1, ::-1])[-1][::-1]
            Bn = np.append(B[1:], math.inf)
            assert np.min(np.maximum(F, np.minimum(B, Bn))) == want, (n, m, n1)


def test_batch_driver_matches_single_calls():
    from paper_2404_05708_gb300 import workloads
    b = workloads.ragged_int_batch(n_pairs=64, len_lo=1, len_hi=40, seed=21)
    out, used = oracle.batch(b.points, b.offsets, b.pairs, nthreads=4)
    assert used >= 1
    for k, (a, c) in enumerate(b.pairs):
        assert out[k] == oracle.dfd2_linear(b.curve(a), b.curve(c))


# ------------------------------------------------------------ appendix variants

def _dtw_brute(p, q):
    tab = brute._d2_table(np.asarray(p, np.float32), np.asarray(q, np.float32))
    n, m = len(tab), len(tab[0])
    return min(sum(tab[i][j] for i, j in path) for path in brute.couplings(n, m))


def test_dtw_bruteforce():
    rng = np.random.default_rng(18)
    for _ in range(60):
        n, m = int(rng.integers(1, 6)), int(rng.integers(1, 6))
        p = rand_int_curve(rng, n, 2).astype(np.float32)
        q = rand_int_curve(rng, m, 2).astype(np.float32)
        assert oracle.dtw(p, q) == _dtw_brute(p, q)


def test_dtw_f32mirror_exact_on_integers_and_bounded_otherwise():
    """The float32 DTW mirror equals the float64 DTW (pinned by brute force
    above) exactly when every value is an integer below 2^24, and is within
    the summation bound otherwise: a path has at most n+m-1 non-negative
    terms, each with dim+1 roundings, plus one rounding per addition."""
    rng = np.random.default_rng(19)
    for _ in range(40):
        n, m = int(rng.integers(1, 40)), int(rng.integers(1, 40))
        p = rand_int_curve(rng, n, 2).astype(np.float32)
        q = rand_int_curve(rng, m, 2).astype(np.float32)
        assert oracle.dtw_f32mirror(p, q) == oracle.dtw(p, q)
    for dim in (1, 3, 16):
        for _ in range(10):
            n, m = int(rng.integers(1, 300)), int(rng.integers(1, 300))
            p = np.cumsum(rng.normal(size=(n, dim)), 0).astype(np.float32)
            q = np.cumsum(rng.normal(size=(m, dim)), 0).astype(np.float32)
            ref = oracle.dtw(p, q)
            bound = (n + m + dim + 2) * 2.0 ** -24 * ref
            assert abs(oracle.dtw_f32mirror(p, q) - ref) <= bound


def test_dtw_f32mirror_planted_mistake_is_caught():
    """A DTW cell that kept the maximum of the Frechet recurrence instead of
    the sum would not match: the mirror differs from the Frechet mirror."""
    rng = np.random.default_rng(20)
    p = rand_int_curve(rng, 12, 2).astype(np.float32)
    q = rand_int_curve(rng, 9, 2).astype(np.float32)
    assert oracle.dtw_f32mirror(p, q) > oracle.dfd2_f32mirror(p, q)


def test_perturb_single_rounding():
    """x + sigma*z with one rounding: exact where the exact value is a
    float32; where the float64 sum of x and the (exact) float64 product is
    itself exact, equal to that sum rounded once to float32."""
    rng = np.random.default_rng(23)
    x = rng.integers(-1000, 1000, size=500).astype(np.float32)
    z = rng.integers(-64, 64, size=500).astype(np.float32) / np.float32(8)
    out = oracle.perturb(x, z, 0.25)
    assert np.array_equal(out, x + np.float32(0.25) * z)      # all exact
    x = rng.normal(size=2000).astype(np.float32)
    z = rng.normal(size=2000).astype(np.float32)
    sigma = np.float32(0.3)
    prod = z.astype(np.float64) * np.float64(sigma)            # exact in float64
    s64 = x.astype(np.float64) + prod
    exact = (s64 - x.astype(np.float64)) == prod                # the float64 sum did not round
    assert exact.sum() > 100
    assert np.array_equal(oracle.perturb(x, z, sigma)[exact], s64[exact].astype(np.float32))
    # planted mistake: two roundings (product first) differ somewhere
    two = (np.float32(sigma) * z) + x
    assert not np.array_equal(two, oracle.perturb(x, z, sigma))


def test_levenshtein_known_and_brute():
    enc = lambda s: np.array([ord(c) for c in s], np.int32)
    assert oracle.levenshtein(enc("kitten"), enc("sitting")) == 3
    assert oracle.levenshtein(enc("flaw"), enc("lawn")) == 2
    assert oracle.levenshtein(enc("a"), enc("a")) == 0
    assert oracle.levenshtein(enc("a"), enc("b")) == 1

    def lev_rec(a, b):   # direct recursive definition
        from functools import lru_cache

        @lru_cache(None)
        def L(i, j):
            if i == 0:
                return j
            if j == 0:
                return i
            return min(L(i - 1, j) + 1, L(i, j - 1) + 1, L(i - 1, j - 1) + (a[i - 1] != b[j - 1]))
        return L(len(a), len(b))

    rng = np.random.default_rng(19)
    for _ in range(100):
        a = rng.integers(0, 3, size=int(rng.integers(1, 9))).astype(np.int32)
        b = rng.integers(0, 3, size=int(rng.integers(1, 9))).astype(np.int32)
        assert oracle.levenshtein(a, b) == lev_rec(tuple(a), tuple(b))


# ------------------------------------------------------------ planted mistakes

@pytest.mark.parametrize("mutant,fname", [(1, "dfd2_linear"), (2, "dfd2_linear"), (3, "dfd2_full"),
                                          (4, "dfd2_memo"), (5, "dfd2_linear")])
def test_pins_catch_planted_mistakes(tmp_path, mutant, fname):
    """Each planted mistake in the oracle must fail the brute-force pin."""
    path = oracle.build(str(tmp_path / f"mut{mutant}.so"), mutant=mutant, force=True)
    lib = oracle.load(path)
    f = getattr(oracle, fname)
    rng = np.random.default_rng(20)
    caught = False
    for _ in range(200):
        n, m = int(rng.integers(1, 6)), int(rng.integers(1, 6))
        p, q = rand_f32_curve(rng, n, 2), rand_f32_curve(rng, m, 2)
        if f(p, q, lib=lib) != brute.dfd2_bruteforce(p, q):
            caught = True
            break
    assert caught, f"mutant {mutant} survived the pins"
