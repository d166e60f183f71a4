"""GPU parity of the threshold decider (dfd_batch_decide) and the exact k-NN
search (dfd_knn), both with early abandon.

Expected values come from the oracle only: float32 delta^2 from its float32
selection mirror (the kernels' distance order), int32 delta^2 exact in int64.
Pruning must never change a result: ties (delta^2 == eps^2) are never
abandoned, abandoned pairs have delta^2 > eps^2, and the k-NN answer equals
the k smallest (delta^2, position) over all candidates.
"""
import numpy as np
import pytest

import oracle
from paper_2404_05708_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def walk_batch(rng, n_curves, lo, hi, dim, dtype):
    lens = rng.integers(lo, hi + 1, size=n_curves)
    off = np.zeros(n_curves + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    if dtype == "f32":
        pts = np.cumsum(rng.normal(0, 1, size=(off[-1], dim)), axis=0).astype(np.float32)
        # restart every curve near the origin so that distances vary
        for c in range(n_curves):
            pts[off[c]:off[c + 1]] -= pts[off[c]] - rng.normal(0, 3, size=dim).astype(np.float32)
    else:
        pts = np.zeros((off[-1], dim), np.int32)
        for c in range(n_curves):
            pts[off[c]:off[c + 1]] = np.cumsum(rng.integers(-40, 41, size=(lens[c], dim)), axis=0) + \
                rng.integers(-200, 201, size=dim)
    return pts, off


def expected(pts, off, pairs, dtype):
    d2, _ = oracle.batch(pts, off, pairs, mirror=(dtype == "f32"))
    return d2.astype(np.float32) if dtype == "f32" else d2.astype(np.int64)


def f32_at_most(x):
    """Largest float32 <= x (how the decider reads a float64 threshold)."""
    f = np.float32(x)
    return np.nextafter(f, np.float32(-np.inf)) if float(f) > x else f


@pytest.mark.parametrize("dtype,dim", [("f32", 2), ("f32", 3), ("f32", 16), ("i32", 2), ("i32", 3)])
def test_decide_global_threshold(dctx, dtype, dim):
    rng = np.random.default_rng(11 + dim)
    pts, off = walk_batch(rng, 400, 8, 300, dim, dtype)
    pairs = rng.integers(0, 400, size=(3000, 2)).astype(np.int32)
    want = expected(pts, off, pairs, dtype)
    eps2 = float(np.median(want))
    d2, within, ab = dctx.decide(dev(pts), dev(off), dev(pairs), eps2)
    torch.cuda.synchronize()
    d2, within, ab = d2.cpu().numpy(), within.cpu().numpy(), int(ab.item())
    limit = f32_at_most(eps2) if dtype == "f32" else np.floor(eps2)
    truth = want <= limit
    assert np.array_equal(within.astype(bool), truth)
    computed = d2 != (np.inf if dtype == "f32" else np.iinfo(np.int64).max)
    assert np.array_equal(d2[computed], want[computed])
    assert np.all(want[~computed] > limit)
    assert ab == int((~computed).sum()) and ab > 0, ab   # the median threshold abandons some pairs


@pytest.mark.parametrize("dtype", ["f32", "i32"])
def test_decide_per_pair_ties_and_one_below(dctx, dtype):
    """eps2 = delta^2 exactly: within, never abandoned; one unit below: not within."""
    rng = np.random.default_rng(5)
    pts, off = walk_batch(rng, 200, 1, 600, 2, dtype)
    pairs = rng.integers(0, 200, size=(1500, 2)).astype(np.int32)
    want = expected(pts, off, pairs, dtype)
    at = want.copy()
    below = (np.nextafter(want.astype(np.float32), np.float32(-1)) if dtype == "f32" else want - 1)
    for eps, is_within in ((at, True), (below, False)):
        d2, within, ab = dctx.decide(dev(pts), dev(off), dev(pairs), dev(eps))
        torch.cuda.synchronize()
        w = within.cpu().numpy().astype(bool)
        assert np.all(w == is_within), np.nonzero(w != is_within)[0][:10]
        if is_within:
            assert np.array_equal(d2.cpu().numpy(), want) and int(ab.item()) == 0


def test_decide_int_value_classes(dctx):
    """Pairs in both int32 value classes (uint32 bits and int64) decide exactly."""
    rng = np.random.default_rng(8)
    small, so = walk_batch(rng, 60, 20, 200, 2, "i32")
    big = (np.cumsum(rng.integers(-(1 << 18), (1 << 18) + 1, size=(60 * 120, 2)), axis=0) +
           (1 << 27)).astype(np.int32)
    bo = np.arange(0, 60 * 120 + 1, 120, dtype=np.int64)
    pts = np.concatenate([small, big])
    off = np.concatenate([so, so[-1] + bo[1:]])
    pairs = np.concatenate([rng.integers(0, 60, size=(300, 2)), rng.integers(60, 120, size=(300, 2)),
                            np.stack([rng.integers(0, 60, 300), rng.integers(60, 120, 300)], 1)]).astype(np.int32)
    want = expected(pts, off, pairs, "i32")
    for q in (0.1, 0.5, 0.9):
        eps2 = float(np.quantile(want, q))
        d2, within, _ = dctx.decide(dev(pts), dev(off), dev(pairs), eps2)
        torch.cuda.synchronize()
        assert np.array_equal(within.cpu().numpy().astype(bool), want <= np.floor(eps2))
        d2 = d2.cpu().numpy()
        done = d2 != np.iinfo(np.int64).max
        assert np.array_equal(d2[done], want[done])


def knn_truth(qry, pts, off, cand, k):
    n_c = len(off) - 1
    ids = np.arange(n_c) if cand is None else cand
    allp = np.concatenate([qry, pts])
    allo = np.concatenate([[0], off + len(qry)])
    pairs = np.stack([np.zeros(len(ids), np.int32), ids.astype(np.int32) + 1], 1)
    d2, _ = oracle.batch(allp, allo, pairs, mirror=True)
    order = np.lexsort((np.arange(len(ids)), d2))[:k]
    return ids[order], d2[order]


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 10), (3, 64), (2, 1024), (8, 5)])
def test_knn_matches_brute_force(dctx, dim, k):
    rng = np.random.default_rng(21 + k)
    pts, off = walk_batch(rng, 2500, 16, 320, dim, "f32")
    qry = pts[off[7]:off[8]] + rng.normal(0, 0.3, size=(off[8] - off[7], dim)).astype(np.float32)
    want_ids, want_d2 = knn_truth(qry, pts, off, None, k)
    ids, d2, ab = dctx.knn(dev(qry), dev(pts), dev(off), k)
    torch.cuda.synchronize()
    assert np.array_equal(ids.cpu().numpy(), want_ids), (ids.cpu().numpy()[:10], want_ids[:10])
    assert np.array_equal(d2.cpu().numpy(), want_d2)
    n_ab, evaluated = (int(x) for x in ab.cpu().numpy())
    total_cells = len(qry) * int(off[-1])
    assert 0 < evaluated <= total_cells
    if k <= 64:
        assert n_ab > 0 and evaluated < total_cells   # small k prunes


def test_knn_candidate_subset_ties_and_padding(dctx):
    """A candidate list with duplicates (exact ties, broken by position) and
    fewer candidates than k (padded with -1 / +inf)."""
    rng = np.random.default_rng(3)
    pts, off = walk_batch(rng, 300, 10, 200, 2, "f32")
    qry = pts[off[0]:off[1]].copy()
    cand = np.array([5, 9, 5, 17, 0, 9, 250], np.int32)
    k = 10
    ids, d2, _ = dctx.knn(dev(qry), dev(pts), dev(off), k, cand=dev(cand))
    torch.cuda.synchronize()
    want_ids, want_d2 = knn_truth(qry, pts, off, cand, len(cand))
    got_ids, got_d2 = ids.cpu().numpy(), d2.cpu().numpy()
    assert np.array_equal(got_ids[:len(cand)], want_ids)
    assert np.array_equal(got_d2[:len(cand)], want_d2)
    assert np.all(got_ids[len(cand):] == -1) and np.all(np.isinf(got_d2[len(cand):]))
    assert got_ids[0] == 0 and got_d2[0] == 0.0   # the query itself
