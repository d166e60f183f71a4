"""GPU parity of the appendix variants (dfd_batch_variant): DTW bit-identical
to the oracle's float32 DTW mirror (and within the derived bound of the
float64 DTW), Levenshtein exact against the textbook table."""
import numpy as np
import pytest

import oracle
from paper_2404_05708_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EDGES = [1, 2, 31, 32, 33, 63, 64, 65, 255, 256, 257, 300, 513]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def edge_pairs(rng, gen):
    lens, pairs = [], []
    for a in EDGES:
        for b in rng.choice(EDGES, size=4, replace=False):
            pairs.append((len(lens), len(lens) + 1))
            lens += [a, int(b)]
    lens = np.array(lens, np.int64)
    off = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    return gen(int(off[-1])), off, np.array(pairs, np.int32)


@pytest.mark.parametrize("dim", [1, 2, 3, 8, 16])
def test_dtw_matches_mirror_and_bound(dctx, dim):
    rng = np.random.default_rng(60 + dim)
    pts, off, pairs = edge_pairs(rng, lambda t: np.cumsum(rng.normal(size=(t, dim)), 0).astype(np.float32))
    got = dctx.dtw(dev(pts), dev(off), dev(pairs)).cpu().numpy()
    for k, (a, b) in enumerate(pairs):
        p, q = pts[off[a]:off[a + 1]], pts[off[b]:off[b + 1]]
        mirror = np.float32(oracle.dtw_f32mirror(p, q))
        assert got[k] == mirror, (k, len(p), len(q), got[k], mirror)
        ref = oracle.dtw(p, q)
        assert abs(float(got[k]) - ref) <= (len(p) + len(q) + dim + 2) * 2.0 ** -24 * ref


def test_dtw_integer_inputs_exact(dctx):
    """Integer coordinates with sums below 2^24: the float32 DTW is exact."""
    rng = np.random.default_rng(70)
    pts, off, pairs = edge_pairs(rng, lambda t: rng.integers(-3, 4, size=(t, 2)).astype(np.float32))
    got = dctx.dtw(dev(pts), dev(off), dev(pairs)).cpu().numpy()
    for k, (a, b) in enumerate(pairs):
        assert float(got[k]) == oracle.dtw(pts[off[a]:off[a + 1]], pts[off[b]:off[b + 1]])


@pytest.mark.parametrize("alphabet", [2, 4, 26, 1 << 20])
def test_levenshtein_exact(dctx, alphabet):
    rng = np.random.default_rng(80 + alphabet % 97)
    sym, off, pairs = edge_pairs(rng, lambda t: rng.integers(0, alphabet, size=t).astype(np.int32))
    got = dctx.levenshtein(dev(sym), dev(off), dev(pairs)).cpu().numpy()
    for k, (a, b) in enumerate(pairs):
        assert got[k] == oracle.levenshtein(sym[off[a]:off[a + 1]], sym[off[b]:off[b + 1]]), k


def test_levenshtein_known_values(dctx):
    words = ["kitten", "sitting", "flaw", "lawn", "a", "b", "", "abc"]
    words = [w for w in words if w]
    seqs = [np.array([ord(c) for c in w], np.int32) for w in words]
    off = np.zeros(len(seqs) + 1, np.int64)
    np.cumsum([len(s) for s in seqs], out=off[1:])
    pairs = np.array([(0, 1), (2, 3), (4, 4), (4, 5), (6, 0), (1, 0)], np.int32)
    got = dctx.levenshtein(dev(np.concatenate(seqs)), dev(off), dev(pairs)).cpu().numpy()
    assert list(got) == [3, 2, 0, 1, 6, 3]


def test_variant_argument_errors(dctx):
    from paper_2404_05708_gb300 import dfd
    pts = np.zeros((4, 2), np.int32)
    off = np.array([0, 2, 4], np.int64)
    pairs = np.array([[0, 1]], np.int32)
    with pytest.raises(dfd.DFDError):
        dctx.dtw(dev(pts), dev(off), dev(pairs))            # DTW needs float32
    with pytest.raises(dfd.DFDError):
        dctx.levenshtein(dev(pts), dev(off), dev(pairs))    # Levenshtein needs one symbol per position


@pytest.mark.parametrize("dim", [2, 3])
def test_mc_pair_samples_match_oracle(dctx, dim):
    """Each Monte Carlo sample equals the oracle's float32 mirror on the
    oracle's own perturbation (one rounding) of the same noise."""
    rng = np.random.default_rng(90 + dim)
    n, m, S = 300, 200, 40
    p = np.cumsum(rng.normal(size=(n, dim)), 0).astype(np.float32)
    q = np.cumsum(rng.normal(size=(m, dim)), 0).astype(np.float32)
    zp = rng.normal(size=(S, n, dim)).astype(np.float32)
    zq = rng.normal(size=(S, m, dim)).astype(np.float32)
    sp, sq = 0.3, 0.7
    d, d2 = dctx.mc_pair(dev(p), dev(q), dev(zp), dev(zq), sp, sq)
    torch.cuda.synchronize()
    d2 = d2.cpu().numpy()
    for s in range(S):
        ps = oracle.perturb(p, zp[s], sp)
        qs = oracle.perturb(q, zq[s], sq)
        assert d2[s] == np.float32(oracle.dfd2_f32mirror(ps, qs)), s
    # sigma = 0: every sample is the unperturbed distance
    d0, d20 = dctx.mc_pair(dev(p), dev(q), dev(zp[:3]), dev(zq[:3]), 0.0, 0.0)
    torch.cuda.synchronize()
    assert np.all(d20.cpu().numpy() == np.float32(oracle.dfd2_f32mirror(p, q)))
