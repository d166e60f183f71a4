"""GPU parity of the ragged batch (dfd_batch) and the all-pairs matrix (dfd_matrix).

int32: bit-exact against the int64 oracle; float32: delta^2 bit-identical to
the float32 selection mirror and delta within 1e-6 of the float64 oracle
(tolerance derivation in test_gpu_pair.py).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2404_05708_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_TOL = 1e-6


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_batch(ctx, b, **kw):
    d, d2 = ctx.batch(dev(b.points), dev(b.offsets), dev(b.pairs), **kw)
    torch.cuda.synchronize()
    return d.cpu().numpy(), d2.cpu().numpy()


def check_f32(d, d2, b):
    mirror, _ = oracle.batch(b.points, b.offsets, b.pairs, mirror=True)
    ref, _ = oracle.batch(b.points, b.offsets, b.pairs)
    assert np.array_equal(d2, mirror), np.nonzero(d2 != mirror)[0][:10]
    want = np.sqrt(ref)
    err = np.abs(d.astype(np.float64) - want)
    assert np.all(err <= REL_TOL * np.maximum(want, 1e-300)), err.max()


def ragged_edges(dtype, dim, seed):
    """Lengths at warp/stripe edges (1, 31..33, 127..129, 255..257, 511..513)
    and lengths whose rows are spread over several stripes of fewer than
    32 * Rmax rows (160, 300, 384, 385, 600, 767, 769, 1000)."""
    rng = np.random.default_rng(seed)
    edges = [1, 2, 31, 32, 33, 63, 64, 65, 127, 128, 129, 160, 255, 256, 257, 300, 384, 385, 511, 512, 513, 600,
             767, 769, 1000]
    lens = []
    pairs = []
    for a in edges:
        for bb in edges:
            pairs.append((len(lens), len(lens) + 1))
            lens += [a, bb]
    lens = np.array(lens, np.int64)
    off = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    if dtype == "i32":
        pts = np.cumsum(rng.integers(-64, 65, size=(off[-1], dim)), axis=0).astype(np.int32)
    else:
        pts = np.cumsum(rng.normal(0, 1, size=(off[-1], dim)), axis=0).astype(np.float32)
    return workloads.Batch(points=pts, offsets=off, pairs=np.array(pairs, np.int32))


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_batch_int_edges(dctx, dim):
    b = ragged_edges("i32", dim, 80 + dim)
    _, d2 = run_batch(dctx, b)
    ref, _ = oracle.batch(b.points, b.offsets, b.pairs)
    assert np.array_equal(d2, ref), np.nonzero(d2 != ref)[0][:10]


def value_class_batch(dim, seed):
    """int32 pairs on both sides of the exact-uint32 class bound: union
    bounding boxes with one coordinate range near 46340 (int64 class: its
    square alone passes the bound), squared ranges summing just below /
    above 0x7F7FFFFF, wide curves (|c| near 2^28) that only the int64 path
    can take, and ordinary narrow pairs of one or several row stripes."""
    rng = np.random.default_rng(seed)
    curves, pairs = [], []

    def walk(n, step, start):
        return (np.cumsum(rng.integers(-step, step + 1, size=(n, dim)), axis=0) + start).astype(np.int64)

    def add_pair(a, b):
        pairs.append((len(curves), len(curves) + 1))
        curves.extend([a, b])

    for span in (46339, 46340, 46341, 46342):
        for n, m in ((40, 70), (300, 33), (513, 257)):
            a = walk(n, 50, 0)
            b = walk(m, 50, 0)
            a[0, 0], b[-1, 0] = -span // 2, span - span // 2   # fixes the union range of coordinate 0
            a[:, 0] = np.clip(a[:, 0], -span // 2, span - span // 2)
            b[:, 0] = np.clip(b[:, 0], -span // 2, span - span // 2)
            add_pair(a, b)
    # sum of squared ranges around the limit (each range < 46340)
    r = int(math.isqrt(0x7F7FFFFF // dim))
    for delta in (-1, 0, 1, 2):
        a = walk(64, 20, 0)
        b = walk(96, 20, 0)
        for k in range(dim):
            lo, hi = -(r // 2), r - r // 2 + (delta if k == 0 else 0)
            a[:, k] = np.clip(a[:, k], lo, hi)
            b[:, k] = np.clip(b[:, k], lo, hi)
            a[0, k], b[-1, k] = lo, hi
        add_pair(a, b)
    for n, m in ((50, 60), (400, 700)):
        add_pair(walk(n, 1 << 20, 1 << 28), walk(m, 1 << 20, -(1 << 28)))
    # ordinary narrow pairs, one and several row stripes
    for n, m in ((1, 5), (32, 33), (257, 300), (600, 900), (1000, 40)):
        add_pair(walk(n, 64, 0), walk(m, 64, 0))
    lens = np.array([len(c) for c in curves], np.int64)
    off = np.zeros(len(curves) + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    pts = np.concatenate(curves).astype(np.int32)
    return workloads.Batch(points=pts, offsets=off, pairs=np.array(pairs, np.int32))


@pytest.mark.parametrize("dim", [1, 2, 3, 4])
def test_batch_int_value_classes_bit_exact(dctx, dim):
    """Pairs on both sides of the uint32-bits class bound (and far beyond)
    give the int64 oracle's values bit for bit, through the batch and the
    matrix entry points."""
    b = value_class_batch(dim, 30 + dim)
    ref, _ = oracle.batch(b.points, b.offsets, b.pairs)
    d, d2 = run_batch(dctx, b)
    assert np.array_equal(d2, ref), np.nonzero(d2 != ref)[0][:10]
    assert np.all(d == np.sqrt(ref.astype(np.float64)))
    # the matrix over the last 24 curves mixes both classes
    nc = 24
    c0 = len(b.offsets) - 1 - nc
    sub = workloads.Batch(points=b.points[b.offsets[c0]:], offsets=b.offsets[c0:] - b.offsets[c0],
                          pairs=np.zeros((0, 2), np.int32))
    md, md2 = dctx.matrix(dev(sub.points), dev(sub.offsets))
    torch.cuda.synchronize()
    iu = np.triu_indices(nc, 1)
    want, _ = oracle.batch(sub.points, sub.offsets, np.stack(iu, 1).astype(np.int32))
    assert np.array_equal(md2.cpu().numpy(), want)


@pytest.mark.parametrize("dim", [2, 3, 5, 8, 16])
def test_batch_float_edges(dctx, dim):
    b = ragged_edges("f32", dim, 90 + dim)
    d, d2 = run_batch(dctx, b)
    check_f32(d, d2, b)


def test_batch_ragged_int_full_size(dctx):
    """65,536 pairs, lengths U{16..512}, int32 2-D walks: every pair bit-exact."""
    b = workloads.ragged_int_batch()
    d, d2 = run_batch(dctx, b)
    ref, _ = oracle.batch(b.points, b.offsets, b.pairs)
    assert np.array_equal(d2, ref), np.nonzero(d2 != ref)[0][:10]
    assert np.array_equal(d, np.sqrt(ref.astype(np.float64)))


def test_batch_host_equals_device_batch(dctx):
    """dfd_batch_host (points copied in slices, pairs run per slice) equals
    dfd_batch bit for bit, from page-locked and from pageable points."""
    b = workloads.ragged_int_batch()   # 277 MB of points: several copy slices
    d_dev, d2_dev = run_batch(dctx, b)
    pinned = torch.from_numpy(b.points).pin_memory().numpy()
    for pts in (pinned, b.points):
        d, d2 = dctx.batch_host(pts, b.offsets, b.pairs)
        assert np.array_equal(d2, d2_dev), np.nonzero(d2 != d2_dev)[0][:10]
        assert np.array_equal(d, d_dev)


def test_batch_host_boxes_across_slices(dctx):
    """A pair whose curves sit in two copy slices takes its int32 value class
    from boxes that two launches build (on two streams).  The same context
    first runs small coordinates (every pair narrow), then the same curves
    with every third one scaled by 4096 (pairs with it need the int64 class):
    a launch that read the first call's boxes would take the narrow class and
    overflow."""
    b = workloads.ragged_int_batch(n_pairs=32768)   # 138 MB of points: three copy slices
    n = b.n_curves
    pairs = np.stack([np.arange(0, n - 1), np.arange(1, n)], 1).astype(np.int32)   # neighbours: every boundary
    d, d2 = dctx.batch_host(b.points, b.offsets, pairs)
    d_dev, d2_dev = run_batch(dctx, workloads.Batch(points=b.points, offsets=b.offsets, pairs=pairs))
    assert np.array_equal(d2, d2_dev)
    big = b.points.copy()
    ln = np.diff(b.offsets)
    scale = np.repeat(np.where(np.arange(n) % 3 == 0, 4096, 1), ln).astype(np.int32)
    big *= scale[:, None]
    bb = workloads.Batch(points=big, offsets=b.offsets, pairs=pairs)
    d, d2 = dctx.batch_host(big, b.offsets, pairs)
    d_dev, d2_dev = run_batch(dctx, bb)
    assert np.array_equal(d2, d2_dev), np.nonzero(d2 != d2_dev)[0][:10]
    # the pairs across each third of the points, against the oracle
    cuts = np.searchsorted(b.offsets, [b.offsets[-1] * k // 3 for k in (1, 2)])
    idx = np.unique(np.concatenate([np.arange(c - 3, c + 3) for c in cuts]))
    want, _ = oracle.batch(big, b.offsets, pairs[idx])
    assert np.array_equal(d2[idx], want)
    scaled = (pairs[idx] % 3 == 0).any(axis=1)
    assert scaled.any() and np.all(want[scaled] > 2 ** 31)   # these need the int64 class


@pytest.mark.parametrize("dtype", ["f32", "i32"])
def test_batch_wide_pairs_row_buffer(dtype):
    """Pairs that run several stripes (2-D: more than 256 rows) with a row
    wider than one warp's buffer (4096 columns by default) in both
    orientations run as CTA teams, whose wrap-around row has the CTA's eight
    warp buffers; the other long pairs take the long curve as their rows,
    so that their columns fit (e.g. 300 x 5000, 4097 x 520).  With the
    default buffer every pair equals the oracle and the error word stays
    clear; widened buffers (the pairs then run one warp each) and
    dfd_batch_host give the same bits."""
    from paper_2404_05708_gb300 import dfd
    ctx = dfd.Context(0)
    rng = np.random.default_rng(31)
    lens = np.array([300, 5000, 6100, 280, 100, 9000, 700, 4096, 4097, 520])
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    if dtype == "f32":
        pts = np.cumsum(rng.normal(0, 1, size=(int(off[-1]), 2)), axis=0).astype(np.float32)
    else:
        pts = np.cumsum(rng.integers(-64, 65, size=(int(off[-1]), 2)), axis=0).astype(np.int32)
    pairs = np.array([[0, 1], [1, 2], [3, 5], [4, 5], [6, 7], [6, 8], [8, 9], [2, 1], [7, 9]], np.int32)
    ln = lens[pairs]
    long_ = (ln.min(axis=1) > 256) & (ln.max(axis=1) > 4096)   # several stripes, one curve wider than 4096
    wide = ln.min(axis=1) > 4096                                # wider than 4096 both ways
    assert long_.sum() == 6 and wide.sum() == 2
    b = workloads.Batch(points=pts, offsets=off, pairs=pairs)
    want, _ = oracle.batch(pts, off, pairs, mirror=(dtype == "f32"))
    code = dfd.DFD_F32 if dtype == "f32" else dfd.DFD_I32
    for mode in (1, 2):   # only the wide pairs as teams / every multi-stripe pair
        ctx.set_batch_team(code, 2, mode)
        d, d2 = run_batch(ctx, b)
        assert ctx.get_error() == 0
        assert np.array_equal(d2, want)
    ctx.set_batch_team(code, 2, 0)
    with pytest.raises(dfd.DFDError):
        ctx.set_batch_row_buffer(1000)
    ctx.set_batch_row_buffer(9000)
    d, d2 = run_batch(ctx, b)
    assert ctx.get_error() == 0
    assert np.array_equal(d2, want)
    ctx.close()
    ctx = dfd.Context(0)
    d, d2 = ctx.batch_host(pts, off, pairs)
    assert np.array_equal(d2, want)
    ctx.close()


def team_edges(dtype, dim, seed):
    """Pairs on both sides of every size-class edge of the ragged batch
    (2-D: 32 * Rmax = 256 rows per stripe; a team of 8 warps spreads up to
    8 stripes of up to 256 rows, 2048 rows, one stripe each, and cycles
    beyond; one warp's row buffer holds 4096 columns, a CTA's 32,768):
    rows 255 / 256 (one stripe), 257 (two), 1024 (8 stripes of 128), 2047,
    2048 (8 of 256), 2049 and 2600 (cycling through the CTA buffer), against
    columns 260 .. 40,000; 2049 x 33,000 and 2600 x 40,000 run with the long
    curve as their rows (129 and 157 stripes of one warp), and 32,800 x
    33,000 is wider than a CTA's buffers both ways: it runs last, on every
    buffer of the launch."""
    rng = np.random.default_rng(seed)
    rows = [255, 256, 257, 1024, 2047, 2048, 2049, 2600]
    cols = [260, 1500, 4095, 4097, 9000]
    shapes = [(r, c) for r in rows for c in cols if c >= r] + [(2048, 2049), (2049, 2049), (2600, 2601),
                                                                  (257, 32768), (2049, 33000), (2600, 40000),
                                                                  (32800, 33000)]
    lens, pairs = [], []
    for k, (r, c) in enumerate(shapes):
        a, bb = (r, c) if k % 2 == 0 else (c, r)   # both orders of (rows, cols)
        pairs.append((len(lens), len(lens) + 1))
        lens += [a, bb]
    lens = np.array(lens, np.int64)
    off = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=off[1:])
    if dtype == "i32":
        pts = np.cumsum(rng.integers(-64, 65, size=(off[-1], dim)), axis=0).astype(np.int32)
        # two pairs in the exact int64 value class: 255 x 1500 (one warp) and 1024 x 4097 (a team)
        for k in (1, shapes.index((1024, 4097))):
            pts[off[2 * k]:off[2 * k + 2]] *= 4096
    else:
        pts = np.cumsum(rng.normal(0, 1, size=(off[-1], dim)), axis=0).astype(np.float32)
    return workloads.Batch(points=pts, offsets=off, pairs=np.array(pairs, np.int32))


@pytest.mark.parametrize("dtype,dim", [("i32", 2), ("f32", 2), ("f32", 3)])
def test_batch_team_modes_bit_identical(dctx, dtype, dim):
    """Every team mode (auto; only wide pairs; every multi-stripe pair)
    gives every pair the oracle's value bit for bit (float32: the selection
    mirror), on both sides of each size-class edge, with a clear error word."""
    from paper_2404_05708_gb300 import dfd
    code = dfd.DFD_I32 if dtype == "i32" else dfd.DFD_F32
    b = team_edges(dtype, dim, 150 + dim)
    want, _ = oracle.batch(b.points, b.offsets, b.pairs, mirror=(dtype == "f32"))
    outs = []
    for mode in (0, 1, 2):
        dctx.set_batch_team(code, dim, mode)
        d, d2 = run_batch(dctx, b)
        assert dctx.get_error() == 0
        assert np.array_equal(d2, want), (mode, np.nonzero(d2 != want)[0][:10])
        outs.append(d)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    dctx.set_batch_team(code, dim, 0)


@pytest.mark.parametrize("n_team", [32, 76, 77])
def test_batch_team_halves_on_two_ctas(dctx, n_team):
    """When every team pair's two halves fit one per SM (at most 76 team
    pairs on 152 SMs), each half runs on its own CTA and the CTA that
    finishes second meets the rows; 77 team pairs run whole in one CTA
    each.  Team pairs (every multi-stripe pair: 600 to 1,100 rows) beside
    one-warp pairs (40 to 250 rows), float32 against the selection mirror
    and int32 (both value classes) against the oracle, bit for bit."""
    from paper_2404_05708_gb300 import dfd
    rng = np.random.default_rng(170 + n_team)
    team_lens = rng.integers(600, 1101, size=2 * n_team)
    warp_lens = rng.integers(40, 251, size=2 * 200)
    lens = np.concatenate([team_lens, warp_lens]).astype(np.int64)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    pairs = np.arange(len(lens), dtype=np.int32).reshape(-1, 2)
    for dtype in ("f32", "i32"):
        if dtype == "f32":
            pts = np.cumsum(rng.normal(0, 1, size=(int(off[-1]), 2)), axis=0).astype(np.float32)
        else:
            pts = np.cumsum(rng.integers(-64, 65, size=(int(off[-1]), 2)), axis=0).astype(np.int32)
            pts[off[2]:off[4]] *= 4096   # team pair 1 in the exact int64 class
        b = workloads.Batch(points=pts, offsets=off, pairs=pairs)
        want, _ = oracle.batch(pts, off, pairs, mirror=(dtype == "f32"))
        code = dfd.DFD_F32 if dtype == "f32" else dfd.DFD_I32
        dctx.set_batch_team(code, 2, 2)
        for _ in range(2):   # the meet words start at zero in every launch
            d, d2 = run_batch(dctx, b)
            assert dctx.get_error() == 0
            assert np.array_equal(d2, want), np.nonzero(d2 != want)[0][:10]
        dctx.set_batch_team(code, 2, 0)


def test_batch_team_16d_float(dctx):
    """16-D points (4 rows per lane, 128-column team rings): a team of 8
    stripes of 128 rows, one cycling through 9 stripes, and one pair wider
    than a warp's row buffer both ways (4200 x 5000)."""
    from paper_2404_05708_gb300 import dfd
    rng = np.random.default_rng(160)
    lens = np.array([1024, 1100, 1025, 1200, 4200, 5000, 130, 700])
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    pts = np.cumsum(rng.normal(0, 1, size=(int(off[-1]), 16)), axis=0).astype(np.float32)
    pairs = np.array([[0, 1], [2, 3], [4, 5], [6, 7], [1, 2]], np.int32)
    b = workloads.Batch(points=pts, offsets=off, pairs=pairs)
    for mode in (1, 2):
        dctx.set_batch_team(dfd.DFD_F32, 16, mode)
        d, d2 = run_batch(dctx, b)
        assert dctx.get_error() == 0
        check_f32(d, d2, b)
    dctx.set_batch_team(dfd.DFD_F32, 16, 0)


def test_batch_host_slices_without_pairs_and_checks():
    """Pairs that reference only late curves (early copy slices run no
    launch) still see every curve boxed and checked: results equal
    dfd_batch's, and a NaN in a curve no pair references is rejected as by
    dfd_batch."""
    from paper_2404_05708_gb300 import dfd
    ctx = dfd.Context(0)
    rng = np.random.default_rng(21)
    lens = rng.integers(200, 700, size=30000)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    pts = np.cumsum(rng.normal(0, 1, size=(int(off[-1]), 2)), axis=0).astype(np.float32)   # ~108 MB
    hi = np.arange(27000, 30000)
    pairs = np.stack([rng.choice(hi, 600), rng.choice(hi, 600)], 1).astype(np.int32)
    pairs = np.concatenate([pairs, [[0, 29999], [5, 12]]]).astype(np.int32)
    b = workloads.Batch(points=pts, offsets=off, pairs=pairs)
    d_dev, d2_dev = run_batch(ctx, b)
    d, d2 = ctx.batch_host(pts, off, pairs)
    assert np.array_equal(d2, d2_dev) and np.array_equal(d, d_dev)
    mirror, _ = oracle.batch(pts, off, pairs[-2:], mirror=True)
    assert np.array_equal(d2[-2:], mirror)
    bad = pts.copy()
    bad[off[100] + 3, 1] = np.nan   # curve 100: in no pair
    with pytest.raises(dfd.DFDError):
        ctx.batch_host(bad, off, pairs[:600])
    with pytest.raises(dfd.DFDError):
        ctx.batch_host(pts, off, np.array([[0, 30000]], np.int32))   # id out of range: host check
    ctx.close()


@pytest.mark.parametrize("dtype,dim", [("i32", 2), ("f32", 3)])
def test_batch_packing_orders_agree_and_autotune(dctx, dtype, dim):
    """Both packing orders give identical results; the autotuner keeps one."""
    from paper_2404_05708_gb300 import dfd
    code = dfd.DFD_I32 if dtype == "i32" else dfd.DFD_F32
    b = ragged_edges(dtype, dim, 140 + dim)
    outs = []
    for order in (0, 1):
        dctx.set_batch_order(code, dim, order)
        outs.append(run_batch(dctx, b))
    assert np.array_equal(outs[0][1], outs[1][1]) and np.array_equal(outs[0][0], outs[1][0])
    best = dctx.batch_autotune(dev(b.points), dev(b.offsets), dev(b.pairs))
    assert best in (0, 1)
    d, d2 = run_batch(dctx, b)
    assert np.array_equal(d2, outs[0][1])
    if dtype == "i32":
        ref, _ = oracle.batch(b.points, b.offsets, b.pairs)
        assert np.array_equal(d2, ref)
    else:
        check_f32(d, d2, b)
    dctx.set_batch_order(code, dim, 0)


def test_batch_graph_replay_updates_with_buffers(dctx):
    b = workloads.ragged_int_batch(n_pairs=3000, seed=41)
    pts, off, pr = dev(b.points), dev(b.offsets), dev(b.pairs)
    g, d, d2 = dctx.batch(pts, off, pr, capture=True)
    torch.cuda.synchronize()
    ref, _ = oracle.batch(b.points, b.offsets, b.pairs)
    assert np.array_equal(d2.cpu().numpy(), ref)
    # new contents in the same buffers, then replay
    b2 = workloads.ragged_int_batch(n_pairs=3000, seed=41)
    b2.points = (b2.points * 3 - 7).astype(np.int32)
    pts.copy_(dev(b2.points))
    d2.zero_()
    g.launch()
    g.launch()
    torch.cuda.synchronize()
    ref2, _ = oracle.batch(b2.points, b2.offsets, b2.pairs)
    assert np.array_equal(d2.cpu().numpy(), ref2)
    g.close()


def test_batch_invalid_ids_are_reported(dctx):
    b = ragged_edges("i32", 2, 7)
    pairs = b.pairs.copy()
    pairs[5, 1] = 10 ** 6
    d, d2 = dctx.batch(dev(b.points), dev(b.offsets), dev(pairs))
    torch.cuda.synchronize()
    assert dctx.get_error() == 1          # DFD_ERR_INVALID_ARG
    assert dctx.get_error() == 0


def test_batch_host_invalid_ids_are_reported():
    """dfd_batch_host returns DFD_ERR_INVALID_ARG for an id out of range:
    found by the last launch's device-side plan when every curve fits the
    row buffers, and by the host pass when one is longer; a good call after
    either returns the oracle's values."""
    from paper_2404_05708_gb300 import dfd
    ctx = dfd.Context(0)
    try:
        b = ragged_edges("i32", 2, 9)
        want, _ = oracle.batch(b.points, b.offsets, b.pairs)
        for lens_long in (False, True):
            off, pts = b.offsets, b.points
            if lens_long:   # one extra curve of 5,000 points (> 4,096 columns), not in any pair
                extra = np.cumsum(np.ones((5000, 2), np.int64), axis=0).astype(np.int32)
                pts = np.concatenate([pts, extra])
                off = np.concatenate([off, [off[-1] + 5000]]).astype(np.int64)
            pairs = b.pairs.copy()
            pairs[3, 0] = len(off) + 7
            with pytest.raises(dfd.DFDError) as e:
                ctx.batch_host(pts, off, pairs)
            assert e.value.status == dfd.STATUS_CODE["DFD_ERR_INVALID_ARG"], lens_long
            d, d2 = ctx.batch_host(pts, off, b.pairs)
            assert np.array_equal(d2, want), lens_long
    finally:
        ctx.close()


@pytest.mark.parametrize("dim", [2, 3, 8])
def test_batch_int_range_check(dctx, dim):
    # |c| <= 2^30 - 1 (dim 2) or less is required of every coordinate; the
    # per-curve boxes decide it, so a coordinate outside must be reported
    # wherever it sits: the first point, past the first load round of a long
    # curve, the last point, either sign.
    lens = np.array([5, 300, 700, 33, 1000], np.int64)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    rng = np.random.default_rng(60 + dim)
    base = np.cumsum(rng.integers(-64, 65, size=(off[-1], dim)), axis=0).astype(np.int32)
    pairs = np.array([[0, 1], [2, 3], [4, 0], [1, 2]], np.int32)
    outside = (1 << 30) + 5
    for row, k, val in [(0, 0, outside), (off[1] + 299, dim - 1, -outside), (off[2] + 650, 1, outside),
                        (off[-1] - 1, 0, -outside), (off[4] + 513, dim - 1, 2 ** 31 - 1)]:
        pts = base.copy()
        pts[row, k] = val
        dctx.batch(dev(pts), dev(off), dev(pairs))
        torch.cuda.synchronize()
        assert dctx.get_error() == 2, (row, k, val)   # DFD_ERR_RANGE, then cleared
        assert dctx.get_error() == 0
    # large coordinates inside the limit run (int64 class) and stay exact
    pts = base.copy()
    pts[off[1] + 299, 0] = 1 << 28
    pts[off[4] + 999, dim - 1] = -(1 << 28)
    b = workloads.Batch(points=pts, offsets=off, pairs=pairs)
    d, d2 = run_batch(dctx, b)
    assert dctx.get_error() == 0
    want, _ = oracle.batch(b.points, b.offsets, b.pairs)
    assert np.array_equal(d2, want)


# ----------------------------------------------------------------- matrix

def condensed_oracle(b):
    n = b.n_curves
    ii, jj = np.triu_indices(n, k=1)
    pairs = np.stack([ii, jj], axis=1).astype(np.int32)
    return oracle.batch(b.points, b.offsets, pairs), oracle.batch(b.points, b.offsets, pairs, mirror=True)


def test_matrix_small_float16d(dctx):
    b = workloads.ar1_curves(n_curves=70, seed=51)
    d, d2 = dctx.matrix(dev(b.points), dev(b.offsets))
    torch.cuda.synchronize()
    (ref, _), (mirror, _) = condensed_oracle(b)
    assert np.array_equal(d2.cpu().numpy(), mirror)
    assert np.all(np.abs(d.cpu().numpy() - np.sqrt(ref)) <= REL_TOL * np.sqrt(ref))


def test_matrix_small_int(dctx):
    rng = np.random.default_rng(52)
    lens = rng.integers(1, 300, size=45)
    off = np.zeros(46, np.int64)
    np.cumsum(lens, out=off[1:])
    pts = np.cumsum(rng.integers(-100, 101, size=(off[-1], 3)), axis=0).astype(np.int32)
    b = workloads.Batch(points=pts, offsets=off, pairs=np.zeros((0, 2), np.int32))
    _, d2 = dctx.matrix(dev(pts), dev(off))
    torch.cuda.synchronize()
    (ref, _), _ = condensed_oracle(b)
    assert np.array_equal(d2.cpu().numpy(), ref)


@pytest.mark.parametrize("dtype,dim", [("i32", 2), ("f32", 3), ("f32", 16)])
def test_batch_tile_shapes_bit_identical(dctx, dtype, dim):
    """Every tile shape of the one-warp pairs (rows per lane cap 1 .. Rmax,
    CTAs per SM 1 or all) gives every pair the same bits, on both sides of
    the stripe edges; the autotuner records a valid shape that reproduces them."""
    from paper_2404_05708_gb300 import dfd
    code = dfd.DFD_I32 if dtype == "i32" else dfd.DFD_F32
    b = ragged_edges(dtype, dim, 170 + dim)
    want, _ = oracle.batch(b.points, b.offsets, b.pairs, mirror=(dtype == "f32"))
    rm_full = 8 if dim <= 4 else 4
    for rm in (1, 2, 3, rm_full):
        for cp in (0, 1):
            dctx.set_batch_shape(code, dim, rm, cp)
            for team in (1, 2):
                dctx.set_batch_team(code, dim, team)
                _, d2 = run_batch(dctx, b)
                assert dctx.get_error() == 0
                assert np.array_equal(d2, want), (rm, cp, team, np.nonzero(d2 != want)[0][:10])
    dctx.set_batch_shape(code, dim, 0, 0)
    dctx.set_batch_team(code, dim, 0)
    order = dctx.batch_autotune(dev(b.points), dev(b.offsets), dev(b.pairs))
    o, team, rm, cp = dctx.batch_tuned(code, dim)
    assert o == order and team in (1, 2) and rm in (rm_full // 2, rm_full) and cp in (1, 2)
    _, d2 = run_batch(dctx, b)
    assert np.array_equal(d2, want)
    dctx.set_batch_shape(code, dim, 0, 0)
    dctx.set_batch_team(code, dim, 0)
    dctx.set_batch_order(code, dim, 0)


def test_matrix_tile_shapes_bit_identical(dctx):
    """The matrix under every tile shape equals the oracle bit for bit
    (float32 16-D: the selection mirror; int32 3-D: exact), including curves
    of 300 points that a cap of one row per lane splits into 10 stripes,
    and the autotuner records a shape."""
    from paper_2404_05708_gb300 import dfd
    bf = workloads.ar1_curves(n_curves=40, seed=53)
    _, mirror_f = condensed_oracle(bf)
    rng = np.random.default_rng(54)
    lens = rng.integers(1, 300, size=36)
    off = np.zeros(37, np.int64)
    np.cumsum(lens, out=off[1:])
    pts = np.cumsum(rng.integers(-100, 101, size=(off[-1], 3)), axis=0).astype(np.int32)
    bi = workloads.Batch(points=pts, offsets=off, pairs=np.zeros((0, 2), np.int32))
    (ref_i, _), _ = condensed_oracle(bi)
    for rm in (1, 2, 4, 8):
        for cp in (0, 1):
            dctx.set_matrix_shape(dfd.DFD_F32, 16, min(rm, 4), cp)
            dctx.set_matrix_shape(dfd.DFD_I32, 3, rm, cp)
            _, d2 = dctx.matrix(dev(bf.points), dev(bf.offsets))
            _, e2 = dctx.matrix(dev(pts), dev(off))
            torch.cuda.synchronize()
            assert dctx.get_error() == 0
            assert np.array_equal(d2.cpu().numpy(), mirror_f[0]), (rm, cp)
            assert np.array_equal(e2.cpu().numpy(), ref_i), (rm, cp)
    rm, cp = dctx.matrix_autotune(dev(pts), dev(off))
    assert (rm, cp) == dctx.matrix_tuned(dfd.DFD_I32, 3) and rm in (2, 4, 8) and cp in (1, 2)
    for code, dim in ((dfd.DFD_F32, 16), (dfd.DFD_I32, 3)):
        dctx.set_matrix_shape(code, dim, 0, 0)


def test_matrix_full_size_sampled(dctx):
    """4096 curves, 16-D AR(1), lengths U{64..256}: 8,386,560 pairs, 400 sampled entries vs the oracle."""
    b = workloads.ar1_curves()
    d, d2 = dctx.matrix(dev(b.points), dev(b.offsets))
    torch.cuda.synchronize()
    n = b.n_curves
    rng = np.random.default_rng(53)
    ks = rng.integers(0, n * (n - 1) // 2, size=400)
    # decode k -> (i, j) on the host, independently of the kernel
    starts = np.array([i * (2 * n - i - 1) // 2 for i in range(n)], np.int64)
    ii = np.searchsorted(starts, ks, side="right") - 1
    jj = ks - starts[ii] + ii + 1
    pairs = np.stack([ii, jj], axis=1).astype(np.int32)
    ref, _ = oracle.batch(b.points, b.offsets, pairs)
    mirror, _ = oracle.batch(b.points, b.offsets, pairs, mirror=True)
    got2 = d2.cpu().numpy()[ks]
    got = d.cpu().numpy()[ks]
    assert np.array_equal(got2, mirror)
    assert np.all(np.abs(got - np.sqrt(ref)) <= REL_TOL * np.sqrt(ref))


def test_wide_pairs_outside_the_batch_get_nan_and_an_error(dctx):
    """The decider, the DTW / Levenshtein variants and the matrix run one warp
    per pair with a 4096-column row buffer: a pair of several stripes that is
    wider than the buffer in both orientations gets NaN (float) / -1 (int64)
    outputs, never stale memory, and DFD_ERR_UNSUPPORTED in the error word;
    the other pairs are exact, among them 260 x 5000 points, which runs with
    the long curve as its rows (its columns then fit)."""
    from paper_2404_05708_gb300 import dfd
    rng = np.random.default_rng(180)
    lens = np.array([4200, 5000, 100, 260])
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    pts = np.cumsum(rng.normal(0, 1, size=(int(off[-1]), 2)), axis=0).astype(np.float32)
    pairs = np.array([[0, 1], [0, 2], [2, 3], [3, 1]], np.int32)   # pair 0 is wide both ways
    wide = np.array([True, False, False, False])
    P, O, Q = dev(pts), dev(off), dev(pairs)
    mirror, _ = oracle.batch(pts, off, pairs, mirror=True)
    unsupported = dfd.STATUS_CODE["DFD_ERR_UNSUPPORTED"]

    d2, within, _ = dctx.decide(P, O, Q, 1e12)
    torch.cuda.synchronize()
    assert dctx.get_error() == unsupported
    d2, within = d2.cpu().numpy(), within.cpu().numpy()
    assert np.all(np.isnan(d2[wide])) and np.all(within[wide] == 0)
    assert np.array_equal(d2[~wide], mirror[~wide]) and np.all(within[~wide] == 1)

    out = dctx.dtw(P, O, Q)
    torch.cuda.synchronize()
    assert dctx.get_error() == unsupported
    out = out.cpu().numpy()
    want = np.array([oracle.dtw_f32mirror(pts[off[a]:off[a + 1]], pts[off[b]:off[b + 1]]) for a, b in pairs],
                    np.float32)
    assert np.all(np.isnan(out[wide])) and np.array_equal(out[~wide], want[~wide])

    sym = rng.integers(0, 4, size=(int(off[-1]), 1)).astype(np.int32)
    lev = dctx.levenshtein(dev(sym), O, Q)
    torch.cuda.synchronize()
    assert dctx.get_error() == unsupported
    lev = lev.cpu().numpy()
    assert np.all(lev[wide] == -1)
    for k in np.nonzero(~wide)[0]:
        a, b = pairs[k]
        assert lev[k] == oracle.levenshtein(sym[off[a]:off[a + 1], 0], sym[off[b]:off[b + 1], 0])

    d, dm2 = dctx.matrix(P, O)
    torch.cuda.synchronize()
    assert dctx.get_error() == unsupported
    ii, jj = np.triu_indices(4, k=1)
    mat_pairs = np.stack([ii, jj], 1).astype(np.int32)
    mwant, _ = oracle.batch(pts, off, mat_pairs, mirror=True)
    mwide = np.minimum(lens[ii], lens[jj]) > 4096
    dm2 = dm2.cpu().numpy()
    assert mwide.sum() == 1 and np.all(np.isnan(dm2[mwide])) and np.array_equal(dm2[~mwide], mwant[~mwide])
