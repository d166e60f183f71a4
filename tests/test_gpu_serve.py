"""GPU tests of the continuous-batching server (dfd_server_*).

Each request's distances must be bit-identical whether it runs alone or in a
mix of other requests (and across tick boundaries, where long pairs pause
with their row state on the device), equal to dfd_pair on the same curves,
and match the oracle (float32 mirror bit-exact, float64 within 1e-6).
"""
import numpy as np
import pytest

import oracle
from paper_2404_05708_gb300 import dfd, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def pools(n=600, seed=100, hi=1500):
    p2 = workloads.serving_pool(n_curves=n, dim=2, len_lo=8, len_hi=hi, seed=seed)
    p3 = workloads.serving_pool(n_curves=n, dim=3, len_lo=8, len_hi=hi, seed=seed + 1)
    return {2: p2, 3: p3}


def make_server(ctx, pl, **kw):
    srv = dfd.Server(ctx, **kw)
    for d, b in pl.items():
        assert srv.add_candidates(b.points, b.offsets) == 0
    return srv


def requests(pl, count, seed, kmax=64, qhi=1500):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        d = int(rng.choice([2, 3]))
        n = int(rng.integers(8, qhi))
        q = np.cumsum(rng.normal(0, 1, size=(n, d)), axis=0).astype(np.float32)
        ids = rng.integers(0, pl[d].n_curves, size=int(rng.integers(1, kmax))).astype(np.int64)
        out.append((q, ids))
    return out


def expected(pl, q, ids):
    b = pl[q.shape[1]]
    pts = np.concatenate([q, b.points])
    off = np.concatenate([[0], q.shape[0] + b.offsets]).astype(np.int64)
    pairs = np.stack([np.zeros_like(ids), ids + 1], 1).astype(np.int32)
    mirror, _ = oracle.batch(pts, off, pairs, mirror=True)
    ref, _ = oracle.batch(pts, off, pairs)
    return np.sqrt(mirror.astype(np.float32)), np.sqrt(ref)


def test_alone_equals_in_mix_and_oracle(dctx):
    pl = pools()
    # long query against long candidates: several row stripes, paused between ticks
    rng = np.random.default_rng(7)
    q = np.cumsum(rng.normal(0, 1, size=(1400, 3)), axis=0).astype(np.float32)
    lens = np.diff(pl[3].offsets)
    ids = np.argsort(-lens)[:40].astype(np.int64)
    srv = make_server(dctx, pl, tick_cells=5e6, stripes_per_tick=1)
    t = srv.submit(q, ids)
    st, alone = srv.wait(t)
    assert st == 0
    alone = alone.copy()
    others = requests(pl, 60, seed=8)
    tickets = [srv.submit(a, b) for a, b in others[:30]]
    t2 = srv.submit(q, ids)
    tickets += [srv.submit(a, b) for a, b in others[30:]]
    st2, mixed = srv.wait(t2)
    assert st2 == 0
    assert np.array_equal(alone, mixed)
    for tk, (a, b) in zip(tickets, others):
        st, out = srv.wait(tk)
        assert st == 0
        mirror, ref = expected(pl, a, b)
        assert np.array_equal(out, mirror)
        assert np.all(np.abs(out - ref) <= 1e-6 * ref + 1e-30)
    mirror, ref = expected(pl, q, ids)
    assert np.array_equal(alone, mirror)
    # the same pairs through dfd_pair
    b = pl[3]
    qd = torch.from_numpy(q).cuda()
    for k in range(0, 40, 7):
        c = ids[k]
        cd = torch.from_numpy(b.points[b.offsets[c]:b.offsets[c + 1]]).cuda()
        d, _ = dctx.pair(qd, cd)
        assert d.item() == alone[k]
    s = srv.stats()
    assert s["completed"] == 62 and s["p99_ms"] >= s["p50_ms"] > 0
    srv.close()


def mixed_pool(dim, seed, n=240):
    """Mostly short curves, one in ten longer than a warp's 4096-point row buffer."""
    rng = np.random.default_rng(seed)
    lens = np.where(rng.random(n) < 0.1, rng.integers(4097, 4400, n), rng.integers(8, 600, n))
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    pts = np.cumsum(rng.normal(0, 1, size=(int(off[-1]), dim)), axis=0).astype(np.float32)
    return workloads.Batch(points=pts, offsets=off, pairs=np.zeros((0, 2), np.int32))


def test_slices_across_ticks_classes_and_long_pairs(dctx):
    # short pairs go out as per-request slices (one per cost class, split at
    # tick boundaries), multi-stripe short pairs use the warp row buffer, and
    # pairs with more stripes than a tick runs -- or wider than the buffer --
    # go out as items; every result must equal the float32 mirror bit for bit
    pl = {d: mixed_pool(d, seed=40 + d) for d in (2, 3)}
    srv = make_server(dctx, pl, tick_cells=3e7, stripes_per_tick=3, max_slots=1024)
    rng = np.random.default_rng(11)
    reqs = []
    for i in range(160):
        d = int(rng.choice([2, 3]))
        u = rng.random()
        n = int(rng.integers(8, 500)) if u < 0.6 else int(rng.integers(500, 1100)) if u < 0.95 else \
            int(rng.integers(4100, 4300))
        q = np.cumsum(rng.normal(0, 1, size=(n, d)), axis=0).astype(np.float32)
        k = int(rng.integers(1, 48)) if n < 4000 else 6
        ids = rng.integers(0, len(pl[d].offsets) - 1, size=k).astype(np.int64)
        reqs.append((q, ids))
    tickets = [srv.submit(a, b) for a, b in reqs]
    for tk, (a, b) in zip(tickets, reqs):
        st, out = srv.wait(tk, timeout_ms=120000)
        assert st == 0
        bb = pl[a.shape[1]]
        pts = np.concatenate([a, bb.points])
        off = np.concatenate([[0], a.shape[0] + bb.offsets]).astype(np.int64)
        pairs = np.stack([np.zeros_like(b), b + 1], 1).astype(np.int32)
        mirror, _ = oracle.batch(pts, off, pairs, mirror=True)
        assert np.array_equal(out, np.sqrt(mirror.astype(np.float32)))
    s = srv.stats()
    assert s["completed"] == len(reqs) and s["ticks"] > 1
    srv.close()


def test_small_memory_budget_and_few_slots_still_finish(dctx):
    pl = pools(n=300, seed=110, hi=600)
    srv = make_server(dctx, pl, mem_budget_bytes=1 << 20, max_slots=3, tick_cells=2e6, stripes_per_tick=2)
    reqs = requests(pl, 80, seed=9, kmax=20, qhi=600)
    tickets = [srv.submit(a, b) for a, b in reqs]
    for tk, (a, b) in zip(tickets, reqs):
        st, out = srv.wait(tk, timeout_ms=60000)
        assert st == 0
        mirror, _ = expected(pl, a, b)
        assert np.array_equal(out, mirror)
    srv.close()


def test_cancel(dctx):
    pl = pools(n=200, seed=120, hi=1500)
    srv = make_server(dctx, pl, tick_cells=1e6, stripes_per_tick=1, max_slots=2)
    reqs = requests(pl, 6, seed=10, kmax=200)
    tickets = [srv.submit(a, b) for a, b in reqs]
    assert srv.cancel(tickets[-1]) == 0     # still pending: cancelled at once
    assert srv.cancel(tickets[0]) == 0      # running: cancelled at the next tick boundary
    results = [srv.wait(t, timeout_ms=60000)[0] for t in tickets]
    assert results[-1] == dfd.STATUS_CODE["DFD_ERR_CANCELLED"]
    assert results[0] in (0, dfd.STATUS_CODE["DFD_ERR_CANCELLED"])
    assert all(r == 0 for r in results[1:-1])
    srv.close()


def test_invalid_requests_rejected(dctx):
    pl = pools(n=50, seed=130, hi=100)
    srv = make_server(dctx, pl)
    q = np.zeros((5, 2), np.float32)
    with pytest.raises(dfd.DFDError):
        srv.submit(q, np.array([10 ** 6], np.int64))          # unknown candidate
    with pytest.raises(dfd.DFDError):
        srv.submit(np.zeros((5, 4), np.float32), np.array([0], np.int64))   # no pool of that dim
    bad = q.copy()
    bad[2, 1] = np.inf
    with pytest.raises(dfd.DFDError):
        srv.submit(bad, np.array([0], np.int64))
    srv.close()


def test_request_and_tick_logs(dctx):
    """The per-request log has one record per completed request, its times
    in order (arrival <= submit <= lock <= admission <= first launch <=
    completion) and its cells; the per-tick log covers every tick, with
    device time and the cells of the completed requests; a stats reset
    clears both."""
    pl = pools(n=200, seed=130)
    srv = make_server(dctx, pl, tick_cells=2e6)
    reqs = requests(pl, 12, seed=131, kmax=40, qhi=600)
    t0 = srv.now()
    tickets = [srv.submit(q, ids, arrival_s=t0) for q, ids in reqs]
    for t in tickets:
        assert srv.wait(t)[0] == 0
    st = srv.stats()
    log = srv.request_log()
    assert len(log) == 12 == st["completed"]
    assert sorted(log["ticket"].tolist()) == sorted(tickets)
    eps = 1e-9
    assert np.all(log["arrival_s"] <= log["submit_s"] + eps)
    assert np.all(log["submit_s"] <= log["locked_s"] + eps)
    assert np.all(log["locked_s"] <= log["admit_s"] + eps)
    assert np.all(log["admit_s"] <= log["launch_s"] + eps)
    assert np.all(log["launch_s"] <= log["done_s"] + eps)
    by_ticket = {int(r["ticket"]): r for r in log}
    for t, (q, ids) in zip(tickets, reqs):
        r = by_ticket[t]
        lens = np.diff(pl[q.shape[1]].offsets)[ids]
        assert r["cells"] == float(np.sum(q.shape[0] * lens)) and r["k"] == len(ids) and r["n"] == q.shape[0]
    ticks = srv.tick_log()
    assert len(ticks) == st["ticks"] >= 1
    assert np.all(ticks["gpu_ms"] > 0) and np.all(ticks["build_s"] <= ticks["launched_s"])
    assert np.all(ticks["launched_s"] <= ticks["retired_s"])
    assert abs(ticks["cells"].sum() - st["cells"]) <= 1e-6 * st["cells"]
    srv.reset_stats()
    assert len(srv.request_log()) == 0 and len(srv.tick_log()) == 0
    srv.close()
