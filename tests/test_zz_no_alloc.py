"""dfd_pair_noalloc: the distance without any device allocation.

Some users of this library cannot let it call cudaMalloc: their process's
device memory is reserved up front by another allocator (a framework's
caching pool, a serving engine under a fixed HBM budget), or they call it
from latency-critical loops where a cudaMalloc / cudaFree, which can
synchronise the whole device, is not acceptable.  dfd_pair_noalloc serves
them: no context, no allocation, its scratch in a fixed array inside the
library's device image.  These tests call it through the C ABI and check it
against the ordinary entry point, dfd_pair, on consecutive calls.

This file is named to be collected last, so a run that stops at the first
failure has already run every other test; it also passes on its own.
"""
import numpy as np
import pytest

from paper_2404_05708_gb300 import dfd, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(p, q, dtype_code, d_out, d2_out):
    s = torch.cuda.current_stream().cuda_stream
    st = dfd.dfd_pair_noalloc(0, dtype_code, p.shape[1], p.data_ptr(), p.shape[0], q.data_ptr(), q.shape[0],
                              d_out.data_ptr(), d2_out.data_ptr(), s)
    torch.cuda.synchronize()
    return st


def _existing(ctx, p, q):
    d, d2 = ctx.pair(p, q)
    torch.cuda.synchronize()
    return d.item(), d2.item()


def test_noalloc_matches_dfd_pair_on_consecutive_calls(dctx):
    rng = np.random.default_rng(70)
    # call 1: float32, 3-D
    p1, q1 = workloads.warped_long_pair(3001, 2500, dim=3, seed=71)
    P1, Q1 = torch.from_numpy(p1).cuda(), torch.from_numpy(q1).cuda()
    d1 = torch.empty(1, dtype=torch.float32, device="cuda")
    d21 = torch.empty(1, dtype=torch.float32, device="cuda")
    assert _noalloc(P1, Q1, dfd.DFD_F32, d1, d21) == 0
    want_d, want_d2 = _existing(dctx, P1, Q1)
    assert d21.item() == want_d2 and d1.item() == want_d

    # call 2: int32, 2-D, different sizes (the array keeps the last call's contents)
    p2 = np.cumsum(rng.integers(-64, 65, size=(1800, 2)), axis=0).astype(np.int32)
    q2 = np.cumsum(rng.integers(-64, 65, size=(2200, 2)), axis=0).astype(np.int32)
    P2, Q2 = torch.from_numpy(p2).cuda(), torch.from_numpy(q2).cuda()
    d2 = torch.empty(1, dtype=torch.float64, device="cuda")
    d22 = torch.empty(1, dtype=torch.int64, device="cuda")
    assert _noalloc(P2, Q2, dfd.DFD_I32, d2, d22) == 0
    want_d, want_d2 = _existing(dctx, P2, Q2)
    assert d22.item() == want_d2 and d2.item() == want_d

    # call 3: call 1 again; device free memory must not move across it
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    assert _noalloc(P1, Q1, dfd.DFD_F32, d1, d21) == 0
    free_after = torch.cuda.mem_get_info()[0]
    assert free_after == free_before
    want_d, want_d2 = _existing(dctx, P1, Q1)
    assert d21.item() == want_d2 and d1.item() == want_d


def test_noalloc_falls_back_to_one_front(dctx):
    """300,000 columns of 3-D float32: one front's scratch fits the fixed
    array, two fronts' (two packed q streams) does not, so the wavefront
    runs one front; q = p + t gives delta^2 = |t|^2 exactly."""
    rng = np.random.default_rng(72)
    n = 300_000
    p = np.cumsum(rng.integers(-1, 2, size=(n, 3)), axis=0).astype(np.float32)
    t = np.array([3.0, -4.0, 12.0], np.float32)
    P, Q = torch.from_numpy(p).cuda(), torch.from_numpy(p + t).cuda()
    d = torch.empty(1, dtype=torch.float32, device="cuda")
    d2 = torch.empty(1, dtype=torch.float32, device="cuda")
    assert _noalloc(P, Q, dfd.DFD_F32, d, d2) == 0
    torch.cuda.synchronize()
    assert d2.item() == 169.0 and d.item() == 13.0
    e, e2 = dctx.pair(P, Q)   # the context path runs two fronts
    assert e2.item() == d2.item() and e.item() == d.item()


def test_noalloc_rejects_inputs_beyond_its_fixed_capacity():
    # float32 3-D needs ~36 bytes per column of q: 600,000 columns exceed 16 MiB.
    p = torch.zeros((10, 3), dtype=torch.float32, device="cuda")
    q = torch.zeros((600_000, 3), dtype=torch.float32, device="cuda")
    d = torch.empty(1, dtype=torch.float32, device="cuda")
    d2 = torch.empty(1, dtype=torch.float32, device="cuda")
    assert _noalloc(p, q, dfd.DFD_F32, d, d2) == dfd.STATUS_CODE["DFD_ERR_CAPACITY"]


def test_noalloc_device_error_leaves_outputs_unset_after_a_good_call(dctx):
    """A rejected coordinate found on the device must not yield a distance.
    The caller has no context to read the error from, so the outputs keep
    their NaN / -1 fill -- also on a pair of several bands (two fronts and
    the combine pass), right after a good call left its rows in the array."""
    p, q = workloads.warped_long_pair(3001, 2500, dim=3, seed=73)
    P, Q = torch.from_numpy(p).cuda(), torch.from_numpy(q).cuda()
    d = torch.empty(1, dtype=torch.float32, device="cuda")
    d2 = torch.empty(1, dtype=torch.float32, device="cuda")
    assert _noalloc(P, Q, dfd.DFD_F32, d, d2) == 0
    want_d, want_d2 = _existing(dctx, P, Q)
    assert d2.item() == want_d2 and d.item() == want_d
    bad = p.copy()
    bad[1700, 2] = np.nan
    assert _noalloc(torch.from_numpy(bad).cuda(), Q, dfd.DFD_F32, d, d2) == 0
    assert np.isnan(d.item()) and np.isnan(d2.item())

    rng = np.random.default_rng(74)
    pi = np.cumsum(rng.integers(-64, 65, size=(1800, 2)), axis=0).astype(np.int32)
    qi = np.cumsum(rng.integers(-64, 65, size=(2200, 2)), axis=0).astype(np.int32)
    Pi, Qi = torch.from_numpy(pi).cuda(), torch.from_numpy(qi).cuda()
    di = torch.empty(1, dtype=torch.float64, device="cuda")
    d2i = torch.empty(1, dtype=torch.int64, device="cuda")
    assert _noalloc(Pi, Qi, dfd.DFD_I32, di, d2i) == 0
    want_d, want_d2 = _existing(dctx, Pi, Qi)
    assert d2i.item() == want_d2 and di.item() == want_d
    badi = qi.copy()
    badi[5, 1] = 1 << 30   # outside the exact int32 range
    assert _noalloc(Pi, torch.from_numpy(badi).cuda(), dfd.DFD_I32, di, d2i) == 0
    assert np.isnan(di.item()) and d2i.item() == -1
    # and the next good call is unaffected
    assert _noalloc(Pi, Qi, dfd.DFD_I32, di, d2i) == 0
    assert d2i.item() == want_d2 and di.item() == want_d
