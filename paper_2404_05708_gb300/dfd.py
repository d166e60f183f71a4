"""Thin Python binding of libdfd.so (include/dfd.h).

Argument marshalling only: every step of the distance computation runs in
the CUDA library.  If the library has not been built, or no CUDA device is
usable, the calls raise; there is no CPU fallback.

Low-level functions keep the C names and take raw integers (device
pointers, sizes, a cudaStream_t handle).  ``Context`` wraps them for torch
tensors: ``ctx.pair(p, q)`` with float32 or int32 CUDA tensors of shape
``[n, dim]`` / ``[m, dim]`` returns ``(dist, dist2)`` tensors on the device.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_build", "libdfd.so")

DFD_F32, DFD_I32 = 0, 1
DFD_VARIANT_DTW, DFD_VARIANT_LEVENSHTEIN = 1, 2
STATUS = {
    0: "DFD_OK", 1: "DFD_ERR_INVALID_ARG", 2: "DFD_ERR_RANGE", 3: "DFD_ERR_NONFINITE", 4: "DFD_ERR_OOM",
    5: "DFD_ERR_CUDA", 6: "DFD_ERR_TIMEOUT", 7: "DFD_ERR_BUSY", 8: "DFD_ERR_CANCELLED", 9: "DFD_ERR_NOT_READY",
    10: "DFD_ERR_UNSUPPORTED", 11: "DFD_ERR_CAPACITY",
}
STATUS_CODE = {v: k for k, v in STATUS.items()}


class DFDError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = int(status)
        super().__init__(f"{where}: {STATUS.get(self.status, self.status)}")


class Options(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_size_t), ("mem_budget_bytes", ctypes.c_size_t),
                ("max_slots", ctypes.c_int), ("wait_timeout_ms", ctypes.c_double), ("check_inputs", ctypes.c_int)]


class WaveShape(ctypes.Structure):
    _fields_ = [("rows_per_lane", ctypes.c_int), ("warps", ctypes.c_int), ("ctas", ctypes.c_int)]


class ServerOptions(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_size_t), ("mem_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int),
                ("tick_cells", ctypes.c_double), ("stripes_per_tick", ctypes.c_int)]


class RequestRecord(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("arrival_s", ctypes.c_double), ("submit_s", ctypes.c_double),
                ("admit_s", ctypes.c_double), ("launch_s", ctypes.c_double), ("done_s", ctypes.c_double),
                ("cells", ctypes.c_double), ("n", ctypes.c_int), ("k", ctypes.c_int), ("dim", ctypes.c_int),
                ("pad", ctypes.c_int), ("locked_s", ctypes.c_double)]


class ServingStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("cancelled", ctypes.c_uint64), ("ticks", ctypes.c_uint64),
                ("cells", ctypes.c_double), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("gpu_busy_ms", ctypes.c_double), ("gcups_busy", ctypes.c_double),
                ("gcups_wall", ctypes.c_double), ("arena_used_bytes", ctypes.c_size_t)]


_lock = threading.Lock()
_lib = None

_VP = ctypes.c_void_p
_I64 = ctypes.c_int64
_INT = ctypes.c_int

# name -> argtypes (all return int status unless listed in _RESTYPE)
_SIGS = {
    "dfd_options_default": [ctypes.POINTER(Options)],
    "dfd_status_string": [_INT],
    "dfd_context_create": [ctypes.POINTER(_VP), _INT, ctypes.POINTER(Options)],
    "dfd_context_destroy": [_VP],
    "dfd_get_error": [_VP],
    "dfd_pair": [_VP, _INT, _INT, _VP, _I64, _VP, _I64, _VP, _VP, _VP],
    "dfd_pair_reference": [_VP, _INT, _INT, _VP, _I64, _VP, _I64, _VP, _VP, _VP],
    "dfd_pair_host": [_VP, _INT, _INT, _VP, _I64, _VP, _I64, _VP, _VP],
    "dfd_pair_shaped": [_VP, _INT, _INT, _VP, _I64, _VP, _I64, _VP, _VP, _VP, ctypes.POINTER(WaveShape)],
    "dfd_pair_plan": [_VP, _INT, _INT, _I64, _I64, ctypes.POINTER(WaveShape)],
    "dfd_pair_autotune": [_VP, _INT, _INT, _VP, _I64, _VP, _I64, _VP, ctypes.POINTER(WaveShape)],
    "dfd_autotune_save": [_VP, ctypes.c_char_p],
    "dfd_autotune_load": [_VP, ctypes.c_char_p],
    "dfd_debug_bounded_wait": [_VP, ctypes.c_double],
    "dfd_pair_noalloc": [_INT, _INT, _INT, _VP, _I64, _VP, _I64, _VP, _VP, _VP],
    "dfd_batch": [_VP, _INT, _INT, _VP, _VP, _I64, _VP, _I64, _VP, _VP, _VP],
    "dfd_batch_host": [_VP, _INT, _INT, _VP, _VP, _I64, _VP, _I64, _VP, _VP],
    "dfd_batch_autotune": [_VP, _INT, _INT, _VP, _VP, _I64, _VP, _I64, _VP, _VP, ctypes.POINTER(ctypes.c_int), _VP],
    "dfd_batch_set_order": [_VP, _INT, _INT, _INT],
    "dfd_batch_set_row_buffer": [_VP, _INT],
    "dfd_batch_set_team": [_VP, _INT, _INT, _INT],
    "dfd_batch_tuned": [_VP, _INT, _INT, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
    "dfd_batch_set_shape": [_VP, _INT, _INT, _INT, _INT],
    "dfd_matrix_set_shape": [_VP, _INT, _INT, _INT, _INT],
    "dfd_matrix_tuned": [_VP, _INT, _INT, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
    "dfd_matrix_autotune": [_VP, _INT, _INT, _VP, _VP, _I64, _VP, _VP, ctypes.POINTER(ctypes.c_int),
                            ctypes.POINTER(ctypes.c_int), _VP],
    "dfd_matrix": [_VP, _INT, _INT, _VP, _VP, _I64, _VP, _VP, _VP],
    "dfd_batch_decide": [_VP, _INT, _INT, _VP, _VP, _I64, _VP, _I64, _VP, ctypes.c_double, _VP, _VP, _VP, _VP],
    "dfd_mc_pair": [_VP, _INT, _VP, _I64, _VP, _I64, _VP, _VP, ctypes.c_float, ctypes.c_float, _I64, _VP, _VP, _VP],
    "dfd_batch_variant": [_VP, _INT, _INT, _INT, _VP, _VP, _I64, _VP, _I64, _VP, _VP],
    "dfd_knn": [_VP, _INT, _VP, _I64, _VP, _VP, _I64, _VP, _I64, _INT, _VP, _VP, _VP, _VP, _VP, _VP],
    "dfd_batch_capture": [_VP, _INT, _INT, _VP, _VP, _I64, _VP, _I64, _VP, _VP, ctypes.POINTER(_VP)],
    "dfd_matrix_capture": [_VP, _INT, _INT, _VP, _VP, _I64, _VP, _VP, ctypes.POINTER(_VP)],
    "dfd_graph_launch": [_VP, _VP],
    "dfd_graph_destroy": [_VP],
    "dfd_server_options_default": [ctypes.POINTER(ServerOptions)],
    "dfd_server_create": [_VP, ctypes.POINTER(ServerOptions), ctypes.POINTER(_VP)],
    "dfd_server_destroy": [_VP],
    "dfd_server_add_candidates": [_VP, _INT, _VP, _VP, _I64, ctypes.POINTER(_I64)],
    "dfd_server_submit": [_VP, _INT, _VP, _I64, _VP, _I64, _VP, ctypes.c_double, ctypes.POINTER(ctypes.c_uint64)],
    "dfd_server_wait": [_VP, ctypes.c_uint64, ctypes.c_double],
    "dfd_server_cancel": [_VP, ctypes.c_uint64],
    "dfd_server_stats": [_VP, ctypes.POINTER(ServingStats)],
    "dfd_server_stats_reset": [_VP],
    "dfd_server_request_log": [_VP, _VP, _I64, ctypes.POINTER(_I64)],
    "dfd_server_tick_log": [_VP, _VP, _I64, ctypes.POINTER(_I64)],
    "dfd_server_now": [_VP],
    "dfd_timing_enable": [_VP, _INT],
    "dfd_timing_last": [_VP, ctypes.POINTER(ctypes.c_double)],
    "dfd_microbench": [_VP, _INT, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
}

MICRO_OPS = {"ffma": 0, "ffma2": 1, "fmnmx": 2, "fmnmx3": 3, "imnmx": 4, "imnmx64": 5, "imad_wide": 6,
             "shfl": 7, "cell_f32_d3": 8, "cell_i32_d2": 9, "distonly_f32_d3": 10,
             "lat_fmnmx": 11, "lat_cell": 12, "lat_shfl": 13, "lat_ffma2": 14, "lat_mnmx64": 15,
             "cell_f32_d16": 16, "cell_i32b_d2": 17, "cell_dtw_f32_d2": 18, "cell_lev_i32": 19,
             "cell_f32_d2": 20}
_RESTYPE = {"dfd_status_string": ctypes.c_char_p, "dfd_server_now": ctypes.c_double}


def declared_symbols():
    return list(_SIGS)


def load_library(path: str | None = None):
    """Load libdfd.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library not built: {p} (run __graft_entry__.build())")
        lib = ctypes.CDLL(p)
        for name, args in _SIGS.items():
            f = getattr(lib, name, None)
            if f is None:
                continue
            f.argtypes = args
            f.restype = _RESTYPE.get(name, _INT)
        if path is None:
            _lib = lib
        return lib


def _check(st: int, where: str):
    if st != 0:
        raise DFDError(st, where)


# ------------------------------------------------------------ C-named calls

def dfd_options_default() -> Options:
    o = Options()
    _check(load_library().dfd_options_default(ctypes.byref(o)), "dfd_options_default")
    return o


def dfd_status_string(status: int) -> str:
    return load_library().dfd_status_string(int(status)).decode()


def dfd_context_create(device: int = 0, opt: Options | None = None) -> int:
    h = _VP()
    _check(load_library().dfd_context_create(ctypes.byref(h), int(device), ctypes.byref(opt) if opt else None),
           "dfd_context_create")
    return h.value


def dfd_context_destroy(ctx: int) -> int:
    return load_library().dfd_context_destroy(ctx)


def dfd_get_error(ctx: int) -> int:
    return load_library().dfd_get_error(ctx)


def dfd_pair(ctx, dtype, dim, p, n, q, m, out_dist, out_dist2, stream) -> int:
    return load_library().dfd_pair(ctx, dtype, dim, p, n, q, m, out_dist, out_dist2, stream)


def dfd_pair_reference(ctx, dtype, dim, p, n, q, m, out_dist, out_dist2, stream) -> int:
    return load_library().dfd_pair_reference(ctx, dtype, dim, p, n, q, m, out_dist, out_dist2, stream)


def dfd_pair_host(ctx, dtype, dim, p, n, q, m, out_dist, out_dist2) -> int:
    return load_library().dfd_pair_host(ctx, dtype, dim, p, n, q, m, out_dist, out_dist2)


def dfd_batch_host(ctx, dtype, dim, points, offsets, n_curves, pairs, n_pairs, out_dist, out_dist2) -> int:
    return load_library().dfd_batch_host(ctx, dtype, dim, points, offsets, n_curves, pairs, n_pairs, out_dist,
                                         out_dist2)


def dfd_pair_noalloc(device, dtype, dim, p, n, q, m, out_dist, out_dist2, stream) -> int:
    """dfd_pair without a context and without any device allocation (fixed scratch array)."""
    return load_library().dfd_pair_noalloc(device, dtype, dim, p, n, q, m, out_dist, out_dist2, stream)


def dfd_batch(ctx, dtype, dim, points, offsets, n_curves, pairs, n_pairs, out_dist, out_dist2, stream) -> int:
    return load_library().dfd_batch(ctx, dtype, dim, points, offsets, n_curves, pairs, n_pairs, out_dist, out_dist2,
                                    stream)


def dfd_matrix(ctx, dtype, dim, points, offsets, n_curves, out_condensed, out_dist2, stream) -> int:
    return load_library().dfd_matrix(ctx, dtype, dim, points, offsets, n_curves, out_condensed, out_dist2, stream)


def dfd_batch_decide(ctx, dtype, dim, points, offsets, n_curves, pairs, n_pairs, eps2, eps2_all, out_dist2,
                     out_within, abandoned, stream) -> int:
    return load_library().dfd_batch_decide(ctx, dtype, dim, points, offsets, n_curves, pairs, n_pairs, eps2,
                                           float(eps2_all), out_dist2, out_within, abandoned, stream)


def dfd_mc_pair(ctx, dim, p, n, q, m, noise_p, noise_q, sigma_p, sigma_q, n_samples, out_dist2, out_dist,
                stream) -> int:
    return load_library().dfd_mc_pair(ctx, dim, p, n, q, m, noise_p, noise_q, float(sigma_p), float(sigma_q),
                                      n_samples, out_dist2, out_dist, stream)


def dfd_batch_variant(ctx, variant, dtype, dim, points, offsets, n_curves, pairs, n_pairs, out, stream) -> int:
    return load_library().dfd_batch_variant(ctx, variant, dtype, dim, points, offsets, n_curves, pairs, n_pairs, out,
                                            stream)


def dfd_knn(ctx, dim, query, n, points, offsets, n_curves, cand, n_cand, k, out_ids, out_dist2, out_dist, abandoned,
            evaluated, stream) -> int:
    return load_library().dfd_knn(ctx, dim, query, n, points, offsets, n_curves, cand, n_cand, k, out_ids, out_dist2,
                                  out_dist, abandoned, evaluated, stream)


def dfd_batch_capture(ctx, dtype, dim, points, offsets, n_curves, pairs, n_pairs, out_dist, out_dist2) -> int:
    g = _VP()
    _check(load_library().dfd_batch_capture(ctx, dtype, dim, points, offsets, n_curves, pairs, n_pairs, out_dist,
                                            out_dist2, ctypes.byref(g)), "dfd_batch_capture")
    return g.value


def dfd_matrix_capture(ctx, dtype, dim, points, offsets, n_curves, out_condensed, out_dist2) -> int:
    g = _VP()
    _check(load_library().dfd_matrix_capture(ctx, dtype, dim, points, offsets, n_curves, out_condensed, out_dist2,
                                             ctypes.byref(g)), "dfd_matrix_capture")
    return g.value


def dfd_graph_launch(graph, stream) -> int:
    return load_library().dfd_graph_launch(graph, stream)


def dfd_graph_destroy(graph) -> int:
    return load_library().dfd_graph_destroy(graph)


def dfd_pair_shaped(ctx, dtype, dim, p, n, q, m, out_dist, out_dist2, stream, shape: WaveShape | None) -> int:
    return load_library().dfd_pair_shaped(ctx, dtype, dim, p, n, q, m, out_dist, out_dist2, stream,
                                          ctypes.byref(shape) if shape is not None else None)


def dfd_timing_enable(ctx, on: bool) -> int:
    return load_library().dfd_timing_enable(ctx, 1 if on else 0)


def dfd_timing_last(ctx) -> float:
    ms = ctypes.c_double()
    _check(load_library().dfd_timing_last(ctx, ctypes.byref(ms)), "dfd_timing_last")
    return ms.value


def dfd_microbench(ctx, op: int):
    """(per-clock-per-SM rate, SM MHz) of one measurement kernel."""
    r, mhz = ctypes.c_double(), ctypes.c_double()
    _check(load_library().dfd_microbench(ctx, int(op), ctypes.byref(r), ctypes.byref(mhz)), "dfd_microbench")
    return r.value, mhz.value


def dfd_debug_bounded_wait(ctx, timeout_ms: float) -> int:
    return load_library().dfd_debug_bounded_wait(ctx, float(timeout_ms))


def dfd_pair_plan(ctx, dtype, dim, n, m) -> WaveShape:
    s = WaveShape()
    _check(load_library().dfd_pair_plan(ctx, dtype, dim, n, m, ctypes.byref(s)), "dfd_pair_plan")
    return s


def dfd_pair_autotune(ctx, dtype, dim, p, n, q, m, stream) -> WaveShape:
    s = WaveShape()
    _check(load_library().dfd_pair_autotune(ctx, dtype, dim, p, n, q, m, stream, ctypes.byref(s)),
           "dfd_pair_autotune")
    return s


def dfd_autotune_save(ctx, path: str) -> int:
    return load_library().dfd_autotune_save(ctx, str(path).encode())


def dfd_autotune_load(ctx, path: str) -> int:
    return load_library().dfd_autotune_load(ctx, str(path).encode())


# -------------------------------------------------------- torch convenience

def _torch():
    import torch
    return torch


def _dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.float32:
        return DFD_F32
    if t.dtype == torch.int32:
        return DFD_I32
    raise TypeError(f"curves must be float32 or int32, got {t.dtype}")


def _curve(t):
    if t.dim() == 1:
        t = t.unsqueeze(1)
    if t.dim() != 2:
        raise ValueError("a curve is an [n, dim] tensor")
    return t.contiguous()


def dfd_server_create(ctx, opt: ServerOptions) -> int:
    h = _VP()
    _check(load_library().dfd_server_create(ctx, ctypes.byref(opt), ctypes.byref(h)), "dfd_server_create")
    return h.value


def dfd_server_options_default() -> ServerOptions:
    o = ServerOptions()
    _check(load_library().dfd_server_options_default(ctypes.byref(o)), "dfd_server_options_default")
    return o


def dfd_server_destroy(server) -> int:
    return load_library().dfd_server_destroy(server)


def dfd_server_add_candidates(server, dim, points, offsets, n_curves) -> int:
    first = _I64()
    _check(load_library().dfd_server_add_candidates(server, dim, points, offsets, n_curves, ctypes.byref(first)),
           "dfd_server_add_candidates")
    return first.value


def dfd_server_submit(server, dim, query, n, cand_ids, k, out, arrival_s=-1.0) -> int:
    t = ctypes.c_uint64()
    _check(load_library().dfd_server_submit(server, dim, query, n, cand_ids, k, out, float(arrival_s),
                                            ctypes.byref(t)), "dfd_server_submit")
    return t.value


def dfd_server_wait(server, ticket, timeout_ms=-1.0) -> int:
    return load_library().dfd_server_wait(server, ticket, float(timeout_ms))


def dfd_server_cancel(server, ticket) -> int:
    return load_library().dfd_server_cancel(server, ticket)


def dfd_server_stats(server) -> ServingStats:
    st = ServingStats()
    _check(load_library().dfd_server_stats(server, ctypes.byref(st)), "dfd_server_stats")
    return st


def dfd_server_stats_reset(server) -> int:
    return load_library().dfd_server_stats_reset(server)


def dfd_server_now(server) -> float:
    return load_library().dfd_server_now(server)


class Server:
    """Continuous-batching search server (query vs resident candidates)."""

    def __init__(self, ctx: "Context", mem_budget_bytes: int = 1 << 30, max_slots: int = 256,
                 tick_cells: float = 4e9, stripes_per_tick: int = 8):
        opt = dfd_server_options_default()
        opt.mem_budget_bytes = int(mem_budget_bytes)
        opt.max_slots = int(max_slots)
        opt.tick_cells = float(tick_cells)
        opt.stripes_per_tick = int(stripes_per_tick)
        self.ctx = ctx
        self.handle = dfd_server_create(ctx.handle, opt)
        self._keep = {}

    def add_candidates(self, points, offsets) -> int:
        import numpy as np
        points = np.ascontiguousarray(points, np.float32)
        offsets = np.ascontiguousarray(offsets, np.int64)
        return dfd_server_add_candidates(self.handle, points.shape[1], points.ctypes.data, offsets.ctypes.data,
                                         offsets.shape[0] - 1)

    def submit(self, query, cand_ids, out=None, arrival_s=-1.0) -> int:
        import numpy as np
        query = np.ascontiguousarray(query, np.float32)
        if query.ndim == 1:
            query = query[:, None]
        cand_ids = np.ascontiguousarray(cand_ids, np.int64)
        if out is None:
            out = np.zeros(cand_ids.shape[0], np.float32)
        t = dfd_server_submit(self.handle, query.shape[1], query.ctypes.data, query.shape[0], cand_ids.ctypes.data,
                              cand_ids.shape[0], out.ctypes.data, arrival_s)
        self._keep[t] = out
        return t

    def wait(self, ticket, timeout_ms=-1.0):
        """(status, out array); the out array is final when status is 0."""
        st = dfd_server_wait(self.handle, ticket, timeout_ms)
        out = self._keep.get(ticket)
        if st != STATUS_CODE["DFD_ERR_NOT_READY"]:
            self._keep.pop(ticket, None)
        return st, out

    def cancel(self, ticket) -> int:
        return dfd_server_cancel(self.handle, ticket)

    def stats(self) -> dict:
        s = dfd_server_stats(self.handle)
        return {f: getattr(s, f) for f, _ in ServingStats._fields_}

    def reset_stats(self):
        dfd_server_stats_reset(self.handle)

    def request_log(self):
        """Per-request times of the requests completed since the last reset: a
        numpy structured array (ticket, arrival_s, submit_s, admit_s, launch_s,
        done_s, cells, n, k, dim)."""
        import numpy as np
        lib = load_library()
        n = _I64(0)
        _check(lib.dfd_server_request_log(self.handle, None, 0, ctypes.byref(n)), "dfd_server_request_log")
        recs = (RequestRecord * max(n.value, 1))()
        _check(lib.dfd_server_request_log(self.handle, ctypes.cast(recs, _VP), n.value, ctypes.byref(n)),
               "dfd_server_request_log")
        dt = np.dtype([("ticket", "<u8"), ("arrival_s", "<f8"), ("submit_s", "<f8"), ("admit_s", "<f8"),
                       ("launch_s", "<f8"), ("done_s", "<f8"), ("cells", "<f8"), ("n", "<i4"), ("k", "<i4"),
                       ("dim", "<i4"), ("pad", "<i4"), ("locked_s", "<f8")])
        return np.frombuffer(bytes(recs), dtype=dt, count=n.value).copy()

    def tick_log(self):
        """Per-tick record of the ticks retired since the last reset: a numpy
        structured array (build_s, launched_s, retired_s, gpu_ms, cells,
        n_items, n_slices, n_outs, n_admitted, admit_ms, build_ms,
        slow_call_ms, slow_call)."""
        import numpy as np
        lib = load_library()
        dt = np.dtype([("build_s", "<f8"), ("launched_s", "<f8"), ("retired_s", "<f8"), ("gpu_ms", "<f8"),
                       ("cells", "<f8"), ("n_items", "<i4"), ("n_slices", "<i4"), ("n_outs", "<i4"),
                       ("n_admitted", "<i4"), ("admit_ms", "<f8"), ("build_ms", "<f8"), ("slow_call_ms", "<f8"),
                       ("slow_call", "<i4"), ("pad", "<i4"), ("sync_s", "<f8"), ("synced_s", "<f8"),
                       ("locked_s", "<f8")])
        n = _I64(0)
        _check(lib.dfd_server_tick_log(self.handle, None, 0, ctypes.byref(n)), "dfd_server_tick_log")
        buf = np.zeros(max(n.value, 1), dtype=dt)
        _check(lib.dfd_server_tick_log(self.handle, buf.ctypes.data, n.value, ctypes.byref(n)),
               "dfd_server_tick_log")
        return buf[: n.value].copy()

    def now(self) -> float:
        return dfd_server_now(self.handle)

    def close(self):
        if self.handle:
            dfd_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    """A captured dfd_batch / dfd_matrix call; keeps its buffers alive."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def launch(self, stream=None):
        torch = _torch()
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        _check(dfd_graph_launch(self.handle, s), "dfd_graph_launch")

    def close(self):
        if self.handle:
            dfd_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """A libdfd context bound to one CUDA device."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, wait_timeout_ms: float = 2000.0,
                 check_inputs: bool = True):
        opt = dfd_options_default()
        opt.mem_budget_bytes = int(mem_budget_bytes)
        opt.wait_timeout_ms = float(wait_timeout_ms)
        opt.check_inputs = 1 if check_inputs else 0
        self.device = int(device)
        self.handle = dfd_context_create(self.device, opt)

    def close(self):
        if self.handle:
            dfd_context_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_error(self) -> int:
        return dfd_get_error(self.handle)

    def _outs(self, dt, out_dist, out_dist2):
        torch = _torch()
        dev = torch.device("cuda", self.device)
        if out_dist is None:
            out_dist = torch.empty(1, dtype=torch.float32 if dt == DFD_F32 else torch.float64, device=dev)
        if out_dist2 is None:
            out_dist2 = torch.empty(1, dtype=torch.float32 if dt == DFD_F32 else torch.int64, device=dev)
        return out_dist, out_dist2

    def pair(self, p, q, out_dist=None, out_dist2=None, stream=None, shape=None, reference=False):
        """delta and delta^2 of two device curves; enqueued on `stream` (default: current)."""
        torch = _torch()
        p, q = _curve(p), _curve(q)
        dt = _dtype_code(p)
        if _dtype_code(q) != dt or p.shape[1] != q.shape[1]:
            raise ValueError("p and q must share dtype and dim")
        out_dist, out_dist2 = self._outs(dt, out_dist, out_dist2)
        s = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        args = (self.handle, dt, p.shape[1], p.data_ptr(), p.shape[0], q.data_ptr(), q.shape[0],
                out_dist.data_ptr(), out_dist2.data_ptr(), s)
        if reference:
            st = dfd_pair_reference(*args)
        elif shape is not None:
            st = dfd_pair_shaped(*args, WaveShape(*shape))
        else:
            st = dfd_pair(*args)
        _check(st, "dfd_pair")
        return out_dist, out_dist2

    def _batch_outs(self, dt, count, out_dist, out_dist2):
        torch = _torch()
        dev = torch.device("cuda", self.device)
        if out_dist is None:
            out_dist = torch.empty(count, dtype=torch.float32 if dt == DFD_F32 else torch.float64, device=dev)
        if out_dist2 is None:
            out_dist2 = torch.empty(count, dtype=torch.float32 if dt == DFD_F32 else torch.int64, device=dev)
        return out_dist, out_dist2

    def batch(self, points, offsets, pairs, out_dist=None, out_dist2=None, stream=None, capture=False):
        """Distances of pairs[k] = (a, b) of CSR curves; returns (dist, dist2) or a Graph if capture."""
        torch = _torch()
        points = _curve(points)
        dt = _dtype_code(points)
        offsets = offsets.contiguous()
        pairs = pairs.contiguous()
        if offsets.dtype != torch.int64 or pairs.dtype != torch.int32:
            raise TypeError("offsets must be int64 and pairs int32")
        n_pairs = pairs.numel() // 2
        out_dist, out_dist2 = self._batch_outs(dt, n_pairs, out_dist, out_dist2)
        args = (self.handle, dt, points.shape[1], points.data_ptr(), offsets.data_ptr(), offsets.numel() - 1,
                pairs.data_ptr(), n_pairs, out_dist.data_ptr(), out_dist2.data_ptr())
        if capture:
            return Graph(dfd_batch_capture(*args), (points, offsets, pairs, out_dist, out_dist2)), out_dist, out_dist2
        s = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        _check(dfd_batch(*args, s), "dfd_batch")
        return out_dist, out_dist2

    def batch_autotune(self, points, offsets, pairs, stream=None):
        """Time both packing orders of the ragged batch on these pairs (device
        tensors), keep the faster for their (dtype, dim class); returns it (0 or 1)."""
        torch = _torch()
        points = _curve(points)
        dt = _dtype_code(points)
        offsets, pairs = offsets.contiguous(), pairs.contiguous()
        if offsets.dtype != torch.int64 or pairs.dtype != torch.int32:
            raise TypeError("offsets must be int64 and pairs int32")
        n_pairs = pairs.numel() // 2
        out_dist, out_dist2 = self._batch_outs(dt, n_pairs, None, None)
        best = ctypes.c_int(0)
        s = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        _check(load_library().dfd_batch_autotune(self.handle, dt, points.shape[1], points.data_ptr(),
                                                 offsets.data_ptr(), offsets.numel() - 1, pairs.data_ptr(), n_pairs,
                                                 out_dist.data_ptr(), out_dist2.data_ptr(), ctypes.byref(best), s),
               "dfd_batch_autotune")
        return best.value

    def set_batch_order(self, dtype: int, dim: int, order: int):
        """Set the ragged batch's packing order (0 variant-major, 1 cost-descending)."""
        _check(load_library().dfd_batch_set_order(self.handle, dtype, dim, order), "dfd_batch_set_order")

    def set_batch_team(self, dtype: int, dim: int, mode: int):
        """Which ragged-batch pairs run as CTA teams: 0 auto, 1 only pairs too wide
        for one warp's row buffer, 2 every pair of several stripes."""
        _check(load_library().dfd_batch_set_team(self.handle, dtype, dim, mode), "dfd_batch_set_team")

    def batch_tuned(self, dtype: int, dim: int):
        """(packing order, team mode, rows per lane cap, CTAs per SM) recorded for
        (dtype, dim class); 0 = the default."""
        o, t, r, c = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        _check(load_library().dfd_batch_tuned(self.handle, dtype, dim, ctypes.byref(o), ctypes.byref(t),
                                              ctypes.byref(r), ctypes.byref(c)), "dfd_batch_tuned")
        return o.value, t.value, r.value, c.value

    def set_batch_shape(self, dtype: int, dim: int, rows_per_lane: int, ctas_per_sm: int):
        """Tile shape of the ragged batch's one-warp pairs (0, 0 = defaults)."""
        _check(load_library().dfd_batch_set_shape(self.handle, dtype, dim, rows_per_lane, ctas_per_sm),
               "dfd_batch_set_shape")

    def set_matrix_shape(self, dtype: int, dim: int, rows_per_lane: int, ctas_per_sm: int):
        """Tile shape of the all-pairs matrix (0, 0 = defaults)."""
        _check(load_library().dfd_matrix_set_shape(self.handle, dtype, dim, rows_per_lane, ctas_per_sm),
               "dfd_matrix_set_shape")

    def matrix_tuned(self, dtype: int, dim: int):
        r, c = ctypes.c_int(0), ctypes.c_int(0)
        _check(load_library().dfd_matrix_tuned(self.handle, dtype, dim, ctypes.byref(r), ctypes.byref(c)),
               "dfd_matrix_tuned")
        return r.value, c.value

    def matrix_autotune(self, points, offsets, stream=None):
        """Time the matrix's tile shapes on these curves (device tensors), keep
        the fastest; returns (rows per lane cap, CTAs per SM)."""
        torch = _torch()
        points = _curve(points)
        dt = _dtype_code(points)
        offsets = offsets.contiguous()
        n = offsets.numel() - 1
        npairs = n * (n - 1) // 2
        od, od2 = self._batch_outs(dt, npairs, None, None)
        r, c = ctypes.c_int(0), ctypes.c_int(0)
        s = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        _check(load_library().dfd_matrix_autotune(self.handle, dt, points.shape[1], points.data_ptr(),
                                                  offsets.data_ptr(), n, od.data_ptr(), od2.data_ptr(),
                                                  ctypes.byref(r), ctypes.byref(c), s), "dfd_matrix_autotune")
        return r.value, c.value

    def set_batch_row_buffer(self, cols: int):
        """Widen the ragged batch's per-warp row buffer (columns, >= 4096): pairs
        that run several stripes may then have longer curves of up to `cols` points."""
        _check(load_library().dfd_batch_set_row_buffer(self.handle, cols), "dfd_batch_set_row_buffer")

    def batch_host(self, points, offsets, pairs, out_dist=None, out_dist2=None):
        """dfd_batch on host (numpy) arrays, synchronous; returns (dist, dist2).
        Page-locked points (e.g. a pinned tensor's numpy view) are copied to the
        device directly, slice by slice, overlapping the computation."""
        import numpy as np
        points = np.ascontiguousarray(points)
        if points.ndim == 1:
            points = points[:, None]
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        pairs = np.ascontiguousarray(pairs, dtype=np.int32)
        n_pairs = pairs.size // 2
        # (outputs need no zero fill: every entry is written)
        if points.dtype == np.float32:
            dt = DFD_F32
            d1 = out_dist if out_dist is not None else np.empty(n_pairs, np.float32)
            d2 = out_dist2 if out_dist2 is not None else np.empty(n_pairs, np.float32)
        elif points.dtype == np.int32:
            dt = DFD_I32
            d1 = out_dist if out_dist is not None else np.empty(n_pairs, np.float64)
            d2 = out_dist2 if out_dist2 is not None else np.empty(n_pairs, np.int64)
        else:
            raise TypeError("curves must be float32 or int32")
        _check(dfd_batch_host(self.handle, dt, points.shape[1], points.ctypes.data, offsets.ctypes.data,
                              offsets.size - 1, pairs.ctypes.data, n_pairs, d1.ctypes.data, d2.ctypes.data),
               "dfd_batch_host")
        return d1, d2

    def decide(self, points, offsets, pairs, eps2, out_dist2=None, out_within=None, stream=None):
        """Threshold decision delta^2 <= eps2 per pair with early abandon.  eps2 is a
        number (all pairs) or a device tensor (float32 / int64 per pair).
        Returns (dist2, within, abandoned): exact delta^2 of pairs computed to
        the end (+inf / INT64_MAX when abandoned), 0/1 flags, abandoned count."""
        torch = _torch()
        points = _curve(points)
        dt = _dtype_code(points)
        offsets, pairs = offsets.contiguous(), pairs.contiguous()
        if offsets.dtype != torch.int64 or pairs.dtype != torch.int32:
            raise TypeError("offsets must be int64 and pairs int32")
        n_pairs = pairs.numel() // 2
        dev = points.device
        if out_dist2 is None:
            out_dist2 = torch.empty(n_pairs, dtype=torch.float32 if dt == DFD_F32 else torch.int64, device=dev)
        if out_within is None:
            out_within = torch.empty(n_pairs, dtype=torch.int32, device=dev)
        ab = torch.zeros(1, dtype=torch.int64, device=dev)
        if isinstance(eps2, (int, float)):
            eps_ptr, eps_all = None, float(eps2)
        else:
            want = torch.float32 if dt == DFD_F32 else torch.int64
            eps2 = eps2.contiguous()
            if eps2.dtype != want or eps2.numel() != n_pairs:
                raise TypeError(f"eps2 must be {want} with one value per pair")
            eps_ptr, eps_all = eps2.data_ptr(), 0.0
        s = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        st = dfd_batch_decide(self.handle, dt, points.shape[1], points.data_ptr(), offsets.data_ptr(),
                              offsets.numel() - 1, pairs.data_ptr(), n_pairs, eps_ptr, eps_all, out_dist2.data_ptr(),
                              out_within.data_ptr(), ab.data_ptr(), s)
        _check(st, "dfd_batch_decide")
        return out_dist2, out_within, ab

    def mc_pair(self, p, q, noise_p, noise_q, sigma_p, sigma_q, stream=None):
        """Monte Carlo samples of delta for uncertain float32 curves: returns
        (dist, dist2), float32[n_samples], sample s perturbing p and q by
        sigma * noise[s] (noise_p: [S, n, dim], noise_q: [S, m, dim])."""
        torch = _torch()
        p, q = _curve(p), _curve(q)
        noise_p, noise_q = noise_p.contiguous(), noise_q.contiguous()
        if p.dtype != torch.float32 or q.dtype != torch.float32 or noise_p.dtype != torch.float32 or \
                noise_q.dtype != torch.float32:
            raise TypeError("curves and noise must be float32")
        S = noise_p.shape[0]
        if tuple(noise_p.shape) != (S, p.shape[0], p.shape[1]) or tuple(noise_q.shape) != (S, q.shape[0], q.shape[1]):
            raise ValueError("noise_p must be [S, n, dim] and noise_q [S, m, dim]")
        d = torch.empty(S, dtype=torch.float32, device=p.device)
        d2 = torch.empty(S, dtype=torch.float32, device=p.device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        st = dfd_mc_pair(self.handle, p.shape[1], p.data_ptr(), p.shape[0], q.data_ptr(), q.shape[0],
                         noise_p.data_ptr(), noise_q.data_ptr(), sigma_p, sigma_q, S, d2.data_ptr(), d.data_ptr(), s)
        _check(st, "dfd_mc_pair")
        return d, d2

    def dtw(self, points, offsets, pairs, out=None, stream=None):
        """DTW (appendix variant, squared-distance ground cost) of float32 CSR pairs."""
        return self._variant(DFD_VARIANT_DTW, points, offsets, pairs, out, stream)

    def levenshtein(self, symbols, offsets, pairs, out=None, stream=None):
        """Edit distance of int32 symbol sequences (CSR, one symbol per position)."""
        return self._variant(DFD_VARIANT_LEVENSHTEIN, symbols, offsets, pairs, out, stream)

    def _variant(self, var, points, offsets, pairs, out, stream):
        torch = _torch()
        points = points.reshape(-1, 1) if points.dim() == 1 else points
        points = _curve(points)
        dt = _dtype_code(points)
        offsets, pairs = offsets.contiguous(), pairs.contiguous()
        if offsets.dtype != torch.int64 or pairs.dtype != torch.int32:
            raise TypeError("offsets must be int64 and pairs int32")
        n_pairs = pairs.numel() // 2
        if out is None:
            out = torch.empty(n_pairs, dtype=torch.float32 if var == DFD_VARIANT_DTW else torch.int64,
                              device=points.device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        st = dfd_batch_variant(self.handle, var, dt, points.shape[1], points.data_ptr(), offsets.data_ptr(),
                               offsets.numel() - 1, pairs.data_ptr(), n_pairs, out.data_ptr(), s)
        _check(st, "dfd_batch_variant")
        return out

    def knn(self, query, points, offsets, k, cand=None, stream=None):
        """k nearest candidates of a float32 query curve.  Returns (ids, dist2,
        counters): int32[k], float32[k] ascending, device int64[2] = (candidates
        abandoned or skipped, recurrence cells evaluated)."""
        torch = _torch()
        query, points = _curve(query), _curve(points)
        if query.dtype != torch.float32 or points.dtype != torch.float32 or query.shape[1] != points.shape[1]:
            raise TypeError("query and candidates must be float32 curves of one dim")
        offsets = offsets.contiguous()
        if offsets.dtype != torch.int64:
            raise TypeError("offsets must be int64")
        n_curves = offsets.numel() - 1
        if cand is not None:
            cand = cand.contiguous()
            if cand.dtype != torch.int32:
                raise TypeError("cand must be int32")
        n_cand = cand.numel() if cand is not None else n_curves
        dev = points.device
        ids = torch.empty(k, dtype=torch.int32, device=dev)
        d2 = torch.empty(k, dtype=torch.float32, device=dev)
        ab = torch.zeros(2, dtype=torch.int64, device=dev)   # [abandoned, cells evaluated]
        s = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        st = dfd_knn(self.handle, query.shape[1], query.data_ptr(), query.shape[0], points.data_ptr(),
                     offsets.data_ptr(), n_curves, cand.data_ptr() if cand is not None else None, n_cand, int(k),
                     ids.data_ptr(), d2.data_ptr(), None, ab.data_ptr(), ab.data_ptr() + 8, s)
        _check(st, "dfd_knn")
        return ids, d2, ab

    def matrix(self, points, offsets, out_dist=None, out_dist2=None, stream=None, capture=False):
        """Condensed upper-triangle distance matrix of CSR curves."""
        torch = _torch()
        points = _curve(points)
        dt = _dtype_code(points)
        offsets = offsets.contiguous()
        if offsets.dtype != torch.int64:
            raise TypeError("offsets must be int64")
        n = offsets.numel() - 1
        count = n * (n - 1) // 2
        out_dist, out_dist2 = self._batch_outs(dt, count, out_dist, out_dist2)
        args = (self.handle, dt, points.shape[1], points.data_ptr(), offsets.data_ptr(), n, out_dist.data_ptr(),
                out_dist2.data_ptr())
        if capture:
            return Graph(dfd_matrix_capture(*args), (points, offsets, out_dist, out_dist2)), out_dist, out_dist2
        s = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        _check(dfd_matrix(*args, s), "dfd_matrix")
        return out_dist, out_dist2

    def pair_host(self, p, q):
        """delta and delta^2 of two host (numpy) curves; synchronous."""
        import numpy as np
        p = np.ascontiguousarray(p)
        q = np.ascontiguousarray(q)
        if p.ndim == 1:
            p = p[:, None]
        if q.ndim == 1:
            q = q[:, None]
        if p.dtype == np.float32:
            dt, d1, d2 = DFD_F32, np.zeros(1, np.float32), np.zeros(1, np.float32)
        elif p.dtype == np.int32:
            dt, d1, d2 = DFD_I32, np.zeros(1, np.float64), np.zeros(1, np.int64)
        else:
            raise TypeError("curves must be float32 or int32")
        st = dfd_pair_host(self.handle, dt, p.shape[1], p.ctypes.data, p.shape[0], q.ctypes.data, q.shape[0],
                           d1.ctypes.data, d2.ctypes.data)
        _check(st, "dfd_pair_host")
        return d1[0], d2[0]

    def plan(self, dtype: int, dim: int, n: int, m: int):
        s = dfd_pair_plan(self.handle, dtype, dim, n, m)
        return s.rows_per_lane, s.warps, s.ctas

    def autotune(self, p, q, stream=None):
        """Time every candidate wavefront shape on device curves (p, q) and
        keep the fastest for their size class; returns (rows_per_lane, warps, ctas)."""
        torch = _torch()
        p, q = _curve(p), _curve(q)
        dt = _dtype_code(p)
        if _dtype_code(q) != dt or p.shape[1] != q.shape[1]:
            raise ValueError("p and q must share dtype and dim")
        st = stream if stream is not None else torch.cuda.current_stream(self.device).cuda_stream
        s = dfd_pair_autotune(self.handle, dt, p.shape[1], p.data_ptr(), p.shape[0], q.data_ptr(), q.shape[0], st)
        return s.rows_per_lane, s.warps, s.ctas

    def save_tuning(self, path):
        _check(dfd_autotune_save(self.handle, path), "dfd_autotune_save")

    def load_tuning(self, path):
        _check(dfd_autotune_load(self.handle, path), "dfd_autotune_load")
