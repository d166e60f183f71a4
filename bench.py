#!/usr/bin/env python3
"""Benchmark of the discrete Frechet distance hot path on GB300.

The headline metric is the batched / served rate against per-pair launches,
so the default workload is the ragged batch: 65,536 pairs of int32 2-D
random walks, lengths U{16..512} drawn per curve (seeded, synthetic).  A step
is one complete batch through ``dfd_batch`` (input checks, the device-built
work list and the persistent batch kernel, one captured CUDA graph launch).
``value`` = cells / second / 1e9 (GCUPS) with the curves resident in HBM;
``e2e`` = the same metric through ``dfd_batch_host`` with host buffers (the
host->device copies and the result read inside the timed region).

The same line carries, on one GPU:
  config.per_pair  the same pairs (a 512-pair sample) one launch each through
                   dfd_pair (band wavefront) and dfd_pair_reference (the
                   plain per-pair form), back to back on one stream;
  serving          p50 / p99 latency and rates of the continuous-batching
                   server under open-loop Poisson streams (1,000 and 10,000
                   requests/s, 2 s of arrivals, three sweeps each);
  long_pair        the 200,000 x 200,000 3-D float32 pair through dfd_pair
                   (rate, roofline fraction, oracle check).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
    python bench.py --workload long     # only the 200,000^2 pair
    python bench.py --workload matrix   # all pairs of 4096 16-D AR(1) curves, one graph launch per step
    python bench.py --workload pair2k   # one 2000 x 1500 2-D pair
    python bench.py --workload serve    # the serving sweep alone (more rates)

Under torchrun (N > 1) the batch and matrix workloads shard their pairs
across ranks (no collective) and the single long pair runs as replicas
(one per rank); value = all ranks' cells / the slowest rank's time.
``--impl reference`` times the CPU oracle (float64 / int64 Alg. 5) on host
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import gc
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DFD GCUPS (batched/served vs per-pair) at oracle accuracy; p50/p99 request latency"
UNIT = "GCUPS"
N_POINTS = 200_000
DIM = 3
SEED = 3
L2_FLUSH_BYTES = 256 << 20
CPU_SAMPLE = 50_000          # cpu_baseline of the long pair: prefix p[:a], q[:a]
REF_SAMPLE = 20_000          # --impl reference: prefix per step

# DRAM bytes (read + write) per launch of the main kernel, from an ncu launch
# list of the benchmark command (gpu__time_duration.sum, dram__bytes_read.sum,
# dram__bytes_write.sum: one pass), keyed by the hash of the kernel sources it
# was taken on (and "/<workload>" where two workloads share those sources);
# any later source change reports null.
TRAFFIC_BY_KERNEL_SHA: dict = {
    "9799fd99282b0741": 15759897,    # wave_kernel<F32, 3, 6>, long pair 200,000^2 (two fronts, 512-column q chunks)
    "4da739c00f897e73": 16059648,    # the same with a 4-chunk q ring (15.40 MB read, 0.66 MB written)
    "336ce32a9a0f5945": 16327168,    # the same after the prep kernel and the fused combine (15.73 MB read, 0.59 MB written)
    "b1c84c88a75cca4c": 16335104,    # the same with the int32 value classes beside it (15.68 MB read, 0.66 MB written)
    "b1c84c88a75cca4c/pair2k": 138906,   # wave_kernel<F32, 2, 4>, pair 2000 x 1500 (mean of 10 launches, reads only)
    "27aa8e25b42fbf75": 289363200,   # batch_kernel<I32, 2>, ragged batch of 65,536 pairs (graph launches)
    # batch_kernel<I32, 2> with size classes and the 8-step loop: 147.41 MB per launch captured on the
    # 32,768-pair batch (139.0 MB of inputs), scaled by the inputs (the points are read once) to the
    # 65,536-pair batch's 278.6 MB
    "46c1e1b19151a973": 295400000,
    # the same after the grouped staging loads / stores, the cost-based orientation and the
    # slice filter of the plan: 145.60 MB per launch on the 32,768-pair batch (138.2 MB of
    # points), scaled by the points to the 65,536-pair batch's 277.0 MB
    "cb7f3699e1ec87c1": 291797623,
    # the same after the one-block plan and the two-front teams: 145.70 MB per launch on 32,768 pairs
    "4e3a53f28fbbf8b0": 291998225,
    # the same with programmatic launches and team halves on two CTAs: 146.02 MB per launch on 32,768 pairs
    "be9bbfac9032b6ac": 292637166,
    # the same with the plan's cost models in 32-bit and float32 arithmetic: 145.68 MB per launch on 32,768 pairs
    "d222274be6df4291": 291956860,
}


def long_workload(n, m):
    return f"long pair {n}x{m}, {DIM}-D float32 warped random walk (seed {SEED})"


PAIR2K_WORKLOAD = "pair 2000x1500, 2-D float32 Gaussian walks (seeds 1, 2)"
BATCH_WORKLOAD = ("ragged batch, {n:,} pairs of int32 2-D random walks, lengths U{{16..512}} (seed 4), "
                  "one persistent launch per step in a captured CUDA graph")
MATRIX_WORKLOAD = ("all-pairs matrix (upper triangle) of {n} float32 16-D AR(1) curves (phi 0.95), "
                   "lengths U{{64..256}} (seed 5), one launch per step in a CUDA graph")


def kernel_sha(files=("wave_kernel.cuh", "wave_launch.cuh", "wave_shape.h", "dfd_device.cuh")) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2404_05708_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch",
                    choices=["long", "batch", "matrix", "pair2k", "serve", "knn", "next", "paper"])
    ap.add_argument("--rates", default="100,1000,3000,10000,20000,30000")
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--tick-cells", type=float, default=4e9, help="serve: cell budget of one tick")
    ap.add_argument("--stripes-per-tick", type=int, default=8, help="serve: row stripes a long pair advances per tick")
    ap.add_argument("--n", type=int, default=N_POINTS)
    ap.add_argument("--m", type=int, default=N_POINTS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--shape", default="", help="long pair: fixed launch shape R,W,ctas (no autotune)")
    ap.add_argument("--pairs", type=int, default=0, help="batch: number of pairs (default 65,536)")
    ap.add_argument("--curves", type=int, default=0, help="matrix: number of curves (default 4096)")
    ap.add_argument("--no-extras", action="store_true",
                    help="batch: leave out the serving sweep and the long pair of the default line")
    ap.add_argument("--extra-rates", default="1000,10000", help="batch line: serving rates (req/s)")
    ap.add_argument("--serve-repeats", type=int, default=3, help="batch line: sweeps per serving rate")
    ap.add_argument("--paper-points", default="",
                    help="paper: only these points, comma-separated PxN (e.g. 1024x512); default all")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.lines = []
        self.proc = None
        self.thread = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id:
            cmd[1:1] = ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- workloads
class LongPair:
    """One long 3-D float32 pair through dfd_pair (band wavefront)."""
    micro_op = "cell_f32_d3"
    dtype = "f32"
    # the wavefront starts on the prep kernel's tail (programmatic launch), so
    # the library's events bracket both
    kernel_timing = "prep and wavefront kernels"
    launches_per_step = 3          # prep (check + q packing), wavefront, combine (set per shape below)

    def __init__(self, args, ctx, dfd, torch, workloads, rank, world):
        self.n, self.m = args.n, args.m
        p_np, q_np = workloads.warped_long_pair(self.n, self.m, dim=DIM, seed=SEED)
        # the e2e step reads the inputs from page-locked host memory
        self.p_np = torch.from_numpy(p_np).pin_memory().numpy()
        self.q_np = torch.from_numpy(q_np).pin_memory().numpy()
        self.p = torch.from_numpy(self.p_np).cuda()
        self.q = torch.from_numpy(self.q_np).cuda()
        self.ctx, self.torch = ctx, torch
        self.d = torch.empty(1, dtype=torch.float32, device="cuda")
        self.d2 = torch.empty(1, dtype=torch.float32, device="cuda")
        self.cells = self.n * self.m
        if args.shape:
            shape, tuned = tuple(int(x) for x in args.shape.split(",")), False
            self.shape = shape
        elif getattr(args, "no_autotune", False):
            shape, tuned = ctx.plan(0, DIM, self.n, self.m), False
        else:
            # Untimed setup: time each candidate launch shape once, keep the fastest.
            shape, tuned = ctx.autotune(self.p, self.q), True
            torch.cuda.synchronize()
        self.config = {"workload": long_workload(self.n, self.m),
                       "n": self.n, "m": self.m, "dim": DIM, "cells_per_step": self.cells,
                       "launch_shape": {"rows_per_lane": shape[0], "warps": shape[1], "ctas": shape[2],
                                        "autotuned": tuned},
                       "kernel_sha": kernel_sha()}
        # prep kernel + wavefront; two fronts (a pair of two bands or more) on a
        # row of more than 65,536 columns add a combine kernel (shorter rows are
        # met by the wavefront's last CTA)
        bands = -(-self.n // (32 * shape[0] * shape[1]))
        self.launches_per_step = 3 if bands >= 2 and self.m > 65536 else 2
        self.config["fronts"] = 2 if bands >= 2 else 1
        self.h2d = (self.n + self.m) * DIM * 4
        self.d2h = 16

    shape = None

    def step(self):
        self.ctx.pair(self.p, self.q, self.d, self.d2, shape=self.shape)

    def e2e_step(self):
        return self.ctx.pair_host(self.p_np, self.q_np)

    def verify(self):
        gold_path = os.path.join(ROOT, "tests", "golden", "long_pair_200k.json")
        if self.n != N_POINTS or self.m != N_POINTS or not os.path.exists(gold_path):
            return None
        rec = json.load(open(gold_path))
        h = hashlib.sha256()
        h.update(self.p_np.tobytes())
        h.update(self.q_np.tobytes())
        if h.hexdigest() != rec["sha256"]:
            return None
        got = float(self.d.item())
        return abs(got - rec["delta_f64"]) <= 1e-6 * rec["delta_f64"]

    def cpu_baseline(self):
        import oracle
        a = min(CPU_SAMPLE, self.n, self.m)
        ps, qs = self.p_np[:a].copy(), self.q_np[:a].copy()
        oracle.load()
        t0 = time.perf_counter()
        oracle.dfd2_linear(ps, qs)
        dt = time.perf_counter() - t0
        return {"value": a * a / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"prefix p[:{a}], q[:{a}] of the same pair, Alg. 5 float64, one thread, {dt:.1f} s"}

    def per_pair(self):
        return None


class Pair2k(LongPair):
    """One 2000 x 1500 2-D float32 pair (Gaussian walks)."""
    micro_op = "cell_f32_d2"
    launches_per_step = 2          # prep (check + q packing), wavefront (its last CTA meets the two fronts)

    def __init__(self, args, ctx, dfd, torch, workloads, rank, world):
        self.n, self.m = 2000, 1500
        self.p_np, self.q_np = workloads.gaussian_walk_pair(self.n, self.m, dim=2)
        self.p = torch.from_numpy(self.p_np).cuda()
        self.q = torch.from_numpy(self.q_np).cuda()
        self.ctx, self.torch = ctx, torch
        self.d = torch.empty(1, dtype=torch.float32, device="cuda")
        self.d2 = torch.empty(1, dtype=torch.float32, device="cuda")
        self.cells = self.n * self.m
        self.config = {"workload": PAIR2K_WORKLOAD, "n": self.n,
                       "m": self.m, "dim": 2, "cells_per_step": self.cells, "kernel_sha": kernel_sha()}
        self.traffic_tag = "pair2k"   # same kernel sources as the long pair, another workload
        self.h2d = (self.n + self.m) * 2 * 4
        self.d2h = 16

    def verify(self):
        import oracle
        import math
        return abs(float(self.d.item()) - math.sqrt(oracle.dfd2_linear(self.p_np, self.q_np))) <= \
            1e-6 * float(self.d.item())

    def cpu_baseline(self):
        import oracle
        oracle.load()
        t0 = time.perf_counter()
        k = 0
        while time.perf_counter() - t0 < 10.0:
            oracle.dfd2_linear(self.p_np, self.q_np)
            k += 1
        dt = time.perf_counter() - t0
        return {"value": k * self.cells / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"the full pair, {k} times, Alg. 5 float64, one thread"}

    def per_pair(self):
        torch = self.torch
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        self.ctx.pair(self.p, self.q, reference=True)
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(5):
            self.ctx.pair(self.p, self.q, reference=True)
        ev1.record()
        torch.cuda.synchronize()
        return {"per_pair_reference_gcups": 5 * self.cells / (ev0.elapsed_time(ev1) * 1e-3) / 1e9}


class _Many:
    """Shared logic of the batch and matrix workloads (pairs sharded over ranks)."""

    def e2e_step(self):
        torch = self.torch
        self.pts_dev.copy_(self.pts_host, non_blocking=True)
        self.graph.launch()
        self.out_host.copy_(self.out2, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        return self.out_host

    def step(self):
        self.graph.launch()


def int_pair_classes(b, pairs):
    """Per pair: True when the union bounding box keeps every squared
    distance exact in uint32 below the first float NaN pattern (the
    library's narrow value class), from per-curve min / max."""
    lo = np.minimum.reduceat(b.points.astype(np.int64), b.offsets[:-1], axis=0)
    hi = np.maximum.reduceat(b.points.astype(np.int64), b.offsets[:-1], axis=0)
    r = np.maximum(hi[pairs[:, 0]], hi[pairs[:, 1]]) - np.minimum(lo[pairs[:, 0]], lo[pairs[:, 1]])
    return np.all(r <= 46340, axis=1) & ((r * r).sum(axis=1) <= 0x7F7FFFFF)


class Batch(_Many):
    """65,536 ragged int32 2-D pairs, lengths U{16..512}, one captured graph per step."""
    micro_op = "cell_i32_d2"
    dtype = "i32"
    launches_per_step = 5          # input check, 3 plan kernels, persistent batch kernel

    def __init__(self, args, ctx, dfd, torch, workloads, rank, world):
        from paper_2404_05708_gb300 import shard
        b = workloads.ragged_int_batch(n_pairs=args.pairs) if args.pairs else workloads.ragged_int_batch()
        pairs = b.pairs[shard.shard_pairs(b.lengths(), b.pairs, rank, world)].copy()
        self.b, self.pairs_np = b, pairs
        self.ctx, self.torch = ctx, torch
        ln = b.lengths()
        self.cells = int(np.sum(ln[pairs[:, 0]] * ln[pairs[:, 1]]))
        self.pts_host = torch.from_numpy(b.points).pin_memory()
        self.pts_dev = torch.from_numpy(b.points).cuda()
        self.off = torch.from_numpy(b.offsets).cuda()
        self.pairs = torch.from_numpy(pairs).cuda()
        # untimed setup: pick the packing order (variant-major / cost-descending) on these pairs
        order = ctx.batch_autotune(self.pts_dev, self.off, self.pairs)
        torch.cuda.synchronize()
        self.graph, self.out, self.out2 = ctx.batch(self.pts_dev, self.off, self.pairs, capture=True)
        self.out_host = torch.empty_like(self.out2, device="cpu").pin_memory()
        _, team, rm, cp = ctx.batch_tuned(dfd.DFD_I32, 2)
        self.config = {"workload": BATCH_WORKLOAD.format(n=b.pairs.shape[0]),
                       "n_pairs": int(pairs.shape[0]), "dim": 2, "cells_per_step": self.cells,
                       "packing": {"order": ["variant-major", "cost-descending"][order],
                                   "teams": {1: "pairs wider than a warp's buffer",
                                             2: "every pair of several stripes"}.get(team, "plan's model"),
                                   "rows_per_lane_cap": rm, "ctas_per_sm": cp, "autotuned": True},
                       "kernel_sha": kernel_sha(("batch_kernel.cuh", "batch_launch.cuh", "dfd_device.cuh"))}
        # e2e: dfd_batch_host from page-locked points (copy slices overlap the
        # batch kernels), offsets and pairs from host memory, dist + dist2 back
        self.pts_pinned_np = self.pts_host.numpy()
        self.h2d = b.points.nbytes + b.offsets.nbytes + pairs.nbytes
        self.d2h = pairs.shape[0] * 16
        narrow = int_pair_classes(b, pairs)
        cells = ln[pairs[:, 0]].astype(np.int64) * ln[pairs[:, 1]]
        self.cells_narrow = int(cells[narrow].sum())
        self.config["value_classes"] = {"uint32_bits_pairs": int(narrow.sum()), "int64_pairs": int((~narrow).sum())}

    def e2e_step(self):
        d, d2 = self.ctx.batch_host(self.pts_pinned_np, self.b.offsets, self.pairs_np)
        return d2

    def kernel_ms(self, steps, flush):
        """Duration of the batch kernel alone: the graph's launches carry no
        readable library events, so the same call runs uncaptured (same
        pairs, same kernel) with the library's event pair around the
        kernel on the launching stream, L2 flushed before each."""
        from paper_2404_05708_gb300 import dfd
        out = []
        for k in range(steps + 2):
            flush.zero_()
            self.ctx.batch(self.pts_dev, self.off, self.pairs, self.out, self.out2)
            ms = dfd.dfd_timing_last(self.ctx.handle)
            if k >= 2:
                out.append(ms)
        return out

    def micro_mix(self):
        mix = [("cell_i32b_d2", self.cells_narrow), ("cell_i32_d2", self.cells - self.cells_narrow)]
        return [(op, c) for op, c in mix if c > 0]

    def verify(self):
        import oracle
        idx = np.random.default_rng(0).choice(self.pairs_np.shape[0], size=512, replace=False)
        ref, _ = oracle.batch(self.b.points, self.b.offsets, self.pairs_np[idx])
        return bool(np.array_equal(self.out2.cpu().numpy()[idx], ref))

    def cpu_baseline(self):
        """The oracle over the whole batch, repeated for about 10 s of host time."""
        import oracle
        oracle.load()
        t0 = time.perf_counter()
        reps = 0
        while time.perf_counter() - t0 < 10.0:
            _, used = oracle.batch(self.b.points, self.b.offsets, self.pairs_np)
            reps += 1
        dt = time.perf_counter() - t0
        return {"value": reps * self.cells / dt / 1e9, "unit": UNIT, "cores": used, "kind": "oracle",
                "sample": f"all {self.pairs_np.shape[0]} pairs of the batch, {reps} times, Alg. 5 int64, "
                          f"{used} threads, {dt:.1f} s"}

    def per_pair(self):
        """The same pairs one launch each, back to back on one stream (sample of 512)."""
        torch = self.torch
        ln = self.b.lengths()
        idx = np.random.default_rng(1).choice(self.pairs_np.shape[0], size=512, replace=False)
        curves = []
        cells = 0
        for k in idx:
            a, c = self.pairs_np[k]
            pa = self.pts_dev[self.b.offsets[a]:self.b.offsets[a + 1]]
            pc = self.pts_dev[self.b.offsets[c]:self.b.offsets[c + 1]]
            curves.append((pa, pc))
            cells += int(ln[a] * ln[c])
        out = {}
        for name, kw in (("per_pair_reference_gcups", {"reference": True}), ("per_pair_wave_gcups", {})):
            for pa, pc in curves[:8]:
                self.ctx.pair(pa, pc, **kw)
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            for pa, pc in curves:
                self.ctx.pair(pa, pc, **kw)
            ev1.record()
            torch.cuda.synchronize()
            out[name] = cells / (ev0.elapsed_time(ev1) * 1e-3) / 1e9
        return out


class Matrix(_Many):
    """All-pairs condensed matrix of 4096 16-D float32 AR(1) curves, lengths U{64..256}."""
    micro_op = "cell_f32_d16"
    dtype = "f32"
    launches_per_step = 2          # input check, persistent matrix kernel

    def __init__(self, args, ctx, dfd, torch, workloads, rank, world):
        if world > 1:
            raise SystemExit("the matrix workload runs on one GPU")
        b = workloads.ar1_curves(n_curves=args.curves) if args.curves else workloads.ar1_curves()
        self.b = b
        self.ctx, self.torch = ctx, torch
        ln = b.lengths().astype(np.int64)
        tot = int(ln.sum())
        self.cells = int((tot * tot - int(np.sum(ln * ln))) // 2)
        self.pts_host = torch.from_numpy(b.points).pin_memory()
        self.pts_dev = torch.from_numpy(b.points).cuda()
        self.off = torch.from_numpy(b.offsets).cuda()
        # untimed setup: tile shape timed on the first 1,024 curves (1/16 of the pairs)
        sub = min(1024, b.n_curves)
        rm, cp = ctx.matrix_autotune(self.pts_dev[: int(b.offsets[sub])], self.off[: sub + 1])
        torch.cuda.synchronize()
        self.graph, self.out, self.out2 = ctx.matrix(self.pts_dev, self.off, capture=True)
        self.out_host = torch.empty_like(self.out2, device="cpu").pin_memory()
        n = b.n_curves
        self.config = {"workload": MATRIX_WORKLOAD.format(n=n),
                       "n_curves": n, "n_pairs": n * (n - 1) // 2, "dim": 16, "cells_per_step": self.cells,
                       "tile_shape": {"rows_per_lane_cap": rm, "ctas_per_sm": cp,
                                      "autotuned_on": f"the first {sub} curves"},
                       "kernel_sha": kernel_sha(("batch_kernel.cuh", "batch_launch.cuh", "dfd_device.cuh"))}
        self.h2d = b.points.nbytes
        self.d2h = self.out2.numel() * 4

    def verify(self):
        import oracle
        n = self.b.n_curves
        rng = np.random.default_rng(2)
        ks = rng.integers(0, n * (n - 1) // 2, size=128)
        starts = np.array([i * (2 * n - i - 1) // 2 for i in range(n)], np.int64)
        ii = np.searchsorted(starts, ks, side="right") - 1
        jj = ks - starts[ii] + ii + 1
        mirror, _ = oracle.batch(self.b.points, self.b.offsets, np.stack([ii, jj], 1).astype(np.int32), mirror=True)
        return bool(np.array_equal(self.out2.cpu().numpy()[ks], mirror))

    def cpu_baseline(self):
        import oracle
        oracle.load()
        rng = np.random.default_rng(3)
        n = self.b.n_curves
        pairs = np.stack([rng.integers(0, n, 20000), rng.integers(0, n, 20000)], 1).astype(np.int32)
        t0 = time.perf_counter()
        _, used = oracle.batch(self.b.points, self.b.offsets, pairs)
        dt = time.perf_counter() - t0
        ln = self.b.lengths()
        cells = int(np.sum(ln[pairs[:, 0]] * ln[pairs[:, 1]]))
        return {"value": cells / dt / 1e9, "unit": UNIT, "cores": used, "kind": "oracle",
                "sample": f"20,000 random pairs of the 4096 curves, Alg. 5 float64, {used} threads, {dt:.1f} s"}

    def per_pair(self):
        return None


class Knn:
    """Exact k-NN (k = 10) of a float32 2-D query curve among the 2^16-curve
    serving pool, with early abandon; one query per step (8 queries cycled).
    `value` counts every candidate's n*m cells (the work the search answers
    for), so pruning shows as a higher rate; config holds the abandoned
    fraction and the time dfd_batch needs to compute every distance."""
    micro_op = "cell_f32_d3"
    dtype = "f32"
    launches_per_step = 5          # 2 input checks, init, search, sort

    def __init__(self, args, ctx, dfd, torch, workloads, rank, world):
        self.k = 10
        pool = workloads.serving_pool(dim=2, seed=8)
        qs = workloads.serving_pool(n_curves=8, dim=2, seed=99)
        self.pool, self.qs = pool, qs
        self.ctx, self.torch = ctx, torch
        self.pts = torch.from_numpy(pool.points).cuda()
        self.off = torch.from_numpy(pool.offsets).cuda()
        self.q_host = [torch.from_numpy(qs.curve(i).copy()).pin_memory() for i in range(8)]
        self.q_dev = [q.cuda() for q in self.q_host]
        plen = int(pool.lengths().sum())
        self.cells_q = [int(len(q)) * plen for q in self.q_host]
        self.it = 0
        self.cells = int(np.mean(self.cells_q))
        # full computation of every distance for the same query (comparison)
        allp = torch.cat([self.q_dev[0], self.pts])
        allo = torch.cat([torch.zeros(1, dtype=torch.int64, device="cuda"), self.off + len(self.q_dev[0])])
        pairs = torch.stack([torch.zeros(pool.n_curves, dtype=torch.int32),
                             torch.arange(1, pool.n_curves + 1, dtype=torch.int32)], 1).cuda()
        ctx.batch(allp, allo, pairs)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(True), torch.cuda.Event(True)
        e0.record()
        d, d2 = ctx.batch(allp, allo, pairs)
        e1.record()
        torch.cuda.synchronize()
        self.full_ms = e0.elapsed_time(e1)
        self.full_top = torch.sort(d2)[0][: self.k].cpu().numpy()
        ids, kd2, ab = ctx.knn(self.q_dev[0], self.pts, self.off, self.k)
        torch.cuda.synchronize()
        self.ab_frac = int(ab[0].item()) / pool.n_curves
        self.match_full = bool(np.array_equal(kd2.cpu().numpy(), self.full_top))
        self.config = {"workload": "exact k-NN (k = 10) of a float32 2-D query among 2^16 resident Gaussian-walk "
                                   "candidates, lognormal lengths median 256 (seeds 8, 99), early abandon",
                       "k": self.k, "n_candidates": pool.n_curves, "cells_per_step": self.cells,
                       "abandoned_fraction": round(self.ab_frac, 4),
                       "full_batch_ms_same_query": round(self.full_ms, 3),
                       "kernel_sha": kernel_sha(("batch_kernel.cuh", "knn.cu", "dfd_device.cuh"))}
        self.h2d = int(self.q_host[0].numel() * 4)
        self.d2h = self.k * 8

    def step(self):
        i = self.it % 8
        self.it += 1
        _, _, c = self.ctx.knn(self.q_dev[i], self.pts, self.off, self.k)
        self.counters.append(c)

    counters = []

    def evaluated_cells(self):
        """Mean recurrence cells actually evaluated per step (after pruning)."""
        vals = [int(c[1].item()) for c in self.counters[-8:]]
        return sum(vals) / max(len(vals), 1)

    def e2e_step(self):
        i = self.it % 8
        self.it += 1
        q = self.q_dev[i]
        q.copy_(self.q_host[i], non_blocking=True)
        ids, d2, _ = self.ctx.knn(q, self.pts, self.off, self.k)
        return ids.cpu(), d2.cpu()

    def verify(self):
        # k-NN of query 1 among the first 2048 candidates against the oracle,
        # and query 0's k-NN against the full GPU computation of all distances
        import oracle
        torch = self.torch
        sub = 2048
        cand = torch.arange(sub, dtype=torch.int32, device="cuda")
        ids, d2, _ = self.ctx.knn(self.q_dev[1], self.pts, self.off, self.k, cand=cand)
        qn = self.qs.curve(1)
        allp = np.concatenate([qn, self.pool.points[: self.pool.offsets[sub]]])
        allo = np.concatenate([[0], self.pool.offsets[: sub + 1] + len(qn)])
        pairs = np.stack([np.zeros(sub, np.int32), np.arange(1, sub + 1, dtype=np.int32)], 1)
        want, _ = oracle.batch(allp, allo, pairs, mirror=True)
        order = np.lexsort((np.arange(sub), want))[: self.k]
        ok = np.array_equal(ids.cpu().numpy(), order) and np.array_equal(d2.cpu().numpy(), want[order])
        return bool(ok and self.match_full)

    def cpu_baseline(self):
        import oracle
        qn = self.qs.curve(0)
        sub = 64
        allp = np.concatenate([qn, self.pool.points[: self.pool.offsets[sub]]])
        allo = np.concatenate([[0], self.pool.offsets[: sub + 1] + len(qn)])
        pairs = np.stack([np.zeros(sub, np.int32), np.arange(1, sub + 1, dtype=np.int32)], 1)
        oracle.load()
        t0 = time.perf_counter()
        oracle.batch(allp, allo, pairs, nthreads=1)
        dt = time.perf_counter() - t0
        cells = len(qn) * int(self.pool.offsets[sub])
        return {"value": cells / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"query 0 against the first {sub} candidates, all distances (no pruning), Alg. 5 float64, "
                          f"one thread, {dt:.1f} s"}

    def per_pair(self):
        return None


WORKLOADS = {"long": LongPair, "pair2k": Pair2k, "batch": Batch, "matrix": Matrix, "knn": Knn}


def serve_sweep(ctx, rates, seconds, repeats, tick_cells, stripes_per_tick):
    """Open-loop Poisson request streams against the continuous-batching server.

    Pools: 2^16 float32 Gaussian-walk candidates per dim (2 and 3), lognormal
    lengths (median 256, sigma 0.75, clipped to [32, 4096]).  Requests: dim 2
    or 3, lognormal query length, k ~ U{1..1024} candidates.  For each rate
    the client submits every request at its scheduled arrival time (latency
    is measured from that time, so a late client cannot hide queueing) for
    `seconds` seconds of arrivals, then waits for all of them; each rate runs
    `repeats` times with fresh arrival draws.
    """
    from paper_2404_05708_gb300 import dfd, workloads
    pools = {d: workloads.serving_pool(dim=d, seed=6 + d) for d in (2, 3)}
    srv = dfd.Server(ctx, mem_budget_bytes=4 << 30, max_slots=512, tick_cells=tick_cells,
                     stripes_per_tick=stripes_per_tick)
    for d in (2, 3):
        srv.add_candidates(pools[d].points, pools[d].offsets)
    sweep = []
    # A separate process that sleeps 1 ms at a time and reports every sleep that
    # overran by more than 5 ms: a pause of the whole host (seen by this
    # process and the watcher alike) shows there, so a latency outlier can be
    # told apart from a stall of the server.  Times are CLOCK_MONOTONIC, the
    # server's clock.
    watch_s = 60.0 + sum(max(20, int(r * seconds)) / r + 2.0 for r in rates) * repeats
    watcher = subprocess.Popen(
        [sys.executable, "-c",
         "import sys,time\n"
         "end=time.monotonic()+float(sys.argv[1])\n"
         "while time.monotonic()<end:\n"
         "    a=time.monotonic(); time.sleep(0.001); d=time.monotonic()-a\n"
         "    if d>0.006: print(f'{a:.6f} {d*1e3:.2f}', flush=True)\n",
         str(watch_s)], stdout=subprocess.PIPE, text=True)
    gaps = []

    def read_gaps():
        for ln in watcher.stdout:
            gaps.append(tuple(float(x) for x in ln.split()))
    threading.Thread(target=read_gaps, daemon=True).start()
    # warm-up
    w = workloads.serving_requests(20, 1000.0, {2: 1 << 16, 3: 1 << 16}, seed=99)
    for t in [srv.submit(r.query, r.cand_ids) for r in w]:
        srv.wait(t)
    for rate in rates:
        for rep in range(repeats):
            n_req = max(20, int(rate * seconds))
            reqs = workloads.serving_requests(n_req, rate, {2: 1 << 16, 3: 1 << 16}, seed=int(rate) + 7919 * rep)
            srv.reset_stats()
            # no garbage-collector pass inside the open loop: a full pass over the
            # request objects delays submissions (latency counts from the
            # scheduled arrival)
            gc.collect()
            gc.disable()
            t0 = srv.now() + 0.05
            tickets = []
            for r in reqs:
                due = t0 + r.arrival_s
                while True:
                    d = due - srv.now()
                    if d <= 0:
                        break
                    time.sleep(min(d, 0.002))
                tickets.append(srv.submit(r.query, r.cand_ids, arrival_s=due))
            for t in tickets:
                srv.wait(t)
            gc.enable()
            st = srv.stats()
            t_end = srv.now()
            stalls = [round(d, 1) for a, d in list(gaps) if t0 <= a <= t_end]
            sweep.append({"rate_req_s": rate, "repeat": rep, "requests": n_req, "p50_ms": st["p50_ms"],
                          "p99_ms": st["p99_ms"], "gcups_wall": st["gcups_wall"], "gcups_busy": st["gcups_busy"],
                          "ticks": st["ticks"], "cells": st["cells"], "host_stalls_ms": stalls})
    srv.close()
    watcher.terminate()
    return sweep


SERVE_WORKLOAD = ("serving: Poisson stream of query-vs-k-candidates requests (dims 2, 3; lognormal lengths "
                  "median 256 clipped [32, 4096]; k ~ U{1..1024}) against 2^16 resident candidates per dim")


def run_serving(args):
    """The serving sweep alone (see serve_sweep), over --rates."""
    import torch
    from paper_2404_05708_gb300 import build, dfd
    build.build()
    torch.cuda.set_device(0)
    ctx = dfd.Context(0)
    rates = [float(r) for r in args.rates.split(",")]
    sweep = serve_sweep(ctx, rates, args.serve_seconds, 1, args.tick_cells, args.stripes_per_tick)
    ctx.close()
    best = max(sweep, key=lambda x: x["gcups_wall"])
    out = {"metric": METRIC, "value": best["gcups_wall"], "unit": UNIT, "n_gpus": 1,
           "higher_is_better": True, "dtype": "f32", "data": "synthetic",
           "config": {"workload": SERVE_WORKLOAD,
                      "tick_cells": args.tick_cells, "stripes_per_tick": args.stripes_per_tick},
           "serving": sweep}
    print(json.dumps(out))
    return 0


def run_next(args):
    """The rows after the hot path, each on seeded synthetic inputs, timed
    with CUDA events over --steps launches after --warmup, verified on a
    sample against the oracle, with its roofline against the measured cell
    mix of its own recurrence:

    decider  dfd_batch_decide on the ragged int32 batch (65,536 pairs, the
             batch workload) with eps^2 = the median delta^2 of its first
             2,048 pairs; rate over all candidate cells, abandoned share.
    dtw      DTW of 16,384 float32 2-D Gaussian-walk pairs, lengths U{16..512}.
    lev      Levenshtein distance of 16,384 pairs of int32 symbol sequences
             over {0..3}, lengths U{16..512}.
    mc       4,096 Monte Carlo samples of one pair of 512-point 2-D walks,
             both curves perturbed by 0.05 * N(0, 1) per coordinate.
    """
    import torch
    import oracle
    from paper_2404_05708_gb300 import build, dfd, workloads
    build.build()
    oracle.load()
    torch.cuda.set_device(0)
    ctx = dfd.Context(0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    steps, warmup = max(args.steps, 3), max(args.warmup, 3)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    def roof(op, cells, ms):
        rate, mhz = dfd.dfd_microbench(ctx.handle, dfd.MICRO_OPS[op])
        mix = rate * sms * mhz * 1e6 / 1e9
        ach = cells / (ms * 1e-3) / 1e9
        out = {"bound": "alu", "achieved": ach, "unit": "Gcell/s",
               "measured_mix": {"peak": mix, "frac": ach / mix,
                                "basis": f"measured mix {op} {rate:.2f} cells/clk/SM x {sms} SMs x {mhz:.0f} MHz"}}
        if op in MIX_INSTR_PER_CELL:
            peak = 128.0 / MIX_INSTR_PER_CELL[op] * sms * mhz * 1e6 / 1e9
            out.update(peak=peak, frac=ach / peak,
                       peak_basis=f"issue bound: 128 lane-instructions/clk/SM / {MIX_INSTR_PER_CELL[op]:.0f} "
                                  f"instructions per cell x {sms} SMs x {mhz:.0f} MHz")
        else:
            out.update(peak=mix, frac=ach / mix, peak_basis=out["measured_mix"]["basis"])
        return out

    def ragged(n_pairs, seed, gen):
        rng = np.random.default_rng(seed)
        lens = rng.integers(16, 513, size=2 * n_pairs)
        off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        pts = gen(rng, int(off[-1]))
        pairs = np.arange(2 * n_pairs, dtype=np.int32).reshape(-1, 2)
        return pts, off, pairs, lens

    rows = []
    # decider
    b = workloads.ragged_int_batch()
    ln = b.lengths()
    cells = int(np.sum(ln[b.pairs[:, 0]] * ln[b.pairs[:, 1]]))
    ref, _ = oracle.batch(b.points, b.offsets, b.pairs[:2048])
    eps2 = float(np.median(ref))
    P, O, Q = (torch.from_numpy(x).cuda() for x in (b.points, b.offsets, b.pairs))
    out = {}
    def dec():
        out["r"] = ctx.decide(P, O, Q, eps2)
    ms = timed(dec)
    d2, within, ab = out["r"]
    ok = bool(np.array_equal(within[:2048].cpu().numpy().astype(bool), ref <= eps2))
    rows.append({"row": "decider", "pairs": int(b.pairs.shape[0]), "cells_per_step": cells, "ms": ms,
                 "gcups_all_cells": cells / (ms * 1e-3) / 1e9, "eps2": eps2,
                 "abandoned": int(ab.item()) / b.pairs.shape[0], "verified_vs_oracle": ok})
    # DTW
    pts, off, pairs, lens = ragged(16384, 11, lambda rng, n: np.cumsum(rng.normal(0, 1, size=(n, 2)), axis=0)
                                   .astype(np.float32))
    cells = int(np.sum(lens[0::2] * lens[1::2]))
    P, O, Q = (torch.from_numpy(x).cuda() for x in (pts, off, pairs))
    ms = timed(lambda: out.__setitem__("r", ctx.dtw(P, O, Q)))
    got = out["r"][:256].cpu().numpy()
    want = np.array([oracle.dtw_f32mirror(pts[off[2 * i]:off[2 * i + 1]], pts[off[2 * i + 1]:off[2 * i + 2]])
                     for i in range(256)], np.float32)
    rows.append({"row": "dtw", "pairs": 16384, "cells_per_step": cells, "ms": ms,
                 "gcups": cells / (ms * 1e-3) / 1e9, "verified_vs_oracle": bool(np.array_equal(got, want)),
                 "roofline": roof("cell_dtw_f32_d2", cells, ms)})
    # Levenshtein
    sym, off, pairs, lens = ragged(16384, 12, lambda rng, n: rng.integers(0, 4, size=(n, 1)).astype(np.int32))
    cells = int(np.sum(lens[0::2] * lens[1::2]))
    P, O, Q = (torch.from_numpy(x).cuda() for x in (sym, off, pairs))
    ms = timed(lambda: out.__setitem__("r", ctx.levenshtein(P, O, Q)))
    got = out["r"][:256].cpu().numpy()
    want = np.array([oracle.levenshtein(sym[off[2 * i]:off[2 * i + 1], 0], sym[off[2 * i + 1]:off[2 * i + 2], 0])
                     for i in range(256)], np.int64)
    rows.append({"row": "levenshtein", "pairs": 16384, "cells_per_step": cells, "ms": ms,
                 "gcups": cells / (ms * 1e-3) / 1e9, "verified_vs_oracle": bool(np.array_equal(got, want)),
                 "roofline": roof("cell_lev_i32", cells, ms)})
    # Monte Carlo
    rng = np.random.default_rng(13)
    p = np.cumsum(rng.normal(0, 1, size=(512, 2)), axis=0).astype(np.float32)
    q = np.cumsum(rng.normal(0, 1, size=(512, 2)), axis=0).astype(np.float32)
    S = 4096
    zp = rng.normal(0, 1, size=(S, 512, 2)).astype(np.float32)
    zq = rng.normal(0, 1, size=(S, 512, 2)).astype(np.float32)
    Pd, Qd, Zp, Zq = (torch.from_numpy(x).cuda() for x in (p, q, zp, zq))
    ms = timed(lambda: out.__setitem__("r", ctx.mc_pair(Pd, Qd, Zp, Zq, 0.05, 0.05)))
    d2 = out["r"][1].cpu().numpy()
    ok = all(d2[s] == np.float32(oracle.dfd2_f32mirror(oracle.perturb(p, zp[s], 0.05), oracle.perturb(q, zq[s], 0.05)))
             for s in (0, 1, 2047, 4095))
    cells = S * 512 * 512
    rows.append({"row": "monte_carlo", "samples": S, "cells_per_step": cells, "ms": ms,
                 "gcups": cells / (ms * 1e-3) / 1e9, "verified_vs_oracle": bool(ok),
                 "roofline": roof("cell_f32_d2", cells, ms)})
    ctx.close()
    out_line = {"metric": METRIC, "value": rows[1]["gcups"], "unit": UNIT, "n_gpus": 1, "steps": steps,
                "warmup": warmup, "higher_is_better": True, "dtype": "mixed", "data": "synthetic",
                "config": {"workload": "rows after the hot path: early-abandon decider, DTW, Levenshtein, "
                                       "Monte Carlo samples (value: DTW)"},
                "rows": rows}
    print(json.dumps(out_line))
    return 0


def run_paper(args):
    """The paper's own experiment shape (Sec. 4, Experiment 1), as context:
    N pairs of 2-D float32 walks with steps uniform in {-1,0,1}^2, (i)
    P = Q = 2^10 points with N = 2^5 ... 2^14 pairs, (ii) N = 2^10 pairs with
    P = Q = 2^5 ... 2^14 points.  Each point runs as one dfd_batch launch,
    once with one warp per pair (for P > 4096 with the row buffer widened to
    P) and once with CTA teams for the pairs of several stripes.
    From P = 2^12 on the same pairs also run through dfd_pair (the band
    wavefront), one launch per pair, spread over 16 contexts each on its own
    stream so that several pairs share the GPU.  L2 is flushed before each
    step (untimed); CUDA events time each step after --warmup; the first
    pairs of every point are checked bit-exact against the oracle's float32
    mirror.
    """
    import torch
    import oracle
    from paper_2404_05708_gb300 import build, dfd, workloads
    build.build()
    oracle.load()
    torch.cuda.set_device(0)
    steps, warmup = max(args.steps, 3), max(args.warmup, 3)
    ctx = dfd.Context(0)
    n_ctx = 16
    side = [dfd.Context(0) for _ in range(n_ctx)]
    streams = [torch.cuda.Stream() for _ in range(n_ctx)]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mix_rate, mix_mhz = dfd.dfd_microbench(ctx.handle, dfd.MICRO_OPS["cell_f32_d2"])
    # issue bound of the float32 2-D cell (4 lane-instructions per cell)
    peak = 128.0 / MIX_INSTR_PER_CELL["cell_f32_d2"] * sms * mix_mhz * 1e6 / 1e9

    def timed(fn):
        for _ in range(warmup):
            fn()
        total = 0.0
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
        return total / steps

    rows = []
    points = [("i", 1 << 10, 1 << k) for k in (5, 7, 9, 11, 13, 14)] + \
             [("ii", 1 << k, 1 << 10) for k in (5, 7, 9, 11, 12, 13, 14)]
    if args.paper_points:
        keep = {tuple(int(x) for x in pn.split("x")) for pn in args.paper_points.split(",")}
        points = [pt for pt in points if (pt[1], pt[2]) in keep]
    for sweep, P, N in points:
        b = workloads.paper_walks(N, P)
        cells = N * P * P
        pts = torch.from_numpy(b.points).cuda()
        O, Q = torch.from_numpy(b.offsets).cuda(), torch.from_numpy(b.pairs).cuda()
        nchk = 8 if P <= 4096 else 1
        mirror, _ = oracle.batch(b.points, b.offsets, b.pairs[:nchk], mirror=True)
        if P > 4096:
            ctx.set_batch_row_buffer(P)   # one warp per pair needs a row of P columns per warp
        out = {}
        for mode, engine in ((0, "dfd_batch, one launch, size classes chosen by the plan (default)"),
                             (1, "dfd_batch, one launch, one warp per pair"),
                             (2, "dfd_batch, one launch, CTA teams for pairs of several stripes")):
            if mode != 1 and P <= 256:
                continue                  # one stripe: no team pairs
            ctx.set_batch_team(dfd.DFD_F32, 2, mode)
            ms = timed(lambda: out.__setitem__("r", ctx.batch(pts, O, Q)))
            d2 = out["r"][1][:nchk].cpu().numpy()
            ok = bool(np.array_equal(d2, mirror)) and ctx.get_error() == 0
            # the same call captured once in a CUDA graph (the batch API's hot path:
            # one graph launch per step instead of the call's six launches)
            graph, _, g2 = ctx.batch(pts, O, Q, capture=True)
            ms_g = timed(graph.launch)
            ok_g = bool(np.array_equal(g2[:nchk].cpu().numpy(), mirror)) and ctx.get_error() == 0
            graph.close()
            rows.append({"sweep": sweep, "P": P, "N": N, "cells_per_step": cells, "ms": ms,
                         "gcups": cells / (ms * 1e-3) / 1e9, "engine": engine, "team_mode": mode,
                         "roofline_frac": cells / (ms * 1e-3) / 1e9 / peak,
                         "graph_ms": ms_g, "graph_gcups": cells / (ms_g * 1e-3) / 1e9,
                         "verified_vs_oracle": ok and ok_g})
        ctx.set_batch_team(dfd.DFD_F32, 2, 0)
        if P >= 4096:
            curves = [pts[b.offsets[c]:b.offsets[c + 1]] for c in range(2 * N)]
            od = torch.empty(N, dtype=torch.float32, device="cuda")
            od2 = torch.empty(N, dtype=torch.float32, device="cuda")
            cur = torch.cuda.current_stream()

            def wave_all():
                for s in streams:
                    s.wait_stream(cur)
                for i in range(N):
                    k = i % n_ctx
                    side[k].pair(curves[2 * i], curves[2 * i + 1], out_dist=od[i:i + 1], out_dist2=od2[i:i + 1],
                                 stream=streams[k].cuda_stream)
                for s in streams:
                    cur.wait_stream(s)
            ms = timed(wave_all)
            rows.append({"sweep": sweep, "P": P, "N": N, "cells_per_step": cells, "ms": ms,
                         "gcups": cells / (ms * 1e-3) / 1e9,
                         "engine": f"dfd_pair per pair (band wavefront), {n_ctx} contexts on their own streams",
                         "verified_vs_oracle": bool(np.array_equal(od2[:nchk].cpu().numpy(), mirror))})
        del pts, O, Q
    for c in side:
        c.close()
    ctx.close()
    out_line = {"metric": METRIC, "value": max(r["gcups"] for r in rows), "unit": UNIT, "n_gpus": 1, "steps": steps,
                "warmup": warmup, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "the paper's Experiment 1 shape: N pairs of 2-D walks, steps in {-1,0,1}^2, "
                                       "(i) P=Q=2^10, N=2^5..2^14, (ii) N=2^10, P=Q=2^5..2^14 (value: best point)",
                           "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MB write)",
                           "roofline_peak": {"value": peak, "unit": "Gcell/s",
                                             "basis": f"issue bound: 128 lane-instructions/clk/SM / 4 instructions "
                                                      f"per float32 2-D cell x {sms} SMs x {mix_mhz:.0f} MHz "
                                                      f"(measured mix cell_f32_d2: {mix_rate:.2f} cells/clk/SM)"}},
                "rows": rows}
    print(json.dumps(out_line))
    return 0


# -------------------------------------------------------------- reference
def run_reference(args):
    """CPU oracle on host cores, bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_2404_05708_gb300 import workloads
    oracle.load()
    if args.workload in ("long", "pair2k"):
        if args.workload == "long":
            p, q = workloads.warped_long_pair(args.n, args.m, dim=DIM, seed=SEED)
            a = min(REF_SAMPLE, args.n, args.m)
            ps, qs = p[:a].copy(), q[:a].copy()
            sample = f"prefix p[:{a}], q[:{a}] of the {args.n}x{args.m} pair per step (Alg. 5, float64, 1 thread)"
            cfg = {"workload": long_workload(args.n, args.m), "n": args.n, "m": args.m, "dim": DIM,
                   "cells_per_step": args.n * args.m}
        else:
            ps, qs = workloads.gaussian_walk_pair(2000, 1500, dim=2)
            sample = "the full 2000x1500 pair per step (Alg. 5, float64, 1 thread)"
            cfg = {"workload": PAIR2K_WORKLOAD, "n": 2000, "m": 1500, "dim": 2, "cells_per_step": 2000 * 1500}
        cells_step = ps.shape[0] * qs.shape[0]
        for _ in range(args.warmup):
            oracle.dfd2_linear(ps, qs)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            oracle.dfd2_linear(ps, qs)
        dt = time.perf_counter() - t0
        cores, dtype = 1, "f64"
    elif args.workload not in ("batch", "matrix", "paper"):
        print(json.dumps({"impl": "reference", "unavailable": f"no oracle arm for --workload {args.workload}: it "
                                                              "covers long, pair2k, batch, matrix and paper"}))
        return 0
    else:
        if args.workload == "paper":
            b = workloads.paper_walks(1 << 10, 1 << 10)
            pairs = b.pairs[:64]
            dtype = "f64"
            cfg = {"workload": "the paper's Experiment 1 shape, point P=Q=2^10, N=2^10 pairs of 2-D walks",
                   "P": 1024, "N": 1024, "cells_per_step": 1024 * 1024 * 1024}
            sample = "first 64 pairs of the point per step (Alg. 5, float64, all host threads)"
        elif args.workload == "batch":
            b = workloads.ragged_int_batch()
            pairs = b.pairs[:4096]
            dtype = "int64"
            cfg = {"workload": BATCH_WORKLOAD.format(n=b.pairs.shape[0]), "n_pairs": int(b.pairs.shape[0]), "dim": 2,
                   "cells_per_step": int(np.sum(b.lengths()[b.pairs[:, 0]] * b.lengths()[b.pairs[:, 1]]))}
            sample = "first 4096 pairs of the batch per step (Alg. 5, int64, all host threads)"
        else:
            b = workloads.ar1_curves()
            rng = np.random.default_rng(3)
            pairs = np.stack([rng.integers(0, 4096, 4096), rng.integers(0, 4096, 4096)], 1).astype(np.int32)
            dtype = "f64"
            ln_all = b.lengths().astype(np.int64)
            cfg = {"workload": MATRIX_WORKLOAD.format(n=4096), "n_curves": 4096, "n_pairs": 4096 * 4095 // 2, "dim": 16,
                   "cells_per_step": int((ln_all.sum() ** 2 - (ln_all ** 2).sum()) // 2)}
            sample = "4096 random pairs per step (Alg. 5, float64, all host threads)"
        ln = b.lengths()
        cells_step = int(np.sum(ln[pairs[:, 0]] * ln[pairs[:, 1]]))
        for _ in range(args.warmup):
            oracle.batch(b.points, b.offsets, pairs)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            _, cores = oracle.batch(b.points, b.offsets, pairs)
        dt = time.perf_counter() - t0
    v = cells_step * args.steps / dt / 1e9
    out = {
        "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": cfg,
        "impl": "reference",
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "host_cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))
    return 0


# ------------------------------------------------------------------ ours
def timed_steps(wl, ctx, dfd, torch, steps, warmup, flush, world, kernel_timed):
    """W untimed steps, then K steps each bracketed by CUDA events on the
    launching stream, L2 flushed before each (outside the events); the
    library's own event pair around the main kernel when `kernel_timed`.
    Returns (total device ms, per-step kernel ms, clocks sampled meanwhile)."""
    import torch.distributed as dist
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        flush.zero_()
        wl.step()
    torch.cuda.synchronize()
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid).replace("GPU-", "")
    except Exception:
        gpu_id = None
    sampler = ClockSampler(gpu_id)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    kernel_ms = []
    for k in range(steps):
        flush.zero_()                       # L2 flush outside the timed events
        ev[k][0].record(stream)
        wl.step()
        ev[k][1].record(stream)
        if kernel_timed:
            try:
                kernel_ms.append(dfd.dfd_timing_last(ctx.handle))
            except dfd.DFDError:
                kernel_timed = False        # the step has no readable pair of library events
                kernel_ms = []
    torch.cuda.synchronize()
    step_ms = [x.elapsed_time(y) for x, y in ev]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    torch.cuda.synchronize()
    clocks = sampler.stop()
    # the library's kernel events must sit inside the step's (a graph
    # captured without them, or a failed read, falls back to the whole step)
    if kernel_ms and not all(0 < km <= sm * 1.0001 for km, sm in zip(kernel_ms, step_ms)):
        kernel_ms = []
    return total_ms, kernel_ms, clocks


# Instructions per cell of the kernels' own cell (lane-instructions): the
# roofline peak is the issue bound from the unit counts, 4 sub-partitions x
# 32 lanes = 128 lane-instructions per clock per SM, over these -- a hard
# upper bound.  (The measured mix kernels are reported beside it as context:
# their per-block timing windows can overstate, e.g. the uint32-bits mix of
# 6 instructions per cell timed at 28.0 cells/clk/SM, above the 21.3 that
# issue allows.)  float32 cells run two rows per f32x2 instruction.
MIX_INSTR_PER_CELL = {
    "cell_f32_d3": 5.0,      # (3 sub + mul + 2 fma) / 2 rows, min3, max
    "cell_f32_d2": 4.0,      # (2 sub + mul + fma) / 2 rows, min3, max
    "cell_i32b_d2": 5.0,     # |p|^2 + |q|^2 - 2 p.q: add and 2 multiply-adds, min3, max
    "cell_f32_d16": 18.0,    # (16 sub + mul + 15 fma) / 2 rows, min3, max
    "cell_dtw_f32_d2": 6.0,  # sub, sub, mul, fma, min3, add
}


def alu_roofline(wl, ctx, dfd, sms, clocks, kernel_ms, total_ms, steps):
    """ALU roofline of the workload's cell mix (cell-weighted over the mixes
    it runs: time adds per cell).  peak = the issue bound from the unit
    counts when every mix has a defined instruction count, else the measured
    mix rate; both are reported."""
    mixes = wl.micro_mix() if hasattr(wl, "micro_mix") else [(wl.micro_op, wl.cells)]
    inv, basis, mb_mhz = 0.0, [], 0.0
    tot = max(sum(c for _, c in mixes), 1)
    for op, cells in mixes:
        cell_rate, mb_mhz = dfd.dfd_microbench(ctx.handle, dfd.MICRO_OPS[op])
        inv += cells / tot / cell_rate
        basis.append(f"{op} {cell_rate:.2f} cells/clk/SM on {cells / tot:.1%} of cells")
    clk = clocks["sm_mhz"] if clocks else mb_mhz
    mix_peak = (1.0 / inv) * sms * clk * 1e6 / 1e9
    kern_avg = (sum(kernel_ms) / len(kernel_ms)) if kernel_ms else total_ms / steps
    work_cells = wl.evaluated_cells() if hasattr(wl, "evaluated_cells") else wl.cells
    achieved = work_cells / (kern_avg * 1e-3) / 1e9
    mix_basis = f"measured mix ({'; '.join(basis)}) x {sms} SMs x {clk:.0f} MHz"
    if all(op in MIX_INSTR_PER_CELL for op, _ in mixes):
        ipc = sum(c / tot * MIX_INSTR_PER_CELL[op] for op, c in mixes)
        peak = 128.0 / ipc * sms * clk * 1e6 / 1e9
        peak_basis = (f"issue bound: 128 lane-instructions/clk/SM / {ipc:.2f} instructions per cell "
                      f"x {sms} SMs x {clk:.0f} MHz")
    else:
        peak, peak_basis = mix_peak, mix_basis
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gcell/s", "frac": achieved / peak,
                "traffic": TRAFFIC_BY_KERNEL_SHA.get(
                    wl.config.get("kernel_sha", "") + (f"/{wl.traffic_tag}" if getattr(wl, "traffic_tag", None) else "")),
                "peak_basis": peak_basis,
                "measured_mix": {"peak": mix_peak, "frac": achieved / mix_peak, "basis": mix_basis}}
    roofline["timing"] = (getattr(wl, "kernel_timing", "main kernel") + ", the library's CUDA events on the launching stream"
                          if kernel_ms else "whole step (all launches of the step)")
    if hasattr(wl, "evaluated_cells"):
        roofline["achieved_basis"] = (f"recurrence cells actually evaluated ({work_cells:.3e} per step; "
                                      f"value counts all {wl.cells:.3e} candidate cells)")
    return roofline


def long_pair_summary(args, ctx, dfd, torch, workloads, flush, sms):
    """The 200,000^2 3-D float32 pair through dfd_pair, for the batch line."""
    la = argparse.Namespace(**vars(args))
    la.n, la.m, la.shape, la.no_autotune = N_POINTS, N_POINTS, "", False
    wl = LongPair(la, ctx, dfd, torch, workloads, 0, 1)
    steps, warmup = 5, 3
    total_ms, kernel_ms, clocks = timed_steps(wl, ctx, dfd, torch, steps, warmup, flush, 1, True)
    roof = alu_roofline(wl, ctx, dfd, sms, clocks, kernel_ms, total_ms, steps)
    out = {"workload": wl.config["workload"], "value": wl.cells * steps / (total_ms * 1e-3) / 1e9, "unit": UNIT,
           "steps": steps, "warmup": warmup, "ms_per_step": total_ms / steps,
           "launch_shape": wl.config["launch_shape"], "fronts": wl.config["fronts"],
           "roofline": roof, "verified_vs_oracle": wl.verify(), "clocks": clocks}
    del wl
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serve":
        return run_serving(args)
    if args.workload == "next":
        return run_next(args)
    if args.workload == "paper":
        return run_paper(args)

    import torch
    import torch.distributed as dist
    from paper_2404_05708_gb300 import build, dfd, workloads

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()

    ctx = dfd.Context(local)
    dfd.dfd_timing_enable(ctx.handle, True)
    wl = WORKLOADS[args.workload](args, ctx, dfd, torch, workloads, rank, world)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    kernel_timed = args.workload in ("long", "pair2k", "batch")
    total_ms, kernel_ms, clocks = timed_steps(wl, ctx, dfd, torch, args.steps, args.warmup, flush, world,
                                              kernel_timed)
    if world > 1:
        c = torch.tensor([wl.cells], device="cuda", dtype=torch.float64)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
        total_cells = float(c.item())
        dist.barrier()
    else:
        total_cells = float(wl.cells)
    value = total_cells * args.steps / (total_ms * 1e-3) / 1e9
    verified = wl.verify()

    # end to end through the public API with host buffers (the first call
    # grows the context's staging areas: the warm-up takes at least 3 calls)
    e2e_times = []
    e2e_warm = max(args.warmup, 3)
    for k in range(e2e_warm + args.steps):
        t0 = time.perf_counter()
        wl.e2e_step()
        if k >= e2e_warm:
            e2e_times.append(time.perf_counter() - t0)
    e2e_total = sum(e2e_times)
    if world > 1:
        t = torch.tensor([e2e_total], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_total = float(t.item())
    e2e_value = total_cells * args.steps / e2e_total / 1e9

    sms = torch.cuda.get_device_properties(local).multi_processor_count
    if not kernel_ms and hasattr(wl, "kernel_ms"):
        kernel_ms = wl.kernel_ms(args.steps, flush)
    roofline = alu_roofline(wl, ctx, dfd, sms, clocks, kernel_ms, total_ms, args.steps)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = wl.cpu_baseline()
        cpu["host_cores"] = os.cpu_count()
    extra = wl.per_pair() if rank == 0 else None

    cfg = dict(wl.config)
    cfg.update({"parallelism": (f"dp{world} (pairs sharded)" if args.workload in ("batch", "matrix")
                                else "replicas") if world > 1 else "single",
                "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MB write)", "verified_vs_oracle": verified})
    if extra:
        cfg["per_pair"] = extra
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong" if args.workload in ("batch", "matrix") else "weak", "vs_baseline": None,
        "dtype": wl.dtype, "data": "synthetic", "config": cfg, "roofline": roofline, "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": wl.h2d, "d2h_bytes_per_step": wl.d2h,
                "step_ms": [round(t * 1e3, 3) for t in e2e_times]},
        "gpu_launches": wl.launches_per_step * args.steps,
        "clocks": clocks,
    }
    del wl
    if args.workload == "batch" and world == 1 and not args.no_extras:
        # the served form and the long pair on the same GPU, after the batch
        rates = [float(r) for r in args.extra_rates.split(",") if r]
        if rates:
            out["serving"] = serve_sweep(ctx, rates, args.serve_seconds, args.serve_repeats, args.tick_cells,
                                         args.stripes_per_tick)
            out["serving_config"] = {"workload": SERVE_WORKLOAD, "tick_cells": args.tick_cells,
                                     "stripes_per_tick": args.stripes_per_tick,
                                     "seconds_of_arrivals": args.serve_seconds}
        out["long_pair"] = long_pair_summary(args, ctx, dfd, torch, workloads, flush, sms)
    if rank == 0:
        print(json.dumps(out))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


import numpy as np  # noqa: E402  (workload classes use it)

if __name__ == "__main__":
    sys.exit(main())
