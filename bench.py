#!/usr/bin/env python
"""Benchmark of the inter-visibility hot path on GB300.

Headline workload: the 25k-facet city (4 km square, 5,000 box buildings,
25,001 facets, 3 x 3 samples per facet, 100,000 Rx snapshots at 350 km/h
every 1 ms along a serpentine, rooftop Tx, reflection order 3).  One step =
one pass of the whole path over it: ivm_build_matrix (ingest, BVH, facing
screen, sample-pair occlusion), ivm_build_table (Tx and Rx rows and the
direct path per snapshot) and ivm_expand_image_tree (orders 0..3, counts
and fingerprints).

Metric: visibility pair-tests per second: the N^2 ordered facet pairs the
matrix decides plus the 2 N S Tx/Rx-facet pairs the table decides, per step,
divided by the step time.  Snapshot tables per second (S / step time) is
reported beside it.  Three forms run on the same step: fast (FP32 filter with
exact fallback, persistent queues, occluder caches, row deduplication, graph
replay, autotuned shape), plain (exact integer tests, one warp per item, no
caches) and learned (fast + the trained cluster ranker); their outputs are
compared bit for bit.

`value` is device time (CUDA events on the library's stream) with inputs
resident in HBM; L2 is flushed between steps by writing a 512 MB buffer
outside the timed events.  `e2e` is the same metric through the same C-ABI
calls with pinned host buffers (every copy inside the timed region).
Beside the headline: the roofline of the dominant kernel (FP32 work per
Sec. 8(d)'s count of the method's tests), the precision form on the
degenerate district (undecided fraction, mismatches against stored
brute-force oracle bits), the 64-scene batch (one batched, persistent,
graph-replayed call per phase against the plain form), the district step and
the district's further outputs (visibility ranges, ray validation, edges,
interface relations), and the CPU oracle on the host cores.
`--impl reference` times the CPU oracle on the city instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "visibility pair-tests/s and Tx/Rx snapshot tables/s, bit-exact, vs plain GPU form"
UNIT = "pair-tests/s"
CITY = ("city: 4 km x 4 km, 5,000 box buildings (8-40 m footprint, 6-60 m high), 25,001 facets, "
        "3x3 samples per facet, 100,000 Rx snapshots at 350 km/h every 1 ms along a serpentine, "
        "rooftop Tx, reflection order <= 3, seed 5")
DISTRICT = ("district: 1 km x 1 km, 200 box buildings (8-40 m footprint, 6-60 m high), "
            "1,001 facets, 5x5 samples per facet, 10,000 Rx snapshots at 120 km/h every 1 ms, "
            "rooftop Tx, reflection order <= 3, seed 2")
# FP32 work per test, as the method's algorithmic count: a segment-box slab
# test about 12 FLOP, a segment-facet test about 50 FLOP; a fused multiply-add
# counts as 2 FLOP in the peak.
FLOP_PER_BOX_TEST = 12
FLOP_PER_FACET_TEST = 50
GOLDEN = os.path.join(ROOT, "tests", "golden")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    # profiling case: one phase of one form on a slice of a workload (no JSON contract line)
    p.add_argument("--profile", choices=["matrix", "table", "tree", "step"], default=None)
    p.add_argument("--workload", choices=["city", "district"], default="city")
    p.add_argument("--form", choices=["fast", "fast_edge_filter", "plain", "learned"],
                   default="fast")
    p.add_argument("--snapshots", type=int, default=None)
    p.add_argument("--rows", type=int, default=None,
                   help="profiling: decide only the pairs of the first ROWS matrix rows")
    p.add_argument("--shape", default=None,
                   help="profiling: launch shape tile,warps_per_block,table_tile[,proof_tile"
                        "[,corner proof 0/1]] instead of the autotuner's")
    return p.parse_args()


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "25"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # the sampler takes a moment to start: wait for its first sample so that
        # the samples cover the timed region that follows
        t0 = time.time()
        while time.time() - t0 < 5.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.05)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        with open(self.path) as fh:
            lines = fh.readlines()
        os.unlink(self.path)
        return Clocks.summarize(lines)

    @staticmethod
    def summarize(lines):
        """Median SM clock, the highest max clock and the throttle reasons seen
        in nvidia-smi's CSV lines (the FIELDS order, no header, no units)."""
        rows = []
        for line in lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------------ CPU oracle

def oracle_sample(sc, n_rows, n_snaps, seed, threads, mode):
    """Oracle on a bounded sample of the workload; returns (pair tests, s)."""
    import numpy as np

    import oracle
    rng = np.random.default_rng(seed)
    rows = rng.choice(sc.n_facets, n_rows, replace=False)
    snaps = rng.choice(sc.n_snap, n_snaps, replace=False)
    t0 = time.perf_counter()
    oracle.matrix(sc.facets, sc.samples_per_side, rows=rows, threads=threads, mode=mode)
    oracle.table(sc.facets, sc.samples_per_side, sc.tx, sc.rx, snaps=snaps, threads=threads,
                 mode=mode)
    dt = time.perf_counter() - t0
    units = n_rows * sc.n_facets + 2 * n_snaps * sc.n_facets
    return units, dt


ORACLE_GRID = ("oracle/ivm_oracle.c in grid mode: the brute-force definition's exact int128 "
               "triangle test, each segment tested against the triangles an exact xy grid "
               "cannot rule out (bit-identical to brute force, which is infeasible at this "
               "size: about 3e16 triangle tests for the matrix)")


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle
    from paper_2501_02747_gb300 import scenegen as sg
    oracle.build()
    sc = sg.city()
    threads = os.cpu_count() or 1
    for k in range(args.warmup):
        oracle_sample(sc, 1, 2, 100 + k, threads, "grid")
    units = 0
    secs = 0.0
    for k in range(args.steps):
        u, dt = oracle_sample(sc, 16, 32, 200 + k, threads, "grid")
        units += u
        secs += dt
    value = units / secs
    sample = ("per step: 16 seeded matrix rows (16 x 25,001 ordered pairs) and 32 seeded "
              "snapshots (32 x 2 x 25,001 Tx/Rx-facet pairs) of the city workload")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "int128",
        "data": "synthetic",
        "config": {"workload": CITY, "oracle": ORACLE_GRID},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ------------------------------------------------------------------ GPU arm

def traffic_from_profiles(kernel):
    """dram bytes per launch of `kernel` from profiles/, if taken on the current sources."""
    from paper_2501_02747_gb300 import build
    path = os.path.join(ROOT, "profiles", f"traffic_{kernel}.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_digest") != build._digest():
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def fp32_flop(st):
    """The method's algorithmic FP32 work in one call's traversal, from its own
    counters: box tests x 12 plus facet tests x 50."""
    return st["node_tests"] * FLOP_PER_BOX_TEST + st["leaf_tests"] * FLOP_PER_FACET_TEST


def popcount(a):
    import numpy as np
    return int(np.unpackbits(np.ascontiguousarray(a).view(np.uint8)).sum())


def fast_flags(ivm):
    """The fast form: persistent queues, occluder caches, row deduplication,
    graph replay and the rectangle test for axis-aligned facets."""
    return (ivm.IVM_FLAG_PERSISTENT | ivm.IVM_FLAG_OCCLUDER_CACHE | ivm.IVM_FLAG_DEDUP_SOURCES |
            ivm.IVM_FLAG_GRAPH | ivm.IVM_FLAG_ALIGNED_FACETS)


def runs(pos):
    """Runs of equal consecutive positions in an [S][3] trajectory."""
    import numpy as np
    if len(pos) == 0:
        return 0
    return 1 + int((np.diff(pos, axis=0) != 0).any(axis=1).sum())


class Path:
    """Device buffers and the three calls of one step over one scene; with
    ws > 1 this rank's share (its matrix rows, the all-reduce of the parts,
    then the table and tree of its snapshot range)."""

    def __init__(self, ivm, shard, ctx, sc, dev, ws, rank, tuned, stream):
        import torch
        self.ivm, self.shard, self.ctx, self.sc, self.ws = ivm, shard, ctx, sc, ws
        self.stream = stream
        N, S = sc.n_facets, sc.n_snap
        self.N, self.S, self.K, self.s = N, S, sc.max_order, sc.samples_per_side
        self.W = ivm.words(N)
        self.units = N * N + 2 * N * S   # the whole job's units (split across ranks)
        self.rows = shard.row_ranges(N, ws)[rank]
        self.snap = shard.snapshot_ranges(S, ws)[rank]
        self.fac = torch.from_numpy(sc.facets).to(dev)
        self.tx = torch.from_numpy(sc.tx).to(dev)
        self.rx = torch.from_numpy(sc.rx).to(dev)
        self.M = torch.empty((N, self.W), dtype=torch.int32, device=dev)
        self.T = torch.empty((S, 2, self.W), dtype=torch.int32, device=dev)
        self.L = torch.empty((S,), dtype=torch.uint8, device=dev)
        self.summ = torch.empty((S, self.K + 1, 3), dtype=torch.int64, device=dev)
        # the autotuner's choice of the matrix's corner proof joins the fast flags
        fast = fast_flags(ivm) | (tuned.get("flags", 0) & ivm.IVM_FLAG_NO_CORNER_PROOF)
        self.forms = {"plain": dict(mode=ivm.IVM_MODE_EXACT, flags=0),
                      "fast": dict(mode=ivm.IVM_MODE_FILTERED, flags=fast),
                      "fast_edge_filter": dict(mode=ivm.IVM_MODE_FILTERED,
                                               flags=fast & ~ivm.IVM_FLAG_ALIGNED_FACETS),
                      "learned": dict(mode=ivm.IVM_MODE_LEARNED, flags=fast)}
        self.tuned = tuned
        sm = {"tile": tuned["tile"], "warps_per_block": tuned["warps_per_block"]}
        stt = {"tile": tuned["table_tile"], "warps_per_block": tuned["warps_per_block"],
               "proof_tile": tuned.get("proof_tile", 0)}
        self.shape = {"plain": ({}, {}), "fast": (sm, stt), "fast_edge_filter": (sm, stt),
                      "learned": (sm, stt)}
        # rows the table actually traces: one per run of equal positions per side
        self.traced = N * N + N * sum(runs(p) for p in (sc.tx[self.snap[0]:self.snap[1]],
                                                        sc.rx[self.snap[0]:self.snap[1]]))

    def outputs(self):
        return (self.M, self.T, self.L, self.summ)

    def step(self, form, bufs=None, marks=None):
        """The three calls; `marks` (4 CUDA events) bracket them on the stream."""
        ivm = self.ivm
        fac, tx, rx, M, T, L, summ = bufs or (self.fac, self.tx, self.rx) + self.outputs()
        kw = self.forms[form]
        kw_m, kw_t = self.shape[form]
        if marks:
            marks[0].record(self.stream)
        if self.ws == 1:
            _, stm = ivm.ivm_build_matrix(self.ctx, fac, self.s, out=M, **kw, **kw_m)
        else:
            _, stm = ivm.ivm_build_matrix_rows(self.ctx, fac, self.s, self.rows, out=M, **kw,
                                               **kw_m)
            self.shard.exchange_matrix(M)
        if marks:
            marks[1].record(self.stream)
        a, b = self.snap
        _, stt = ivm.ivm_build_table(self.ctx, fac, self.s, tx[a:b], rx[a:b],
                                     out=(T[a:b], L[a:b]), **kw, **kw_t)
        if marks:
            marks[2].record(self.stream)
        ivm.ivm_expand_image_tree(self.ctx, M, T[a:b], L[a:b], self.N, self.K,
                                  summary=summ[a:b])
        if marks:
            marks[3].record(self.stream)
        return stm, stt


def timed(path, form, steps, warmup, flush, ws, clocks=None):
    """W untimed steps, then K steps timed with CUDA events on the library's
    stream, L2 flushed between them (outside the events); the max over ranks."""
    import torch
    ivm = path.ivm
    for _ in range(warmup):
        path.step(form)
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    launches0 = ivm.kernel_launches()
    times = []
    calls = {"matrix": 0.0, "table": 0.0, "tree": 0.0}
    kern = {"matrix": 0.0, "table": 0.0}
    flop = {"matrix": 0.0, "table": 0.0}
    stats = None
    torch.cuda.nvtx.range_push(f"timed_{form}")
    for _ in range(steps):
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        stm, stt = path.step(form, marks=ev)
        torch.cuda.synchronize()
        times.append(ev[0].elapsed_time(ev[3]))
        for k, name in enumerate(("matrix", "table", "tree")):
            calls[name] += ev[k].elapsed_time(ev[k + 1]) / steps
        stats = {"matrix": stm.as_dict(), "table": stt.as_dict()}
        for name in ("matrix", "table"):
            kern[name] += stats[name]["ms_traverse"] / steps
            flop[name] += fp32_flop(stats[name]) / steps
    torch.cuda.nvtx.range_pop()
    launches = ivm.kernel_launches() - launches0
    clk = clocks.stop() if clocks else None
    torch.cuda.synchronize()
    barrier(ws)
    ms = max_over_ranks(ws, sum(times)) / steps
    return {"ms": ms, "steps": steps, "warmup": warmup, "calls": calls, "kern": kern,
            "flop": flop, "stats": stats, "launches": launches, "clocks": clk}


def same_outputs(path, forms):
    """Runs one step per form and compares every output with the first's."""
    import torch
    ref = None
    agree = True
    for form in forms:
        path.step(form)
        torch.cuda.synchronize()
        now = tuple(x.clone() for x in path.outputs())
        if ref is None:
            ref = now
        else:
            agree &= all(bool((a == b).all()) for a, b in zip(ref, now))
        del now
    return agree


def roofline(t, ivm, ctx, n_sm, traffic_name):
    """Roofline of the dominant traversal kernel of a timed form `t`."""
    peaks = {}
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        peaks = json.load(open(p))
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    dom = "table" if t["kern"]["table"] >= t["kern"]["matrix"] else "matrix"
    kname = {"table": "k_table", "matrix": "k_matrix"}[dom]
    peak = n_sm * 128 * 2 * sm_max * 1e6 / 1e12
    ms = t["kern"][dom]
    achieved = t["flop"][dom] / (ms / 1e3) / 1e12 if ms > 0 else 0.0
    st = t["stats"][dom]
    ffma = 2 * ivm.ivm_fp32_peak(ctx) / 1e12
    return {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak if peak else None,
            "traffic": traffic_from_profiles(f"{kname}_{traffic_name}"),
            "peak_basis": f"nominal FP32: {n_sm} SMs x 128 lanes x 2 FLOP per FMA x "
                          f"{sm_max:.0f} MHz (sm_max_mhz of MEASURED_PEAKS.json)",
            "work_basis": f"{FLOP_PER_BOX_TEST} FLOP per segment-box test (node_tests) + "
                          f"{FLOP_PER_FACET_TEST} FLOP per segment-facet test (leaf_tests), per "
                          "launch: the method's tests counted by the library, each at the "
                          "FLOP of its plain FP32 form",
            "ms_per_launch": ms, "flop_per_launch": t["flop"][dom],
            "node_tests": st["node_tests"], "leaf_tests": st["leaf_tests"],
            "exact_tests": st["exact_tests"], "segments": st["segments"],
            "peak_measured_ffma": ffma,
            "frac_of_measured_ffma": achieved / ffma if ffma else None,
            "kernel_ms_per_step": dict(t["kern"])}


def profile_case(args, ivm, shard, sg, ctx, dev, stream):
    """One phase of one form on a slice of a workload (launch shape as timed);
    the calls after the warm-up run inside the NVTX range "profile_<phase>"
    (ncu --nvtx --nvtx-include).  Prints the last call's counters."""
    import dataclasses

    import torch
    sc = sg.city() if args.workload == "city" else sg.district()
    Sp = min(sc.n_snap, args.snapshots or sc.n_snap)
    sc = dataclasses.replace(sc, tx=sc.tx[:Sp], rx=sc.rx[:Sp])   # buffers for the slice only
    fd = torch.from_numpy(sc.facets).to(dev)
    tx = torch.from_numpy(sc.tx).to(dev)
    rx = torch.from_numpy(sc.rx).to(dev)
    if args.shape:
        v = [int(x) for x in args.shape.split(",")]
        tuned = {"tile": v[0], "warps_per_block": v[1], "table_tile": v[2],
                 "proof_tile": v[3] if len(v) > 3 else 0,
                 "flags": ivm.IVM_FLAG_NO_CORNER_PROOF if len(v) > 4 and v[4] == 0 else 0}
    else:
        tuned = ivm.ivm_autotune(ctx, fd, sc.samples_per_side, tx, rx,
                                 mode=ivm.IVM_MODE_FILTERED, flags=fast_flags(ivm))
    path = Path(ivm, shard, ctx, sc, dev, 1, 0, tuned, stream)
    if args.form == "learned":
        ivm.ivm_ranker_train(ctx, [sg.tiny().facets, sg.degenerate(n_snap=16).facets],
                             sc.samples_per_side, epochs=12, lr=2e-3)
    kw = path.forms[args.form]
    kw_m, kw_t = path.shape[args.form]
    s, N, K = path.s, path.N, path.K
    rows = (0, min(N, args.rows)) if args.rows else None
    st = None
    for it in range(args.warmup + args.steps):
        if it == args.warmup:
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_push(f"profile_{args.profile}")
        if args.profile in ("matrix", "step") or (args.profile == "tree" and it == 0):
            if rows:
                _, st = ivm.ivm_build_matrix_rows(ctx, fd, s, rows, out=path.M, **kw, **kw_m)
            else:
                _, st = ivm.ivm_build_matrix(ctx, fd, s, out=path.M, **kw, **kw_m)
        if args.profile in ("table", "step") or (args.profile == "tree" and it == 0):
            _, st = ivm.ivm_build_table(ctx, fd, s, tx, rx, out=(path.T, path.L), **kw, **kw_t)
        if args.profile in ("tree", "step"):
            ivm.ivm_expand_image_tree(ctx, path.M, path.T, path.L, N, K, summary=path.summ)
    torch.cuda.synchronize()
    if args.steps:
        torch.cuda.nvtx.range_pop()
    if args.profile in ("step", "tree"):
        st = None
    print(json.dumps({"profile": args.profile, "workload": args.workload, "form": args.form,
                      "snapshots": Sp, "rows": rows, "tuned": tuned,
                      "stats": st.as_dict() if st is not None else None}))


def district_block(args, ivm, shard, sg, ctx, dev, stream, flush):
    """The district step (fast and plain) and the district's further outputs,
    each timed on its own: visibility ranges with their blockers and the
    coherence time (Sec. III-C/D), image-method validation of image-tree
    candidates (Sec. IV-B), edge rows and the nearest edge (Sec. III-B), edges
    as matrix rows and columns, interface relations (Sec. II-B)."""
    import numpy as np
    import torch
    sc = sg.district()
    fd = torch.from_numpy(sc.facets).to(dev)
    tuned = ivm.ivm_autotune(ctx, fd, sc.samples_per_side, torch.from_numpy(sc.tx).to(dev),
                             torch.from_numpy(sc.rx).to(dev), mode=ivm.IVM_MODE_FILTERED,
                             flags=fast_flags(ivm))
    p = Path(ivm, shard, ctx, sc, dev, 1, 0, tuned, stream)
    tf = timed(p, "fast", args.steps, args.warmup, flush, 1)
    tp = timed(p, "plain", args.steps, args.warmup, flush, 1)
    agree = same_outputs(p, ["plain", "fast"])
    N, s = p.N, p.s
    p.step("fast")
    torch.cuda.synchronize()
    reps = max(3, min(args.steps, 10))

    def med(fn):
        ts = []
        for it in range(1 + reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = fn()
            torch.cuda.synchronize()
            if it:
                ts.append(1e3 * (time.perf_counter() - t0))
        return statistics.median(ts), r

    ms, (recs, rsum) = med(lambda: ivm.ivm_visibility_ranges(ctx, p.fac, s, p.tx, p.rx, p.T))
    tc = [rsum["snapshots"][x] / rsum["ranges"][x] if rsum["ranges"][x] else None
          for x in range(2)]   # snapshots 1 ms apart
    ranges_out = {
        "what": "visibility ranges (maximal runs of each table bit), first blocker at both ends "
                "of each, coherence time per Eq. (8)-(9); C-ABI call ivm_visibility_ranges on "
                "the step's table, records copied to host",
        "ms_per_call": ms, "ranges": int(len(recs)), "ranges_per_side": rsum["ranges"],
        "coherence_time_ms": {"tx": tc[0], "rx": tc[1],
                              "scenario": min(x for x in tc if x is not None) if any(tc) else None}}
    a0, a1, rk = 0, 4, 2
    _, n_cand = ivm.ivm_expand_image_tree(ctx, p.M, p.T[a0:a1], p.L[a0:a1], N, rk,
                                          count_paths=True)
    _, cand, n_cand, _ = ivm.ivm_expand_image_tree(ctx, p.M, p.T[a0:a1], p.L[a0:a1], N, rk,
                                                   paths_capacity=max(n_cand, 1))
    cand = cand[:n_cand]
    flags = torch.zeros(max(n_cand, 1), dtype=torch.uint8, device=dev)
    ms, _ = med(lambda: ivm.ivm_validate_paths(ctx, p.fac, s, p.tx[a0:a1], p.rx[a0:a1], cand,
                                               rk, out=flags[:n_cand]))
    rays_out = {"what": "image-method validation of image-tree candidates (orders 0-2) as "
                        "specular rays, C-ABI call ivm_validate_paths, snapshots 0..3",
                "candidates": int(n_cand), "valid_rays": int(flags[:n_cand].sum().item()),
                "ms_per_call": ms}
    E = torch.from_numpy(sg.edges_of(sc)).to(dev)
    ms, (etab, _) = med(lambda: ivm.ivm_build_edge_table(ctx, p.fac, s, E, p.tx, p.rx,
                                                         mode=ivm.IVM_MODE_FILTERED))
    ne = int(E.shape[0])
    edges_out = {"what": "edge rows (the 8 convex edges of every building, s samples each) and "
                         "the nearest visible edge per source, C-ABI call ivm_build_edge_table",
                 "edges": ne, "ms_per_call": ms,
                 "edge_tests_per_s": 2 * ne * p.S / (ms / 1e3)}
    EF = torch.from_numpy(sg.edge_faces_of(sc)).to(dev)
    fe = torch.zeros((N, (ne + 31) // 32), dtype=torch.int32, device=dev)
    ee = torch.zeros((ne, (ne + 31) // 32), dtype=torch.int32, device=dev)
    ms, _ = med(lambda: ivm.ivm_build_edge_matrix(ctx, p.fac, s, E, EF, out=(fe, ee)))
    edge_matrix_out = {"what": "edges as matrix rows and columns (facet-edge and edge-edge "
                               "bits), C-ABI call ivm_build_edge_matrix",
                       "facet_edge_pairs": N * ne, "edge_edge_pairs": ne * (ne - 1) // 2,
                       "ms_per_call": ms,
                       "facet_edge_bits": popcount(fe.cpu().numpy()),
                       "edge_edge_bits": popcount(ee.cpu().numpy())}
    ms, (rp, rr, _) = med(lambda: ivm.ivm_interface_relations(ctx, p.fac, s, p.M))
    relations_out = {"what": "PAR/PER relation and angular bouncing ranges of every visible "
                             "ordered pair, C-ABI call ivm_interface_relations",
                     "pairs": int(len(rp)), "par": int((rr == 1).sum()),
                     "per": int((rr == 2).sum()), "ms_per_call": ms}
    return {"workload": DISTRICT, "autotuned_shape": tuned,
            "fast": {"ms_per_step": tf["ms"], "value": p.units / (tf["ms"] / 1e3),
                     "ms_per_call": tf["calls"]},
            "plain": {"ms_per_step": tp["ms"], "value": p.units / (tp["ms"] / 1e3),
                      "ms_per_call": tp["calls"]},
            "speedup_vs_plain": tp["ms"] / tf["ms"], "forms_bit_identical": agree,
            "steps": args.steps, "warmup": args.warmup,
            "visibility_ranges": ranges_out, "ray_validation": rays_out, "edges": edges_out,
            "edge_matrix": edge_matrix_out, "interface_relations": relations_out}


def precision_block(ivm, sg, ctx, dev):
    """The precision form on the degenerate district: the fraction of FP32
    facet tests the filter could not decide (settled by exact integers), and
    mismatches against stored brute-force oracle bits: the full matrix and
    the table rows within 16 snapshots of each near-grazing snapshot."""
    import numpy as np
    import torch
    from tests.golden.make_oracle_matrices import digest, grazing_window
    sc = sg.degenerate()
    s = sc.samples_per_side
    fd = torch.from_numpy(sc.facets).to(dev)
    # the four-edge FP32 filter on every facet (no rectangle test): the precision form
    fast = fast_flags(ivm) & ~ivm.IVM_FLAG_ALIGNED_FACETS
    M, stm = ivm.ivm_build_matrix(ctx, fd, s, mode=ivm.IVM_MODE_FILTERED, flags=fast)
    (T, L), stt = ivm.ivm_build_table(ctx, fd, s, torch.from_numpy(sc.tx).to(dev),
                                      torch.from_numpy(sc.rx).to(dev),
                                      mode=ivm.IVM_MODE_FILTERED, flags=fast)
    torch.cuda.synchronize()
    out = {"workload": "degenerate district: the district family with 10 of 200 buildings "
                       "placed degenerately (shared wall spans, aligned facades, equal "
                       "heights, vertical edges on Tx-Rx lines at snapshots "
                       f"{sc.meta['grazing_snapshots']}), 5x5 samples, 10,000 snapshots",
           "form": "four-edge FP32 filter with a proven error bound on every facet test, exact "
                   "int64/int128 fallback where it cannot decide (+ persistent, caches, graph)"}
    for name, st in (("matrix", stm.as_dict()), ("table", stt.as_dict())):
        out[name] = {"facet_tests": st["leaf_tests"], "undecided": st["undecided"],
                     "undecided_fraction": st["undecided"] / st["leaf_tests"]
                     if st["leaf_tests"] else 0.0,
                     "ms_per_call": st["ms_total"]}
    zm = np.load(os.path.join(GOLDEN, "oracle_matrix_degenerate.npz"))
    zt = np.load(os.path.join(GOLDEN, "oracle_table_degenerate.npz"))
    snaps = grazing_window(sc)
    fresh = (str(zm["digest"]) == digest(sc.facets, s) and
             str(zt["digest"]) == digest(sc.facets, s, sc.tx[snaps], sc.rx[snaps]) and
             (zt["snaps"] == snaps).all())
    Mg = M.cpu().numpy().view(np.uint32)
    Tg = T.cpu().numpy().view(np.uint32)[snaps]
    Lg = L.cpu().numpy()[snaps]
    out["mismatches_vs_oracle"] = {
        "matrix_bits": popcount(Mg ^ zm["matrix"]) if fresh else None,
        "table_bits": popcount(Tg ^ zt["table"]) if fresh else None,
        "los": int((Lg != zt["los"]).sum()) if fresh else None,
        "checked": f"all {sc.n_facets}^2 matrix bits and the {len(snaps)} table rows and "
                   "direct paths within 16 snapshots of each near-grazing snapshot",
        "oracle": "brute force (every sample segment against every triangle, exact int128), "
                  "stored by tests/golden/make_oracle_matrices.py",
        "oracle_current": bool(fresh)}
    return out


def batch_block(args, ivm, sg, ctx, dev, stream, flush):
    """The 64-scene batch: each phase as one batched call (persistent queues
    over all scenes, graph replay, autotuned shape) against the plain form."""
    import torch
    scenes = sg.batch()
    s = 3
    fd = [torch.from_numpy(x.facets).to(dev) for x in scenes]
    tx = [torch.from_numpy(x.tx).to(dev) for x in scenes]
    rx = [torch.from_numpy(x.rx).to(dev) for x in scenes]
    fast = fast_flags(ivm)
    t0 = time.perf_counter()
    tuned = ivm.ivm_autotune(ctx, fd, s, tx, rx, mode=ivm.IVM_MODE_FILTERED, flags=fast)
    tune_s = time.perf_counter() - t0

    def bufs():
        Ms = [torch.empty((x.n_facets, ivm.words(x.n_facets)), dtype=torch.int32, device=dev)
              for x in scenes]
        Ts = [(torch.empty((x.n_snap, 2, ivm.words(x.n_facets)), dtype=torch.int32, device=dev),
               torch.empty((x.n_snap,), dtype=torch.uint8, device=dev)) for x in scenes]
        return Ms, Ts

    fast |= tuned["flags"] & ivm.IVM_FLAG_NO_CORNER_PROOF
    forms = {"fast": (dict(mode=ivm.IVM_MODE_FILTERED, flags=fast,
                           tile=tuned["tile"], warps_per_block=tuned["warps_per_block"]),
                      dict(mode=ivm.IVM_MODE_FILTERED, flags=fast,
                           tile=tuned["table_tile"], warps_per_block=tuned["warps_per_block"],
                           proof_tile=tuned["proof_tile"])),
             "plain": (dict(mode=ivm.IVM_MODE_EXACT), dict(mode=ivm.IVM_MODE_EXACT))}
    res, outs = {}, {}
    for form, steps, warm in (("fast", min(args.steps, 3), 1), ("plain", 1, 0)):
        Ms, Ts = bufs()
        kw_m, kw_t = forms[form]
        ms_m, ms_t = [], []
        for it in range(warm + steps):
            flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            ivm.ivm_build_matrix(ctx, fd, s, out=Ms, **kw_m)
            ev[1].record(stream)
            ivm.ivm_build_table(ctx, fd, s, tx, rx, out=Ts, **kw_t)
            ev[2].record(stream)
            torch.cuda.synchronize()
            if it >= warm:
                ms_m.append(ev[0].elapsed_time(ev[1]))
                ms_t.append(ev[1].elapsed_time(ev[2]))
        res[form] = {"steps": steps, "warmup": warm,
                     "matrix_ms_per_call": statistics.mean(ms_m),
                     "table_ms_per_call": statistics.mean(ms_t)}
        outs[form] = (Ms, Ts)
    agree = all(bool((a == b).all()) for a, b in zip(outs["fast"][0], outs["plain"][0]))
    agree &= all(bool((a[0] == b[0]).all()) and bool((a[1] == b[1]).all())
                 for a, b in zip(outs["fast"][1], outs["plain"][1]))
    units = sum(x.n_facets ** 2 + 2 * x.n_facets * x.n_snap for x in scenes)
    for form in res:
        ms = res[form]["matrix_ms_per_call"] + res[form]["table_ms_per_call"]
        res[form]["ms_per_step"] = ms
        res[form]["value"] = units / (ms / 1e3)
    return {"workload": "64 seeded scenes of 50-2,000 box buildings (251-9,786 facets, sum of "
                        "N^2 = 9.06e8), 791,715 snapshots in all, 3x3 samples",
            "form": "one batched call per phase over all 64 scenes: FP32 filter + exact "
                    "fallback, persistent work queues, caches, row deduplication, CUDA-graph "
                    "replay, launch shape from the autotuner",
            "autotuned_shape": tuned, "autotune_s": tune_s, "pair_tests_per_step": units,
            "fast": res["fast"], "plain": res["plain"],
            "speedup_vs_plain": res["plain"]["ms_per_step"] / res["fast"]["ms_per_step"],
            "forms_bit_identical": agree}


def run_ours(args, ws, rank, local):
    import torch

    from paper_2501_02747_gb300 import build, ivm, shard
    from paper_2501_02747_gb300 import scenegen as sg
    build.build()
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    stream = torch.cuda.current_stream(local)
    ctx = ivm.Context(local, stream)
    if args.profile:
        profile_case(args, ivm, shard, sg, ctx, dev, stream)
        ctx.close()
        return
    sc = sg.city()
    fast = fast_flags(ivm)
    # launch shape of the fast form from the library's autotuner (untimed)
    tuned = ivm.ivm_autotune(ctx, torch.from_numpy(sc.facets).to(dev), sc.samples_per_side,
                             torch.from_numpy(sc.tx).to(dev), torch.from_numpy(sc.rx).to(dev),
                             mode=ivm.IVM_MODE_FILTERED, flags=fast)
    path = Path(ivm, shard, ctx, sc, dev, ws, rank, tuned, stream)
    # the cluster ranker of the learned form, trained (untimed) on the exact
    # method's logged hits in the tiny and degenerate scenes
    t0 = time.perf_counter()
    train_loss = ivm.ivm_ranker_train(ctx, [sg.tiny().facets, sg.degenerate(n_snap=16).facets],
                                      path.s, epochs=12, lr=2e-3)
    train_s = time.perf_counter() - t0
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    tf = timed(path, "fast", args.steps, args.warmup, flush, ws, clocks=Clocks(local))
    # the plain and learned forms: fewer steps (plain takes about 12x longer)
    tl = timed(path, "learned", min(args.steps, 5), min(args.warmup, 2), flush, ws)
    te = timed(path, "fast_edge_filter", min(args.steps, 5), min(args.warmup, 2), flush, ws)
    tp = timed(path, "plain", min(args.steps, 2), min(args.warmup, 1), flush, ws)
    agree = same_outputs(path, ["plain", "fast", "fast_edge_filter", "learned"])
    N, S = path.N, path.S
    units = path.units
    value = units / (tf["ms"] / 1e3)
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count

    def per_seg(st, key):
        return st[key] / st["segments"] if st["segments"] else None

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tf["ms"], "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "int64/int128 + fp32 filter",
        "data": "synthetic",
        "config": {"workload": CITY,
                   "form": "fast: FP32 facet tests with proven error bounds (plane-crossing "
                           "test for axis-aligned rectangles, four-edge filter otherwise) and "
                           "exact fallback, persistent work queue, occluder cache, one row per "
                           "run of equal source positions, CUDA-graph replay of each call, "
                           "launch shape from the autotuner",
                   "l2": "flushed between steps (512 MB write)",
                   "facets": N, "snapshots": S, "samples_per_side": path.s,
                   "max_order": path.K, "pair_tests_per_step": units,
                   "autotuned_shape": tuned,
                   "parallelism": "one workload split over ranks: matrix rows of about equal "
                                  "pair counts, one all-reduce of the matrix parts, snapshot "
                                  "ranges for the table and tree" if ws > 1 else "1 GPU"},
        "snapshot_tables_per_s": S / (tf["ms"] / 1e3),
        "traced_pair_tests_per_step": path.traced,
        "value_traced": path.traced / (tf["ms"] / 1e3),
        "units_note": "pair tests per step = N^2 matrix pairs + 2 N S table pairs; the Tx is "
                      "static, so the table traces one Tx row and copies it over the route "
                      "(row deduplication): traced_pair_tests_per_step counts one row per run "
                      "of equal positions, value_traced is the rate on those",
        "ms_per_call": tf["calls"],
        "plain": {"ms_per_step": tp["ms"], "value": units / (tp["ms"] / 1e3),
                  "steps": tp["steps"], "warmup": tp["warmup"], "ms_per_call": tp["calls"],
                  "form": "exact int64/int128 facet tests, one warp per work item, no caches"},
        "speedup_vs_plain": tp["ms"] / tf["ms"],
        "fast_edge_filter": {
            "form": "the fast form with the four-edge FP32 filter on every facet (no rectangle "
                    "test for axis-aligned facets)",
            "ms_per_step": te["ms"], "value": units / (te["ms"] / 1e3), "steps": te["steps"],
            "warmup": te["warmup"], "ms_per_call": te["calls"]},
        "learned": {
            "form": "fast + learned cluster order in the matrix call (BF16 MLP ranking of 64 BVH "
                    "subtrees per candidate pair, tensor-core inference)",
            "ms_per_step": tl["ms"], "value": units / (tl["ms"] / 1e3),
            "steps": tl["steps"], "warmup": tl["warmup"],
            "speedup_vs_plain": tp["ms"] / tl["ms"],
            "matrix_ms_per_call": tl["calls"]["matrix"],
            "matrix_ms_per_call_without_ranker": tf["calls"]["matrix"],
            "matrix_node_tests_per_segment": per_seg(tl["stats"]["matrix"], "node_tests"),
            "matrix_node_tests_per_segment_without_ranker":
                per_seg(tf["stats"]["matrix"], "node_tests"),
            "matrix_leaf_tests_per_segment": per_seg(tl["stats"]["matrix"], "leaf_tests"),
            "matrix_leaf_tests_per_segment_without_ranker":
                per_seg(tf["stats"]["matrix"], "leaf_tests"),
            "first_proposal_hits": tl["stats"]["matrix"]["ranker_hits"],
            "hits_at_8": tl["stats"]["matrix"]["ranker_hits8"],
            "hits_note": "segments blocked inside the first proposed cluster / inside any of "
                         "the up to 8 proposals walked first, of the matrix call's segments",
            "train": {"scenes": "tiny (41 facets) + degenerate district (1,001 facets)",
                      "epochs": 12, "final_loss": train_loss, "seconds": train_s}},
        "forms_bit_identical": agree,
        "gpu_launches": tf["launches"],
        "clocks": tf["clocks"],
        "stats": tf["stats"],
        "roofline": roofline(tf, ivm, ctx, n_sm, "city"),
    }

    if not args.no_e2e:
        fac_h = torch.from_numpy(sc.facets).pin_memory()
        tx_h = torch.from_numpy(sc.tx).pin_memory()
        rx_h = torch.from_numpy(sc.rx).pin_memory()
        W, K = path.W, path.K
        M_h = torch.empty((N, W), dtype=torch.int32).pin_memory()
        T_h = torch.empty((S, 2, W), dtype=torch.int32).pin_memory()
        L_h = torch.empty((S,), dtype=torch.uint8).pin_memory()
        summ_h = torch.empty((S, K + 1, 3), dtype=torch.int64).pin_memory()
        a, b = path.snap

        def e2e_step():
            if ws == 1:   # the library copies host buffers in and out itself
                path.step("fast", bufs=(fac_h, tx_h, rx_h, M_h, T_h, L_h, summ_h))
                return
            # the all-reduce needs device buffers: stage this rank's inputs and outputs
            path.fac.copy_(fac_h, non_blocking=True)
            path.tx[a:b].copy_(tx_h[a:b], non_blocking=True)
            path.rx[a:b].copy_(rx_h[a:b], non_blocking=True)
            path.step("fast")
            M_h.copy_(path.M)
            T_h[a:b].copy_(path.T[a:b])
            L_h[a:b].copy_(path.L[a:b])
            summ_h[a:b].copy_(path.summ[a:b])

        for _ in range(max(1, args.warmup)):
            e2e_step()
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(ws, time.perf_counter() - t0) / args.steps
        Sr = b - a
        if ws == 1:   # facets go in for both calls; the matrix and table go out and back in
            h2d = 2 * fac_h.numel() * 4 + 2 * Sr * 3 * 4 + M_h.numel() * 4 + \
                Sr * 2 * W * 4 + Sr
        else:
            h2d = fac_h.numel() * 4 + 2 * Sr * 3 * 4
        d2h = M_h.numel() * 4 + Sr * 2 * W * 4 + Sr + Sr * (K + 1) * 3 * 8
        out["e2e"] = {"value": units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * e2e_s,
                      "path": "same C-ABI calls with pinned host buffers" + (
                          "" if ws == 1 else ", staged through device buffers for the "
                          "all-reduce (rank 0's bytes)")}
        del fac_h, tx_h, rx_h, M_h, T_h, L_h, summ_h

    if rank == 0 and ws == 1:
        out["precision"] = precision_block(ivm, sg, ctx, dev)
        out["batch"] = batch_block(args, ivm, sg, ctx, dev, stream, flush)
        out["district"] = district_block(args, ivm, shard, sg, ctx, dev, stream, flush)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        u, dt = oracle_sample(sc, 48, 192, 7, threads, "grid")
        out["cpu_baseline"] = {"value": u / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
                               "sample": "48 seeded matrix rows and 192 seeded snapshots of the "
                                         f"city workload ({u} pair tests, {dt:.1f} s); "
                                         + ORACLE_GRID}
    ctx.close()
    if rank == 0:
        print(json.dumps(out))


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
