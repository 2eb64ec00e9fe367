#!/usr/bin/env python
"""Benchmark of the inter-visibility hot path on GB300.

One step = one pass of the whole path over the district workload (1 km
square, 200 box buildings, 1,001 facets, 5 x 5 samples per facet, 10,000
Rx snapshots at 120 km/h every 1 ms, rooftop Tx, reflection order 3):
ivm_build_matrix (ingest, BVH, facing screen, sample-pair occlusion),
ivm_build_table (Tx and Rx rows and the direct path per snapshot) and
ivm_expand_image_tree (orders 0..3, counts and fingerprints).

Metric: visibility pair-tests per second: the N^2 ordered facet pairs the
matrix decides plus the 2 N S Tx/Rx-facet pairs the table decides, per step,
divided by the step time.  Snapshot tables per second (S / step time) is
reported beside it.

`value` is device time (CUDA events on the library's stream) with inputs
resident in HBM; L2 is flushed between steps by writing a 512 MB buffer
outside the timed events.  `e2e` is the same metric through the same C-ABI
calls with pinned host buffers (every copy inside the timed region).
`--impl reference` times the CPU oracle (the brute-force definition) on the
host cores instead.
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
WORKLOAD = ("district: 1 km x 1 km, 200 box buildings (8-40 m footprint, 6-60 m high), "
            "1,001 facets, 5x5 samples per facet, 10,000 Rx snapshots at 120 km/h every 1 ms, "
            "rooftop Tx, reflection order <= 3, seed 2")
FP32_OPS_PER_NODE_TEST = 30      # seg_box: 3 axes x 8 + 6 for the widening
FP32_OPS_PER_FILTERED_LEAF = 104  # 4 edges x 26 (value, permanent, bound, compare)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    # profiling case: one phase of one form on the first N snapshots (no JSON contract line)
    p.add_argument("--profile", choices=["matrix", "table", "tree", "step"], default=None)
    p.add_argument("--form", choices=["fast", "plain", "learned"], default="fast")
    p.add_argument("--snapshots", type=int, default=None)
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

def oracle_sample(sc, n_rows, n_snaps, seed, threads):
    """Oracle on a bounded sample of the workload; returns (pair tests, s)."""
    import numpy as np

    import oracle
    rng = np.random.default_rng(seed)
    rows = rng.choice(sc.n_facets, n_rows, replace=False)
    snaps = rng.choice(sc.n_snap, n_snaps, replace=False)
    t0 = time.perf_counter()
    oracle.matrix(sc.facets, sc.samples_per_side, rows=rows, threads=threads)
    oracle.table(sc.facets, sc.samples_per_side, sc.tx, sc.rx, snaps=snaps, threads=threads)
    dt = time.perf_counter() - t0
    units = n_rows * sc.n_facets + 2 * n_snaps * sc.n_facets
    return units, dt


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle
    from paper_2501_02747_gb300 import scenegen as sg
    oracle.build()
    sc = sg.district()
    threads = os.cpu_count() or 1
    for k in range(args.warmup):
        oracle_sample(sc, 1, 2, 100 + k, threads)
    units = 0
    secs = 0.0
    for k in range(args.steps):
        u, dt = oracle_sample(sc, 4, 16, 200 + k, threads)
        units += u
        secs += dt
    value = units / secs
    sample = (f"per step: 4 seeded matrix rows (4 x 1,001 ordered pairs) and 16 seeded "
              f"snapshots (16 x 2 x 1,001 Tx/Rx-facet pairs) of the district workload")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "int128",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "oracle": "brute force, every segment against every "
                   "triangle, exact int128 (oracle/ivm_oracle.c)"},
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


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    from paper_2501_02747_gb300 import build, ivm, shard
    from paper_2501_02747_gb300 import scenegen as sg
    build.build()
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    stream = torch.cuda.current_stream(local)
    sc = sg.district()
    N, S, K, s = sc.n_facets, sc.n_snap, sc.max_order, sc.samples_per_side
    W = ivm.words(N)
    units = N * N + 2 * N * S   # the whole job's units (split across ranks when ws > 1)
    rows = shard.row_ranges(N, ws)[rank]
    snap_a, snap_b = shard.snapshot_ranges(S, ws)[rank]
    ctx = ivm.Context(local, stream)
    facets_d = torch.from_numpy(sc.facets).to(dev)
    tx_d = torch.from_numpy(sc.tx).to(dev)
    rx_d = torch.from_numpy(sc.rx).to(dev)
    M_d = torch.empty((N, W), dtype=torch.int32, device=dev)
    T_d = torch.empty((S, 2, W), dtype=torch.int32, device=dev)
    L_d = torch.empty((S,), dtype=torch.uint8, device=dev)
    summ_d = torch.empty((S, K + 1, 3), dtype=torch.int64, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    forms = {
        "plain": dict(mode=ivm.IVM_MODE_EXACT, flags=0),
        "fast": dict(mode=ivm.IVM_MODE_FILTERED,
                     flags=ivm.IVM_FLAG_PERSISTENT | ivm.IVM_FLAG_OCCLUDER_CACHE
                     | ivm.IVM_FLAG_DEDUP_SOURCES | ivm.IVM_FLAG_GRAPH),
    }

    forms["learned"] = dict(mode=ivm.IVM_MODE_LEARNED, flags=forms["fast"]["flags"])

    # launch shape of the fast form from the library's autotuner (untimed)
    tuned = ivm.ivm_autotune(ctx, facets_d, s, tx_d, rx_d, mode=forms["fast"]["mode"],
                             flags=forms["fast"]["flags"])
    shape = {"plain": ({}, {}),
             "fast": ({"tile": tuned["tile"], "warps_per_block": tuned["warps_per_block"]},
                      {"tile": tuned["table_tile"], "warps_per_block": tuned["warps_per_block"]})}
    shape["learned"] = shape["fast"]
    # the cluster ranker of the learned form, trained (untimed) on the exact
    # method's logged hits in the tiny and degenerate scenes
    t0 = time.perf_counter()
    train_loss = ivm.ivm_ranker_train(ctx, [sg.tiny().facets, sg.degenerate(n_snap=16).facets],
                                      s, epochs=12, lr=2e-3)
    train_s = time.perf_counter() - t0

    def step(form, fac, tx, rx, M, T, L, summ, marks=None):
        """The three calls; `marks` (4 CUDA events) bracket them on the stream.
        With ws > 1 this rank's share: its matrix rows, the all-reduce of the
        parts, then the table and tree of its snapshot range."""
        kw = forms[form]
        kw_m, kw_t = shape[form]
        if marks:
            marks[0].record(stream)
        if ws == 1:
            _, stm = ivm.ivm_build_matrix(ctx, fac, s, out=M, **kw, **kw_m)
        else:
            _, stm = ivm.ivm_build_matrix_rows(ctx, fac, s, rows, out=M, **kw, **kw_m)
            shard.exchange_matrix(M)
        if marks:
            marks[1].record(stream)
        a, b = snap_a, snap_b
        _, stt = ivm.ivm_build_table(ctx, fac, s, tx[a:b], rx[a:b], out=(T[a:b], L[a:b]),
                                     **kw, **kw_t)
        if marks:
            marks[2].record(stream)
        ivm.ivm_expand_image_tree(ctx, M, T[a:b], L[a:b], N, K, summary=summ[a:b])
        if marks:
            marks[3].record(stream)
        return stm, stt

    if args.profile:
        # profiling case: one phase of one form (launch shape as timed), on the
        # first --snapshots snapshots; the calls after the warm-up run inside
        # the NVTX range "profile_<phase>" (ncu --nvtx --nvtx-include)
        Sp = min(S, args.snapshots or S)
        kw = forms[args.form]
        kw_m, kw_t = shape[args.form]
        st = None
        for it in range(args.warmup + args.steps):
            if it == args.warmup:
                torch.cuda.synchronize()
                torch.cuda.nvtx.range_push(f"profile_{args.profile}")
            if args.profile in ("matrix", "step"):
                _, st = ivm.ivm_build_matrix(ctx, facets_d, s, out=M_d, **kw, **kw_m)
            if args.profile in ("table", "step"):
                _, st = ivm.ivm_build_table(ctx, facets_d, s, tx_d[:Sp], rx_d[:Sp],
                                            out=(T_d[:Sp], L_d[:Sp]), **kw, **kw_t)
            if args.profile in ("tree", "step"):
                if args.profile == "tree" and it == 0:
                    ivm.ivm_build_matrix(ctx, facets_d, s, out=M_d, **kw, **kw_m)
                    ivm.ivm_build_table(ctx, facets_d, s, tx_d[:Sp], rx_d[:Sp],
                                        out=(T_d[:Sp], L_d[:Sp]), **kw, **kw_t)
                ivm.ivm_expand_image_tree(ctx, M_d, T_d[:Sp], L_d[:Sp], N, K, summary=summ_d[:Sp])
        torch.cuda.synchronize()
        if args.steps:
            torch.cuda.nvtx.range_pop()
        if args.profile == "step":
            st = None
        print(json.dumps({"profile": args.profile, "form": args.form, "snapshots": Sp,
                          "stats": st.as_dict() if st is not None else None}))
        ctx.close()
        return

    def timed(form):
        for _ in range(args.warmup):
            step(form, facets_d, tx_d, rx_d, M_d, T_d, L_d, summ_d)
        torch.cuda.synchronize()
        barrier(ws)
        torch.cuda.synchronize()
        launches0 = ivm.kernel_launches()
        times, kern = [], {"matrix": 0.0, "table": 0.0}
        ops, node_tests, leaf_tests = {"matrix": 0, "table": 0}, 0, 0
        calls = {"matrix": 0.0, "table": 0.0, "tree": 0.0}
        stats = None
        torch.cuda.nvtx.range_push(f"timed_{form}")
        for _ in range(args.steps):
            flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            stm, stt = step(form, facets_d, tx_d, rx_d, M_d, T_d, L_d, summ_d, marks=ev)
            torch.cuda.synchronize()
            times.append(ev[0].elapsed_time(ev[3]))
            for k, name in enumerate(("matrix", "table", "tree")):
                calls[name] += ev[k].elapsed_time(ev[k + 1]) / args.steps
            kern["matrix"] += stm.ms_traverse
            kern["table"] += stt.ms_traverse
            for name, st in (("matrix", stm), ("table", stt)):
                leaf_fp = st.leaf_tests - st.exact_tests if forms[form]["mode"] else 0
                ops[name] += st.node_tests * FP32_OPS_PER_NODE_TEST + \
                    leaf_fp * FP32_OPS_PER_FILTERED_LEAF
            stats = (stm.as_dict(), stt.as_dict())
        torch.cuda.nvtx.range_pop()
        launches = ivm.kernel_launches() - launches0
        torch.cuda.synchronize()
        barrier(ws)
        ms = max_over_ranks(ws, sum(times)) / args.steps
        return ms, kern, ops, launches, stats, calls

    clocks = Clocks(local)
    ms_plain, kern_plain, ops_plain, _, stats_plain, calls_plain = timed("plain")
    clocks.start()
    ms_fast, kern_fast, ops_fast, launches, stats_fast, calls_fast = timed("fast")
    clk = clocks.stop()
    ms_lrn, kern_lrn, _, _, stats_lrn, calls_lrn = timed("learned")

    # parity of the forms on this step's outputs (cheap, outside timing)
    step("plain", facets_d, tx_d, rx_d, M_d, T_d, L_d, summ_d)
    ref = (M_d.clone(), T_d.clone(), L_d.clone(), summ_d.clone())
    step("fast", facets_d, tx_d, rx_d, M_d, T_d, L_d, summ_d)
    forms_agree = all(bool((a == b).all()) for a, b in zip(ref, (M_d, T_d, L_d, summ_d)))
    step("learned", facets_d, tx_d, rx_d, M_d, T_d, L_d, summ_d)
    forms_agree &= all(bool((a == b).all()) for a, b in zip(ref, (M_d, T_d, L_d, summ_d)))

    def per_seg(st, key):
        return st[key] / st["segments"] if st["segments"] else None

    # visibility ranges, Blockage column and coherence time of this step's
    # table (Sec. III-C/D), one call after the step, timed on its own
    step("fast", facets_d, tx_d, rx_d, M_d, T_d, L_d, summ_d)
    torch.cuda.synchronize()
    rng_ms = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        recs, rsum = ivm.ivm_visibility_ranges(ctx, facets_d, s, tx_d[snap_a:snap_b],
                                               rx_d[snap_a:snap_b], T_d[snap_a:snap_b])
        if it >= args.warmup:
            rng_ms.append(1e3 * (time.perf_counter() - t0))
    dt_ms = 1.0   # snapshots are 1 ms apart (120 km/h, 10/3 cm per step)
    tc = [dt_ms * rsum["snapshots"][x] / rsum["ranges"][x] if rsum["ranges"][x] else None
          for x in range(2)]
    ranges_out = {
        "what": "visibility ranges (maximal runs of each table bit), first blocker at both ends "
                "of each, coherence time per Eq. (8)-(9); C-ABI call ivm_visibility_ranges on "
                "this step's table, records copied to host",
        "ms_per_call": statistics.median(rng_ms),
        "ranges": int(len(recs)),
        "ranges_per_side": rsum["ranges"],
        "snapshots_per_side": rsum["snapshots"],
        "coherence_time_ms": {"tx": tc[0], "rx": tc[1],
                              "scenario": min(x for x in tc if x is not None) if any(tc) else None},
        "table_bits_per_s": 2 * N * (snap_b - snap_a) / (statistics.median(rng_ms) / 1e3),
    }

    # image-method validation of the step's image-tree candidates (Sec. IV-B),
    # orders 0..2 at the first snapshots of this rank's range, timed on its own
    ray_snaps, ray_K = min(4, snap_b - snap_a), 2
    a0, a1 = snap_a, snap_a + ray_snaps
    _, n_cand = ivm.ivm_expand_image_tree(ctx, M_d, T_d[a0:a1], L_d[a0:a1], N, ray_K,
                                          count_paths=True)
    _, cand, n_cand, _ = ivm.ivm_expand_image_tree(ctx, M_d, T_d[a0:a1], L_d[a0:a1], N, ray_K,
                                                   paths_capacity=max(n_cand, 1))
    cand = cand[:n_cand]
    flags = torch.zeros(max(n_cand, 1), dtype=torch.uint8, device=dev)
    ray_ms = []
    for it in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ivm.ivm_validate_paths(ctx, facets_d, s, tx_d[a0:a1], rx_d[a0:a1], cand, ray_K,
                               out=flags[:n_cand])
        if it >= args.warmup:
            ray_ms.append(1e3 * (time.perf_counter() - t0))
    n_valid = int(flags[:n_cand].sum().item()) if n_cand else 0
    # edges as visible nodes and the edge nearest each source (Sec. III-B), timed on its own
    E_d = torch.from_numpy(sg.edges_of(sc)).to(dev)
    edge_ms = []
    for it in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        etab, enear = ivm.ivm_build_edge_table(ctx, facets_d, s, E_d, tx_d[snap_a:snap_b],
                                               rx_d[snap_a:snap_b], mode=ivm.IVM_MODE_FILTERED)
        if it >= args.warmup:
            edge_ms.append(1e3 * (time.perf_counter() - t0))
    ebits = np.unpackbits(etab.view(np.uint8), axis=-1, bitorder="little")[..., :E_d.shape[0]]
    edges_out = {
        "what": "edge rows (the 8 convex edges of every building as visible nodes, s samples "
                "each) and the nearest visible edge per source, C-ABI call ivm_build_edge_table, "
                "results copied to host",
        "edges": int(E_d.shape[0]), "ms_per_call": statistics.median(edge_ms),
        "edge_tests_per_s": 2 * int(E_d.shape[0]) * (snap_b - snap_a) /
                            (statistics.median(edge_ms) / 1e3),
        "visible_edges_mean": [float(ebits[:, 0].sum(axis=1).mean()),
                               float(ebits[:, 1].sum(axis=1).mean())],
    }
    # edges as matrix rows and columns: facet-edge and edge-edge visibility
    # (Sec. I-II, Sec. III-B), timed on its own, outputs left on the device
    EF_d = torch.from_numpy(sg.edge_faces_of(sc)).to(dev)
    ne = int(E_d.shape[0])
    fe_d = torch.zeros((N, (ne + 31) // 32), dtype=torch.int32, device=dev)
    ee_d = torch.zeros((ne, (ne + 31) // 32), dtype=torch.int32, device=dev)
    em_ms = []
    for it in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ivm.ivm_build_edge_matrix(ctx, facets_d, s, E_d, EF_d, out=(fe_d, ee_d))
        if it >= args.warmup:
            em_ms.append(1e3 * (time.perf_counter() - t0))
    fe_bits = int(np.unpackbits(fe_d.cpu().numpy().view(np.uint8)).sum())
    ee_bits = int(np.unpackbits(ee_d.cpu().numpy().view(np.uint8)).sum())
    edge_matrix_out = {
        "what": "edges as matrix rows and columns: facet-edge bits fe [N][WE] and edge-edge "
                "bits ee [E][WE], C-ABI call ivm_build_edge_matrix, outputs on the device",
        "facet_edge_pairs": N * ne, "edge_edge_pairs": ne * (ne - 1) // 2,
        "ms_per_call": statistics.median(em_ms),
        "pair_tests_per_s": (N * ne + ne * (ne - 1) // 2) / (statistics.median(em_ms) / 1e3),
        "facet_edge_bits": fe_bits, "edge_edge_bits": ee_bits,
    }
    # interface relations and angular bouncing ranges of the step's visible
    # pairs (Sec. II-B, Eq. (1)-(2)), timed on its own
    rel_ms = []
    for it in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rpairs, rrel, _ = ivm.ivm_interface_relations(ctx, facets_d, s, M_d)
        if it >= args.warmup:
            rel_ms.append(1e3 * (time.perf_counter() - t0))
    relations_out = {
        "what": "PAR/PER relation and the four edges' angular bouncing ranges of every "
                "visible ordered pair of the step's matrix, C-ABI call ivm_interface_relations, "
                "results copied to host",
        "pairs": int(len(rpairs)), "par": int((rrel == 1).sum()), "per": int((rrel == 2).sum()),
        "ms_per_call": statistics.median(rel_ms),
        "pairs_per_s": len(rpairs) / (statistics.median(rel_ms) / 1e3),
    }
    rays_out = {
        "what": "image-method validation of image-tree candidates (orders 0-2) as specular "
                f"rays, C-ABI call ivm_validate_paths, snapshots {a0}..{a1 - 1}",
        "candidates": int(n_cand), "valid_rays": n_valid,
        "ms_per_call": statistics.median(ray_ms),
        "candidates_per_s": n_cand / (statistics.median(ray_ms) / 1e3) if ray_ms else None,
    }

    value = units / (ms_fast / 1e3)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_fast, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "int64/int128 + fp32 filter",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "form": "fast: FP32 filter + exact fallback, "
                   "persistent work queue, occluder cache, one row per run of equal "
                   "source positions, CUDA-graph replay of each call",
                   "l2": "flushed between steps (512 MB write)",
                   "facets": N, "snapshots": S, "samples_per_side": s, "max_order": K,
                   "pair_tests_per_step": units, "autotuned_shape": tuned,
                   "parallelism": "one workload split over ranks: matrix rows of about equal "
                                  "pair counts, one all-reduce of the matrix parts, snapshot "
                                  "ranges for the table and tree" if ws > 1 else "1 GPU"},
        "snapshot_tables_per_s": S / (ms_fast / 1e3),
        "plain": {"ms_per_step": ms_plain, "value": units / (ms_plain / 1e3),
                  "form": "exact int64/int128 facet tests, one warp per work item"},
        "speedup_vs_plain": ms_plain / ms_fast,
        "learned": {
            "form": "fast + learned cluster order in the matrix call (BF16 MLP ranking of "
                    "64 BVH subtrees per candidate pair, tensor-core inference)",
            "ms_per_step": ms_lrn, "value": units / (ms_lrn / 1e3),
            "speedup_vs_plain": ms_plain / ms_lrn,
            "matrix_ms_per_call": calls_lrn["matrix"],
            "matrix_ms_per_call_without_ranker": calls_fast["matrix"],
            "matrix_node_tests_per_segment": per_seg(stats_lrn[0], "node_tests"),
            "matrix_node_tests_per_segment_without_ranker": per_seg(stats_fast[0], "node_tests"),
            "matrix_leaf_tests_per_segment": per_seg(stats_lrn[0], "leaf_tests"),
            "matrix_leaf_tests_per_segment_without_ranker": per_seg(stats_fast[0], "leaf_tests"),
            "first_proposal_hits": stats_lrn[0]["ranker_hits"],
            "train": {"scenes": "tiny (41 facets) + degenerate district (1,001 facets)",
                      "epochs": 12, "final_loss": train_loss, "seconds": train_s}},
        "ms_per_call": {"fast": calls_fast, "plain": calls_plain, "learned": calls_lrn},
        "visibility_ranges": ranges_out,
        "ray_validation": rays_out,
        "edges": edges_out,
        "edge_matrix": edge_matrix_out,
        "interface_relations": relations_out,
        "forms_bit_identical": forms_agree,
        "gpu_launches": launches,
        "clocks": clk,
        "stats": {"matrix": stats_fast[0], "table": stats_fast[1]},
    }
    # roofline of the dominant kernel (FP32 issue of the traversal)
    dom = "table" if kern_fast["table"] >= kern_fast["matrix"] else "matrix"
    kname = {"table": "k_table", "matrix": "k_matrix"}[dom]
    import json as _json
    peaks = _json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    peak = n_sm * 128 * sm_max * 1e6 / 1e12
    achieved = ops_fast[dom] / (kern_fast[dom] / 1e3) / 1e12 if kern_fast[dom] > 0 else 0.0
    out["roofline"] = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak,
                       "unit": "Tops/s", "frac": achieved / peak if peak else None,
                       "traffic": traffic_from_profiles(kname),
                       "peak_basis": f"{n_sm} SMs x 128 FP32 lanes x {sm_max:.0f} MHz "
                                     "(sm_max_mhz of MEASURED_PEAKS.json)",
                       "ms_per_launch": kern_fast[dom] / args.steps,
                       "ms_per_step_matrix": kern_fast["matrix"] / args.steps,
                       "ms_per_step_table": kern_fast["table"] / args.steps}
    # the same fraction against this GPU's measured FMA issue rate (eight
    # independent FMA chains per thread, full occupancy: ivm_fp32_peak)
    ffma = ivm.ivm_fp32_peak(ctx) / 1e12
    out["roofline"]["peak_measured_ffma"] = ffma
    out["roofline"]["frac_of_measured_ffma"] = achieved / ffma if ffma else None

    if not args.no_e2e:
        fac_h = torch.from_numpy(sc.facets).pin_memory()
        tx_h = torch.from_numpy(sc.tx).pin_memory()
        rx_h = torch.from_numpy(sc.rx).pin_memory()
        M_h = torch.empty((N, W), dtype=torch.int32).pin_memory()
        T_h = torch.empty((S, 2, W), dtype=torch.int32).pin_memory()
        L_h = torch.empty((S,), dtype=torch.uint8).pin_memory()
        summ_h = torch.empty((S, K + 1, 3), dtype=torch.int64).pin_memory()
        a, b = snap_a, snap_b

        def e2e_step():
            if ws == 1:   # the library copies host buffers in and out itself
                step("fast", fac_h, tx_h, rx_h, M_h, T_h, L_h, summ_h)
                return
            # the all-reduce needs device buffers: stage this rank's inputs and outputs
            facets_d.copy_(fac_h, non_blocking=True)
            tx_d[a:b].copy_(tx_h[a:b], non_blocking=True)
            rx_d[a:b].copy_(rx_h[a:b], non_blocking=True)
            step("fast", facets_d, tx_d, rx_d, M_d, T_d, L_d, summ_d)
            M_h.copy_(M_d)
            T_h[a:b].copy_(T_d[a:b])
            L_h[a:b].copy_(L_d[a:b])
            summ_h[a:b].copy_(summ_d[a:b])

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
        if ws == 1:   # facets go in for both calls; the matrix goes out and back in
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

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        u, dt = oracle_sample(sc, 32, 96, 7, threads)
        out["cpu_baseline"] = {"value": u / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
                               "sample": "32 seeded matrix rows and 96 seeded snapshots of the "
                                         f"district workload ({u} pair tests, {dt:.1f} s)"}
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
