#!/usr/bin/env python3
"""Benchmark of the dynamic graph store's hot path on the power-law workload.

Workload (R-MAT scale 20: V = 1,048,576, 16,777,216 draws with a/b/c/d =
0.57/0.19/0.19/0.05, duplicates and self-loops dropped, weights U[1,100];
buckets from the load-factor rule with load factor 0.7).  One step is one
pass of the whole path on one batch size B (default 2^20):

    insert B new R-MAT edges -> incremental BFS, SSSP (from the max-degree
    vertex) and WCC -> commit -> delete B live edges -> BFS, SSSP (decremental)
    and WCC (static recompute) -> commit -> query B edges (half present)

WCC and the query batch only read the graph, as BFS and SSSP do: they run
on a second stream (default priority) forked after each update batch and
joined before the next change, beside BFS/SSSP on the main stream (high
priority); the step's phases are timed on the main stream and the second
stream's calls by their own events.

value = 3B edges (inserted + deleted + queried) / step time, in Medges/s,
with inputs resident in device memory; `e2e` is the same through the C-ABI
with the inputs copied from pinned host buffers and the results (flags,
bitmap, SSSP distances) copied back inside the timed region.  L2 is flushed
between steps by writing a 512 MiB buffer.

`--impl reference` times the CPU oracle (plain single-threaded C++,
recomputing everything from scratch) on the same workload and metric.
Under torchrun each rank runs an independent replica (weak scaling); rank 0
prints one JSON line.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "batched edge insert/delete/query Medges/s; incr-SSSP ms; % of HBM roofline"
UNIT = "Medges/s"
L2_FLUSH_BYTES = 512 << 20


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--batch", type=int, default=1 << 20)
    p.add_argument("--scale", type=int, default=20)
    p.add_argument("--draws", type=int, default=1 << 24)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--workload", choices=["powerlaw", "growth", "served", "road"], default="powerlaw",
                   help="powerlaw: the benchmark line; growth: the learned-sizing study on the R-MAT "
                        "scale-22 growth stream; served: plain vs continuous-batching serving on the R-MAT "
                        "scale-21 request stream; road: incremental SSSP on the 4096^2 road-like grid "
                        "(each prints its own JSON line)")
    return p.parse_args(argv)


# ----------------------------------------------------------------- ranks

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world, use_cuda):
    if world <= 1:
        return None
    import torch.distributed as dist

    dist.init_process_group(backend="nccl" if use_cuda else "gloo")
    return dist


def reduce_across(values, op, dist, device):
    """all_reduce of a list of floats (op: 'max' or 'sum'); identity at N=1."""
    if dist is None:
        return list(values)
    import torch

    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return t.cpu().tolist()


def barrier(dist, device=None):
    if dist is not None:
        if device is not None and device.type == "cuda":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# -------------------------------------------------------------- workload

def make_workload(args, n_batches):
    import synth

    t0 = time.time()
    G = synth.powerlaw_graph(scale=args.scale, draws=args.draws)
    deg = np.bincount(G.src, minlength=G.V)
    source = int(np.argmax(deg))
    batches = [synth.powerlaw_batch(G, k, args.batch) for k in range(n_batches)]
    return G, source, batches, time.time() - t0


def workload_config(args, G):
    return {
        "workload": "R-MAT scale %d power-law graph (V=%d, %d edges after dropping duplicates and self-loops, "
                    "weights U[1,100]); step = insert %d + incr BFS/SSSP/WCC + delete %d + decr BFS/SSSP + "
                    "static WCC + query %d" % (args.scale, G.V, len(G.src), args.batch, args.batch, args.batch),
        "vertices": G.V,
        "edges": int(len(G.src)),
        "batch": args.batch,
        "buckets": "load-factor rule, load factor 0.7",
        "l2": "flushed between timed steps (512 MiB write)",
        "parallelism": "independent replica per GPU",
    }


# ------------------------------------------------------------- clocks

class ClockSampler:
    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self, gpu_index=0):
        if self.proc is None or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or f[0] != str(gpu_index):
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        busy = [x for x in sm if x > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------- roofline model

def algorithmic_bytes(family, ctr, n_per_launch, launches):
    """Bytes the method must move for one kernel family over the timed
    region, from the work counters: slabs are 128 B, an index gather counts
    one 32 B sector, a random 8 B read-modify-write counts 8 B each way."""
    if family == "query":
        return launches * n_per_launch * (8 + 32 + 0.125) + 128 * ctr["query_slabs"]
    if family == "insert":
        return launches * n_per_launch * (12 + 32 + 32) + 128 * (ctr["insert_slabs"] + ctr["insert_new_slabs"])
    if family == "delete":
        return launches * n_per_launch * (8 + 32 + 32) + 128 * ctr["delete_slabs"]
    if family == "sssp_rounds":
        # rounds, then the tree nodes unpacked into the caller's dist/parent
        return (ctr["relax_lists"] * (4 + 4 + 8) + 128 * ctr["relax_slabs"] + 16 * ctr["relax_edges"]
                + ctr["relax_improved"] * (8 + 4 + 8) + ctr.get("unpacked", 0) * (8 + 4 + 4))
    if family == "sssp_relax_into_invalid":
        return 4 * ctr["scan_owners"] + (128 + 8) * ctr["scan_slabs"] + 16 * ctr["scan_targets"]
    if family == "sssp_enqueue_invalid":
        return ctr["scan_improved"] * (8 + 8 + 8 + 4)
    if family == "sssp_relax_updated":
        return (ctr["seed_lists"] * (4 + 8 + 8) + 128 * ctr["seed_slabs"] + 16 * ctr["seed_edges"]
                + ctr["seed_improved"] * (8 + 4 + 8))
    if family == "sssp_invalidate_walk":
        return ctr["walk_vertices"] * 8 + ctr["invalidated"] * 8
    if family == "wcc_hook_all":
        return 128 * ctr["wcc_slabs"] + 16 * ctr["wcc_edges"]
    if family == "wcc_hook_updated":
        return 128 * ctr["wcc_upd_slabs"] + 16 * ctr["wcc_upd_edges"]
    return None


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
# kernel families, from the ncu launch list of this benchmark summarised in
# profiles/launches_powerlaw_rmat20_b1M.md (full workload, one pass), and
# the SHA-256 of the kernel sources (csrc/) it was taken with.  A figure is
# reported only while those sources are unchanged; otherwise traffic is null.
NCU_TRAFFIC_SOURCES_SHA = "7c40a5cb5cbb9d2ac94b78f631250ad2c8dc2c74747ed419265b0b6764bb4f3a"
NCU_TRAFFIC = {
    "sssp_rounds": 49446528,
    "sssp_relax_into_invalid": 281274624,
    "sssp_enqueue_invalid": 11139072,
    "sssp_relax_updated": 149913216,
    "sssp_invalidate_walk": 8524096,
    "sssp_invalidate": 13739968,
    "wcc_hook_all": 351008128,
    "wcc_hook_updated": 139749504,
    "insert": 241921792,
    "delete": 198795904,
    "query": 130562048,
    "stage_dedup": 40166336,
    "update_slab_pointers": 60561856,
}


def kernel_sources_sha():
    import hashlib

    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2305_17813_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode() + b"\0" + fh.read())
    return h.hexdigest()


def ncu_traffic(family):
    """DRAM bytes per launch of `family` from the committed ncu capture, or
    None when there is none or the kernel sources changed since."""
    if family not in NCU_TRAFFIC or NCU_TRAFFIC_SOURCES_SHA is None:
        return None
    return NCU_TRAFFIC[family] if kernel_sources_sha() == NCU_TRAFFIC_SOURCES_SHA else None


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ----------------------------------------------------------------- GPU arm

def run_ours(args, world, rank, local):
    import torch

    import paper_2305_17813_gb300 as mk

    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist = dist_init(world, True)
    lib = mk.load()
    W, K, B = args.warmup, args.steps, args.batch
    n_e2e = 0 if args.no_e2e else K
    G, source, batches, gen_s = make_workload(args, W + K + n_e2e)
    V, E = G.V, len(G.src)
    # the step runs on a high-priority stream; WCC, which only reads the
    # graph, runs beside it on a default-priority stream (see step())
    stream = torch.cuda.Stream(device=device, priority=-1)
    torch.cuda.set_stream(stream)
    sp = ctypes.c_void_p(stream.cuda_stream)

    def u32(a):
        return mk.to_device_u32(a, device)

    src_d = u32(G.src)
    buckets = mk.bucket_rule(V, src_d, 0.7)
    g = mk.Graph(V, edge_capacity_hint=E + (W + K + n_e2e + 2) * B, buckets=buckets)
    h = g.handle
    chunk = 1 << 22
    dst_d, w_d = u32(G.dst), u32(G.w)
    for i in range(0, E, chunk):
        mk.check(lib.mk_insert_batch(h, ctypes.c_void_p(src_d[i:i + chunk].data_ptr()),
                                     ctypes.c_void_p(dst_d[i:i + chunk].data_ptr()),
                                     ctypes.c_void_p(w_d[i:i + chunk].data_ptr()), min(chunk, E - i), None, sp),
                 "load")
    del src_d, dst_d, w_d
    g.commit()
    out = {k: torch.empty(V, dtype=torch.int32, device=device) for k in
           ("bd", "bp", "sd", "sp", "lab")}
    fl_i = torch.empty(B, dtype=torch.uint8, device=device)
    fl_d = torch.empty(B, dtype=torch.uint8, device=device)
    bm = torch.empty((B + 31) // 32, dtype=torch.int32, device=device)
    P = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    for fn, a, b in ((lib.mk_incr_bfs, "bd", "bp"), (lib.mk_incr_sssp, "sd", "sp")):
        mk.check(fn(h, source, P(out[a]), P(out[b]), sp), "static")
    mk.check(lib.mk_incr_wcc(h, P(out["lab"]), sp), "static wcc")
    g.commit()
    torch.cuda.synchronize()
    st = g.last_error()
    if st != mk.MK_OK:
        raise RuntimeError("device status %d after the load" % st)

    # X2 autotuner: kernel shapes for this graph (untimed setup)
    tb = batches[0]
    tuning = g.autotune(tb["q_src"], tb["q_dst"], source)
    g.commit()
    dev_batches = []
    for bt in batches[:W + K]:
        dev_batches.append({k: u32(bt[k]) for k in ("ins_src", "ins_dst", "ins_w", "del_src", "del_dst",
                                                     "q_src", "q_dst")})
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=device)
    # phases on the main stream; wcc1_wait / wcc2_wait / query_wait are what
    # is left of the calls on the second stream after BFS and SSSP (the
    # joins); their own durations come from events on that stream
    names = ["insert", "bfs1", "sssp1", "wcc1_wait", "commit1", "delete", "bfs2", "sssp2", "wcc2_wait", "commit2",
             "query_wait"]

    # WCC only reads the graph, as BFS and SSSP do: it runs on a second
    # stream, forked after each update batch and joined before the commit,
    # so its kernels overlap the BFS/SSSP kernels (a user of the library
    # can do the same: calls on one graph may overlap when none of them
    # changes it).
    ws = torch.cuda.Stream(device=device)
    wsp = ctypes.c_void_p(ws.cuda_stream)

    def step(bt, ev, hooks=None, wev=None):
        hooks = hooks or {}
        wev = wev or [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record(stream)
        mk.check(lib.mk_insert_batch(h, P(bt["ins_src"]), P(bt["ins_dst"]), P(bt["ins_w"]), B, P(fl_i), sp), "ins")
        ev[1].record(stream)
        if "after_insert" in hooks:
            hooks["after_insert"]()
        ws.wait_event(ev[1])
        wev[0].record(ws)
        mk.check(lib.mk_incr_wcc(h, P(out["lab"]), wsp), "wcc")
        wev[1].record(ws)
        mk.check(lib.mk_incr_bfs(h, source, P(out["bd"]), P(out["bp"]), sp), "bfs")
        ev[2].record(stream)
        mk.check(lib.mk_incr_sssp(h, source, P(out["sd"]), P(out["sp"]), sp), "sssp")
        ev[3].record(stream)
        stream.wait_event(wev[1])
        ev[4].record(stream)
        mk.check(lib.mk_commit_batch(h, sp), "commit")
        ev[5].record(stream)
        if "before_delete" in hooks:
            hooks["before_delete"]()
        mk.check(lib.mk_delete_batch(h, P(bt["del_src"]), P(bt["del_dst"]), B, P(fl_d), sp), "del")
        ev[6].record(stream)
        ws.wait_event(ev[6])
        wev[2].record(ws)
        mk.check(lib.mk_incr_wcc(h, P(out["lab"]), wsp), "wcc")
        wev[3].record(ws)
        # the query batch only reads the graph too: after the delete, beside
        # the decremental BFS/SSSP (a commit moves only update markers)
        mk.check(lib.mk_query_batch(h, P(bt["q_src"]), P(bt["q_dst"]), B, P(bm), None, wsp), "query")
        wev[4].record(ws)
        mk.check(lib.mk_incr_bfs(h, source, P(out["bd"]), P(out["bp"]), sp), "bfs")
        ev[7].record(stream)
        mk.check(lib.mk_incr_sssp(h, source, P(out["sd"]), P(out["sp"]), sp), "sssp")
        ev[8].record(stream)
        stream.wait_event(wev[3])
        ev[9].record(stream)
        mk.check(lib.mk_commit_batch(h, sp), "commit")
        ev[10].record(stream)
        stream.wait_event(wev[4])
        ev[11].record(stream)

    def events():
        return [torch.cuda.Event(enable_timing=True) for _ in range(12)]

    for k in range(W):
        flush.fill_(k)
        torch.cuda.nvtx.range_push("step")  # lets a profiler select the steps' kernels
        step(dev_batches[k], events())
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if g.last_error() != mk.MK_OK:
        raise RuntimeError("device status after warm-up")
    g.counters(reset=True)
    g.profile(True)
    launches0 = g.launch_count()
    evs = [events() for _ in range(K)]
    wevs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(K)]
    clock = ClockSampler(os.path.join(ROOT, "gpurun_out", "bench_clocks_rank%d.csv" % rank)
                         if os.path.isdir(os.path.join(ROOT, "gpurun_out")) else "/tmp/bench_clocks_rank%d.csv" % rank)
    barrier(dist, device)
    torch.cuda.synchronize()
    wall0 = time.time()
    with clock:
        for k in range(K):
            flush.fill_(k + 1)
            torch.cuda.nvtx.range_push("step")
            step(dev_batches[W + k], evs[k], wev=wevs[k])
            torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
    wall = time.time() - wall0
    barrier(dist, device)
    launches = g.launch_count() - launches0
    prof = g.profile_read()
    g.profile(False)
    ctr = g.counters()
    status = g.last_error()
    if status != mk.MK_OK:
        raise RuntimeError("device status %d in the timed region" % status)
    step_ms = [evs[k][0].elapsed_time(evs[k][11]) for k in range(K)]
    phase = {n: statistics.mean(evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(K))
             for i, n in enumerate(names)}
    wcc_incr = statistics.mean(wevs[k][0].elapsed_time(wevs[k][1]) for k in range(K))
    wcc_static = statistics.mean(wevs[k][2].elapsed_time(wevs[k][3]) for k in range(K))
    query_ms = statistics.mean(wevs[k][3].elapsed_time(wevs[k][4]) for k in range(K))
    local_ms = statistics.mean(step_ms)
    ms_max, = reduce_across([local_ms], "max", dist, device)
    units_total, = reduce_across([3.0 * B], "sum", dist, device)
    value = units_total / (ms_max / 1e3) / 1e6

    # roofline: kernel family with the largest share of the timed region
    fam_time = {name: t for name, (n, t) in prof.items()}
    fam_launch = {name: n for name, (n, t) in prof.items()}
    dom = max(fam_time, key=fam_time.get)
    per_launch_n = B
    bytes_total = algorithmic_bytes(dom, ctr, per_launch_n, fam_launch[dom])
    peak, peak_kind = measured_peak()
    roof = None
    if bytes_total is not None and fam_time[dom] > 0:
        per_launch_bytes = bytes_total / fam_launch[dom]
        avg_ms = fam_time[dom] / fam_launch[dom]
        achieved = per_launch_bytes / (avg_ms / 1e3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_source": peak_kind, "traffic": ncu_traffic(dom),
                "algorithmic_bytes_per_launch": int(per_launch_bytes), "avg_launch_ms": round(avg_ms, 4),
                "launches": fam_launch[dom]}
    # every family's share and achieved bandwidth, for the record
    kernels = {}
    total_prof = sum(fam_time.values()) or 1.0
    for name in sorted(fam_time, key=fam_time.get, reverse=True):
        bt = algorithmic_bytes(name, ctr, B, fam_launch[name])
        kernels[name] = {"launches": fam_launch[name], "ms": round(fam_time[name], 3),
                         "share": round(fam_time[name] / total_prof, 4)}
        if bt is not None and fam_time[name] > 0:
            kernels[name]["gbs"] = round(bt / (fam_time[name] / 1e3) / 1e9, 1)

    result = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": round(ms_max, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic", "config": workload_config(args, G),
        "insert_medges_s": round(B / phase["insert"] / 1e3, 1),
        "delete_medges_s": round(B / phase["delete"] / 1e3, 1),
        "query_medges_s": round(B / query_ms / 1e3, 1),
        "incr_sssp_ms": round(phase["sssp1"], 3), "decr_sssp_ms": round(phase["sssp2"], 3),
        "incr_bfs_ms": round(phase["bfs1"], 3), "decr_bfs_ms": round(phase["bfs2"], 3),
        "incr_wcc_ms": round(wcc_incr, 3), "static_wcc_ms": round(wcc_static, 3),
        "wcc_overlap": "WCC and the query batch run on a second stream beside BFS/SSSP; their ms and rates are "
                       "their own durations there",
        "phases_ms": {k: round(v, 3) for k, v in phase.items()},
        "roofline": roof, "kernels": kernels, "counters": ctr,
        "gpu_launches": int(launches), "wall_s_timed": round(wall, 3), "gen_s": round(gen_s, 1),
        "tuning": {k: tuning[k] for k in ("query_group", "query_block", "rounds_blocks_per_sm")},
        "clocks": clock.summary(local),
    }

    # end to end through the C ABI with host buffers
    if n_e2e:
        host = []
        for bt in batches[W + K:W + K + n_e2e]:
            host.append({k: torch.from_numpy(np.ascontiguousarray(bt[k]).view(np.int32)).pin_memory()
                         for k in ("ins_src", "ins_dst", "ins_w", "del_src", "del_dst", "q_src", "q_dst")})
        stage = {k: torch.empty(B, dtype=torch.int32, device=device) for k in host[0]}
        h_fl_i = torch.empty(B, dtype=torch.uint8).pin_memory()
        h_fl_d = torch.empty(B, dtype=torch.uint8).pin_memory()
        h_bm = torch.empty((B + 31) // 32, dtype=torch.int32).pin_memory()
        h_sd = torch.empty(V, dtype=torch.int32).pin_memory()
        h_spar = torch.empty(V, dtype=torch.int32).pin_memory()
        # Every step copies its inputs in and its results out inside the timed
        # region; the copies that later phases need overlap the earlier
        # phases on a second stream: the delete and query inputs come in
        # while the insert and the algorithms run, and the insert flags go
        # out while the algorithms run.
        copy = torch.cuda.Stream(device=device)
        e2e_ms = []
        for k in range(n_e2e):
            flush.fill_(100 + k)
            e = events()
            torch.cuda.synchronize()
            e[0].record(stream)
            for key in ("ins_src", "ins_dst", "ins_w"):
                stage[key].copy_(host[k][key], non_blocking=True)
            copy.wait_event(e[0])
            ready = torch.cuda.Event()
            with torch.cuda.stream(copy):
                for key in ("del_src", "del_dst", "q_src", "q_dst"):
                    stage[key].copy_(host[k][key], non_blocking=True)
                ready.record(copy)
            inserted = torch.cuda.Event()

            def after_insert():
                inserted.record(stream)
                copy.wait_event(inserted)
                with torch.cuda.stream(copy):
                    h_fl_i.copy_(fl_i, non_blocking=True)

            step(stage, e[1:] + [torch.cuda.Event(enable_timing=True)],
                 {"after_insert": after_insert, "before_delete": lambda: stream.wait_event(ready)})
            h_fl_d.copy_(fl_d, non_blocking=True)
            h_bm.copy_(bm, non_blocking=True)
            h_sd.copy_(out["sd"], non_blocking=True)
            h_spar.copy_(out["sp"], non_blocking=True)
            stream.wait_stream(copy)
            e[11].record(stream)
            torch.cuda.synchronize()
            e2e_ms.append(e[0].elapsed_time(e[11]))
        if g.last_error() != mk.MK_OK:
            raise RuntimeError("device status in the e2e pass")
        e2e_local = statistics.mean(e2e_ms)
        e2e_max, = reduce_across([e2e_local], "max", dist, device)
        result["e2e"] = {"value": round(units_total / (e2e_max / 1e3) / 1e6, 2), "unit": UNIT,
                         "h2d_bytes_per_step": int(B * 4 * 7), "d2h_bytes_per_step": int(2 * B + 4 * ((B + 31) // 32)
                                                                                         + 8 * V),
                         "ms_per_step": round(e2e_max, 3)}
    g.close()
    return result, dist, G, source, batches


# ------------------------------------------------------- learned sizing

def growth_experiment(S, split=32, horizon=8, epochs=20, lr=3e-3, load_factor=0.7, keep_graphs=False):
    """Learned slab sizing on a growth stream S (synth.growth_stream).

    A graph sized by the load-factor rule at the initial load runs batches
    1..split while a degree trace records every applied insert and delete.
    The network is trained on (features at batch t, edges gained per batch
    over the next `horizon` batches) for every t with a full window, then
    predicts each vertex's growth over the remaining batches.  Two graphs are
    rebuilt from the live edges at `split`: one with the learned bucket
    counts, one with the load-factor rule on the current degrees (the baseline
    the learned counts are measured against).
    Both run the remaining batches; the insert time, a query batch over live
    edges, chain lengths and slabs walked per query are compared."""
    import torch

    import paper_2305_17813_gb300 as mk
    from paper_2305_17813_gb300 import sizing

    V = S.V
    n_batches = len(S.batches)
    u = lambda a: mk.to_device_u32(a)  # noqa: E731
    total_edges = len(S.init.src) + sum(len(b.ins_src) for b in S.batches)
    b0 = mk.bucket_rule(V, u(S.init.src), load_factor)
    g = mk.Graph(V, edge_capacity_hint=2 * total_edges, buckets=b0)
    trace = sizing.DegreeTrace(V)
    s0, d0 = u(S.init.src), u(S.init.dst)
    f = g.insert(s0, d0, u(S.init.w))
    trace.apply(s0, d0, f, +1)
    g.commit()
    trace.snapshot()
    snaps = {0: trace.out_deg.clone()}
    feats = {}
    for k in range(split):
        b = S.batches[k]
        si, di = u(b.ins_src), u(b.ins_dst)
        trace.apply(si, di, g.insert(si, di, u(b.ins_w)), +1)
        sd, dd = u(b.del_src), u(b.del_dst)
        trace.apply(sd, dd, g.delete(sd, dd), -1)
        g.commit()
        trace.snapshot()
        t = k + 1
        snaps[t] = trace.out_deg.clone()
        if t >= 4 and t + horizon <= split:
            feats[t] = trace.features(b0)
    X = torch.cat([feats[t] for t in sorted(feats)])
    T = torch.cat([sizing.growth_targets(snaps[t], snaps[t + horizon], horizon) for t in sorted(feats)])
    model = sizing.SizingModel(seed=0)
    t0 = time.time()
    losses = model.train(X, T, epochs=epochs, lr=lr)
    train_s = time.time() - t0
    x_now = trace.features(b0)
    learned_b, _ = model.buckets(x_now, trace.out_deg, horizon=n_batches - split, load_factor=load_factor)
    es, ed, ew = g.export()
    rule_b = mk.bucket_rule(V, es, load_factor)
    source = int(torch.argmax(trace.out_deg).item())
    g.close()
    out = {"vertices": V, "batches": n_batches, "split": split, "horizon": horizon, "train_samples": int(X.shape[0]),
           "train_losses": [round(x, 5) for x in losses], "train_s": round(train_s, 2), "source": source}
    graphs = []
    rng = np.random.default_rng(7)
    for name, bk in (("learned", learned_b), ("rule", rule_b)):
        gg = mk.Graph(V, edge_capacity_hint=2 * total_edges, buckets=bk)
        gg.insert(es, ed, ew, flags=False)
        gg.commit()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ins_ms = 0.0
        n_ins = 0
        for k in range(split, n_batches):
            b = S.batches[k]
            si, di, wi = u(b.ins_src), u(b.ins_dst), u(b.ins_w)
            sd, dd = u(b.del_src), u(b.del_dst)
            ev[0].record()
            gg.insert(si, di, wi, flags=False)
            ev[1].record()
            torch.cuda.synchronize()
            ins_ms += ev[0].elapsed_time(ev[1])
            n_ins += len(b.ins_src)
            gg.delete(sd, dd, flags=False)
            gg.commit()
        ls, ld, _ = gg.export()
        pick = torch.from_numpy(rng.integers(0, ls.numel(), min(ls.numel(), 1 << 20)))
        qs, qd = ls[pick.cuda()].contiguous(), ld[pick.cuda()].contiguous()
        gg.counters(reset=True)
        q_times = []
        for _ in range(7):
            ev[0].record()
            gg.query(qs, qd, weights=False)
            ev[1].record()
            torch.cuda.synchronize()
            q_times.append(ev[0].elapsed_time(ev[1]))
        q_ms = statistics.median(q_times)
        ctr = gg.counters()
        st = gg.stats()
        out[name] = {"lists": int(st["lists"]), "chain_mean": round(st["chain_mean"], 4), "chain_max": int(st["chain_max"]),
                     "device_bytes": int(st["device_bytes"]),
                     "query_slabs_per_query": round(ctr["query_slabs"] / 7 / qs.numel(), 4),
                     "insert_medges_s": round(n_ins / ins_ms / 1e3, 1), "query_medges_s": round(qs.numel() / q_ms / 1e3, 1)}
        if keep_graphs:
            graphs.append(gg)
        else:
            gg.close()
    model.close()
    if keep_graphs:
        out["graphs"] = graphs
    return out


# ---------------------------------------------------------------- serving

def serve_experiment(G, R, rate_fracs=(0.5, 0.9), max_inflight=64, commit_every=8, retain_every=16,
                     retain_sssp_every=64, n_req=None, log=None, keep_outputs=False, query_pool=1 << 21,
                     insert_pool=1 << 22):
    """Plain one-launch-per-request execution against the continuous-batching
    server on the same request stream R (synth.request_stream) over graph G.
    First both run with every request available at once (capacity), then
    with Poisson arrivals at each fraction of the plain capacity; latency =
    completion - arrival.  The outputs of a deterministic sample of requests
    (every retain_every-th; every retain_sssp_every-th SSSP) are kept and
    must be identical between the two modes."""
    import torch

    import paper_2305_17813_gb300 as mk
    import synth

    lib = mk.load()
    V, E = G.V, len(G.src)
    N = n_req or len(R.kind)
    kinds, sizes, offs, srcs = R.kind[:N], R.size[:N], R.offset[:N], R.source[:N]
    u = lambda a: mk.to_device_u32(a)  # noqa: E731
    QP, IP = query_pool, insert_pool
    rng = np.random.default_rng(11)
    pick = rng.integers(0, E, QP)
    live = rng.random(QP) < 0.5
    qs = u(np.where(live, G.src[pick], rng.integers(0, V, QP)).astype(np.uint32))
    qd = u(np.where(live, G.dst[pick], rng.integers(0, V, QP)).astype(np.uint32))
    is_, id_ = synth.rmat_pairs(int(np.log2(V)), IP, synth.substream(3100, 1))
    is_, id_ = u(is_), u(id_)
    iw = u(synth.weights(IP, synth.substream(3100, 2), 1, 100))
    perm = synth.permutation(E, synth.substream(3100, 3))
    ds, dd = u(G.src[perm]), u(G.dst[perm])
    P_ = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())  # noqa: E731
    maxn = int(sizes.max()) if N else 1
    ring = []
    for _ in range(max_inflight):
        ring.append({"bm": torch.empty((maxn + 31) // 32, dtype=torch.int32, device="cuda"),
                     "fl": torch.empty(maxn, dtype=torch.uint8, device="cuda"),
                     "dist": torch.empty(V, dtype=torch.int32, device="cuda")})
    retained = {}

    def outputs(i, store):
        """(out0, out1) for request i; retained requests get their own."""
        k, n = int(kinds[i]), int(sizes[i])
        keep = (i % retain_every == 0) if k != 3 else (i % retain_sssp_every == 0)
        if keep:
            if k == 0:
                t = (torch.empty((n + 31) // 32, dtype=torch.int32, device="cuda"), None)
            elif k in (1, 2):
                t = (torch.empty(n, dtype=torch.uint8, device="cuda"), None)
            else:
                t = (torch.empty(V, dtype=torch.int32, device="cuda"), torch.empty(V, dtype=torch.int32, device="cuda"))
            store[i] = t
            return t
        slot = ring[i % max_inflight]
        if k == 0:
            return slot["bm"], None
        if k in (1, 2):
            return slot["fl"], None
        return slot["dist"], None

    def inputs(i):
        k, n, o = int(kinds[i]), int(sizes[i]), int(offs[i])
        if k == 0:
            return qs[o:o + n], qd[o:o + n], None
        if k == 1:
            return is_[o:o + n], id_[o:o + n], iw[o:o + n]
        if k == 2:
            o %= E
            if o + n > E:
                o = 0
            return ds[o:o + n], dd[o:o + n], None
        return None, None, None

    pool = int((E + IP) / 15 * 1.3) + (1 << 21)

    def fresh():
        b = mk.bucket_rule(V, u(G.src), 0.7)
        g = mk.Graph(V, buckets=b, pool_slabs=pool)
        g.insert(G.src, G.dst, G.w, flags=False)
        g.commit()
        torch.cuda.synchronize()
        return g

    def run_plain(arrivals, store):
        g = fresh()
        h = g.handle
        sp = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        lat = np.zeros(N)
        n_upd = 0
        t0 = time.perf_counter()
        for i in range(N):
            while time.perf_counter() - t0 < arrivals[i]:
                pass
            k, n = int(kinds[i]), int(sizes[i])
            a, b, w = inputs(i)
            o0, o1 = outputs(i, store)
            if k == 0:
                rc = lib.mk_query_batch(h, P_(a), P_(b), n, P_(o0), None, sp)
            elif k == 1:
                rc = lib.mk_insert_batch(h, P_(a), P_(b), P_(w), n, P_(o0), sp)
            elif k == 2:
                rc = lib.mk_delete_batch(h, P_(a), P_(b), n, P_(o0), sp)
            else:
                rc = lib.mk_incr_sssp(h, int(srcs[i]), P_(o0), P_(o1), sp)
            mk.check(rc, "plain request")
            if k in (1, 2):
                n_upd += 1
                if commit_every and n_upd % commit_every == 0:
                    mk.check(lib.mk_commit_batch(h, sp), "commit")
            torch.cuda.synchronize()
            lat[i] = time.perf_counter() - t0 - arrivals[i]
        total = time.perf_counter() - t0
        assert g.last_error() == mk.MK_OK
        g.close()
        return total, lat

    def run_served(arrivals, store):
        g = fresh()
        srv = mk.Server(g, max_inflight=max_inflight, commit_every=commit_every)
        lat = np.zeros(N)
        bad = 0
        nxt = done = 0
        t0 = time.perf_counter()
        while done < N:
            now = time.perf_counter() - t0
            while nxt < N and arrivals[nxt] <= now:
                k, n = int(kinds[nxt]), int(sizes[nxt])
                a, b, w = inputs(nxt)
                o0, o1 = outputs(nxt, store)
                srv.submit(k, a, b, w, n, int(srcs[nxt]), o0, o1, tag=nxt)
                nxt += 1
            for tag, st in srv.progress():
                lat[tag] = time.perf_counter() - t0 - arrivals[tag]
                bad += st != 0
                done += 1
        total = time.perf_counter() - t0
        srv.close()
        assert bad == 0, "%d requests refused or failed" % bad
        assert g.last_error() == mk.MK_OK
        g.close()
        return total, lat

    edges = float(sizes.sum())

    def summary(total, lat):
        return {"seconds": round(total, 3), "requests_per_s": round(N / total, 1),
                "medges_per_s": round(edges / total / 1e6, 1),
                "p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 3),
                "p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 3)}

    out = {"requests": N, "edges": int(edges), "max_inflight": max_inflight, "commit_every": commit_every}
    zero = np.zeros(N)
    store_p, store_s = {}, {}
    tp, lp = run_plain(zero, store_p)
    ts, ls = run_served(zero, store_s)
    out["capacity"] = {"plain": summary(tp, lp), "served": summary(ts, ls)}
    if log:
        log(out)
    mism = [i for i in store_p if not all(torch.equal(x, y) for x, y in zip(store_p[i], store_s[i]) if x is not None)]
    out["compared_requests"] = len(store_p)
    out["mismatches"] = len(mism)
    if keep_outputs:
        out["outputs"] = (store_p, store_s)
        out["inputs"] = inputs
    cap = N / tp
    for frac in rate_fracs:
        arr = np.cumsum(R.gaps[:N]) / (frac * cap)
        sp_, ss_ = {}, {}
        t1, l1 = run_plain(arr, sp_)
        t2, l2 = run_served(arr, ss_)
        m = [i for i in sp_ if not all(torch.equal(x, y) for x, y in zip(sp_[i], ss_[i]) if x is not None)]
        out["rate_%d%%" % round(frac * 100)] = {"rate_req_s": round(frac * cap, 1), "plain": summary(t1, l1),
                                                "served": summary(t2, l2), "mismatches": len(m)}
        out["mismatches"] += len(m)
    return out


# ------------------------------------------------------------- CPU oracle

ORACLE_SAMPLE = ("insert, delete and query of the step's B edges each, plus one from-scratch recompute of BFS, "
                 "Dijkstra SSSP and union-find WCC after the insert batch; the step time counts that recompute "
                 "twice, because the full step recomputes after each of its two update batches; single thread")


def oracle_step(o, bt, source):
    """Seconds of one step of the workload on the oracle (bounded sample:
    the recompute after the delete batch is taken to cost the same as the
    one after the insert batch)."""
    t0 = time.perf_counter()
    o.insert(bt["ins_src"], bt["ins_dst"], bt["ins_w"])
    t1 = time.perf_counter()
    o.bfs(source)
    o.sssp(source)
    o.wcc()
    t2 = time.perf_counter()
    o.delete(bt["del_src"], bt["del_dst"])
    o.query(bt["q_src"], bt["q_dst"])
    t3 = time.perf_counter()
    return (t1 - t0) + 2 * (t2 - t1) + (t3 - t2)


def run_oracle_steps(G, batches, source, steps, B):
    import oracle

    o = oracle.OracleGraph(G.V)
    o.insert(G.src, G.dst, G.w)
    secs = [oracle_step(o, batches[k], source) for k in range(steps)]
    return secs


def cpu_baseline(G, batches, source, B):
    secs = run_oracle_steps(G, batches, source, 1, B)
    s = secs[0]
    return {"value": round(3 * B / s / 1e6, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": ORACLE_SAMPLE + "; B = %d; %.1f s per step" % (B, s)}


def run_reference(args, world, rank, local):
    if rank != 0:
        return None
    W, K, B = args.warmup, args.steps, args.batch
    G, source, batches, _ = make_workload(args, W + K)
    import oracle

    o = oracle.OracleGraph(G.V)
    o.insert(G.src, G.dst, G.w)
    for k in range(W):
        # warm-up steps only advance the graph: the oracle recomputes from
        # scratch and has no state a warm-up could prime
        bt = batches[k]
        o.insert(bt["ins_src"], bt["ins_dst"], bt["ins_w"])
        o.delete(bt["del_src"], bt["del_dst"])
    secs = [oracle_step(o, batches[W + k], source) for k in range(K)]
    ms = statistics.mean(secs) * 1e3
    value = 3 * B / (ms / 1e3) / 1e6
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": round(ms, 1), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic", "config": workload_config(args, G),
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": ORACLE_SAMPLE + "; B = %d" % B},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_served(args):
    import torch

    import synth

    torch.cuda.set_device(0)
    t0 = time.time()
    G = synth.powerlaw_graph(scale=21, draws=1 << 25)
    R = synth.request_stream(100000, G.V, len(G.src))
    gen_s = time.time() - t0
    res = serve_experiment(G, R)
    res.update({"workload": "R-MAT scale 21 graph (V=2,097,152, 2^25 draws, duplicates and self-loops dropped, "
                            "weights U[1,100]) under a Poisson stream of 100,000 requests: 60% query, 15% insert, "
                            "15% delete, 10% incremental SSSP from a pool of 16 sources; sizes log-uniform in "
                            "[1, 2^20]; arrival rates 50% and 90% of the measured plain capacity",
                "gen_s": round(gen_s, 1)})
    return res


def run_road(args):
    """Road-like workload: 4,096 x 4,096 grid + 0.1% long-range edges, 64
    mixed batches of 2^16 (half deletes of grid links, half inserts), the
    incremental SSSP from the corner vertex after each batch."""
    import torch

    import paper_2305_17813_gb300 as mk
    import synth

    torch.cuda.set_device(0)
    t0 = time.time()
    R = synth.road_graph(4096, 4096)
    batches = [synth.road_batch(R, k) for k in range(64)]
    gen_s = time.time() - t0
    g = mk.Graph(R.V, edge_capacity_hint=len(R.src) + 64 * (1 << 16), buckets=1)
    chunk = 1 << 22
    for i in range(0, len(R.src), chunk):
        g.insert(R.src[i:i + chunk], R.dst[i:i + chunk], R.w[i:i + chunk], flags=False)
    g.commit()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    torch.cuda.synchronize()
    ev[0].record()
    g.sssp(0)
    ev[1].record()
    torch.cuda.synchronize()
    static_ms = ev[0].elapsed_time(ev[1])
    g.commit()
    dev = [{k: mk.to_device_u32(b[k]) for k in ("ins_src", "ins_dst", "ins_w", "del_src", "del_dst")} for b in batches]
    sssp_ms, del_ms, ins_ms = [], [], []
    for k in range(64):
        b = dev[k]
        ev[0].record()
        g.delete(b["del_src"], b["del_dst"], flags=False)
        ev[1].record()
        g.insert(b["ins_src"], b["ins_dst"], b["ins_w"], flags=False)
        ev[2].record()
        g.sssp(0)
        ev[3].record()
        g.commit()
        torch.cuda.synchronize()
        del_ms.append(ev[0].elapsed_time(ev[1]))
        ins_ms.append(ev[1].elapsed_time(ev[2]))
        sssp_ms.append(ev[2].elapsed_time(ev[3]))
    if g.last_error() != mk.MK_OK:
        raise RuntimeError("device status in the road run")
    nd, ni = len(batches[0]["del_src"]), len(batches[0]["ins_src"])
    g.close()
    return {"workload": "4,096 x 4,096 road-like grid (67,092,480 grid edges + 67,092 long-range edges, weights "
                        "U[1,1000]); 64 mixed batches of 2^16 (2^15 deletes of grid links, 2^15 inserts); "
                        "incremental SSSP from vertex 0 after each batch",
            "static_sssp_ms": round(static_ms, 2),
            "incr_sssp_ms_mean": round(statistics.mean(sssp_ms), 3),
            "incr_sssp_ms_p50": round(statistics.median(sssp_ms), 3),
            "incr_sssp_ms_max": round(max(sssp_ms), 3),
            "delete_medges_s": round(nd / statistics.mean(del_ms) / 1e3, 1),
            "insert_medges_s": round(ni / statistics.mean(ins_ms) / 1e3, 1),
            "gen_s": round(gen_s, 1)}


def run_growth(args):
    import torch

    import synth

    torch.cuda.set_device(0)
    t0 = time.time()
    S = synth.growth_stream(scale=22, draws=1 << 26, n_batches=64)
    gen_s = time.time() - t0
    res = growth_experiment(S, split=32, horizon=8, epochs=20)
    res.update({"workload": "R-MAT scale 22 growth stream (67,108,864 draws; first 50% loaded; 64 insert batches "
                            "with preferential source skew 0.5, each followed by 10% deletes); network trained on "
                            "batches 1-32, graphs rebuilt at batch 32 with learned vs load-factor bucket counts",
                "gen_s": round(gen_s, 1)})
    return res


def main(argv=None):
    args = parse_args(argv)
    world, rank, local = dist_env()
    if args.workload in ("growth", "served", "road"):
        if rank == 0:
            res = {"growth": run_growth, "served": run_served, "road": run_road}[args.workload](args)
            print(json.dumps(res), flush=True)
        return 0
    if args.impl == "reference":
        res = run_reference(args, world, rank, local)
        if res is not None:
            print(json.dumps(res), flush=True)
        return 0
    result, dist, G, source, batches = run_ours(args, world, rank, local)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            result["cpu_baseline"] = cpu_baseline(G, batches, source, args.batch)
        print(json.dumps(result), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
