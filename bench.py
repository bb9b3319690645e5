#!/usr/bin/env python3
"""Benchmark of the dynamic graph store's hot path on the power-law workload.

Workload (R-MAT scale 20: V = 1,048,576, 16,777,216 draws with a/b/c/d =
0.57/0.19/0.19/0.05, duplicates and self-loops dropped, weights U[1,100];
buckets from the load-factor rule with load factor 0.7).  One step is one
pass of the whole path on one batch of size B (default 2^20):

    insert B new R-MAT edges -> incremental BFS, SSSP (from the max-degree
    vertex) and WCC -> commit -> delete B live edges -> BFS, SSSP (decremental)
    and WCC (static recompute) -> commit -> query B edges (half present)

The batches come from synth.PowerlawStream, which draws every delete from
the edges live at that point and exactly half of the queries from the live
edges; after the timed region every timed step is checked from the kernels'
own flags and bitmaps (all deletes applied, exactly B // 2 queries present,
the inserts the stream expects), and the run stops without a value if one
is off.

WCC and the query batch only read the graph, as BFS and SSSP do: they run
on a second stream (default priority) forked after each update batch and
joined before the next change, beside BFS/SSSP on the main stream (high
priority); the step's phases are timed on the main stream and the second
stream's calls by their own events.

value = 3B edges (inserted + deleted + queried) / step time, in Medges/s,
with inputs resident in device memory; `e2e` is the same through the C-ABI
with the inputs copied from pinned host buffers and every result (flags,
bitmap, BFS/SSSP distances and parents, WCC labels) copied back inside the
timed region.  L2 is flushed between steps by writing a 512 MiB buffer.
After them come three steps with every call on one stream (`kernels_solo`:
each kernel family's own GB/s and fraction of the measured copy bandwidth)
and steps at the workload's other batch sizes 2^12, 2^16 and 2^22
(`per_batch`), continuing the same stream of batches.

`--impl reference` times the CPU oracle (plain single-threaded C++,
recomputing everything from scratch) on the same workload and metric, every
part of every step executed (see OracleStep).  Under torchrun each rank runs
an independent replica (weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
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
    p.add_argument("--no-solo", action="store_true", help="skip the steps that time every kernel alone")
    p.add_argument("--no-per-batch", action="store_true",
                   help="skip the steps at the workload's other batch sizes (2^12, 2^16, 2^22)")
    p.add_argument("--workload", choices=["powerlaw", "growth", "served", "road", "analytics", "buckets", "l2", "set"],
                   default="powerlaw",
                   help="powerlaw: the benchmark line; growth: the learned-sizing study on the R-MAT "
                        "scale-22 growth stream; served: plain vs continuous-batching serving on the R-MAT "
                        "scale-21 request stream; road: incremental SSSP on the 4096^2 road-like grid; "
                        "analytics: PageRank and triangle counting; buckets: the power-law step with the "
                        "load-factor bucket rule against one bucket per vertex (hashing off); l2: the step "
                        "with L2 persistence windows over parts of the store; set: the map layout against "
                        "the ConcurrentSet layout (each prints its own JSON line)")
    p.add_argument("--road-size", type=int, default=4096, help="road workload: grid side")
    p.add_argument("--road-batches", type=int, default=64, help="road workload: mixed batches")
    p.add_argument("--road-batch-size", type=int, default=1 << 16, help="road workload: edges a batch")
    p.add_argument("--road-delta", type=int, default=None,
                   help="road workload: one pass with this Near-Far width for every call instead of the "
                        "three passes (plain, ordered static call, ordered every call)")
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

def make_workload(args, max_batch):
    """The R-MAT graph, the BFS/SSSP source (largest out-degree, ties to the
    smallest id) and the batch stream (synth.PowerlawStream)."""
    import synth

    G = synth.powerlaw_graph(scale=args.scale, draws=args.draws)
    deg = np.bincount(G.src, minlength=G.V)
    source = int(np.argmax(deg))
    return G, source, synth.PowerlawStream(G, max_batch=max_batch)


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
        "batches": "deletes drawn from the edges live at the delete, queries exactly half live (checked per step)",
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
        # walk of the updated lists, or the inserted-edge log (16 B an entry
        # plus the 8 B source node)
        return (ctr["seed_lists"] * (4 + 8 + 8) + 128 * ctr["seed_slabs"] + 16 * ctr["seed_edges"]
                + ctr["seed_improved"] * (8 + 4 + 8) + ctr.get("seed_log", 0) * (16 + 8))
    if family == "sssp_invalidate_walk":
        return ctr["walk_vertices"] * 8 + ctr["invalidated"] * 8
    if family == "wcc_hook_all":
        return 128 * ctr["wcc_slabs"] + 16 * ctr["wcc_edges"]
    if family == "wcc_hook_updated":
        # walk of the updated lists, or the inserted-edge log (16 B an entry)
        return 128 * ctr["wcc_upd_slabs"] + 16 * ctr["wcc_upd_edges"] + 16 * ctr.get("wcc_log", 0)
    return None


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
# kernel families, from the committed ncu launch list of this benchmark
# (full workload, one pass), and
# the SHA-256 of the kernel sources (csrc/) it was taken with.  A figure is
# reported only while those sources are unchanged; otherwise traffic is null.
NCU_TRAFFIC_SOURCES_SHA = "23cc176d5d3307aa6d343140c981b5fca75866b242cd4298c6962f3e813fb31d"
NCU_TRAFFIC = {
"sssp_rounds": 49676000,
    "sssp_relax_into_invalid": 280899072,
    "sssp_enqueue_invalid": 11004224,
    "sssp_relax_updated": 26472768,
    "sssp_invalidate_walk": 8524864,
    "sssp_invalidate": 13739456,
    "wcc_hook_all": 350455296,
    "wcc_hook_updated": 19096192,
    "insert": 255002240,
    "delete": 198414976,
    "query": 130889088,
    "stage_dedup": 40148544,
    "update_slab_pointers": 60540224,
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

class StepRunner:
    """One device graph of the power-law workload and the step that the
    benchmark times (see the module docstring), with per-step output buffers
    so that every timed step can be checked afterwards."""

    def __init__(self, args, G, source, capacity_edges, device, buckets=None):
        import torch

        import paper_2305_17813_gb300 as mk

        self.mk, self.torch, self.device = mk, torch, device
        self.lib = lib = mk.load()
        self.V, self.source = G.V, source
        # the step runs on a high-priority stream; the calls that only read
        # the graph (WCC, the query batch) run beside it on a second stream
        self.stream = torch.cuda.Stream(device=device, priority=-1)
        torch.cuda.set_stream(self.stream)
        self.sp = ctypes.c_void_p(self.stream.cuda_stream)
        self.side = torch.cuda.Stream(device=device)
        self.sidep = ctypes.c_void_p(self.side.cuda_stream)
        E = len(G.src)
        src_d = self.u32(G.src)
        if buckets is None:
            buckets = mk.bucket_rule(G.V, src_d, 0.7)
        self.g = mk.Graph(G.V, edge_capacity_hint=capacity_edges, buckets=buckets)
        self.h = self.g.handle
        chunk = 1 << 22
        dst_d, w_d = self.u32(G.dst), self.u32(G.w)
        for i in range(0, E, chunk):
            mk.check(lib.mk_insert_batch(self.h, self.P(src_d[i:i + chunk]), self.P(dst_d[i:i + chunk]),
                                         self.P(w_d[i:i + chunk]), min(chunk, E - i), None, self.sp), "load")
        del src_d, dst_d, w_d
        self.g.commit()
        self.out = {k: torch.empty(G.V, dtype=torch.int32, device=device) for k in ("bd", "bp", "sd", "sp", "lab")}
        P = self.P
        for fn, a, b in ((lib.mk_incr_bfs, "bd", "bp"), (lib.mk_incr_sssp, "sd", "sp")):
            mk.check(fn(self.h, source, P(self.out[a]), P(self.out[b]), self.sp), "static")
        mk.check(lib.mk_incr_wcc(self.h, P(self.out["lab"]), self.sp), "static wcc")
        self.g.commit()
        torch.cuda.synchronize()
        st = self.g.last_error()
        if st != mk.MK_OK:
            raise RuntimeError("device status %d after the load" % st)
        self.flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=device)

    def u32(self, a):
        return self.mk.to_device_u32(a, self.device)

    @staticmethod
    def P(t):
        return ctypes.c_void_p(t.data_ptr())

    def to_device(self, bt):
        return {k: self.u32(bt[k]) for k in BATCH_KEYS}

    def outputs(self, n, steps):
        """Per-step flag and bitmap buffers (insert flags, delete flags,
        query bitmap) for `steps` steps of batch size n."""
        torch = self.torch
        return [(torch.empty(n, dtype=torch.uint8, device=self.device),
                 torch.empty(n, dtype=torch.uint8, device=self.device),
                 torch.empty((n + 31) // 32, dtype=torch.int32, device=self.device)) for _ in range(steps)]

    def step(self, bt, n, outs, ev, wev, hooks=None, solo=False):
        """One step on batch bt (device tensors) of size n.  ev: 12 events
        on the main stream, wev: 5 on the second stream.  solo=True runs
        every call on the main stream (no overlap)."""
        mk, lib, P, h, out, src = self.mk, self.lib, self.P, self.h, self.out, self.source
        stream, sp = self.stream, self.sp
        ws, wsp = (stream, sp) if solo else (self.side, self.sidep)
        fl_i, fl_d, bm = outs
        hooks = hooks or {}
        ev[0].record(stream)
        mk.check(lib.mk_insert_batch(h, P(bt["ins_src"]), P(bt["ins_dst"]), P(bt["ins_w"]), n, P(fl_i), sp), "ins")
        ev[1].record(stream)
        if "after_insert" in hooks:
            hooks["after_insert"]()
        ws.wait_event(ev[1])
        wev[0].record(ws)
        mk.check(lib.mk_incr_wcc(h, P(out["lab"]), wsp), "wcc")
        wev[1].record(ws)
        mk.check(lib.mk_incr_bfs(h, src, P(out["bd"]), P(out["bp"]), sp), "bfs")
        ev[2].record(stream)
        mk.check(lib.mk_incr_sssp(h, src, P(out["sd"]), P(out["sp"]), sp), "sssp")
        ev[3].record(stream)
        stream.wait_event(wev[1])
        ev[4].record(stream)
        mk.check(lib.mk_commit_batch(h, sp), "commit")
        ev[5].record(stream)
        if "before_delete" in hooks:
            hooks["before_delete"]()
        mk.check(lib.mk_delete_batch(h, P(bt["del_src"]), P(bt["del_dst"]), n, P(fl_d), sp), "del")
        ev[6].record(stream)
        if "after_delete" in hooks:
            hooks["after_delete"]()
        ws.wait_event(ev[6])
        wev[2].record(ws)
        mk.check(lib.mk_incr_wcc(h, P(out["lab"]), wsp), "wcc")
        wev[3].record(ws)
        # the query batch only reads the graph too: after the delete, beside
        # the decremental BFS/SSSP (a commit moves only update markers)
        mk.check(lib.mk_query_batch(h, P(bt["q_src"]), P(bt["q_dst"]), n, P(bm), None, wsp), "query")
        wev[4].record(ws)
        if "after_side" in hooks:
            hooks["after_side"](ws)
        mk.check(lib.mk_incr_bfs(h, src, P(out["bd"]), P(out["bp"]), sp), "bfs")
        ev[7].record(stream)
        if "after_bfs" in hooks:
            hooks["after_bfs"]()
        mk.check(lib.mk_incr_sssp(h, src, P(out["sd"]), P(out["sp"]), sp), "sssp")
        ev[8].record(stream)
        stream.wait_event(wev[3])
        ev[9].record(stream)
        mk.check(lib.mk_commit_batch(h, sp), "commit")
        ev[10].record(stream)
        stream.wait_event(wev[4])
        ev[11].record(stream)

    def events(self, n):
        return [self.torch.cuda.Event(enable_timing=True) for _ in range(n)]

    def run(self, batches, n, warmup, flush_tag, solo=False, clock=None, dist=None):
        """Warm-up steps, then the timed steps, each on its own batch; returns
        the timing record and the per-step outputs of the timed steps."""
        torch, mk, g = self.torch, self.mk, self.g
        dev = [self.to_device(bt) for bt in batches]
        warm_outs = self.outputs(n, 1)[0]
        for k in range(warmup):
            self.flush.fill_(flush_tag + k)
            torch.cuda.nvtx.range_push("step")  # lets a profiler select the steps' kernels
            self.step(dev[k], n, warm_outs, self.events(12), self.events(5), solo=solo)
            torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        if g.last_error() != mk.MK_OK:
            raise RuntimeError("device status after warm-up")
        K = len(batches) - warmup
        outs = self.outputs(n, K)
        evs = [self.events(12) for _ in range(K)]
        wevs = [self.events(5) for _ in range(K)]
        g.counters(reset=True)
        g.profile(True)
        g.profile_read()
        launches0 = g.launch_count()
        barrier(dist, self.device)
        torch.cuda.synchronize()
        wall0 = time.time()
        with (clock if clock is not None else _Null()):
            for k in range(K):
                self.flush.fill_(flush_tag + warmup + k)
                torch.cuda.nvtx.range_push("step")
                self.step(dev[warmup + k], n, outs[k], evs[k], wevs[k], solo=solo)
                torch.cuda.nvtx.range_pop()
            torch.cuda.synchronize()
        wall = time.time() - wall0
        barrier(dist, self.device)
        launches = g.launch_count() - launches0
        prof = g.profile_read()
        g.profile(False)
        ctr = g.counters()
        status = g.last_error()
        if status != mk.MK_OK:
            raise RuntimeError("device status %d in the timed region" % status)
        names = ["insert", "bfs1", "sssp1", "wcc1_wait", "commit1", "delete", "bfs2", "sssp2", "wcc2_wait",
                 "commit2", "query_wait"]
        rec = {
            "step_ms": [evs[k][0].elapsed_time(evs[k][11]) for k in range(K)],
            "phase": {nm: statistics.mean(evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(K))
                      for i, nm in enumerate(names)},
            "wcc_incr": statistics.mean(wevs[k][0].elapsed_time(wevs[k][1]) for k in range(K)),
            "wcc_static": statistics.mean(wevs[k][2].elapsed_time(wevs[k][3]) for k in range(K)),
            "query_ms": statistics.mean(wevs[k][3].elapsed_time(wevs[k][4]) for k in range(K)),
            "prof": prof, "ctr": ctr, "launches": int(launches), "wall": wall, "K": K,
        }
        return rec, outs, batches[warmup:]

    def close(self):
        self.g.close()


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


BATCH_KEYS = ("ins_src", "ins_dst", "ins_w", "del_src", "del_dst", "q_src", "q_dst")


def check_steps(outs, batches, n):
    """The workload check of every timed step, from the kernels' own
    outputs: each insert flagged exactly the edges that the stream added to
    its live set, each delete removed all n edges, and exactly n // 2
    queries were present.  Raises when a step was not a step of the
    workload (no value is printed then)."""
    ins, dele, qry = [], [], []
    for (fl_i, fl_d, bm), bt in zip(outs, batches):
        ni = int(fl_i.sum().item())
        nd = int(fl_d.sum().item())
        words = bm.cpu().numpy().view(np.uint32)
        nq = int(np.unpackbits(words.view(np.uint8)).sum())
        if ni != bt["n_inserted"] or nd != n or nq != bt["n_present"]:
            raise RuntimeError("batch %d is off the workload: %d inserted (stream: %d), %d of %d deleted, "
                               "%d of %d queries present (stream: %d)"
                               % (bt["k"], ni, bt["n_inserted"], nd, n, nq, n, bt["n_present"]))
        ins.append(ni / n)
        dele.append(nd / n)
        qry.append(nq / n)
    return {"steps_checked": len(outs), "batches": [int(bt["k"]) for bt in batches],
            "insert_applied_frac": [round(min(ins), 4), round(max(ins), 4)],
            "delete_applied_frac": [round(min(dele), 4), round(max(dele), 4)],
            "query_present_frac": [round(min(qry), 4), round(max(qry), 4)],
            "rule": "every delete removes a live edge and exactly half the queries are present, checked from "
                    "the kernels' flags and bitmaps of every timed step"}


def family_table(prof, ctr, n, peak):
    """Per kernel family: launches, summed CUDA-event ms, share of the summed
    time, and (where a byte model exists) achieved GB/s and its fraction of
    the measured copy bandwidth."""
    fam_time = {name: t for name, (m, t) in prof.items()}
    fam_launch = {name: m for name, (m, t) in prof.items()}
    total = sum(fam_time.values()) or 1.0
    out = {}
    for name in sorted(fam_time, key=fam_time.get, reverse=True):
        bt = algorithmic_bytes(name, ctr, n, fam_launch[name])
        out[name] = {"launches": fam_launch[name], "ms": round(fam_time[name], 3),
                     "share": round(fam_time[name] / total, 4)}
        if bt is not None and fam_time[name] > 0:
            gbs = bt / (fam_time[name] / 1e3) / 1e9
            out[name]["gbs"] = round(gbs, 1)
            out[name]["frac"] = round(gbs / peak, 4)
    return out


def summarize(rec, n, peak, units_factor=3.0):
    ph = rec["phase"]
    ms = statistics.mean(rec["step_ms"])
    return {
        "value": round(units_factor * n / (ms / 1e3) / 1e6, 2), "ms_per_step": round(ms, 3),
        "insert_medges_s": round(n / ph["insert"] / 1e3, 1),
        "delete_medges_s": round(n / ph["delete"] / 1e3, 1),
        "query_medges_s": round(n / rec["query_ms"] / 1e3, 1),
        "incr_sssp_ms": round(ph["sssp1"], 3), "decr_sssp_ms": round(ph["sssp2"], 3),
        "incr_bfs_ms": round(ph["bfs1"], 3), "decr_bfs_ms": round(ph["bfs2"], 3),
        "incr_wcc_ms": round(rec["wcc_incr"], 3), "static_wcc_ms": round(rec["wcc_static"], 3),
    }


def run_ours(args, world, rank, local):
    import torch

    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist = dist_init(world, True)
    W, K, B = args.warmup, args.steps, args.batch
    n_e2e = 0 if args.no_e2e else K
    n_solo = 0 if args.no_solo else 3
    per_batch = [] if args.no_per_batch else [b for b in PER_BATCH if b != B]
    t0 = time.time()
    G, source, S = make_workload(args, max([B] + per_batch))
    main_batches = [S.batch(B) for _ in range(W + K + n_e2e + n_solo)]
    gen_s = time.time() - t0
    V, E = G.V, len(G.src)
    inserted_total = B * len(main_batches) + sum(pb * (PB_WARMUP + pb_steps(pb)) for pb in per_batch)
    R = StepRunner(args, G, source, E + inserted_total, device)
    mk, lib, g = R.mk, R.lib, R.g

    # X2 autotuner: kernel shapes for this graph (untimed setup)
    tb = main_batches[0]
    tuning = g.autotune(tb["q_src"], tb["q_dst"], source)
    g.commit()

    peak, peak_kind = measured_peak()
    clock = ClockSampler(os.path.join(tempfile.gettempdir(), "bench_clocks_rank%d_%d.csv" % (rank, os.getpid())))
    rec, outs, timed = R.run(main_batches[:W + K], B, W, flush_tag=0, clock=clock, dist=dist)
    checks = check_steps(outs, timed, B)
    del outs
    main = summarize(rec, B, peak)
    ms_max, = reduce_across([statistics.mean(rec["step_ms"])], "max", dist, device)
    units_total, = reduce_across([3.0 * B], "sum", dist, device)
    value = units_total / (ms_max / 1e3) / 1e6

    prof, ctr = rec["prof"], rec["ctr"]
    kernels = family_table(prof, ctr, B, peak)
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    roof = None
    bytes_total = algorithmic_bytes(dom, ctr, B, kernels[dom]["launches"])
    if bytes_total is not None and kernels[dom]["ms"] > 0:
        nl = kernels[dom]["launches"]
        per_launch_bytes = bytes_total / nl
        avg_ms = kernels[dom]["ms"] / nl
        achieved = per_launch_bytes / (avg_ms / 1e3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_source": peak_kind, "traffic": ncu_traffic(dom),
                "algorithmic_bytes_per_launch": int(per_launch_bytes), "avg_launch_ms": round(avg_ms, 4),
                "launches": nl}

    result = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": round(ms_max, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic", "config": workload_config(args, G),
        **{k: v for k, v in main.items() if k not in ("value", "ms_per_step")},
        "wcc_overlap": "WCC and the query batch run on a second stream beside BFS/SSSP; their ms and rates are "
                       "their own durations there",
        "phases_ms": {k: round(v, 3) for k, v in rec["phase"].items()},
        "workload_check": checks,
        "roofline": roof, "kernels": kernels, "counters": ctr,
        "gpu_launches": rec["launches"], "wall_s_timed": round(rec["wall"], 3), "gen_s": round(gen_s, 1),
        "tuning": {k: tuning[k] for k in ("query_group", "query_block", "rounds_blocks_per_sm")},
        "clocks": clock.summary(local),
    }
    at = W + K

    # end to end through the C ABI with host buffers
    if n_e2e:
        result["e2e"] = run_e2e(R, main_batches[at:at + n_e2e], B, dist, units_total)
        at += n_e2e

    # every kernel family timed alone: the same step with every call on the
    # main stream, so that no family shares the GPU with another
    if n_solo:
        srec, souts, stimed = R.run(main_batches[at:at + n_solo], B, 0, flush_tag=500, solo=True)
        check_steps(souts, stimed, B)
        del souts
        sk = family_table(srec["prof"], srec["ctr"], B, peak)
        result["kernels_solo"] = {"steps": n_solo, "ms_per_step": round(statistics.mean(srec["step_ms"]), 3),
                                  "peak": peak, "families": sk}
        at += n_solo

    # the other batch sizes of the workload, continuing the same stream
    if per_batch:
        pbr = {str(B): {**main, "steps": K, "warmup": W,
                        "o_e_share": o_e_share(kernels)}}
        for pb in per_batch:
            nW, nK = PB_WARMUP, pb_steps(pb)
            bts = [S.batch(pb) for _ in range(nW + nK)]
            prec, pouts, ptimed = R.run(bts, pb, nW, flush_tag=1000 + pb % 997)
            pchk = check_steps(pouts, ptimed, pb)
            del pouts
            pk = family_table(prec["prof"], prec["ctr"], pb, peak)
            pbr[str(pb)] = {**summarize(prec, pb, peak), "steps": nK, "warmup": nW,
                            "batches": pchk["batches"], "o_e_share": o_e_share(pk),
                            "top_kernels": {k: pk[k] for k in list(pk)[:5]}}
        result["per_batch"] = pbr
    R.close()
    return result, dist, G, source, main_batches


PER_BATCH = (1 << 12, 1 << 16, 1 << 20, 1 << 22)
PB_WARMUP = 3


def pb_steps(pb):
    return 3 if pb >= 1 << 22 else 5


def o_e_share(kernels):
    """Share of the summed kernel time taken by the passes over every edge
    (the decremental relax-into-invalid scan and the static WCC pass), which
    do not shrink with the batch."""
    return round(sum(kernels[k]["share"] for k in ("sssp_relax_into_invalid", "wcc_hook_all", "wcc_init")
                     if k in kernels), 4)


def run_e2e(R, batches, B, dist, units_total):
    """Steps through the C ABI with the inputs in pinned host memory: every
    step copies its inputs in and its results out inside its timed span
    (insert and delete flags, the query bitmap, BFS and SSSP distances and
    parents, WCC labels).  The inputs of later phases come in, and every
    result leaves as soon as the step no longer writes it, on a copy stream
    beside the phases still running; only the SSSP tree leaves at the end.
    The steps are queued back to back, as the device-resident steps are
    (each step's span runs from before its first copy in to after its last
    copy out, and the next step's copies wait for it), and every step's
    results are checked on the host after the last one."""
    torch, mk = R.torch, R.mk
    device, stream, V = R.device, R.stream, R.V
    K = len(batches)
    # a step's seven input arrays sit back to back in one pinned buffer (the
    # insert's three first), so they come in with two copies, not seven
    host = [torch.from_numpy(np.concatenate([np.ascontiguousarray(bt[k]).view(np.int32) for k in BATCH_KEYS]))
            .pin_memory() for bt in batches]
    stage_all = torch.empty(len(BATCH_KEYS) * B, dtype=torch.int32, device=device)
    stage = {k: stage_all[i * B:(i + 1) * B] for i, k in enumerate(BATCH_KEYS)}
    n_ins = 3 * B
    outs = R.outputs(B, 1)[0]
    fl_i, fl_d, bm = outs
    # one set of pinned result buffers per step
    h_out = [{"fl_i": torch.empty(B, dtype=torch.uint8).pin_memory(),
              "fl_d": torch.empty(B, dtype=torch.uint8).pin_memory(),
              "bm": torch.empty((B + 31) // 32, dtype=torch.int32).pin_memory(),
              **{key: torch.empty(V, dtype=torch.int32).pin_memory() for key in R.out}} for _ in range(K)]
    copy = torch.cuda.Stream(device=device)
    evs = [R.events(14) for _ in range(K)]
    wevs = [R.events(5) for _ in range(K)]

    def on_copy(src_stream, pairs):
        """Copy stream waits for src_stream's work so far, then copies."""
        done = torch.cuda.Event()
        done.record(src_stream)
        copy.wait_event(done)
        with torch.cuda.stream(copy):
            for dst, t in pairs:
                dst.copy_(t, non_blocking=True)

    torch.cuda.synchronize()
    for k in range(K):
        e, h = evs[k], h_out[k]
        R.flush.fill_(100 + k)
        e[0].record(stream)
        with torch.cuda.stream(stream):
            stage_all[:n_ins].copy_(host[k][:n_ins], non_blocking=True)
        # the later phases' inputs follow the insert's on the link (copies
        # that share it would delay the insert's), while the insert runs
        ins_in = torch.cuda.Event()
        ins_in.record(stream)
        copy.wait_event(ins_in)
        ready = torch.cuda.Event()
        with torch.cuda.stream(copy):
            stage_all[n_ins:].copy_(host[k][n_ins:], non_blocking=True)
            ready.record(copy)
        hooks = {
            "after_insert": lambda h=h: on_copy(stream, [(h["fl_i"], fl_i)]),
            "before_delete": lambda ready=ready: stream.wait_event(ready),
            "after_delete": lambda h=h: on_copy(stream, [(h["fl_d"], fl_d)]),
            # results that nothing later in the step rewrites leave while
            # the rest of the step runs: the query bitmap and the WCC labels
            # (second stream), the BFS tree (main stream, beside the SSSP)
            "after_side": lambda ws, h=h: on_copy(ws, [(h["bm"], bm), (h["lab"], R.out["lab"])]),
            "after_bfs": lambda h=h: on_copy(stream, [(h["bd"], R.out["bd"]), (h["bp"], R.out["bp"])]),
        }
        R.step(stage, B, outs, e[1:13], wevs[k], hooks)
        for key in ("sd", "sp"):
            h[key].copy_(R.out[key], non_blocking=True)
        # the next step rewrites the device buffers only after every copy
        # of this one
        stream.wait_stream(copy)
        e[13].record(stream)
    torch.cuda.synchronize()
    e2e_ms = [evs[k][0].elapsed_time(evs[k][13]) for k in range(K)]
    parts = [(evs[k][0].elapsed_time(evs[k][1]), evs[k][1].elapsed_time(evs[k][12]),
              evs[k][12].elapsed_time(evs[k][13])) for k in range(K)]
    for k, bt in enumerate(batches):
        h = h_out[k]
        nq = int(np.unpackbits(h["bm"].numpy().view(np.uint8)).sum())
        if (int(h["fl_i"].sum()) != bt["n_inserted"] or int(h["fl_d"].sum()) != B or nq != bt["n_present"]):
            raise RuntimeError("e2e batch %d is off the workload" % bt["k"])
    if R.g.last_error() != mk.MK_OK:
        raise RuntimeError("device status in the e2e pass")
    e2e_max, = reduce_across([statistics.mean(e2e_ms)], "max", dist, device)
    return {"value": round(units_total / (e2e_max / 1e3) / 1e6, 2), "unit": UNIT,
            "h2d_bytes_per_step": int(B * 4 * len(BATCH_KEYS)),
            "d2h_bytes_per_step": int(2 * B + 4 * ((B + 31) // 32) + 4 * V * len(R.out)),
            "ms_per_step": round(e2e_max, 3), "batches": [int(bt["k"]) for bt in batches],
            # the step's own span split in three: the insert inputs coming in
            # before the first call, the calls (with the other copies beside
            # them), and the SSSP tree (with any copy still running) after
            "split_ms": {name: round(statistics.mean(p[i] for p in parts), 3)
                         for i, name in enumerate(("inputs_in", "calls", "tail_out"))},
            "copies": "in: the step's 7 input arrays, back to back in one pinned host buffer (two copies); out: "
                      "insert and delete flags, query bitmap, BFS and SSSP distances and parents, WCC labels, "
                      "into pinned buffers of each step, checked after the run"}


# ------------------------------------------------------- learned sizing

def growth_experiment(S, split=32, horizon=8, epochs=20, lr=3e-3, load_factor=0.7, keep_graphs=False, repeats=1):
    """Learned slab sizing on a growth stream S (synth.growth_stream).

    A graph sized by the load-factor rule at the initial load runs batches
    1..split while a degree trace records every applied insert and delete.
    The network is trained on (features at batch t, edges gained per batch
    over the next `horizon` batches) for every t with a full window, then
    predicts each vertex's growth over the remaining batches.  Three graphs
    are rebuilt from the live edges at `split`: one with the learned bucket
    counts, one with the load-factor rule on the current degrees, and one
    with the rule on the initial load's degrees (the paper's a priori
    sizing).  Each runs the remaining batches `repeats` times on a fresh
    graph; the insert rate, a query batch over live edges (mean and spread
    over the repeats), chain lengths and slabs walked per query are
    compared, and a gain counts only when it exceeds the summed spreads."""
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
    # three layouts rebuilt from the same live edges at `split`: the learned
    # bucket counts, the load-factor rule on the current degrees, and the
    # rule on the initial load's degrees (the paper's a priori sizing, which
    # the first graph ran with); each replays the remaining batches
    # `repeats` times (a fresh graph each time), so the spread of the rates
    # is measured
    for name, bk in (("learned", learned_b), ("rule", rule_b), ("a_priori", b0)):
        ins_rates, q_rates = [], []
        for rep in range(repeats):
            rng = np.random.default_rng(7)
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
            ins_rates.append(n_ins / ins_ms / 1e3)
            q_rates.append(qs.numel() / q_ms / 1e3)
            if rep == 0:
                ctr = gg.counters()
                st = gg.stats()
                out[name] = {"lists": int(st["lists"]), "chain_mean": round(st["chain_mean"], 4),
                             "chain_max": int(st["chain_max"]), "device_bytes": int(st["device_bytes"]),
                             "query_slabs_per_query": round(ctr["query_slabs"] / 7 / qs.numel(), 4)}
            if keep_graphs and rep == 0 and name != "a_priori":
                graphs.append(gg)
            else:
                gg.close()
        out[name].update({
            "repeats": repeats,
            "insert_medges_s": round(statistics.mean(ins_rates), 1),
            "insert_medges_s_std": round(statistics.pstdev(ins_rates), 1),
            "query_medges_s": round(statistics.mean(q_rates), 1),
            "query_medges_s_std": round(statistics.pstdev(q_rates), 1),
            "insert_medges_s_all": [round(x, 1) for x in ins_rates],
            "query_medges_s_all": [round(x, 1) for x in q_rates]})
    for base in ("rule", "a_priori"):
        for op in ("insert", "query"):
            m_l, m_b = out["learned"][op + "_medges_s"], out[base][op + "_medges_s"]
            spread = out["learned"][op + "_medges_s_std"] + out[base][op + "_medges_s_std"]
            out["learned_vs_%s_%s" % (base, op)] = {"gain": round(m_l / m_b - 1.0, 4),
                                                    "beyond_spread": bool(m_l - m_b > spread)}
    model.close()
    if keep_graphs:
        out["graphs"] = graphs
    return out


# ---------------------------------------------------------------- serving

def serve_experiment(G, R, ring, rate_fracs=(0.5, 0.9), max_inflight=64, commit_every=8, retain_every=16,
                     retain_sssp_every=64, n_req=None, log=None, keep_outputs=False):
    """Plain one-launch-per-request execution against the continuous-batching
    server on the same request stream R (synth.request_stream) over graph G,
    its updates and present queries reading the sequence of G's edges (in a
    fixed random order) followed by `ring` (synth.new_edge_pool) and a copy
    of the ring's first R.hi edges.  First both run with every request available at once (capacity), then
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
    perm = synth.permutation(E, synth.substream(3100, 3))
    tail = min(int(R.hi), len(ring.src))
    seq_s = u(np.concatenate([G.src[perm], ring.src, ring.src[:tail]]))
    seq_d = u(np.concatenate([G.dst[perm], ring.dst, ring.dst[:tail]]))
    seq_w = u(np.concatenate([G.w[perm], ring.w, ring.w[:tail]]))
    AP = int(R.absent_pool)
    abs_s, abs_d = (u(x) for x in synth.uniform_pairs(V, AP, synth.substream(3100, 4)))
    qsrc = R.qsrc[:N]
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
            if qsrc[i]:
                return abs_s[o:o + n], abs_d[o:o + n], None
            return seq_s[o:o + n], seq_d[o:o + n], None
        if k == 1:
            return seq_s[o:o + n], seq_d[o:o + n], seq_w[o:o + n]
        if k == 2:
            return seq_s[o:o + n], seq_d[o:o + n], None
        return None, None, None

    # every insert may claim a new slab pair: room for all of them (deleted
    # pairs are never reused)
    pool = int((E + int(R.inserted)) / 15 * 1.3) + (1 << 21)

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
    # what the retained requests applied or found (the share of insert and
    # delete flags set and of queries present), beside what the stream's
    # live window predicts
    tally = {0: [0, 0], 1: [0, 0], 2: [0, 0]}
    for i, outs in store_p.items():
        k, n = int(kinds[i]), int(sizes[i])
        if k in (1, 2) and n:
            tally[k][0] += int(outs[0][:n].sum().item())
            tally[k][1] += n
        elif k == 0 and n:
            words = outs[0].cpu().numpy().view(np.uint32)
            tally[0][0] += int(np.unpackbits(words.view(np.uint8), bitorder="little")[:n].sum())
            tally[0][1] += n
    exp = {k: [int(R.applied[i]) for i in store_p if int(kinds[i]) == k and int(sizes[i])] for k in (1, 2)}
    out["retained_outcomes"] = {"insert_applied_frac": round(tally[1][0] / max(tally[1][1], 1), 4),
                                "delete_applied_frac": round(tally[2][0] / max(tally[2][1], 1), 4),
                                "query_present_frac": round(tally[0][0] / max(tally[0][1], 1), 4),
                                "expected_insert_applied_frac": round(sum(exp[1]) / max(tally[1][1], 1), 4),
                                "expected_delete_applied_frac": round(sum(exp[2]) / max(tally[2][1], 1), 4),
                                "stream_insert_applied_frac": round(float(R.applied[R.kind == 1].sum())
                                                                    / max(float(R.size[R.kind == 1].sum()), 1), 4),
                                "stream_delete_applied_frac": round(float(R.applied[R.kind == 2].sum())
                                                                    / max(float(R.size[R.kind == 2].sum()), 1), 4)}
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

ORACLE_SAMPLE = ("the whole step on the oracle (plain single-threaded C++): insert, delete and query of the step's "
                 "B edges and a from-scratch BFS, Dijkstra SSSP and union-find WCC after each of the two update "
                 "batches; two replicas of the oracle graph (one after the insert batch, one after the delete "
                 "batch) let the six recomputes and the query batch run at once on seven host threads")


class OracleStep:
    """The benchmark step on the CPU oracle, every part of it executed.

    Two replicas of the oracle's edge set are kept: replica `a` is brought
    to the state after the step's insert batch and replica `b` to the state
    after its delete batch, so the six from-scratch recomputes of a step
    (BFS, SSSP and WCC after each update batch) and the query batch, which
    only read a replica, run at once on seven host threads (each oracle call
    is one foreign call, during which ctypes releases the interpreter lock).
    Replica `a` then applies the delete batch to catch up."""

    THREADS = 7

    def __init__(self, G):
        import concurrent.futures as cf

        import oracle

        self.pool = cf.ThreadPoolExecutor(max_workers=self.THREADS)
        self.a, self.b = oracle.OracleGraph(G.V), oracle.OracleGraph(G.V)
        for f in [self.pool.submit(x.insert, G.src, G.dst, G.w) for x in (self.a, self.b)]:
            f.result()

    def advance(self, bt):
        """Apply a batch's updates without timing (warm-up batches)."""
        def upd(x):
            x.insert(bt["ins_src"], bt["ins_dst"], bt["ins_w"])
            x.delete(bt["del_src"], bt["del_dst"])
        for f in [self.pool.submit(upd, x) for x in (self.a, self.b)]:
            f.result()

    def _timed(self, fn, *a):
        t0 = time.perf_counter()
        fn(*a)
        return time.perf_counter() - t0

    def step(self, bt, source):
        """Seconds of one step and of its parts."""
        a, b, pool, T = self.a, self.b, self.pool, self._timed
        t0 = time.perf_counter()
        fa = pool.submit(T, a.insert, bt["ins_src"], bt["ins_dst"], bt["ins_w"])
        fb = pool.submit(lambda: (b.insert(bt["ins_src"], bt["ins_dst"], bt["ins_w"]),
                                  T(b.delete, bt["del_src"], bt["del_dst"]))[1])
        ins_s, del_s = fa.result(), fb.result()
        t1 = time.perf_counter()
        jobs = {"bfs1": (a.bfs, source), "sssp1": (a.sssp, source), "wcc1": (a.wcc,),
                "bfs2": (b.bfs, source), "sssp2": (b.sssp, source), "wcc2": (b.wcc,),
                "query": (b.query, bt["q_src"], bt["q_dst"])}
        futs = {k: pool.submit(T, *v) for k, v in jobs.items()}
        parts = {k: f.result() for k, f in futs.items()}
        t2 = time.perf_counter()
        a.delete(bt["del_src"], bt["del_dst"])
        t3 = time.perf_counter()
        parts.update({"insert": ins_s, "delete": del_s, "updates_wall": t1 - t0, "recompute_wall": t2 - t1,
                      "catch_up": t3 - t2})
        return t3 - t0, parts

    def close(self):
        self.pool.shutdown()


def oracle_summary(secs, parts, B):
    s = statistics.mean(secs)
    mean = lambda k: statistics.mean(p[k] for p in parts)  # noqa: E731
    return {"value": round(3 * B / s / 1e6, 4), "ms_per_step": round(s * 1e3, 1),
            "insert_medges_s": round(B / mean("insert") / 1e6, 3),
            "delete_medges_s": round(B / mean("delete") / 1e6, 3),
            "query_medges_s": round(B / mean("query") / 1e6, 3),
            "incr_sssp_ms": round(mean("sssp1") * 1e3, 1), "decr_sssp_ms": round(mean("sssp2") * 1e3, 1),
            "incr_bfs_ms": round(mean("bfs1") * 1e3, 1), "static_wcc_ms": round(mean("wcc2") * 1e3, 1)}


def cpu_baseline(G, batches, source, B, W, steps=2):
    """The oracle on `steps` steps of the workload (batches W, W + 1, ...
    after W untimed batches), as in the reference arm."""
    o = OracleStep(G)
    for k in range(W):
        o.advance(batches[k])
    res = [o.step(batches[W + k], source) for k in range(steps)]
    o.close()
    summ = oracle_summary([r[0] for r in res], [r[1] for r in res], B)
    cores = min(OracleStep.THREADS, os.cpu_count() or 1)
    return {"value": summ["value"], "unit": UNIT, "cores": cores, "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": ORACLE_SAMPLE + "; B = %d; %d steps (batches %d-%d); %.1f s per step"
                      % (B, steps, W, W + steps - 1, summ["ms_per_step"] / 1e3),
            "phases": summ}


def cpu_all_cores(G, batches, B, W, steps=3):
    """Batched insert, delete and query on all host cores (oracle/sharded:
    the edge set partitioned by source, one thread per shard) over the same
    batches W, W + 1, ... after W untimed batches."""
    from oracle.sharded import ShardedGraph

    p = ShardedGraph(G.V)
    p.insert(G.src, G.dst, G.w)
    for k in range(W):
        p.insert(batches[k]["ins_src"], batches[k]["ins_dst"], batches[k]["ins_w"])
        p.delete(batches[k]["del_src"], batches[k]["del_dst"])
    t = {"insert": 0.0, "delete": 0.0, "query": 0.0}
    for k in range(W, W + steps):
        bt = batches[k]
        for name, fn, a in (("insert", p.insert, (bt["ins_src"], bt["ins_dst"], bt["ins_w"])),
                            ("delete", p.delete, (bt["del_src"], bt["del_dst"])),
                            ("query", p.query, (bt["q_src"], bt["q_dst"]))):
            t0 = time.perf_counter()
            fn(*a)
            t[name] += time.perf_counter() - t0
    return {"kind": "edge set sharded by source, one thread per shard (oracle/sharded.cpp)",
            "cores": p.threads, "steps": steps, "batch": B,
            **{"%s_medges_s" % k: round(steps * B / v / 1e6, 2) for k, v in t.items()}}


def run_reference(args, world, rank, local):
    if rank != 0:
        return None
    W, K, B = args.warmup, args.steps, args.batch
    G, source, S = make_workload(args, B)
    batches = [S.batch(B) for _ in range(W + K)]
    o = OracleStep(G)
    for k in range(W):
        # warm-up steps only advance the graph: the oracle recomputes from
        # scratch and has no state a warm-up could prime
        o.advance(batches[k])
    res = [o.step(batches[W + k], source) for k in range(K)]
    o.close()
    summ = oracle_summary([r[0] for r in res], [r[1] for r in res], B)
    value = summ["value"]
    cores = min(OracleStep.THREADS, os.cpu_count() or 1)
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": summ["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic", "config": workload_config(args, G),
        **{k: v for k, v in summ.items() if k not in ("value", "ms_per_step")},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "host_cores": os.cpu_count(),
                         "kind": "oracle", "sample": ORACLE_SAMPLE + "; B = %d; batches %d-%d" % (B, W, W + K - 1)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_served(args):
    import torch

    import synth

    torch.cuda.set_device(0)
    t0 = time.time()
    G = synth.powerlaw_graph(scale=21, draws=1 << 25)
    ring = synth.new_edge_pool(G, 1 << 27)
    R = synth.request_stream(100000, G.V, len(G.src), len(ring.src))
    gen_s = time.time() - t0
    res = serve_experiment(G, R, ring)
    res.update({"workload": "R-MAT scale 21 graph (V=2,097,152, 2^25 draws, duplicates and self-loops dropped, "
                            "weights U[1,100]) under a Poisson stream of 100,000 requests: 60%% query, 15%% insert, "
                            "15%% delete, 10%% incremental SSSP from a pool of 16 sources; sizes log-uniform in "
                            "[1, 2^20]; inserts of new R-MAT edges, deletes of live edges (a live window over the "
                            "initial edges and a ring of %d new edges), half the queries inside the live window; "
                            "arrival rates 50%% and 90%% of the measured plain capacity" % len(ring.src),
                "gen_s": round(gen_s, 1)})
    return res


def road_pass(R, batches, delta_static, delta_incremental):
    """One pass of the road workload on a fresh graph: the static SSSP from
    vertex 0, then each mixed batch and the incremental SSSP after it."""
    import torch

    import paper_2305_17813_gb300 as mk

    g = mk.Graph(R.V, edge_capacity_hint=len(R.src) + sum(len(b["ins_src"]) for b in batches), buckets=1)
    g.set_sssp_delta(delta_static, delta_incremental)
    chunk = 1 << 22
    for i in range(0, len(R.src), chunk):
        g.insert(R.src[i:i + chunk], R.dst[i:i + chunk], R.w[i:i + chunk], flags=False)
    g.commit()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    torch.cuda.synchronize()
    ev[0].record()
    d0, p0 = g.sssp(0)
    ev[1].record()
    torch.cuda.synchronize()
    static_ms = ev[0].elapsed_time(ev[1])
    g.commit()
    dev = [{k: mk.to_device_u32(b[k]) for k in ("ins_src", "ins_dst", "ins_w", "del_src", "del_dst")} for b in batches]
    sssp_ms, del_ms, ins_ms = [], [], []
    for k in range(len(batches)):
        b = dev[k]
        ev[0].record()
        g.delete(b["del_src"], b["del_dst"], flags=False)
        ev[1].record()
        g.insert(b["ins_src"], b["ins_dst"], b["ins_w"], flags=False)
        ev[2].record()
        d, p = g.sssp(0)
        ev[3].record()
        g.commit()
        torch.cuda.synchronize()
        del_ms.append(ev[0].elapsed_time(ev[1]))
        ins_ms.append(ev[1].elapsed_time(ev[2]))
        sssp_ms.append(ev[2].elapsed_time(ev[3]))
    if g.last_error() != mk.MK_OK:
        raise RuntimeError("device status in the road run")
    result = (mk.to_numpy_u32(d0), mk.to_numpy_u32(p0), mk.to_numpy_u32(d), mk.to_numpy_u32(p))
    g.close()
    nd, ni = len(batches[0]["del_src"]), len(batches[0]["ins_src"])
    return {"static_sssp_ms": round(static_ms, 2),
            "incr_sssp_ms_mean": round(statistics.mean(sssp_ms), 3),
            "incr_sssp_ms_p50": round(statistics.median(sssp_ms), 3),
            "incr_sssp_ms_max": round(max(sssp_ms), 3),
            "delete_medges_s": round(nd / statistics.mean(del_ms) / 1e3, 1),
            "insert_medges_s": round(ni / statistics.mean(ins_ms) / 1e3, 1)}, result


def run_road(args):
    """Road-like workload: 4,096 x 4,096 grid + 0.1% long-range edges, 64
    mixed batches of 2^16 (half deletes of grid links, half inserts), the
    incremental SSSP from the corner vertex after each batch; run with the
    plain frontier rounds, with Near-Far ordered rounds (bucket width 4,000,
    about eight mean weights) for the static call only, and for every call,
    results compared."""
    import torch

    import synth

    torch.cuda.set_device(0)
    t0 = time.time()
    n, nb = args.road_size, args.road_batches
    R = synth.road_graph(n, n)
    batches = [synth.road_batch(R, k, args.road_batch_size) for k in range(nb)]
    gen_s = time.time() - t0
    desc = ("%d x %d road-like grid (%d grid edges + %d long-range edges, weights U[1,1000]); %d mixed batches "
            "of %d (half deletes of grid links, half inserts); incremental SSSP from vertex 0 after each batch"
            % (n, n, R.n_grid, len(R.src) - R.n_grid, nb, args.road_batch_size))
    if args.road_delta is not None:
        one, _ = road_pass(R, batches, args.road_delta, args.road_delta)
        return {"workload": desc, "near_far_width": args.road_delta, **one, "gen_s": round(gen_s, 1)}
    plain, r0 = road_pass(R, batches, 0, 0)
    nf_static, r1 = road_pass(R, batches, 4000, 0)
    nf, r2 = road_pass(R, batches, 4000, 4000)
    if not all(np.array_equal(x, y) and np.array_equal(x, z) for x, y, z in zip(r0, r1, r2)):
        raise RuntimeError("the Near-Far rounds disagree with the plain rounds")
    return {"workload": desc,
            **plain, "near_far_4000_static": nf_static, "near_far_4000_static_and_incremental": nf,
            "results_equal": True, "gen_s": round(gen_s, 1)}


def run_growth(args):
    import torch

    import synth

    torch.cuda.set_device(0)
    t0 = time.time()
    S = synth.growth_stream(scale=22, draws=1 << 26, n_batches=64)
    gen_s = time.time() - t0
    res = growth_experiment(S, split=32, horizon=8, epochs=20, repeats=5)
    res.update({"workload": "R-MAT scale 22 growth stream (67,108,864 draws; first 50% loaded; 64 insert batches "
                            "with preferential source skew 0.5, each followed by 10% deletes); network trained on "
                            "batches 1-32, graphs rebuilt at batch 32 with learned, load-factor (current degrees) and a "
                            "priori (initial degrees) bucket counts, 5 repeats each",
                "gen_s": round(gen_s, 1)})
    return res


def run_analytics(args):
    """PageRank on the power-law graph (static, then warm-started after one
    2^20 update batch) and triangle counting on an undirected R-MAT graph
    (static, then the inclusion-exclusion update after a batch of new
    undirected edges, against a static recount)."""
    import torch

    import paper_2305_17813_gb300 as mk
    import synth

    torch.cuda.set_device(0)
    out = {"workload": "analytics"}
    G = synth.powerlaw_graph(scale=args.scale, draws=args.draws)
    S = synth.PowerlawStream(G, max_batch=args.batch)
    g = mk.Graph(G.V, edge_capacity_hint=len(G.src) + 4 * args.batch, buckets=mk.bucket_rule(G.V, G.src, 0.7))
    g.insert(G.src, G.dst, G.w, flags=False)
    g.commit()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed_ms(fn):
        torch.cuda.synchronize()
        ev[0].record()
        r = fn()
        ev[1].record()
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]), r

    timed_ms(lambda: g.pagerank(eps=1e-7, max_iter=100))  # warm-up (module load, pools)
    st = g.stats()
    g.profile(True)
    g.profile_read()
    ms_static, (pr, it_static, delta) = timed_ms(lambda: g.pagerank(eps=1e-7, max_iter=100))
    prof = g.profile_read()
    g.profile(False)
    bt = S.batch(args.batch)
    g.insert(bt.ins_src, bt.ins_dst, bt.ins_w, flags=False)
    g.delete(bt.del_src, bt.del_dst, flags=False)
    g.commit()
    ms_warm, (_, it_warm, _) = timed_ms(lambda: g.pagerank(pr, eps=1e-7, max_iter=100))
    ms_cold, (_, it_cold, _) = timed_ms(lambda: g.pagerank(eps=1e-7, max_iter=100))
    n_step, t_step = prof.get("pr_step", (0, 0.0))
    slabs_in_use = int(st["chain_slabs"])
    E, V = int(st["live_edges"]), G.V
    # per super-step: every slab in use read once (128 B) with its owner
    # (4 B), one 8-byte contribution gather and one 8-byte atomic add per
    # edge, and the per-vertex passes (rank, degree, contribution and
    # accumulator reads and writes: 44 B per vertex)
    step_bytes = 132 * slabs_in_use + 16 * E + 44 * V
    peak, _ = measured_peak()
    gbs = step_bytes * n_step / (t_step / 1e3) / 1e9 if t_step else None
    out["pagerank"] = {
        "graph": "R-MAT scale %d, %d edges" % (args.scale, E), "damping": 0.85, "eps_l1": 1e-7,
        "static_ms": round(ms_static, 3), "static_iterations": it_static,
        "ms_per_iteration": round(t_step / max(n_step, 1), 4),
        "after_batch_warm_ms": round(ms_warm, 3), "after_batch_warm_iterations": it_warm,
        "after_batch_static_ms": round(ms_cold, 3), "after_batch_static_iterations": it_cold,
        "warm_speedup": round(ms_cold / ms_warm, 2),
        "step_algorithmic_bytes": int(step_bytes), "step_gbs": round(gbs, 1) if gbs else None,
        "step_frac": round(gbs / peak, 4) if gbs else None,
        "batch": "insert %d + delete %d (one power-law stream batch)" % (args.batch, args.batch)}
    g.close()

    # triangles: undirected R-MAT (both directions stored, no self-loops)
    tscale = max(10, args.scale - 2)
    T = synth.powerlaw_graph(scale=tscale, draws=1 << (tscale + 4))
    keep = T.src != T.dst
    us = np.concatenate([T.src[keep], T.dst[keep]]).astype(np.uint32)
    ud = np.concatenate([T.dst[keep], T.src[keep]]).astype(np.uint32)
    gt = mk.Graph(T.V, edge_capacity_hint=len(us) + (1 << 20), buckets=mk.bucket_rule(T.V, us, 0.7))
    gt.insert(us, ud, flags=False)
    gt.commit()
    gt.triangles()  # warm-up
    ms_tc, count = timed_ms(lambda: gt.triangles())
    bs, bd = synth.rmat_pairs(tscale, 1 << 16, synth.substream(4000, 1))
    k2 = bs != bd
    ns = np.concatenate([bs[k2], bd[k2]]).astype(np.uint32)
    nd = np.concatenate([bd[k2], bs[k2]]).astype(np.uint32)
    f = gt.insert(ns, nd).cpu().numpy().astype(bool)
    ns, nd = ns[f], nd[f]
    upd = mk.Graph(T.V, edge_capacity_hint=len(ns) + 64, buckets=1)
    upd.insert(ns, nd, flags=False)
    dns, dnd = mk.to_device_u32(ns), mk.to_device_u32(nd)
    ms_inc, delta_t = timed_ms(lambda: gt.triangle_delta(upd, dns, dnd, False))
    ms_re, count2 = timed_ms(lambda: gt.triangles())
    if count2 != count + delta_t:
        raise RuntimeError("triangle update disagrees with the recount")
    out["triangles"] = {
        "graph": "undirected R-MAT scale %d, %d directed edges" % (tscale, len(us)), "triangles": int(count),
        "static_ms": round(ms_tc, 3), "batch_new_undirected_edges": int(len(ns) // 2),
        "update_ms": round(ms_inc, 3), "new_triangles": int(delta_t), "recount_ms": round(ms_re, 3),
        "update_speedup_vs_recount": round(ms_re / ms_inc, 2)}
    upd.close()
    gt.close()
    return out


def run_buckets(args):
    """The power-law step with the load-factor bucket rule against one bucket
    per vertex (hashing off: every list is a vertex's whole adjacency), on
    the same stream of batches: per-operation rates, BFS/SSSP/WCC times and
    chain statistics (the paper's hashing and iteration-scheme trade-off)."""
    import torch

    torch.cuda.set_device(0)
    device = torch.device("cuda", 0)
    out = {"workload": "buckets"}
    peak, _ = measured_peak()
    for name, rule in (("load_factor_rule", True), ("single_bucket", False)):
        G, source, S = make_workload(args, args.batch)
        W, K = 3, max(3, args.steps)
        bts = [S.batch(args.batch) for _ in range(W + K)]
        R = StepRunner(args, G, source, len(G.src) + (W + K + 2) * args.batch, device,
                       buckets=None if rule else 1)
        st = R.g.stats()
        rec, outs, timed = R.run(bts, args.batch, W, flush_tag=0)
        check_steps(outs, timed, args.batch)
        fam = family_table(rec["prof"], rec["ctr"], args.batch, peak)
        out[name] = {**summarize(rec, args.batch, peak), "lists": int(st["lists"]),
                     "chain_mean": round(st["chain_mean"], 3), "chain_max": int(st["chain_max"]),
                     "device_bytes": int(st["device_bytes"]),
                     "top_kernels": {k: fam[k] for k in list(fam)[:6]}}
        R.close()
        del R
        torch.cuda.empty_cache()
    return out


def run_l2(args):
    """The power-law step (batch 2^20) with an L2 persistence window
    (mk_l2_window) over one part of the store on both of the step's streams.
    The graph changes as the stream of batches goes on, so every window run
    sits between two runs without a window on the next batches, and each is
    reported against the mean of its two neighbours."""
    import torch

    import paper_2305_17813_gb300 as mk

    torch.cuda.set_device(0)
    device = torch.device("cuda", 0)
    peak, _ = measured_peak()
    G, source, S = make_workload(args, args.batch)
    W, K = 2, max(3, args.steps)
    regions = [("vertex_index", mk.MK_L2_VINFO), ("head_slabs", mk.MK_L2_HEADS), ("pool_slabs", mk.MK_L2_POOL)]
    runs = [("none", mk.MK_L2_NONE)]
    for r in regions:
        runs += [r, ("none", mk.MK_L2_NONE)]
    R = StepRunner(args, G, source, len(G.src) + (len(runs) * (W + K) + 2) * args.batch, device)
    out = {"workload": "l2", "persisting_l2_max_bytes": None, "runs": []}
    for name, region in runs:
        info = {}
        for st in (R.stream, R.side):
            info = R.g.l2_window(region, stream=st)
        bts = [S.batch(args.batch) for _ in range(W + K)]
        rec, outs, timed = R.run(bts, args.batch, W, flush_tag=0)
        check_steps(outs, timed, args.batch)
        if region != mk.MK_L2_NONE:
            out["persisting_l2_max_bytes"] = info.get("max_bytes")
        out["runs"].append({"window": name, **summarize(rec, args.batch, peak),
                            "window_bytes": info.get("window_bytes"), "hit_ratio": info.get("hit_ratio")})
    for st in (R.stream, R.side):
        R.g.l2_window(mk.MK_L2_NONE, stream=st)
    R.close()
    for i, (name, _) in enumerate(runs):
        if name != "none":
            base = (out["runs"][i - 1]["ms_per_step"] + out["runs"][i + 1]["ms_per_step"]) / 2
            out[name] = {"ms_per_step": out["runs"][i]["ms_per_step"], "neighbours_ms_per_step": round(base, 3),
                         "step_time_ratio": round(out["runs"][i]["ms_per_step"] / base, 4),
                         "window_bytes": out["runs"][i]["window_bytes"], "hit_ratio": out["runs"][i]["hit_ratio"]}
    return out


def run_set(args):
    """The unweighted power-law graph in the two layouts of the paper's store:
    the ConcurrentMap slabs of the weighted store (15 pairs a slab) and the
    ConcurrentSet slabs (31 keys a slab), same bucket rule (load factor 0.7
    of the slab's capacity): slabs and device bytes, the load, one batch of
    inserts, deletes and queries, static BFS from three sources and static
    WCC, each timed alone after an L2 flush, results compared between the
    layouts."""
    import torch

    import paper_2305_17813_gb300 as mk

    torch.cuda.set_device(0)
    peak, _ = measured_peak()
    G, source, S = make_workload(args, args.batch)
    deg = np.bincount(G.src, minlength=G.V)
    sources = [int(x) for x in np.argsort(-deg, kind="stable")[:3]]
    bt = S.batch(args.batch)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed_ms(fn):
        flush.fill_(1)
        torch.cuda.synchronize()
        ev[0].record()
        r = fn()
        ev[1].record()
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]), r

    cap = len(G.src) + 4 * args.batch
    dev = {k: mk.to_device_u32(getattr(G, k)) for k in ("src", "dst", "w")}
    b = {k: mk.to_device_u32(getattr(bt, k)) for k in ("ins_src", "ins_dst", "ins_w", "del_src", "del_dst",
                                                        "q_src", "q_dst")}
    out = {"workload": "set", "graph": "R-MAT scale %d, %d edges (weights ignored by BFS/WCC)" % (args.scale,
                                                                                                 len(G.src)),
           "batch": "insert %d + delete %d + query %d (one power-law stream batch)" % ((args.batch,) * 3),
           "l2": "flushed before every timed call (512 MiB write)", "bfs_sources": sources}
    res = {}
    for name in ("map", "set"):
        for rep in range(2):  # the first pass loads modules and pools
            if name == "map":
                g = mk.Graph(G.V, edge_capacity_hint=cap, buckets=mk.bucket_rule(G.V, dev["src"], 0.7))
                load = lambda: g.insert(dev["src"], dev["dst"], dev["w"], flags=False)
            else:
                g = mk.SetGraph(G.V, edge_capacity_hint=cap, buckets=mk.set_bucket_rule(G.V, dev["src"], 0.7))
                load = lambda: g.insert(dev["src"], dev["dst"])
            ms_load, _ = timed_ms(load)
            if name == "map":
                g.commit()
            st = g.stats()
            slabs = int(st["chain_slabs"] if name == "map" else st["slabs_in_use"])
            bfs_ms, bfs_out = [], []
            for src in sources:  # a new source: the map store's first call for it is static
                t, r = timed_ms(lambda: g.bfs(src))
                bfs_ms.append(t)
                bfs_out.append(r)
            if name == "map":
                wcc_ms, lab = timed_ms(lambda: g.wcc())  # the graph's first WCC call: the static pass
            else:
                wcc_ms, lab = timed_ms(lambda: g.wcc())
            if name == "map":
                ins = lambda: g.insert(b["ins_src"], b["ins_dst"], b["ins_w"])
                dele = lambda: g.delete(b["del_src"], b["del_dst"])
                qry = lambda: g.query(b["q_src"], b["q_dst"], weights=False)
            else:
                ins = lambda: g.insert(b["ins_src"], b["ins_dst"])
                dele = lambda: g.delete(b["del_src"], b["del_dst"])
                qry = lambda: g.query(b["q_src"], b["q_dst"])
            ms_ins, fi = timed_ms(ins)
            ms_del, fd = timed_ms(dele)
            if name == "map":
                g.commit()
            ms_q, qr = timed_ms(qry)
            bm = qr[0] if isinstance(qr, tuple) else qr
            if g.last_error() != mk.MK_OK:
                raise RuntimeError("%s layout reported a device error" % name)
            if rep == 1:
                res[name] = {
                    "slabs_in_use": slabs, "lists": int(st["lists"]), "device_bytes": int(st["device_bytes"]),
                    "load_ms": round(ms_load, 3), "load_medges_s": round(len(G.src) / ms_load / 1e3, 1),
                    "static_bfs_ms": [round(t, 3) for t in bfs_ms], "static_wcc_ms": round(wcc_ms, 3),
                    "static_wcc_slab_gbs": round(slabs * 132 / (wcc_ms / 1e3) / 1e9, 1),
                    "insert_medges_s": round(args.batch / ms_ins / 1e3, 1),
                    "delete_medges_s": round(args.batch / ms_del / 1e3, 1),
                    "query_medges_s": round(args.batch / ms_q / 1e3, 1),
                    "_out": ([(mk.to_numpy_u32(d), mk.to_numpy_u32(p)) for d, p in bfs_out], mk.to_numpy_u32(lab),
                             fi.cpu().numpy(), fd.cpu().numpy(), mk.to_numpy_u32(bm))}
            g.close()
            del g
            torch.cuda.empty_cache()
    mo, so = res["map"].pop("_out"), res["set"].pop("_out")
    same = all(np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1]) for a, c in zip(mo[0], so[0]))
    same = same and all(np.array_equal(x, y) for x, y in zip(mo[1:], so[1:]))
    if not same:
        raise RuntimeError("the two layouts disagree")
    out.update(res)
    out["results_equal"] = True
    out["set_over_map"] = {
        "slabs": round(res["set"]["slabs_in_use"] / res["map"]["slabs_in_use"], 3),
        "static_wcc_time": round(res["set"]["static_wcc_ms"] / res["map"]["static_wcc_ms"], 3),
        "static_bfs_time": round(sum(res["set"]["static_bfs_ms"]) / sum(res["map"]["static_bfs_ms"]), 3),
        "query_rate": round(res["set"]["query_medges_s"] / res["map"]["query_medges_s"], 3)}
    out["peak_gbs"] = peak
    return out


def main(argv=None):
    args = parse_args(argv)
    world, rank, local = dist_env()
    if args.workload not in ("powerlaw",):
        if rank == 0:
            res = {"growth": run_growth, "served": run_served, "road": run_road, "analytics": run_analytics,
                   "buckets": run_buckets, "l2": run_l2, "set": run_set}[args.workload](args)
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
            result["cpu_baseline"] = cpu_baseline(G, batches, source, args.batch, args.warmup)
            result["cpu_all_cores_ops"] = cpu_all_cores(G, batches, args.batch, args.warmup)
        print(json.dumps(result), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
