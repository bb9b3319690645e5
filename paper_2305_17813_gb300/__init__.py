"""GB300 slab-hash dynamic graph store (Python binding).

A thin layer over the C ABI of ``include/meerkat.h``: it only turns tensors
into device pointers and CUDA streams into handles.  Every step runs in the
CUDA kernels of ``libmeerkat.so``; if that library is missing the import of
``Graph`` still works but any call raises.

Device arrays are torch CUDA tensors; 32-bit ids and weights travel as
``torch.int32`` tensors holding the unsigned bit patterns (numpy ``uint32``
arrays are accepted and copied to the device).
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._native import (MK_ERR_CUDA, MK_ERR_INTERNAL, MK_ERR_INVALID_ARG, MK_ERR_NO_MEMORY, MK_ERR_POOL_EXHAUSTED,
                      MK_ERR_TIMEOUT, MK_INVALID_LANE, MK_L2_HEADS, MK_L2_NONE, MK_L2_POOL, MK_L2_VINFO, MK_NONE, MK_OK,
                      MkError, check, load, mk_config, mk_kernel_time, mk_stats)

__all__ = [
    "Graph", "load", "MkError", "MK_OK", "MK_ERR_INVALID_ARG", "MK_ERR_POOL_EXHAUSTED", "MK_ERR_TIMEOUT",
    "MK_ERR_CUDA", "MK_ERR_NO_MEMORY", "MK_ERR_INTERNAL", "MK_NONE", "MK_INVALID_LANE", "bucket_rule",
    "to_device_u32", "to_numpy_u32", "Batcher", "Server", "SetGraph", "set_bucket_rule", "MK_L2_NONE", "MK_L2_VINFO", "MK_L2_HEADS", "MK_L2_POOL",
]


def _torch():
    import torch

    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def to_device_u32(x, device="cuda"):
    """A contiguous int32 CUDA tensor holding the uint32 values of x."""
    torch = _torch()
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        if x.dtype in (torch.int32, torch.uint32):
            t = x.to(device=device).contiguous()
            return t.view(torch.int32) if t.dtype == torch.uint32 else t
        x = x.cpu().numpy()
    a = np.ascontiguousarray(np.asarray(x))
    if a.dtype != np.uint32:
        if a.size and (a.min() < 0 or a.max() > 0xFFFFFFFF):
            raise ValueError("values do not fit in uint32")
        a = a.astype(np.uint32)
    return torch.from_numpy(a.view(np.int32)).to(device)


def to_numpy_u32(t) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint32)


def bucket_rule(V: int, src, load_factor: float = 0.7, stream=None):
    """Per-vertex bucket counts max(1, ceil(outdeg / (load_factor * 15)))."""
    torch = _torch()
    lib = load()
    s = to_device_u32(src)
    out = torch.empty(V, dtype=torch.int32, device=s.device)
    check(lib.mk_bucket_rule(V, _ptr(s), s.numel(), load_factor, _ptr(out), _stream(stream)), "mk_bucket_rule")
    return out


class Graph:
    """One dynamic graph on the current CUDA device.

    ``buckets`` is either an int (same bucket count for every vertex) or a
    device tensor of V per-vertex counts (see ``bucket_rule``).
    """

    def __init__(self, V: int, edge_capacity_hint: int = 0, buckets=1, pool_slabs: int = 0, stream=None):
        torch = _torch()
        self._lib = load()
        self.V = int(V)
        cfg = mk_config()
        cfg.V = self.V
        cfg.edge_capacity_hint = int(edge_capacity_hint)
        self._bucket_tensor = None
        if isinstance(buckets, int):
            cfg.buckets = buckets
        else:
            self._bucket_tensor = to_device_u32(buckets)
            cfg.d_bucket_per_vertex = self._bucket_tensor.data_ptr()
        cfg.pool_slabs = int(pool_slabs)
        h = ctypes.c_void_p()
        check(self._lib.mk_graph_create_ex(ctypes.byref(cfg), _stream(stream), ctypes.byref(h)), "mk_graph_create")
        self._h = h
        self.device = torch.device("cuda", torch.cuda.current_device())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mk_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # ---------------------------------------------------------- updates
    def insert(self, src, dst, w=None, flags: bool = True, stream=None):
        torch = _torch()
        s, d, ww = to_device_u32(src), to_device_u32(dst), to_device_u32(w)
        n = s.numel()
        f = torch.empty(n, dtype=torch.uint8, device=self.device) if flags else None
        check(self._lib.mk_insert_batch(self._h, _ptr(s), _ptr(d), _ptr(ww), n, _ptr(f), _stream(stream)),
              "mk_insert_batch")
        return f

    def delete(self, src, dst, flags: bool = True, stream=None):
        torch = _torch()
        s, d = to_device_u32(src), to_device_u32(dst)
        n = s.numel()
        f = torch.empty(n, dtype=torch.uint8, device=self.device) if flags else None
        check(self._lib.mk_delete_batch(self._h, _ptr(s), _ptr(d), n, _ptr(f), _stream(stream)), "mk_delete_batch")
        return f

    def query(self, src, dst, weights: bool = True, stream=None):
        torch = _torch()
        s, d = to_device_u32(src), to_device_u32(dst)
        n = s.numel()
        bm = torch.empty((n + 31) // 32, dtype=torch.int32, device=self.device)
        w = torch.empty(n, dtype=torch.int32, device=self.device) if weights else None
        check(self._lib.mk_query_batch(self._h, _ptr(s), _ptr(d), n, _ptr(bm), _ptr(w), _stream(stream)),
              "mk_query_batch")
        return bm, w

    def commit(self, stream=None):
        check(self._lib.mk_commit_batch(self._h, _stream(stream)), "mk_commit_batch")

    # ------------------------------------------------------- algorithms
    def sssp(self, source: int, stream=None):
        torch = _torch()
        dist = torch.empty(self.V, dtype=torch.int32, device=self.device)
        par = torch.empty(self.V, dtype=torch.int32, device=self.device)
        check(self._lib.mk_incr_sssp(self._h, int(source), _ptr(dist), _ptr(par), _stream(stream)), "mk_incr_sssp")
        return dist, par

    def set_sssp_delta(self, delta_static: int, delta_incremental: int = 0):
        """Near-Far bucket widths of the SSSP rounds for static and for
        incremental calls (0 = the plain rounds)."""
        check(self._lib.mk_set_sssp_delta(self._h, int(delta_static), int(delta_incremental)), "mk_set_sssp_delta")

    def bfs(self, source: int, stream=None):
        torch = _torch()
        dist = torch.empty(self.V, dtype=torch.int32, device=self.device)
        par = torch.empty(self.V, dtype=torch.int32, device=self.device)
        check(self._lib.mk_incr_bfs(self._h, int(source), _ptr(dist), _ptr(par), _stream(stream)), "mk_incr_bfs")
        return dist, par

    def incr_multi(self, requests, stream=None):
        """Advance several BFS/SSSP states in one mk_incr_multi call.
        requests: list of ("sssp" | "bfs", source); returns one (dist,
        parent) pair of tensors per request."""
        torch = _torch()
        from ._native import MK_REQ_BFS, MK_REQ_SSSP, mk_algo_req

        arr = (mk_algo_req * max(1, len(requests)))()
        outs = []
        for i, (kind, source) in enumerate(requests):
            dist = torch.empty(self.V, dtype=torch.int32, device=self.device)
            par = torch.empty(self.V, dtype=torch.int32, device=self.device)
            arr[i].kind = {"sssp": MK_REQ_SSSP, "bfs": MK_REQ_BFS}[kind]
            arr[i].source = int(source)
            arr[i].d_dist, arr[i].d_parent = dist.data_ptr(), par.data_ptr()
            outs.append((dist, par))
        check(self._lib.mk_incr_multi(self._h, arr, len(requests), _stream(stream)), "mk_incr_multi")
        return outs

    def wcc(self, stream=None):
        torch = _torch()
        lab = torch.empty(self.V, dtype=torch.int32, device=self.device)
        check(self._lib.mk_incr_wcc(self._h, _ptr(lab), _stream(stream)), "mk_incr_wcc")
        return lab

    def pagerank(self, pr=None, damping: float = 0.85, eps: float = 1e-7, max_iter: int = 100, stream=None):
        """PageRank (mk_pagerank).  pr: None for the static start (1 / V),
        or a float32 CUDA tensor of V ranks to start from (updated in place).
        Returns (ranks, super-steps, last L1 delta)."""
        torch = _torch()
        warm = pr is not None
        if pr is None:
            pr = torch.empty(self.V, dtype=torch.float32, device=self.device)
        it, delta = ctypes.c_uint32(), ctypes.c_float()
        check(self._lib.mk_pagerank(self._h, _ptr(pr), 1 if warm else 0, damping, eps, max_iter, ctypes.byref(it),
                                    ctypes.byref(delta), _stream(stream)), "mk_pagerank")
        return pr, it.value, delta.value

    def l2_window(self, region: int, stream=None) -> dict:
        """Set (or with MK_L2_NONE remove) an L2 persistence window over one
        part of the graph on `stream` (mk_l2_window)."""
        from ._native import mk_l2_info

        info = mk_l2_info()
        check(self._lib.mk_l2_window(self._h, int(region), _stream(stream), ctypes.byref(info)), "mk_l2_window")
        return {"window_bytes": info.window_bytes, "max_bytes": info.max_bytes, "hit_ratio": info.hit_ratio}

    def triangles(self, stream=None) -> int:
        """Triangles of the undirected graph stored with both directions."""
        v = ctypes.c_uint64()
        check(self._lib.mk_tc_static(self._h, ctypes.byref(v), _stream(stream)), "mk_tc_static")
        return v.value

    def triangle_delta(self, upd: "Graph", src, dst, deletion: bool, stream=None) -> int:
        """Change in the triangle count for a batch whose edges (both
        directions, all actually applied) are (src, dst) and are exactly the
        edges of `upd`; self is the graph after the batch (mk_tc_update)."""
        s, d = to_device_u32(src), to_device_u32(dst)
        out = ctypes.c_int64()
        check(self._lib.mk_tc_update(self._h, upd.handle, _ptr(s), _ptr(d), s.numel(), 1 if deletion else 0,
                                     ctypes.byref(out), _stream(stream)), "mk_tc_update")
        return out.value

    # ------------------------------------------------------- inspection
    def export(self, stream=None):
        """Live edges sorted by (src, dst) as three int32 tensors (uint32 bits)."""
        torch = _torch()
        st = self.stats(stream)
        m = int(st["live_edges"])
        s = torch.empty(max(m, 1), dtype=torch.int32, device=self.device)
        d = torch.empty_like(s)
        w = torch.empty_like(s)
        cnt = torch.zeros(1, dtype=torch.int64, device=self.device)
        check(self._lib.mk_graph_export(self._h, m, _ptr(s), _ptr(d), _ptr(w), _ptr(cnt), _stream(stream)),
              "mk_graph_export")
        return s[:m], d[:m], w[:m]

    def stats(self, stream=None) -> dict:
        st = mk_stats()
        check(self._lib.mk_graph_stats(self._h, ctypes.byref(st), _stream(stream)), "mk_graph_stats")
        return {f: getattr(st, f) for f, _ in mk_stats._fields_}

    def pool_free(self, stream=None) -> int:
        v = ctypes.c_uint64()
        check(self._lib.mk_pool_free(self._h, ctypes.byref(v), _stream(stream)), "mk_pool_free")
        return v.value

    def last_error(self) -> int:
        return int(self._lib.mk_last_error(self._h))

    def marker(self, v: int, bucket: int = 0, stream=None):
        a, b, c = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        check(self._lib.mk_list_marker(self._h, v, bucket, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                       _stream(stream)), "mk_list_marker")
        return a.value, b.value, c.value

    def counters(self, reset: bool = False, stream=None) -> dict:
        from ._native import COUNTER_NAMES

        buf = (ctypes.c_uint64 * 32)()
        check(self._lib.mk_counters(self._h, buf, 32, 1 if reset else 0, _stream(stream)), "mk_counters")
        return {name: int(buf[i]) for i, name in enumerate(COUNTER_NAMES)}

    # ----------------------------------------------- batching and tuning
    def query_multi(self, requests, weights: bool = True, stream=None):
        """Answer a list of (src, dst) requests in one launch; returns a list
        of (bitmap, weights) like query()."""
        torch = _torch()
        from ._native import mk_query_req

        keep, outs = [], []
        arr = (mk_query_req * max(1, len(requests)))()
        for i, (src, dst) in enumerate(requests):
            s, d = to_device_u32(src), to_device_u32(dst)
            n = s.numel()
            bm = torch.empty(max(1, (n + 31) // 32), dtype=torch.int32, device=self.device)
            w = torch.empty(max(1, n), dtype=torch.int32, device=self.device) if weights else None
            arr[i].d_src, arr[i].d_dst, arr[i].n = s.data_ptr(), d.data_ptr(), n
            arr[i].d_bitmap = bm.data_ptr()
            arr[i].d_w = w.data_ptr() if w is not None else None
            keep.append((s, d))
            outs.append((bm[:(n + 31) // 32], None if w is None else w[:n]))
        check(self._lib.mk_query_multi(self._h, arr, len(requests), _stream(stream)), "mk_query_multi")
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        del keep
        return outs

    def update_multi(self, requests, flags: bool = True, stream=None):
        """Apply a list of update requests in order with one mk_update_multi
        call.  Each request is ("insert", src, dst, w) or ("delete", src,
        dst); returns one flag tensor per request (None when flags=False)."""
        torch = _torch()
        from ._native import MK_REQ_DELETE, MK_REQ_INSERT, mk_update_req

        keep, outs = [], []
        arr = (mk_update_req * max(1, len(requests)))()
        for i, req in enumerate(requests):
            kind = {"insert": MK_REQ_INSERT, "delete": MK_REQ_DELETE}[req[0]]
            s, d = to_device_u32(req[1]), to_device_u32(req[2])
            w = to_device_u32(req[3]) if kind == MK_REQ_INSERT and len(req) > 3 else None
            n = s.numel()
            f = torch.empty(max(n, 1), dtype=torch.uint8, device=self.device) if flags else None
            arr[i].kind, arr[i].n = kind, n
            arr[i].d_src, arr[i].d_dst = s.data_ptr(), d.data_ptr()
            arr[i].d_w = None if w is None else w.data_ptr()
            arr[i].d_flags = None if f is None else f.data_ptr()
            keep.append((s, d, w))
            outs.append(None if f is None else f[:n])
        check(self._lib.mk_update_multi(self._h, arr, len(requests), _stream(stream)), "mk_update_multi")
        (torch.cuda.current_stream() if stream is None else stream).synchronize()
        del keep
        return outs

    def autotune(self, src, dst, bfs_source: int, stream=None) -> dict:
        from ._native import mk_tuning

        s, d = to_device_u32(src), to_device_u32(dst)
        t = mk_tuning()
        check(self._lib.mk_autotune(self._h, _ptr(s), _ptr(d), s.numel(), int(bfs_source), _stream(stream),
                                    ctypes.byref(t)), "mk_autotune")
        return {"query_group": t.query_group, "query_block": t.query_block,
                "rounds_blocks_per_sm": t.rounds_blocks_per_sm, "query_best_ms": t.query_best_ms,
                "rounds_best_ms": t.rounds_best_ms, "query_ms": list(t.query_ms)[:12],
                "rounds_ms": [x for x in t.rounds_ms if x > 0]}

    def tuning(self) -> dict:
        from ._native import mk_tuning

        t = mk_tuning()
        check(self._lib.mk_get_tuning(self._h, ctypes.byref(t)), "mk_get_tuning")
        return {"query_group": t.query_group, "query_block": t.query_block,
                "rounds_blocks_per_sm": t.rounds_blocks_per_sm}

    def set_tuning(self, query_group=8, query_block=256, rounds_blocks_per_sm=0):
        from ._native import mk_tuning

        t = mk_tuning()
        t.query_group, t.query_block, t.rounds_blocks_per_sm = query_group, query_block, rounds_blocks_per_sm
        check(self._lib.mk_set_tuning(self._h, ctypes.byref(t)), "mk_set_tuning")

    def profile(self, on: bool = True):
        check(self._lib.mk_profile_enable(self._h, 1 if on else 0), "mk_profile_enable")

    def profile_read(self) -> dict:
        buf = (mk_kernel_time * 64)()
        n = ctypes.c_int()
        check(self._lib.mk_profile_read(self._h, buf, 64, ctypes.byref(n)), "mk_profile_read")
        return {buf[i].name.decode(): (buf[i].launches, buf[i].total_ms) for i in range(n.value)}

    def launch_count(self) -> int:
        return int(self._lib.mk_launch_count(self._h))


def set_bucket_rule(V: int, src, load_factor: float = 0.7, stream=None):
    """Per-vertex bucket counts of the set layout, max(1, ceil(outdeg / (lf * 31)))."""
    torch = _torch()
    lib = load()
    s = to_device_u32(src)
    out = torch.empty(V, dtype=torch.int32, device=s.device)
    check(lib.mk_set_bucket_rule(V, _ptr(s), s.numel(), load_factor, _ptr(out), _stream(stream)),
          "mk_set_bucket_rule")
    return out


class SetGraph:
    """An unweighted graph in the ConcurrentSet layout (mk_set_*)."""

    def __init__(self, V: int, edge_capacity_hint: int = 0, buckets=1, stream=None):
        torch = _torch()
        self._lib = load()
        self.V = int(V)
        b = None if isinstance(buckets, int) else to_device_u32(buckets)
        h = ctypes.c_void_p()
        check(self._lib.mk_set_create(self.V, int(edge_capacity_hint), buckets if b is None else 0, _ptr(b),
                                      _stream(stream), ctypes.byref(h)), "mk_set_create")
        self._h = h
        self.device = torch.device("cuda", torch.cuda.current_device())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mk_set_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def _flags(self, fn, name, src, dst, stream):
        torch = _torch()
        s, d = to_device_u32(src), to_device_u32(dst)
        f = torch.empty(s.numel(), dtype=torch.uint8, device=self.device)
        check(fn(self._h, _ptr(s), _ptr(d), s.numel(), _ptr(f), _stream(stream)), name)
        return f

    def insert(self, src, dst, stream=None):
        return self._flags(self._lib.mk_set_insert_batch, "mk_set_insert_batch", src, dst, stream)

    def delete(self, src, dst, stream=None):
        return self._flags(self._lib.mk_set_delete_batch, "mk_set_delete_batch", src, dst, stream)

    def query(self, src, dst, stream=None):
        torch = _torch()
        s, d = to_device_u32(src), to_device_u32(dst)
        bm = torch.empty((s.numel() + 31) // 32, dtype=torch.int32, device=self.device)
        check(self._lib.mk_set_query_batch(self._h, _ptr(s), _ptr(d), s.numel(), _ptr(bm), _stream(stream)),
              "mk_set_query_batch")
        return bm

    def bfs(self, source: int, stream=None):
        torch = _torch()
        dist = torch.empty(self.V, dtype=torch.int32, device=self.device)
        par = torch.empty(self.V, dtype=torch.int32, device=self.device)
        check(self._lib.mk_set_bfs(self._h, int(source), _ptr(dist), _ptr(par), _stream(stream)), "mk_set_bfs")
        return dist, par

    def wcc(self, stream=None):
        torch = _torch()
        lab = torch.empty(self.V, dtype=torch.int32, device=self.device)
        check(self._lib.mk_set_wcc(self._h, _ptr(lab), _stream(stream)), "mk_set_wcc")
        return lab

    def stats(self, stream=None) -> dict:
        a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        check(self._lib.mk_set_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), _stream(stream)),
              "mk_set_stats")
        return {"lists": a.value, "slabs_in_use": b.value, "device_bytes": c.value}

    def last_error(self) -> int:
        return int(self._lib.mk_set_last_error(self._h))


class Batcher:
    """CUDA-graph batcher of query requests (mk_batcher_*)."""

    def __init__(self, graph: "Graph", max_requests: int = 1024):
        self._lib = graph._lib
        self.graph = graph
        h = ctypes.c_void_p()
        check(self._lib.mk_batcher_create(graph.handle, max_requests, ctypes.byref(h)), "mk_batcher_create")
        self._h = h

    def add_query(self, src, dst, bitmap, w=None):
        """src/dst/bitmap/w: device int32 tensors owned by the caller and kept
        alive until the launch has completed."""
        check(self._lib.mk_batcher_add_query(self._h, _ptr(src), _ptr(dst), src.numel(), _ptr(bitmap), _ptr(w)),
              "mk_batcher_add_query")

    def launch(self, stream=None):
        check(self._lib.mk_batcher_launch(self._h, _stream(stream)), "mk_batcher_launch")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mk_batcher_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching serving engine (mk_server_*).  Buffers passed to
    submit() must stay alive until their request is reported done."""

    QUERY, INSERT, DELETE, SSSP, BFS = 0, 1, 2, 3, 4

    def __init__(self, graph: "Graph", max_inflight: int = 64, commit_every: int = 8):
        self._lib = graph._lib
        h = ctypes.c_void_p()
        check(self._lib.mk_server_create(graph.handle, max_inflight, commit_every, ctypes.byref(h)),
              "mk_server_create")
        self._h = h
        self._cap = 4096
        self._tags = (ctypes.c_uint64 * self._cap)()
        self._st = (ctypes.c_int * self._cap)()

    def submit(self, kind, src=None, dst=None, w=None, n=0, source=0, out0=None, out1=None, tag=0):
        from ._native import mk_request

        r = mk_request()
        r.kind, r.n, r.source, r.tag = int(kind), int(n), int(source), int(tag)
        r.d_src = None if src is None else src.data_ptr()
        r.d_dst = None if dst is None else dst.data_ptr()
        r.d_w = None if w is None else w.data_ptr()
        r.d_out0 = None if out0 is None else out0.data_ptr()
        r.d_out1 = None if out1 is None else out1.data_ptr()
        check(self._lib.mk_server_submit(self._h, ctypes.byref(r)), "mk_server_submit")

    def progress(self):
        """[(tag, status)] of the requests completed since the last call."""
        n = ctypes.c_uint32()
        check(self._lib.mk_server_progress(self._h, self._tags, self._st, self._cap, ctypes.byref(n)),
              "mk_server_progress")
        return [(self._tags[i], self._st[i]) for i in range(n.value)]

    def pending(self):
        q, f = ctypes.c_uint64(), ctypes.c_uint64()
        check(self._lib.mk_server_pending(self._h, ctypes.byref(q), ctypes.byref(f)), "mk_server_pending")
        return q.value, f.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mk_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
