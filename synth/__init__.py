"""Seeded synthetic workloads for the slab-hash dynamic graph store.

This package only draws inputs (edge lists, weights, batches, request
streams).  It contains none of the store's or the algorithms' arithmetic:
the CUDA path and the CPU oracle both receive the numpy arrays built here.
The random numbers come from the counter-based SplitMix64 generator in
``synth.c``; every recipe below states its seeds so a run can be replayed.

The paper evaluates on public graphs (Table 5 of the paper: LJournal, Orkut,
Wikipedia, Wiki-talk, BerkStan, Rand10M, USAfull) that are not available
here.  The recipes stand in for them with graphs of the same shape: R-MAT
for the power-law graphs, a 2D grid with 0.1% long-range edges for the road
network, and uniform random pairs for the random graph.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_f64p = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile ``synth.c`` into ``libsynth.so`` next to it (plain C99)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-Wall", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.syn_splitmix_at.restype = ctypes.c_uint64
            lib.syn_splitmix_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.syn_substream.restype = ctypes.c_uint64
            lib.syn_substream.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.syn_uniform_pairs.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, _u32p, _u32p]
            lib.syn_weights.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, _u32p]
            lib.syn_rmat_pairs.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_uint64, _u32p, _u32p]
            lib.syn_skew_sources.argtypes = [ctypes.c_uint64, ctypes.c_double, ctypes.c_uint64, _u32p,
                                             ctypes.c_uint64, _u32p]
            lib.syn_permutation.argtypes = [ctypes.c_uint64, ctypes.c_uint64, _u32p]
            lib.syn_grid_pairs.restype = ctypes.c_uint64
            lib.syn_grid_pairs.argtypes = [ctypes.c_uint32, ctypes.c_uint32, _u32p, _u32p]
            lib.syn_dedup_pairs.restype = ctypes.c_uint64
            lib.syn_dedup_pairs.argtypes = [_u32p, _u32p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int]
            lib.syn_exponential_gaps.argtypes = [ctypes.c_uint64, ctypes.c_double, ctypes.c_uint64, _f64p]
            lib.syn_log_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                            _u64p]
            lib.syn_set_create.restype = ctypes.c_void_p
            lib.syn_set_create.argtypes = [ctypes.c_uint64]
            lib.syn_set_destroy.argtypes = [ctypes.c_void_p]
            lib.syn_set_count.restype = ctypes.c_uint64
            lib.syn_set_count.argtypes = [ctypes.c_void_p]
            for name in ("syn_set_add", "syn_set_remove"):
                getattr(lib, name).restype = ctypes.c_uint64
                getattr(lib, name).argtypes = [ctypes.c_void_p, _u32p, _u32p, ctypes.c_uint64, _u8p]
            lib.syn_set_contains.argtypes = [ctypes.c_void_p, _u32p, _u32p, ctypes.c_uint64, _u8p]
            _lib = lib
    return _lib


def _p32(a: np.ndarray):
    assert a.dtype == np.uint32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_u32p)


# ---------------------------------------------------------------- primitives

def splitmix_at(seed: int, i: int) -> int:
    return int(_load().syn_splitmix_at(seed & (2**64 - 1), i))


def substream(seed: int, tag: int) -> int:
    return int(_load().syn_substream(seed & (2**64 - 1), tag & (2**64 - 1)))


def uniform_pairs(V: int, n: int, seed: int):
    s = np.empty(n, np.uint32)
    d = np.empty(n, np.uint32)
    if n:
        _load().syn_uniform_pairs(V, n, seed, _p32(s), _p32(d))
    return s, d


def weights(n: int, seed: int, lo: int, hi: int) -> np.ndarray:
    w = np.empty(n, np.uint32)
    if n:
        _load().syn_weights(n, seed, lo, hi, _p32(w))
    return w


def rmat_pairs(scale: int, n: int, seed: int, a=0.57, b=0.19, c=0.19):
    s = np.empty(n, np.uint32)
    d = np.empty(n, np.uint32)
    if n:
        _load().syn_rmat_pairs(scale, n, a, b, c, seed, _p32(s), _p32(d))
    return s, d


def skew_sources(src: np.ndarray, skew: float, seed: int, history: np.ndarray) -> np.ndarray:
    out = np.ascontiguousarray(src.copy())
    h = np.ascontiguousarray(history, dtype=np.uint32)
    if len(out) and len(h):
        _load().syn_skew_sources(len(out), skew, seed, _p32(h), len(h), _p32(out))
    return out


def permutation(n: int, seed: int) -> np.ndarray:
    p = np.empty(n, np.uint32)
    if n:
        _load().syn_permutation(n, seed, _p32(p))
    return p


def grid_pairs(rows: int, cols: int):
    m = 2 * (rows * (cols - 1) + cols * (rows - 1))
    s = np.empty(m, np.uint32)
    d = np.empty(m, np.uint32)
    k = _load().syn_grid_pairs(rows, cols, _p32(s), _p32(d))
    assert k == m
    return s, d


def vertex_bits(V: int) -> int:
    return max(1, int(V - 1).bit_length())


def dedup_pairs(src: np.ndarray, dst: np.ndarray, V: int, drop_self: bool):
    """Keep the first occurrence of each (src, dst); optionally drop loops."""
    s = np.ascontiguousarray(src, dtype=np.uint32).copy()
    d = np.ascontiguousarray(dst, dtype=np.uint32).copy()
    m = _load().syn_dedup_pairs(_p32(s), _p32(d), len(s), vertex_bits(V), int(drop_self))
    if m == 2**64 - 1:
        raise MemoryError("dedup_pairs: out of host memory")
    return s[:m].copy(), d[:m].copy()


def exponential_gaps(n: int, rate: float, seed: int) -> np.ndarray:
    g = np.empty(n, np.float64)
    if n:
        _load().syn_exponential_gaps(n, rate, seed, g.ctypes.data_as(_f64p))
    return g


def log_uniform(n: int, lo: int, hi: int, seed: int) -> np.ndarray:
    o = np.empty(n, np.uint64)
    if n:
        _load().syn_log_uniform(n, lo, hi, seed, o.ctypes.data_as(_u64p))
    return o


# ------------------------------------------------------------------ recipes
# Sub-stream tags: each recipe draws from substream(seed, TAG) so that the
# graph, its weights and each batch use non-overlapping streams.
TAG_PAIRS, TAG_W, TAG_PERM, TAG_QRY, TAG_QPERM, TAG_LONG, TAG_LOCAL, TAG_QPRES = 1, 2, 3, 4, 5, 6, 7, 8


class Batch(dict):
    """Plain dict of numpy arrays with attribute access."""

    __getattr__ = dict.__getitem__


def tiny_workload(V: int = 1024, E: int = 8192, n_ins: int = 1024, n_del: int = 1024,
                  n_qry: int = 4096, wlo: int = 1, whi: int = 100) -> Batch:
    """Plain-method tiny workload: uniform directed graph (seed 0), then an
    insert batch (seed 1), a delete batch sampled from the edges live after
    the inserts (seed 2) and a query batch, half live and half uniform
    (seed 3).  Duplicate pairs in the draw collapse by set semantics inside
    the store; self-loops are kept as ordinary edges."""
    gs, gd = uniform_pairs(V, E, substream(0, TAG_PAIRS))
    gw = weights(E, substream(0, TAG_W), wlo, whi)
    is_, id_ = uniform_pairs(V, n_ins, substream(1, TAG_PAIRS))
    iw = weights(n_ins, substream(1, TAG_W), wlo, whi)
    # live edge list after the load and the inserts (first occurrences)
    ls, ld = dedup_pairs(np.concatenate([gs, is_]), np.concatenate([gd, id_]), V, drop_self=False)
    perm = permutation(len(ls), substream(2, TAG_PERM))
    k = min(n_del, len(ls))
    ds, dd = ls[perm[:k]], ld[perm[:k]]
    # queries: half from edges still live after the deletes, half uniform
    half = n_qry // 2
    rest = perm[k:]
    take = rest[:half] if len(rest) >= half else np.resize(rest, half)
    us, ud = uniform_pairs(V, n_qry - half, substream(3, TAG_QRY))
    qs = np.concatenate([ls[take], us])
    qd = np.concatenate([ld[take], ud])
    qp = permutation(n_qry, substream(3, TAG_QPERM))
    return Batch(V=V, g_src=gs, g_dst=gd, g_w=gw, ins_src=is_, ins_dst=id_, ins_w=iw,
                 del_src=ds, del_dst=dd, q_src=qs[qp], q_dst=qd[qp])


def powerlaw_graph(scale: int = 20, draws: int = 1 << 24, seed: int = 0, wlo: int = 1, whi: int = 100,
                   a=0.57, b=0.19, c=0.19) -> Batch:
    """R-MAT graph with duplicates and self-loops dropped, weights U[wlo, whi]."""
    V = 1 << scale
    s, d = rmat_pairs(scale, draws, substream(seed, TAG_PAIRS), a, b, c)
    s, d = dedup_pairs(s, d, V, drop_self=True)
    w = weights(len(s), substream(seed, TAG_W), wlo, whi)
    return Batch(V=V, src=s, dst=d, w=w, scale=scale)


def _initial_perm(g: Batch) -> np.ndarray:
    p = g.get("_perm")
    if p is None:
        p = permutation(len(g.src), substream(0, TAG_PERM))
        g["_perm"] = p
    return p


class EdgeSet:
    """Set of live (src, dst) pairs kept by a batch stream (``syn_set_*`` in
    ``synth.c``).  It only decides which pairs a recipe draws."""

    def __init__(self, capacity: int):
        lib = _load()
        self._lib = lib
        self._h = lib.syn_set_create(int(capacity))
        if not self._h:
            raise MemoryError("EdgeSet: out of host memory")
        self.capacity = int(capacity)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.syn_set_destroy(h)
            self._h = None

    def __len__(self):
        return int(self._lib.syn_set_count(self._h))

    def add(self, src, dst) -> np.ndarray:
        s, d = np.ascontiguousarray(src, np.uint32), np.ascontiguousarray(dst, np.uint32)
        f = np.zeros(len(s), np.uint8)
        if len(s) and self._lib.syn_set_add(self._h, _p32(s), _p32(d), len(s), f.ctypes.data_as(_u8p)) == 2**64 - 1:
            raise OverflowError("EdgeSet: more than %d live pairs" % self.capacity)
        return f.astype(bool)

    def remove(self, src, dst) -> np.ndarray:
        s, d = np.ascontiguousarray(src, np.uint32), np.ascontiguousarray(dst, np.uint32)
        f = np.zeros(len(s), np.uint8)
        if len(s):
            self._lib.syn_set_remove(self._h, _p32(s), _p32(d), len(s), f.ctypes.data_as(_u8p))
        return f.astype(bool)

    def contains(self, src, dst) -> np.ndarray:
        s, d = np.ascontiguousarray(src, np.uint32), np.ascontiguousarray(dst, np.uint32)
        f = np.zeros(len(s), np.uint8)
        if len(s):
            self._lib.syn_set_contains(self._h, _p32(s), _p32(d), len(s), f.ctypes.data_as(_u8p))
        return f.astype(bool)


class PowerlawStream:
    """Batch stream of the power-law workload on a graph from
    `powerlaw_graph`.  Batch k (seed 100 + k, any size B) is drawn against
    the edges live when it runs, in the order the step applies it:

    * inserts: B R-MAT draws of the graph's scale, self-loops dropped
      (a draw of an edge that is already live is a no-op of the store);
    * deletes: B distinct edges live after those inserts, the oldest first:
      the initial edges in a fixed random order (seed 0), then the edges
      that earlier batches actually added, in batch order;
    * queries: exactly B // 2 edges live after the deletes (uniform over
      them, with replacement) and B - B // 2 uniform pairs that are not
      live (a live draw is rejected and drawn again), shuffled.

    So every delete removes an edge and exactly half the queries are
    present, at every batch size and for any number of batches.  The stream
    keeps the live pairs in an `EdgeSet` and the deletion order in a ring;
    batches must be drawn in order, k = 0, 1, 2, ...
    """

    def __init__(self, g: Batch, max_batch: int = 1 << 22, wlo: int = 1, whi: int = 100):
        self.g, self.wlo, self.whi = g, wlo, whi
        E = len(g.src)
        self.max_batch = int(max_batch)
        self.live = EdgeSet(E + self.max_batch)
        if int(self.live.add(g.src, g.dst).sum()) != E:
            raise ValueError("PowerlawStream: the graph has repeated pairs")
        cap = 1 << max(10, int(E + self.max_batch).bit_length())
        self._rs = np.empty(cap, np.uint32)
        self._rd = np.empty(cap, np.uint32)
        perm = _initial_perm(g)
        self._rs[:E] = g.src[perm]
        self._rd[:E] = g.dst[perm]
        self.head, self.n_live, self.k = 0, E, 0

    def _ring(self, first: int, count: int) -> np.ndarray:
        return (first + np.arange(count, dtype=np.int64)) & (len(self._rs) - 1)

    def _append(self, s: np.ndarray, d: np.ndarray):
        if self.n_live + len(s) > len(self._rs):
            raise OverflowError("PowerlawStream: ring full")
        at = self._ring(self.head + self.n_live, len(s))
        self._rs[at] = s
        self._rd[at] = d
        self.n_live += len(s)

    def batch(self, B: int) -> Batch:
        if B > self.max_batch:
            raise ValueError("PowerlawStream: batch %d above max_batch %d" % (B, self.max_batch))
        g, V = self.g, self.g.V
        k = self.k
        seed = 100 + k
        s, d = rmat_pairs(g.scale, B + B // 8 + 64, substream(seed, TAG_PAIRS))
        keep = s != d
        s, d = s[keep][:B], d[keep][:B]
        assert len(s) == B
        w = weights(B, substream(seed, TAG_W), self.wlo, self.whi)
        new = self.live.add(s, d)
        self._append(s[new], d[new])
        if self.n_live < B:
            raise ValueError("PowerlawStream: fewer than %d live edges" % B)
        at = self._ring(self.head, B)
        ds, dd = self._rs[at].copy(), self._rd[at].copy()
        if not self.live.remove(ds, dd).all():
            raise AssertionError("PowerlawStream: a delete is not live")
        self.head = (self.head + B) & (len(self._rs) - 1)
        self.n_live -= B
        half = B // 2
        pick = weights(half, substream(seed, TAG_QPRES), 0, self.n_live - 1).astype(np.int64)
        at = (self.head + pick) & (len(self._rs) - 1)
        ps, pd = self._rs[at], self._rd[at]
        us, ud = _absent_pairs(self.live, V, B - half, substream(seed, TAG_QRY))
        qp = permutation(B, substream(seed, TAG_QPERM))
        qs = np.concatenate([ps, us])[qp]
        qd = np.concatenate([pd, ud])[qp]
        self.k += 1
        return Batch(ins_src=s, ins_dst=d, ins_w=w, del_src=ds, del_dst=dd, q_src=qs, q_dst=qd,
                     k=k, n_inserted=int(new.sum()), n_present=half)


def _absent_pairs(live: EdgeSet, V: int, n: int, seed: int):
    """n uniform pairs over [0, V) that are not in `live` (rejection: a
    live draw is replaced by the next draw of the same stream)."""
    out_s, out_d, got, rnd = [], [], 0, 0
    while got < n:
        m = max(64, 2 * (n - got))
        s, d = uniform_pairs(V, m, substream(seed, rnd))
        ok = ~live.contains(s, d)
        s, d = s[ok][:n - got], d[ok][:n - got]
        out_s.append(s)
        out_d.append(d)
        got += len(s)
        rnd += 1
    if not out_s:
        return np.empty(0, np.uint32), np.empty(0, np.uint32)
    return np.concatenate(out_s), np.concatenate(out_d)


def road_graph(rows: int = 4096, cols: int = 4096, long_frac: float = 0.001, seed: int = 0,
               wlo: int = 1, whi: int = 1000) -> Batch:
    """4-neighbour bidirectional grid plus round(long_frac * grid edges)
    uniform long-range directed edges (self-loops dropped), weights U[wlo, whi]."""
    V = rows * cols
    gs, gd = grid_pairs(rows, cols)
    nl = int(round(long_frac * len(gs)))
    ls, ld = uniform_pairs(V, nl, substream(seed, TAG_LONG))
    keep = ls != ld
    s = np.concatenate([gs, ls[keep]])
    d = np.concatenate([gd, ld[keep]])
    w = weights(len(s), substream(seed, TAG_W), wlo, whi)
    return Batch(V=V, rows=rows, cols=cols, src=s, dst=d, w=w, n_grid=len(gs))


def road_batch(g: Batch, k: int, B: int = 1 << 16, wlo: int = 1, whi: int = 1000) -> Batch:
    """Mixed batch k (seed 1000 + k): B/2 inserts (half diagonal grid links,
    which the 4-neighbour grid lacks, half uniform long-range edges) and B/2
    deletes of grid links drawn without replacement from a fixed permutation
    of the grid edges."""
    rows, cols, V = g.rows, g.cols, g.V
    seed = 1000 + k
    ni = B // 2
    nloc = ni // 2
    r0 = np.empty(nloc, np.uint32)
    # diagonal neighbour of a uniform vertex that is not on the last row/col
    vs, dirs = uniform_pairs((rows - 1) * (cols - 1), nloc, substream(seed, TAG_LOCAL))
    rr = vs // (cols - 1)
    cc = vs % (cols - 1)
    v = (rr * cols + cc).astype(np.uint32)
    diag = (v + cols + 1).astype(np.uint32)
    flip = (dirs & 1).astype(bool)
    r0 = np.where(flip, diag, v).astype(np.uint32)
    r1 = np.where(flip, v, diag).astype(np.uint32)
    ls, ld = uniform_pairs(V, ni - nloc, substream(seed, TAG_LONG))
    keep = ls != ld
    s = np.concatenate([r0, ls[keep]])
    d = np.concatenate([r1, ld[keep]])
    w = weights(len(s), substream(seed, TAG_W), wlo, whi)
    perm = g.get("_gperm")
    if perm is None:
        perm = permutation(g.n_grid, substream(0, TAG_PERM))
        g["_gperm"] = perm
    nd = B - ni
    di = np.take(perm, (k * nd + np.arange(nd)) % g.n_grid)
    return Batch(ins_src=s, ins_dst=d, ins_w=w, del_src=g.src[di], del_dst=g.dst[di])


def growth_stream(scale: int = 22, draws: int = 1 << 26, n_batches: int = 64, del_frac: float = 0.1,
                  skew: float = 0.5, seed: int = 0, wlo: int = 1, whi: int = 100) -> Batch:
    """Learned-sizing workload: an R-MAT growth stream.  `draws` R-MAT pairs
    (seed `seed`), self-loops and duplicates dropped; the first half is the
    initial load and the rest arrives in `n_batches` insert batches.  Batch k
    (seed 2000 + k) is skewed towards vertices that already have edges: with
    probability `skew` an edge's source is replaced by the source of an
    edge drawn uniformly from everything loaded so far (preferential
    attachment).  Each insert batch is followed by a delete batch of
    del_frac x its size, drawn without replacement from the initial edges."""
    V = 1 << scale
    s, d = rmat_pairs(scale, draws, substream(seed, TAG_PAIRS))
    s, d = dedup_pairs(s, d, V, drop_self=True)
    E = len(s)
    half = E // 2
    w = weights(E, substream(seed, TAG_W), wlo, whi)
    init = Batch(src=s[:half].copy(), dst=d[:half].copy(), w=w[:half].copy())
    rest = np.arange(half, E)
    chunks = np.array_split(rest, n_batches)
    perm = permutation(half, substream(seed, TAG_PERM))
    history = s[:half].copy()
    batches = []
    used = 0
    for k, idx in enumerate(chunks):
        bs = skew_sources(s[idx], skew, substream(2000 + k, TAG_PAIRS), history)
        bd = d[idx]
        keep = bs != bd
        bs, bd, bw = bs[keep], bd[keep], w[idx][keep]
        history = np.concatenate([history, bs])
        nd = int(round(del_frac * len(bs)))
        di = perm[used:used + nd]
        used += nd
        batches.append(Batch(ins_src=bs, ins_dst=bd, ins_w=bw, del_src=s[di].copy(), del_dst=d[di].copy()))
    return Batch(V=V, scale=scale, init=init, batches=batches)


def request_stream(n_req: int, V: int, n_edges: int, mix=(0.6, 0.15, 0.15, 0.1), lo: int = 1, hi: int = 1 << 20,
                   n_sources: int = 16, query_pool: int = 1 << 21, insert_pool: int = 1 << 22,
                   seed: int = 3000) -> Batch:
    """Mixed request stream for the serving workload (seed `seed`).

    kinds: 0 query, 1 insert, 2 delete, 3 incremental SSSP with probabilities
    `mix`; sizes log-uniform in [lo, hi] (update and query requests);
    SSSP sources drawn from a fixed pool of n_sources random vertices (so a
    source recurs and its tree is kept incrementally); `gaps`: unit-rate
    exponential inter-arrival times (scale by 1 / rate).  Request inputs are
    slices of pools: queries at a random offset of a query pool, inserts at
    a random offset of an insert pool, deletes at consecutive offsets of a
    fixed permutation of the initial edges (so they hit live edges until it
    wraps around)."""
    u = np.frombuffer(np.ascontiguousarray(weights(n_req, substream(seed, TAG_PAIRS), 0, 999999)).tobytes(),
                      np.uint32).astype(np.float64) / 1e6
    cum = np.cumsum(mix)
    kind = np.searchsorted(cum, u, side="right").astype(np.uint8)
    kind = np.minimum(kind, 3)
    size = log_uniform(n_req, lo, hi, substream(seed, TAG_W)).astype(np.int64)
    srcs = uniform_pairs(V, n_sources, substream(seed, TAG_LONG))[0]
    pick = weights(n_req, substream(seed, TAG_LOCAL), 0, n_sources - 1)
    source = srcs[pick]
    off_raw = uniform_pairs(0xFFFFFFFF, n_req, substream(seed, TAG_QRY))[0].astype(np.int64)
    offset = np.zeros(n_req, np.int64)
    q = kind == 0
    offset[q] = off_raw[q] % np.maximum(query_pool - size[q], 1)
    ins = kind == 1
    offset[ins] = off_raw[ins] % np.maximum(insert_pool - size[ins], 1)
    dl = kind == 2
    offset[dl] = (np.cumsum(np.where(dl, size, 0)) - size)[dl] % max(1, n_edges)
    size[kind == 3] = 0
    gaps = exponential_gaps(n_req, 1.0, substream(seed, TAG_QPERM))
    return Batch(kind=kind, size=size, source=source, offset=offset, gaps=gaps, sources=srcs)
