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


def new_edge_pool(g: Batch, draws: int, seed: int = 3100, wlo: int = 1, whi: int = 100) -> Batch:
    """Distinct R-MAT edges of g's scale that are not edges of g, self-loops
    dropped, in draw order (seed `seed`), with weights U[wlo, whi]."""
    s, d = rmat_pairs(g.scale, draws, substream(seed, TAG_PAIRS))
    s, d = dedup_pairs(s, d, g.V, drop_self=True)
    live = EdgeSet(len(g.src))
    live.add(g.src, g.dst)
    keep = ~live.contains(s, d)
    s, d = s[keep].copy(), d[keep].copy()
    return Batch(src=s, dst=d, w=weights(len(s), substream(seed, TAG_W), wlo, whi))


def request_stream(n_req: int, V: int, E0: int, ring: int, mix=(0.6, 0.15, 0.15, 0.1), lo: int = 1,
                   hi: int = 1 << 20, n_sources: int = 16, absent_pool: int = 1 << 21, seed: int = 3000) -> Batch:
    """Mixed request stream for the serving workload (seed `seed`).

    kinds: 0 query, 1 insert, 2 delete, 3 incremental SSSP with probabilities
    `mix`; sizes log-uniform in [lo, hi] (update and query requests); SSSP
    sources drawn from a fixed pool of n_sources random vertices (so a
    source recurs and its tree is kept incrementally); `gaps`: unit-rate
    exponential inter-arrival times (scale by 1 / rate).

    Update requests and the present queries read slices of one sequence of
    edges: the E0 initial edges in a fixed random order, then a ring of
    `ring` distinct new edges (`new_edge_pool`), stored followed by a copy of
    its first `hi` edges so that every slice of at most `hi` edges starting
    in the ring is contiguous (`seq_index` maps a position of the unrolled
    sequence to the stored one).  In arrival order an insert cursor i
    (starting at E0) and a delete cursor d (starting at 0) walk the unrolled
    sequence, and the live edges are exactly its positions [d, i):

    * an insert takes [i, i + n) and i advances by n: new edges, unless the
      window [d, i) outgrew the ring (`applied` counts the new ones);
    * a delete takes [d, d + n): its first min(n, i - d) edges are live, the
      rest not yet inserted (no-ops); d advances to min(d + n, i);
    * a query takes, with probability 1/2, a slice inside [d, i) (every
      edge present), and otherwise a slice of a pool of `absent_pool`
      uniform pairs (absent but for chance hits); `qsrc` = 0 / 1.

    `offset` is the stored position (sequence or absent pool) of each
    request's slice; `applied` the expected count of applied updates."""
    u = np.frombuffer(np.ascontiguousarray(weights(n_req, substream(seed, TAG_PAIRS), 0, 999999)).tobytes(),
                      np.uint32).astype(np.float64) / 1e6
    cum = np.cumsum(mix)
    kind = np.minimum(np.searchsorted(cum, u, side="right"), 3).astype(np.uint8)
    size = log_uniform(n_req, lo, hi, substream(seed, TAG_W)).astype(np.int64)
    srcs = uniform_pairs(V, n_sources, substream(seed, TAG_LONG))[0]
    pick = weights(n_req, substream(seed, TAG_LOCAL), 0, n_sources - 1)
    source = srcs[pick]
    coin = weights(n_req, substream(seed, TAG_QPERM), 0, 1)
    raw = uniform_pairs(0xFFFFFFFF, n_req, substream(seed, TAG_QRY))[0].astype(np.int64)
    size[kind == 3] = 0
    offset = np.zeros(n_req, np.int64)
    qsrc = np.zeros(n_req, np.uint8)
    applied = np.zeros(n_req, np.int64)
    i_cur, d_cur = E0, 0
    for r in range(n_req):
        k, n = int(kind[r]), int(size[r])
        if k == 1:
            offset[r] = seq_index(i_cur, E0, ring)
            applied[r] = n - min(n, max(0, i_cur + n - ring - d_cur))
            i_cur += n
        elif k == 2:
            offset[r] = seq_index(d_cur, E0, ring)
            applied[r] = min(n, max(0, i_cur - d_cur))
            d_cur = min(d_cur + n, i_cur)
        elif k == 0:
            if coin[r] == 0 and i_cur - d_cur >= n:
                offset[r] = seq_index(d_cur + int(raw[r] % (i_cur - d_cur - n + 1)), E0, ring)
            else:
                qsrc[r] = 1
                offset[r] = int(raw[r] % max(absent_pool - n, 1))
    gaps = exponential_gaps(n_req, 1.0, substream(seed, TAG_QPERM + 16))
    return Batch(kind=kind, size=size, source=source, offset=offset, qsrc=qsrc, applied=applied, gaps=gaps,
                 sources=srcs, inserted=int(size[kind == 1].sum()), E0=E0, ring=ring, hi=hi,
                 absent_pool=absent_pool)


def seq_index(v: int, E0: int, ring: int) -> int:
    """Stored position of position v of the unrolled request sequence."""
    return v if v < E0 else E0 + (v - E0) % ring
