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
TAG_PAIRS, TAG_W, TAG_PERM, TAG_QRY, TAG_QPERM, TAG_LONG, TAG_LOCAL = 1, 2, 3, 4, 5, 6, 7


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


def powerlaw_batch(g: Batch, k: int, B: int, wlo: int = 1, whi: int = 100) -> Batch:
    """Batch k (seed 100 + k) on a graph from `powerlaw_graph`: B new R-MAT
    inserts (self-loops dropped), B deletes drawn without replacement from the
    initial edges (a fixed permutation consumed from the front, so they are
    live as long as no earlier delete batch took them) and B queries, half from
    the initial edges taken from the back of the permutation and half uniform,
    shuffled."""
    V, E = g.V, len(g.src)
    seed = 100 + k
    s, d = rmat_pairs(g.scale, B + B // 8 + 64, substream(seed, TAG_PAIRS))
    keep = s != d
    s, d = s[keep][:B], d[keep][:B]
    w = weights(len(s), substream(seed, TAG_W), wlo, whi)
    perm = _initial_perm(g)
    lo = (k * B) % max(1, E)
    di = np.take(perm, np.arange(lo, lo + B) % E)
    half = B // 2
    qi = np.take(perm, (E - 1 - ((k * half + np.arange(half)) % E)))
    us, ud = uniform_pairs(V, B - half, substream(seed, TAG_QRY))
    qs = np.concatenate([g.src[qi], us])
    qd = np.concatenate([g.dst[qi], ud])
    qp = permutation(B, substream(seed, TAG_QPERM))
    return Batch(ins_src=s, ins_dst=d, ins_w=w, del_src=g.src[di], del_dst=g.dst[di],
                 q_src=qs[qp], q_dst=qd[qp])


def _initial_perm(g: Batch) -> np.ndarray:
    p = g.get("_perm")
    if p is None:
        p = permutation(len(g.src), substream(0, TAG_PERM))
        g["_perm"] = p
    return p


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
