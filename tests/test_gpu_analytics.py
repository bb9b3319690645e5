"""PageRank and triangle counting on the GPU against the oracle.

PageRank: the device works in 64-bit fixed point (scale 2^48) and stops
when the L1 change of a super-step is <= 1e-7; the oracle iterates in
double precision to 1e-13.  The distance to the common fixpoint is then at
most about 1e-7 * d / (1 - d) = 5.7e-7 (d = 0.85) on the device side, plus
its rounding (below 2^-48 per added term, and the float32 output: 2^-24
relative per rank, at most 6e-8 in L1), so the test bound is an L1
distance of 1e-5 between the two rank vectors.  Results are bit-identical
from run to run (integer atomics).  Triangle counts are exact integers:
static counts and the running count after insert and delete batches
(inclusion-exclusion over the batch) equal the oracle's brute-force count.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
L1_TOL = 1e-5


def _mk():
    import paper_2305_17813_gb300 as mk

    mk.load()
    return mk


def test_pagerank_static_incremental_decremental(cuda_lib):
    import torch

    mk = _mk()
    G = synth.powerlaw_graph(scale=14, draws=1 << 18)
    b = mk.bucket_rule(G.V, G.src, 0.7)
    g = mk.Graph(G.V, edge_capacity_hint=len(G.src) * 2, buckets=b)
    g.insert(G.src, G.dst, G.w)
    g.commit()
    o = oracle.OracleGraph(G.V)
    o.insert(G.src, G.dst, G.w)
    pr, it_static, delta = g.pagerank(eps=1e-7, max_iter=300)
    assert delta <= 1e-7 and it_static < 300
    ref, _ = o.pagerank(eps=1e-13, max_iter=3000)
    assert np.abs(pr.cpu().numpy().astype(np.float64) - ref).sum() <= L1_TOL
    assert abs(float(pr.double().sum()) - 1.0) < 1e-4
    # the same bits on a second run
    pr2, it2, _ = g.pagerank(eps=1e-7, max_iter=300)
    assert it2 == it_static and torch.equal(pr, pr2)
    S = synth.PowerlawStream(G, max_batch=1 << 12)
    bt = S.batch(1 << 12)
    for step in ("insert", "delete"):
        if step == "insert":
            g.insert(bt.ins_src, bt.ins_dst, bt.ins_w)
            o.insert(bt.ins_src, bt.ins_dst, bt.ins_w)
        else:
            g.delete(bt.del_src, bt.del_dst)
            o.delete(bt.del_src, bt.del_dst)
        g.commit()
        # warm start from the ranks before the batch (the dynamic case)
        pr, it_warm, _ = g.pagerank(pr, eps=1e-7, max_iter=300)
        ref, _ = o.pagerank(eps=1e-13, max_iter=3000)
        assert np.abs(pr.cpu().numpy().astype(np.float64) - ref).sum() <= L1_TOL, step
        assert it_warm < it_static, (step, it_warm, it_static)
    assert g.last_error() == mk.MK_OK


def _undirected(s, d):
    keep = s != d
    s, d = s[keep], d[keep]
    a = np.concatenate([s, d]).astype(np.uint32)
    b = np.concatenate([d, s]).astype(np.uint32)
    return a, b


def test_triangles_static_and_after_batches(cuda_lib):
    mk = _mk()
    G = synth.powerlaw_graph(scale=12, draws=1 << 15)
    V = G.V
    s, d = _undirected(G.src, G.dst)
    b = mk.bucket_rule(V, s, 0.7)
    g = mk.Graph(V, edge_capacity_hint=len(s) * 3, buckets=b)
    g.insert(s, d)
    g.commit()
    o = oracle.OracleGraph(V)
    o.insert(s, d)
    count = g.triangles()
    assert count == o.triangles() and count > 1000
    rng = np.random.default_rng(3)
    es, ed, _ = o.export()
    for k in range(4):
        deletion = k % 2 == 1
        if not deletion:
            # new edges: random pairs, plus a K4 on four vertices and a fan,
            # so that triangles with two and three new edges occur
            bs = rng.integers(0, V, 3000)
            bd = rng.integers(0, V, 3000)
            q = rng.choice(V, 6, replace=False)
            k4 = [(q[i], q[j]) for i in range(4) for j in range(i + 1, 4)]
            fan = [(q[4], x) for x in (q[0], q[1], q[5])]
            bs = np.concatenate([bs, [a for a, _ in k4 + fan]]).astype(np.uint32)
            bd = np.concatenate([bd, [c for _, c in k4 + fan]]).astype(np.uint32)
            us, ud = _undirected(bs, bd)
            f = g.insert(us, ud).cpu().numpy().astype(bool)
            assert np.array_equal(f, o.insert(us, ud).astype(bool))
        else:
            es, ed, _ = o.export()
            pick = rng.choice(len(es), 2000, replace=False)
            us, ud = _undirected(es[pick], ed[pick])
            f = g.delete(us, ud).cpu().numpy().astype(bool)
            assert np.array_equal(f, o.delete(us, ud).astype(bool))
        # the batch's applied edges, both directions, and a graph of just them
        ns, nd = us[f], ud[f]
        upd = mk.Graph(V, edge_capacity_hint=len(ns) + 64, buckets=1)
        upd.insert(ns, nd)
        delta = g.triangle_delta(upd, ns, nd, deletion)
        upd.close()
        count += delta
        assert count == o.triangles(), (k, delta)
        assert g.triangles() == count
        g.commit()
    assert g.last_error() == mk.MK_OK


def test_analytics_degenerate_graphs(cuda_lib):
    """No edges: every vertex dangles, the teleport term alone gives ranks
    1 / V.  A grid (no triangles) counts 0, and an empty batch changes
    nothing."""
    mk = _mk()
    g = mk.Graph(1000, edge_capacity_hint=16, buckets=1)
    pr, it, _ = g.pagerank(eps=1e-7)
    assert np.allclose(pr.cpu().numpy(), 1e-3, rtol=1e-6) and it <= 2
    g.close()
    s, d = synth.grid_pairs(30, 30)
    grid = mk.Graph(900, edge_capacity_hint=len(s) * 2, buckets=2)
    grid.insert(s, d)
    assert grid.triangles() == 0
    upd = mk.Graph(900, edge_capacity_hint=16, buckets=1)
    assert grid.triangle_delta(upd, np.zeros(0, np.uint32), np.zeros(0, np.uint32), False) == 0
    lib = mk.load()
    assert lib.mk_l2_window(grid.handle, 7, None, None) == mk.MK_ERR_INVALID_ARG
    assert grid.last_error() == mk.MK_OK
    upd.close()
    grid.close()
