"""GPU parity of incremental / decremental BFS and SSSP trees and of WCC
labels with the CPU oracle (which recomputes from scratch after every batch):
distances, min-id tight parents and min-id component labels, bit-exact."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _mk():
    import paper_2305_17813_gb300 as mk

    mk.load()
    return mk


def check_algos(g, o, sources, wcc=True):
    mk = _mk()
    for src in sources:
        d, p = g.sssp(src)
        od, op = o.sssp(src)
        assert np.array_equal(mk.to_numpy_u32(d), od), "sssp dist from %d" % src
        assert np.array_equal(mk.to_numpy_u32(p), op), "sssp parent from %d" % src
        d, p = g.bfs(src)
        od, op = o.bfs(src)
        assert np.array_equal(mk.to_numpy_u32(d), od), "bfs dist from %d" % src
        assert np.array_equal(mk.to_numpy_u32(p), op), "bfs parent from %d" % src
    if wcc:
        assert np.array_equal(mk.to_numpy_u32(g.wcc()), o.wcc()), "wcc labels"
    assert g.last_error() == mk.MK_OK


def test_tiny_workload_incremental_sequence(cuda_lib):
    mk = _mk()
    w = synth.tiny_workload()
    g = mk.Graph(w.V, edge_capacity_hint=16384, buckets=1)
    o = oracle.OracleGraph(w.V)
    g.insert(w.g_src, w.g_dst, w.g_w)
    o.insert(w.g_src, w.g_dst, w.g_w)
    g.commit()
    check_algos(g, o, [0])          # static
    g.commit()
    g.insert(w.ins_src, w.ins_dst, w.ins_w)
    o.insert(w.ins_src, w.ins_dst, w.ins_w)
    check_algos(g, o, [0])          # incremental
    g.commit()
    g.delete(w.del_src, w.del_dst)
    o.delete(w.del_src, w.del_dst)
    check_algos(g, o, [0])          # decremental (WCC recomputes)
    g.commit()


@pytest.mark.parametrize("buckets", [1, 4])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_mixed_epochs_match_recompute(cuda_lib, buckets, seed):
    """Random insert / delete batches; the algorithms run after every batch
    and sometimes twice inside one epoch, commits between some batches."""
    mk = _mk()
    rng = np.random.default_rng(10 + seed)
    V = 600
    g = mk.Graph(V, edge_capacity_hint=50000, buckets=buckets)
    o = oracle.OracleGraph(V)
    s = rng.integers(0, V, 3000).astype(np.uint32)
    d = rng.integers(0, V, 3000).astype(np.uint32)
    w = rng.integers(1, 50, 3000).astype(np.uint32)
    g.insert(s, d, w)
    o.insert(s, d, w)
    srcs = [0, int(rng.integers(0, V))]
    check_algos(g, o, srcs)
    for step in range(8):
        n = int(rng.integers(1, 400))
        if step % 3 == 1:
            ls, ld, _ = o.export()
            pick = rng.integers(0, len(ls), n)
            g.delete(ls[pick], ld[pick])
            o.delete(ls[pick], ld[pick])
        else:
            s = rng.integers(0, V, n).astype(np.uint32)
            d = rng.integers(0, V, n).astype(np.uint32)
            w = rng.integers(1, 50, n).astype(np.uint32)
            g.insert(s, d, w)
            o.insert(s, d, w)
        check_algos(g, o, srcs, wcc=step % 2 == 0)
        if step % 2 == 1:
            g.commit()


def test_delete_then_reinsert_tree_edge(cuda_lib):
    mk = _mk()
    V = 6
    g = mk.Graph(V, buckets=1)
    o = oracle.OracleGraph(V)
    s = np.array([0, 1, 2, 0, 3, 4], np.uint32)
    d = np.array([1, 2, 3, 3, 4, 5], np.uint32)
    w = np.array([1, 1, 1, 10, 1, 1], np.uint32)
    for x in (g, o):
        x.insert(s, d, w)
    check_algos(g, o, [0])
    g.commit()
    for x in (g, o):
        x.delete([1], [2])            # tree edge: 2, 3, 4, 5 lose their paths
    check_algos(g, o, [0])
    for x in (g, o):
        x.insert([1], [2], [2])       # same edge, new weight, same epoch
    check_algos(g, o, [0])
    g.commit()
    for x in (g, o):
        x.delete([0, 0], [1, 3])      # source cut off from everything
    check_algos(g, o, [0])


def test_grid_closed_form_and_single_component(cuda_lib):
    mk = _mk()
    rows, cols = 64, 96
    s, d = synth.grid_pairs(rows, cols)
    g = mk.Graph(rows * cols, buckets=1)
    g.insert(s, d, np.ones(len(s), np.uint32))
    r, c = np.divmod(np.arange(rows * cols), cols)
    dist, _ = g.bfs(0)
    assert np.array_equal(mk.to_numpy_u32(dist), r + c)
    dist, _ = g.sssp(0)
    assert np.array_equal(mk.to_numpy_u32(dist), r + c)
    assert np.all(mk.to_numpy_u32(g.wcc()) == 0)


def test_power_law_with_bucket_rule(cuda_lib):
    """R-MAT scale 14 with the load-factor bucket rule (many buckets for hubs):
    static, then an insert batch and a delete batch with recomputation."""
    mk = _mk()
    G = synth.powerlaw_graph(scale=14, draws=1 << 18)
    b = mk.bucket_rule(G.V, G.src, 0.7)
    g = mk.Graph(G.V, edge_capacity_hint=len(G.src) * 2, buckets=b)
    o = oracle.OracleGraph(G.V)
    g.insert(G.src, G.dst, G.w)
    o.insert(G.src, G.dst, G.w)
    g.commit()
    src = int(np.argmax(o.out_degree()))
    check_algos(g, o, [src])
    g.commit()
    B = synth.PowerlawStream(G, max_batch=1 << 14).batch(1 << 14)
    g.insert(B.ins_src, B.ins_dst, B.ins_w)
    o.insert(B.ins_src, B.ins_dst, B.ins_w)
    check_algos(g, o, [src])
    g.commit()
    g.delete(B.del_src, B.del_dst)
    o.delete(B.del_src, B.del_dst)
    check_algos(g, o, [src])
    g.commit()
    bm, _ = g.query(B.q_src, B.q_dst)
    assert np.array_equal(mk.to_numpy_u32(bm), o.query(B.q_src, B.q_dst)[0])


def test_long_path_and_mixed_frontier_sizes(cuda_lib):
    """A 9,000-vertex path (thousands of one-list rounds, more than one
    solo phase of the round kernel) feeding a dense random block (frontiers
    of thousands of lists), then a delete that cuts the path in the middle."""
    mk = _mk()
    P = 9000
    B = 4000
    rng = np.random.default_rng(5)
    V = P + B
    ps = np.arange(P - 1, dtype=np.uint32)
    pd = ps + 1
    bs = rng.integers(P, V, 120000).astype(np.uint32)
    bd = rng.integers(P, V, 120000).astype(np.uint32)
    s = np.concatenate([ps, [P - 1], bs]).astype(np.uint32)
    d = np.concatenate([pd, [P], bd]).astype(np.uint32)
    w = rng.integers(1, 9, len(s)).astype(np.uint32)
    g = mk.Graph(V, edge_capacity_hint=len(s) * 2, buckets=1)
    o = oracle.OracleGraph(V)
    g.insert(s, d, w)
    o.insert(s, d, w)
    check_algos(g, o, [0], wcc=True)
    g.commit()
    for x in (g, o):
        x.delete([P // 2], [P // 2 + 1])
    check_algos(g, o, [0], wcc=True)
    g.commit()
    for x in (g, o):
        x.insert([P // 2], [P // 2 + 1], [3])
    check_algos(g, o, [0], wcc=True)


@pytest.mark.parametrize("delta", [7, 300])
def test_near_far_sssp_power_law_stream(cuda_lib, delta):
    """Near-Far ordered SSSP on R-MAT batches of inserts and deletes of live
    edges: the tree equals the oracle's after every batch, BFS (never
    ordered) too, and switching the ordering off mid-stream keeps it."""
    mk = _mk()
    G = synth.powerlaw_graph(scale=13, draws=1 << 17)
    S = synth.PowerlawStream(G, max_batch=1 << 12)
    src = int(np.argmax(np.bincount(G.src, minlength=G.V)))
    g = mk.Graph(G.V, edge_capacity_hint=len(G.src) + (1 << 16), buckets=mk.bucket_rule(G.V, G.src, 0.7))
    g.set_sssp_delta(delta, delta)
    o = oracle.OracleGraph(G.V)
    g.insert(G.src, G.dst, G.w, flags=False)
    o.insert(G.src, G.dst, G.w)
    g.commit()
    for k in range(6):
        if k == 4:
            g.set_sssp_delta(0, 0)
        b = S.batch(1 << 12)
        g.insert(b.ins_src, b.ins_dst, b.ins_w, flags=False)
        o.insert(b.ins_src, b.ins_dst, b.ins_w)
        for fn, ofn in ((g.sssp, o.sssp), (g.bfs, o.bfs)):
            d, p = fn(src)
            od, op = ofn(src)
            assert np.array_equal(mk.to_numpy_u32(d), od) and np.array_equal(mk.to_numpy_u32(p), op), k
        g.commit()
        g.delete(b.del_src, b.del_dst, flags=False)
        o.delete(b.del_src, b.del_dst)
        d, p = g.sssp(src)
        od, op = o.sssp(src)
        assert np.array_equal(mk.to_numpy_u32(d), od) and np.array_equal(mk.to_numpy_u32(p), op), k
        g.commit()
        assert g.last_error() == mk.MK_OK
    g.close()
