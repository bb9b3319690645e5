"""The ConcurrentSet layout (31 keys a slab): batched insert, delete and
query flags and bitmaps, static BFS (hop counts and smallest-id tight
parents) and WCC labels against the oracle on the unweighted view, and the
slab count against the weighted store's on the same edges."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _mk():
    import paper_2305_17813_gb300 as mk

    mk.load()
    return mk


def _check_algos(mk, g, o, srcs):
    for s in srcs:
        d, p = g.bfs(s)
        od, op = o.bfs(s)
        assert np.array_equal(mk.to_numpy_u32(d), od), s
        assert np.array_equal(mk.to_numpy_u32(p), op), s
    assert np.array_equal(mk.to_numpy_u32(g.wcc()), o.wcc())


@pytest.mark.parametrize("buckets", [1, 3])
def test_set_graph_tiny_against_oracle(cuda_lib, buckets):
    mk = _mk()
    w = synth.tiny_workload()
    g = mk.SetGraph(w.V, edge_capacity_hint=1 << 15, buckets=buckets)
    o = oracle.OracleGraph(w.V)
    assert np.array_equal(g.insert(w.g_src, w.g_dst).cpu().numpy(), o.insert(w.g_src, w.g_dst))
    _check_algos(mk, g, o, [0, 5])
    assert np.array_equal(g.insert(w.ins_src, w.ins_dst).cpu().numpy(), o.insert(w.ins_src, w.ins_dst))
    assert np.array_equal(g.delete(w.del_src, w.del_dst).cpu().numpy(), o.delete(w.del_src, w.del_dst))
    bm = g.query(w.q_src, w.q_dst)
    assert np.array_equal(mk.to_numpy_u32(bm), o.query(w.q_src, w.q_dst)[0])
    _check_algos(mk, g, o, [0, 17])
    assert g.last_error() == mk.MK_OK
    g.close()


def test_set_graph_power_law_and_slab_count(cuda_lib):
    mk = _mk()
    G = synth.powerlaw_graph(scale=15, draws=1 << 19)
    sb = mk.set_bucket_rule(G.V, G.src, 0.7)
    g = mk.SetGraph(G.V, edge_capacity_hint=2 * len(G.src), buckets=sb)
    o = oracle.OracleGraph(G.V)
    # a hub's edges spread over many warps and pool slabs: the initial load
    # in one batch
    assert np.array_equal(g.insert(G.src, G.dst).cpu().numpy(), o.insert(G.src, G.dst))
    src = int(np.argmax(o.out_degree()))
    _check_algos(mk, g, o, [src])
    S = synth.PowerlawStream(G, max_batch=1 << 14)
    for _ in range(2):
        b = S.batch(1 << 14)
        assert np.array_equal(g.insert(b.ins_src, b.ins_dst).cpu().numpy(), o.insert(b.ins_src, b.ins_dst))
        assert np.array_equal(g.delete(b.del_src, b.del_dst).cpu().numpy(), o.delete(b.del_src, b.del_dst))
        bm = g.query(b.q_src, b.q_dst)
        assert np.array_equal(mk.to_numpy_u32(bm), o.query(b.q_src, b.q_dst)[0])
    _check_algos(mk, g, o, [src])
    # the same edges in the weighted store take more slabs; a list of the set
    # layout holds 31 keys a slab
    m = mk.Graph(G.V, edge_capacity_hint=2 * len(G.src), buckets=mk.bucket_rule(G.V, G.src, 0.7))
    m.insert(G.src, G.dst, G.w, flags=False)
    o2 = oracle.OracleGraph(G.V)
    o2.insert(G.src, G.dst)
    deg = o2.out_degree().astype(np.int64)
    ss = g.stats()
    ms = m.stats()
    assert ss["lists"] == int(sb.cpu().numpy().astype(np.int64).sum())
    assert ss["slabs_in_use"] < ms["chain_slabs"], (ss, ms)
    g2 = mk.SetGraph(G.V, edge_capacity_hint=2 * len(G.src), buckets=sb)
    g2.insert(G.src, G.dst)
    assert g2.stats()["slabs_in_use"] >= int(((deg + 30) // 31).sum()) + int((deg == 0).sum())
    g2.close()
    assert g.last_error() == mk.MK_OK and m.last_error() == mk.MK_OK
    g.close()
    m.close()


@pytest.mark.parametrize("buckets", [1, 12])
def test_set_graph_deep_bfs_and_isolated_source(cuda_lib, buckets):
    """A 150-edge path (150 levels, many groups of level launches) with side
    branches, a vertex without out-edges as source, and an empty graph."""
    mk = _mk()
    V = 400
    s = np.arange(150, dtype=np.uint32)
    d = s + 1
    bs = np.arange(0, 150, 7, dtype=np.uint32)
    src = np.concatenate([s, bs, [300, 300]]).astype(np.uint32)
    dst = np.concatenate([d, bs + 200, [301, 0]]).astype(np.uint32)
    g = mk.SetGraph(V, edge_capacity_hint=1024, buckets=buckets)
    o = oracle.OracleGraph(V)
    e = mk.SetGraph(V, buckets=buckets)
    oe = oracle.OracleGraph(V)
    _check_algos(mk, e, oe, [0, 399])
    assert np.array_equal(g.insert(src, dst).cpu().numpy(), o.insert(src, dst))
    _check_algos(mk, g, o, [0, 300, 399, 150])
    assert np.array_equal(g.delete([75], [76]).cpu().numpy(), o.delete([75], [76]))
    _check_algos(mk, g, o, [0, 300])
    assert g.last_error() == mk.MK_OK and e.last_error() == mk.MK_OK
    g.close()
    e.close()


def test_set_graph_rmat18_against_oracle(cuda_lib):
    """R-MAT scale 18 (about 3.6 M edges, hubs with thousands of lists'
    worth of keys): load, BFS from the three largest out-degree vertices and
    WCC, then a 2^18 stream batch of inserts, deletes of live edges and
    half-present queries, and BFS / WCC again, all against the oracle."""
    mk = _mk()
    G = synth.powerlaw_graph(scale=18, draws=1 << 22)
    g = mk.SetGraph(G.V, edge_capacity_hint=len(G.src) + (1 << 19), buckets=mk.set_bucket_rule(G.V, G.src, 0.7))
    o = oracle.OracleGraph(G.V)
    assert np.array_equal(g.insert(G.src, G.dst).cpu().numpy(), o.insert(G.src, G.dst))
    top = [int(x) for x in np.argsort(-o.out_degree().astype(np.int64), kind="stable")[:3]]
    _check_algos(mk, g, o, top)
    b = synth.PowerlawStream(G, max_batch=1 << 18).batch(1 << 18)
    fi = g.insert(b.ins_src, b.ins_dst).cpu().numpy()
    assert np.array_equal(fi, o.insert(b.ins_src, b.ins_dst))
    fd = g.delete(b.del_src, b.del_dst).cpu().numpy()
    assert np.array_equal(fd, o.delete(b.del_src, b.del_dst)) and fd.all()
    bm, _ = o.query(b.q_src, b.q_dst)
    assert np.array_equal(mk.to_numpy_u32(g.query(b.q_src, b.q_dst)), bm)
    assert int(oracle.bitmap_to_bool(bm, len(b.q_src)).sum()) == b.n_present
    _check_algos(mk, g, o, top[:1])
    assert g.last_error() == mk.MK_OK
    g.close()


def test_set_graph_invalid_ids_and_pool_exhaustion(cuda_lib):
    """Invalid vertex ids set the sticky status; an exhausted pool reports
    MK_ERR_POOL_EXHAUSTED with exactly the flagged edges stored, and the
    traversals still run on what was stored."""
    mk = _mk()
    g = mk.SetGraph(4, buckets=1)
    f = g.insert([0, 5, 1], [1, 2, 2]).cpu().numpy()
    assert f[1] == 0
    assert g.last_error() == mk.MK_ERR_INVALID_ARG
    bm = g.query([0, 1], [1, 2])
    assert g.last_error() == mk.MK_OK
    got = oracle.bitmap_to_bool(mk.to_numpy_u32(bm), 2)
    assert np.array_equal(got, f[[0, 2]].astype(bool))
    g.query([7], [0])
    assert g.last_error() == mk.MK_ERR_INVALID_ARG
    g.close()

    V = 50000
    src = np.repeat(np.arange(40, dtype=np.uint32), V)
    dst = np.tile(np.arange(V, dtype=np.uint32), 40)
    g = mk.SetGraph(V, edge_capacity_hint=0, buckets=1)
    f = g.insert(src, dst).cpu().numpy()
    assert g.last_error() == mk.MK_ERR_POOL_EXHAUSTED
    assert 0 < int(f.sum()) < len(src)
    bm = g.query(src, dst)
    assert np.array_equal(oracle.bitmap_to_bool(mk.to_numpy_u32(bm), len(src)), f.astype(bool))
    o = oracle.OracleGraph(V)
    keep = f.astype(bool)
    o.insert(src[keep], dst[keep])
    _check_algos(mk, g, o, [0, 39])
    assert g.last_error() == mk.MK_OK
    g.close()
