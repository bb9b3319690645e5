"""Full-size workloads in the launch configuration the benchmark times.

Power-law (R-MAT scale 20, 16M edges, load-factor buckets): every batch size
of the workload (2^12, 2^16, 2^20, 2^22) is inserted, deleted and queried with
per-edge flags and bitmaps compared to the oracle, BFS, SSSP and WCC from the
max-degree vertex are compared in full after every insert and every delete
batch, and the final edge set is compared in full.

Road-like (4,096 x 4,096 grid + 0.1% long-range edges, 67M edges): 64 mixed
batches of 2^16 with incremental SSSP from the corner after each batch; each
result is checked against properties that fix it at any size (triangle
inequality on every live edge, every parent edge live and tight, nothing
reachable outside the reachable set), and the first and last against a full
Dijkstra of the oracle.  A 256 x 256 version is compared in full after every
batch.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
NONE = 0xFFFFFFFF


def _mk():
    import paper_2305_17813_gb300 as mk

    mk.load()
    return mk


def u32(t):
    return _mk().to_numpy_u32(t)


def check_tree_properties(es, ed, ew, dist, par, src):
    """Properties that determine the shortest-path tree with min-id parents."""
    reach = dist != NONE
    du = dist[es].astype(np.int64)
    dv = dist[ed].astype(np.int64)
    w = ew.astype(np.int64)
    ru = reach[es]
    assert np.all(reach[ed][ru]), "an edge leaves the reachable set"
    assert np.all(dv[ru] <= du[ru] + w[ru]), "triangle inequality"
    assert dist[src] == 0 and par[src] == src
    assert np.all(par[~reach] == NONE)
    # min tight predecessor for every reachable vertex
    tight = ru & (du + w == dv) & (ed != src)
    best = np.full(len(dist), NONE, np.int64)
    np.minimum.at(best, ed[tight], es[tight].astype(np.int64))
    v = np.nonzero(reach)[0]
    v = v[v != src]
    assert np.array_equal(par[v].astype(np.int64), best[v]), "parent is not the min-id tight predecessor"


def _oracle_algos(o, src):
    """BFS, SSSP and WCC of the oracle, the three run at once (each is one
    foreign call that releases the interpreter lock)."""
    import concurrent.futures as cf

    with cf.ThreadPoolExecutor(3) as ex:
        f = [ex.submit(o.sssp, src), ex.submit(o.bfs, src), ex.submit(o.wcc)]
        return f[0].result(), f[1].result(), f[2].result()


def _compare_algos(g, o, src, what):
    osp, obf, owc = _oracle_algos(o, src)
    for name, (d, p), (od, op) in (("SSSP", g.sssp(src), osp), ("BFS", g.bfs(src), obf)):
        assert np.array_equal(u32(d), od), "%s distances, %s" % (name, what)
        assert np.array_equal(u32(p), op), "%s parents, %s" % (name, what)
    assert np.array_equal(u32(g.wcc()), owc), "WCC labels, %s" % what


def test_powerlaw_full_size_all_batch_sizes(cuda_lib):
    """Every batch size of the workload in turn on one stream of batches
    (deletes from live edges, queries half live): flags, bitmaps and
    weights after every update, BFS/SSSP/WCC after every insert and every
    delete batch, and the final edge set, all against the oracle."""
    mk = _mk()
    G = synth.powerlaw_graph()
    S = synth.PowerlawStream(G)
    src = int(np.argmax(np.bincount(G.src, minlength=G.V)))
    buckets = mk.bucket_rule(G.V, G.src, 0.7)
    g = mk.Graph(G.V, edge_capacity_hint=len(G.src) + (1 << 24), buckets=buckets)
    o = oracle.OracleGraph(G.V)
    chunk = 1 << 22
    for i in range(0, len(G.src), chunk):
        g.insert(G.src[i:i + chunk], G.dst[i:i + chunk], G.w[i:i + chunk], flags=False)
    o.insert(G.src, G.dst, G.w)
    g.commit()
    g.sssp(src)
    g.bfs(src)
    g.wcc()
    g.commit()
    for B in [1 << 12, 1 << 16, 1 << 20, 1 << 22]:
        b = S.batch(B)
        f = g.insert(b.ins_src, b.ins_dst, b.ins_w).cpu().numpy()
        of = o.insert(b.ins_src, b.ins_dst, b.ins_w)
        assert np.array_equal(f, of), "insert flags, batch %d" % B
        assert int(of.sum()) == b.n_inserted
        _compare_algos(g, o, src, "after the insert batch of %d" % B)
        g.commit()
        f = g.delete(b.del_src, b.del_dst).cpu().numpy()
        of = o.delete(b.del_src, b.del_dst)
        assert np.array_equal(f, of), "delete flags, batch %d" % B
        assert of.all(), "the stream's deletes are live"
        _compare_algos(g, o, src, "after the delete batch of %d" % B)
        g.commit()
        bm, w = g.query(b.q_src, b.q_dst)
        obm, ow = o.query(b.q_src, b.q_dst)
        assert np.array_equal(u32(bm), obm) and np.array_equal(u32(w), ow), "query, batch %d" % B
        assert int(oracle.bitmap_to_bool(obm, B).sum()) == B // 2
        assert g.last_error() == mk.MK_OK
    es, ed, ew = g.export()
    os_, od_, ow_ = o.export()
    assert np.array_equal(u32(es), os_) and np.array_equal(u32(ed), od_) and np.array_equal(u32(ew), ow_)
    g.close()


def road_run(rows, cols, batches, full_check_every, delta=0):
    mk = _mk()
    R = synth.road_graph(rows, cols)
    g = mk.Graph(R.V, edge_capacity_hint=len(R.src) + batches * (1 << 16), buckets=1)
    g.set_sssp_delta(delta, delta)
    o = oracle.OracleGraph(R.V)
    chunk = 1 << 22
    for i in range(0, len(R.src), chunk):
        g.insert(R.src[i:i + chunk], R.dst[i:i + chunk], R.w[i:i + chunk], flags=False)
    o.insert(R.src, R.dst, R.w)
    g.commit()
    d, p = g.sssp(0)
    od, op = o.sssp(0)
    assert np.array_equal(u32(d), od) and np.array_equal(u32(p), op)
    g.commit()
    B = 1 << 16 if rows >= 1024 else 1 << 10
    for k in range(batches):
        b = synth.road_batch(R, k, B)
        fd = g.delete(b.del_src, b.del_dst).cpu().numpy()
        assert np.array_equal(fd, o.delete(b.del_src, b.del_dst))
        fi = g.insert(b.ins_src, b.ins_dst, b.ins_w).cpu().numpy()
        assert np.array_equal(fi, o.insert(b.ins_src, b.ins_dst, b.ins_w))
        d, p = g.sssp(0)
        g.commit()
        assert g.last_error() == mk.MK_OK
        dist, par = u32(d), u32(p)
        if full_check_every and (k % full_check_every == 0 or k == batches - 1):
            od, op = o.sssp(0)
            assert np.array_equal(dist, od) and np.array_equal(par, op), "batch %d" % k
        elif k in (0, batches - 1) or k % 16 == 0:
            es, ed, ew = (u32(x) for x in g.export())
            check_tree_properties(es, ed, ew, dist, par, 0)
    if not full_check_every:
        od, op = o.sssp(0)
        assert np.array_equal(u32(d), od) and np.array_equal(u32(p), op)
    g.close()


def test_road_small_every_batch(cuda_lib):
    road_run(256, 256, 16, full_check_every=1)


def test_road_full_size_64_batches(cuda_lib):
    road_run(4096, 4096, 64, full_check_every=0)


@pytest.mark.parametrize("delta", [1, 1500, 1 << 31])
def test_road_small_near_far_every_batch(cuda_lib, delta):
    """Near-Far ordered SSSP rounds (a bucket width of one weight unit, a
    few edges' worth, and wider than every distance) give the oracle's tree
    after every mixed batch."""
    road_run(256, 256, 12, full_check_every=1, delta=delta)


def test_road_near_far_mid_size(cuda_lib):
    road_run(1024, 1024, 8, full_check_every=4, delta=4000)


def test_road_full_size_near_far(cuda_lib):
    road_run(4096, 4096, 6, full_check_every=0, delta=4000)
