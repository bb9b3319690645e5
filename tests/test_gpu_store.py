"""GPU parity of the slab-hash store (insert, delete, query, export) with the
CPU oracle: bit-exact flags, bitmaps, weights and edge sets on seeded inputs,
plus the edge cases of the method (duplicates, empty batches, hubs whose
list is appended by many warps, invalid ids, pool exhaustion)."""
import json
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _mk():
    import paper_2305_17813_gb300 as mk

    mk.load()
    return mk


def assert_same_edges(g, o):
    mk = _mk()
    s, d, w = g.export()
    os_, od, ow = o.export()
    assert np.array_equal(mk.to_numpy_u32(s), os_)
    assert np.array_equal(mk.to_numpy_u32(d), od)
    assert np.array_equal(mk.to_numpy_u32(w), ow)


def run_ops(g, o, ops):
    """Apply (kind, arrays) ops to both; compare every output."""
    mk = _mk()
    for kind, a in ops:
        if kind == "ins":
            f = g.insert(a[0], a[1], a[2]).cpu().numpy()
            assert np.array_equal(f, o.insert(a[0], a[1], a[2])), "insert flags"
        elif kind == "del":
            f = g.delete(a[0], a[1]).cpu().numpy()
            assert np.array_equal(f, o.delete(a[0], a[1])), "delete flags"
        elif kind == "qry":
            bm, w = g.query(a[0], a[1])
            obm, ow = o.query(a[0], a[1])
            assert np.array_equal(mk.to_numpy_u32(bm), obm), "query bitmap"
            assert np.array_equal(mk.to_numpy_u32(w), ow), "query weights"
        elif kind == "commit":
            g.commit()
    assert g.last_error() == mk.MK_OK
    assert_same_edges(g, o)


def test_tiny_workload_bit_exact(cuda_lib):
    mk = _mk()
    w = synth.tiny_workload()
    g = mk.Graph(w.V, edge_capacity_hint=16384, buckets=1)
    o = oracle.OracleGraph(w.V)
    run_ops(g, o, [
        ("ins", (w.g_src, w.g_dst, w.g_w)), ("commit", None),
        ("ins", (w.ins_src, w.ins_dst, w.ins_w)), ("qry", (w.q_src, w.q_dst)),
        ("del", (w.del_src, w.del_dst)), ("qry", (w.q_src, w.q_dst)), ("commit", None),
    ])
    st = g.stats()
    assert st["live_edges"] == o.num_edges


@pytest.mark.parametrize("buckets", [1, 3, 17])
@pytest.mark.parametrize("seed", [0, 1])
def test_random_batches_many_buckets(cuda_lib, buckets, seed):
    mk = _mk()
    rng = np.random.default_rng(seed)
    V = 777
    g = mk.Graph(V, edge_capacity_hint=40000, buckets=buckets)
    o = oracle.OracleGraph(V)
    for step in range(10):
        n = int(rng.integers(1, 5000)) if step else 12345
        s = rng.integers(0, V, n).astype(np.uint32)
        d = rng.integers(0, V, n).astype(np.uint32)
        kind = ["ins", "del", "qry"][step % 3] if step else "ins"
        if kind == "ins":
            op = ("ins", (s, d, rng.integers(1, 1000, n).astype(np.uint32)))
        elif kind == "del":
            # half drawn from the live edges, half random pairs
            ls, ld, _ = o.export()
            pick = rng.integers(0, len(ls), n // 2)
            op = ("del", (np.concatenate([ls[pick], s[: n - n // 2]]), np.concatenate([ld[pick], d[: n - n // 2]])))
        else:
            op = ("qry", (s, d))
        run_ops(g, o, [op] + ([("commit", None)] if step % 4 == 3 else []))


def test_hub_list_appended_by_many_warps(cuda_lib):
    """One vertex receives thousands of new edges in one batch: its single
    list is extended concurrently by ~100 warps (CAS claims and CAS links)."""
    mk = _mk()
    V = 5000
    g = mk.Graph(V, edge_capacity_hint=20000, buckets=1)
    o = oracle.OracleGraph(V)
    rng = np.random.default_rng(3)
    hub = np.full(3000, 42, np.uint32)
    d = rng.permutation(V)[:3000].astype(np.uint32)
    w = rng.integers(1, 100, 3000).astype(np.uint32)
    # interleave other sources so the hub's edges straddle warp boundaries
    s2 = rng.integers(0, V, 2000).astype(np.uint32)
    d2 = rng.integers(0, V, 2000).astype(np.uint32)
    w2 = rng.integers(1, 100, 2000).astype(np.uint32)
    s = np.concatenate([hub, s2])
    dd = np.concatenate([d, d2])
    ww = np.concatenate([w, w2])
    p = rng.permutation(len(s))
    run_ops(g, o, [("ins", (s[p], dd[p], ww[p])), ("qry", (s, dd)), ("del", (hub[:1500], d[:1500])),
                   ("ins", (hub, d, w)), ("qry", (s, dd))])
    st = g.stats()
    assert st["chain_max"] >= 3000 // 15
    # the device pool counter agrees with the bitmap after CAS-link races
    assert g.pool_free() == st["pool_slabs"] - st["pool_used"]


def test_duplicates_first_occurrence_and_repeated_deletes(cuda_lib):
    mk = _mk()
    g = mk.Graph(16, buckets=2)
    o = oracle.OracleGraph(16)
    s = np.array([1, 1, 1, 2, 2, 1, 3], np.uint32)
    d = np.array([2, 2, 2, 3, 3, 2, 3], np.uint32)
    w = np.array([7, 3, 9, 5, 1, 8, 4], np.uint32)
    run_ops(g, o, [("ins", (s, d, w)), ("ins", (s, d, w + 1)), ("del", (s, d)), ("qry", (s, d)),
                   ("ins", (s[::-1].copy(), d[::-1].copy(), w[::-1].copy())), ("qry", (s, d))])


def test_empty_and_ragged_batches(cuda_lib):
    mk = _mk()
    g = mk.Graph(100, buckets=1)
    o = oracle.OracleGraph(100)
    e = np.zeros(0, np.uint32)
    for n in (0, 1, 31, 32, 33, 257):
        s = (np.arange(n) * 7 % 100).astype(np.uint32)
        d = (np.arange(n) * 13 % 100).astype(np.uint32)
        run_ops(g, o, [("ins", (s, d, np.ones(n, np.uint32))), ("qry", (s, d)), ("del", (e, e)), ("qry", (e, e))])


def test_delete_every_edge_leaves_empty_graph(cuda_lib):
    mk = _mk()
    w = synth.tiny_workload()
    g = mk.Graph(w.V, buckets=1)
    o = oracle.OracleGraph(w.V)
    g.insert(w.g_src, w.g_dst, w.g_w)
    o.insert(w.g_src, w.g_dst, w.g_w)
    s, d, _ = o.export()
    p = np.random.default_rng(0).permutation(len(s))
    f = g.delete(s[p], d[p]).cpu().numpy()
    assert f.all()
    st = g.stats()
    assert st["live_edges"] == 0 and st["tombstones"] == len(s)
    assert g.export()[0].numel() == 0


def test_invalid_vertex_rejects_batch(cuda_lib):
    mk = _mk()
    g = mk.Graph(10, buckets=1)
    g.insert([1, 2], [3, 4], [1, 1])
    assert g.last_error() == mk.MK_OK
    f = g.insert([1, 10], [5, 5], [1, 1]).cpu().numpy()
    assert g.last_error() == mk.MK_ERR_INVALID_ARG
    assert f.tolist() == [0, 0]
    f = g.insert([1], [6], [0]).cpu().numpy()  # weight 0 is rejected
    assert g.last_error() == mk.MK_ERR_INVALID_ARG
    s, d, _ = g.export()
    assert mk.to_numpy_u32(s).tolist() == [1, 2] and mk.to_numpy_u32(d).tolist() == [3, 4]
    bm, _ = g.query([1, 2, 99], [3, 4, 1])
    assert g.last_error() == mk.MK_ERR_INVALID_ARG


def test_pool_exhaustion_applies_flagged_edges_only(cuda_lib):
    """A list that outgrows a 32-slab pool: the status reports the exhausted
    pool and exactly the edges flagged as inserted are stored."""
    mk = _mk()
    V = 4096
    g = mk.Graph(V, buckets=1, pool_slabs=32)
    o = oracle.OracleGraph(V)
    s = np.zeros(1000, np.uint32)
    d = np.arange(1000, dtype=np.uint32)
    f = g.insert(s, d, np.ones(1000, np.uint32)).cpu().numpy()
    assert g.last_error() == mk.MK_ERR_POOL_EXHAUSTED
    assert 0 < f.sum() <= 15 * 33
    keep = f.astype(bool)
    o.insert(s[keep], d[keep], np.ones(int(keep.sum()), np.uint32))
    assert_same_edges(g, o)
    st = g.stats()
    assert st["live_edges"] == int(f.sum())
    assert st["pool_used"] <= 32
    assert g.pool_free() == st["pool_slabs"] - st["pool_used"]


def test_update_slab_pointers_figure_cases(cuda_lib):
    """The two cases of the paper's UpdateSlabPointers() figure: a marker at
    lane 14 of the first updated slab moves to lane 22 of the last slab, or to
    INVALID_LANE when the last slab is full; the updated flag is cleared."""
    mk = _mk()
    with open(os.path.join(GOLDEN, "update_slab_pointers.json")) as fh:
        cases = json.load(fh)["cases"]
    for case in cases:
        g = mk.Graph(1 << 12, buckets=1)
        v = 5
        # pairs occupy two lanes: lane L is the key lane of pair L/2
        before_pairs = case["before"]["lane"] // 2
        d0 = np.arange(100, 100 + before_pairs, dtype=np.uint32)
        g.insert(np.full(len(d0), v, np.uint32), d0, np.ones(len(d0), np.uint32))
        g.commit()
        slab0, lane0, upd0 = g.marker(v)
        assert (lane0, upd0) == (case["before"]["lane"], 0)
        # fill the rest of the marked slab, then the next slab up to `after`
        after = case["after"]["lane"]
        after_pairs = 15 if after == "INVALID" else after // 2
        n_new = (15 - before_pairs) + after_pairs
        d1 = np.arange(1000, 1000 + n_new, dtype=np.uint32)
        g.insert(np.full(n_new, v, np.uint32), d1, np.ones(n_new, np.uint32))
        slab1, lane1, upd1 = g.marker(v)
        assert (slab1, lane1, upd1) == (slab0, lane0, 1)
        g.commit()
        slab2, lane2, upd2 = g.marker(v)
        assert slab2 != slab0 and upd2 == 0
        assert lane2 == (mk.MK_INVALID_LANE if after == "INVALID" else after)


def test_duplicates_across_tiles_and_warps(cuda_lib):
    """Repeated (src, dst) pairs far apart in one batch (different 256-edge
    tiles and warps): exactly the first occurrence is applied, with its
    weight; the same for a delete batch with repeated pairs."""
    mk = _mk()
    V = 3000
    rng = np.random.default_rng(11)
    g = mk.Graph(V, edge_capacity_hint=200000, buckets=2)
    o = oracle.OracleGraph(V)
    base_s = rng.integers(0, V, 400).astype(np.uint32)
    base_d = rng.integers(0, V, 400).astype(np.uint32)
    reps = rng.integers(0, 400, 60000)
    s = base_s[reps]
    d = base_d[reps]
    w = rng.integers(1, 1000, len(s)).astype(np.uint32)
    q = rng.integers(0, 400, 5000)
    run_ops(g, o, [("ins", (s, d, w)), ("qry", (base_s, base_d)), ("commit", None),
                   ("del", (s[q].copy(), d[q].copy())), ("qry", (base_s, base_d))])


def test_mixed_single_and_shared_lists_in_warps(cuda_lib):
    """Each 32-edge warp holds both edges whose list appears once in it and
    lists with several edges (one bucket per vertex, a few hot sources), so
    both the 8-lane-group path and the whole-warp path run in one batch."""
    mk = _mk()
    V = 4096
    rng = np.random.default_rng(12)
    g = mk.Graph(V, edge_capacity_hint=100000, buckets=1)
    o = oracle.OracleGraph(V)
    hot = rng.integers(0, V, 8).astype(np.uint32)
    n = 40000
    s = np.where(rng.random(n) < 0.3, hot[rng.integers(0, 8, n)], rng.integers(0, V, n)).astype(np.uint32)
    d = rng.integers(0, V, n).astype(np.uint32)
    w = rng.integers(1, 100, n).astype(np.uint32)
    run_ops(g, o, [("ins", (s, d, w)), ("qry", (s, d)), ("commit", None),
                   ("del", (s[::3].copy(), d[::3].copy())), ("ins", (s[::2].copy(), d[::2].copy(), w[::2] + 1)),
                   ("qry", (s, d))])


def test_large_vertex_count_offsets(cuda_lib):
    """More than 4096 x 4096 vertices: the head offsets come from a
    two-level prefix sum; edges of the last vertices land in their lists."""
    mk = _mk()
    V = 4096 * 4096 + 5000
    g = mk.Graph(V, edge_capacity_hint=4096, buckets=2)
    assert g.stats()["lists"] == 2 * V
    # distinct new pairs: all stored; then all present with their weights
    s = np.array([V - 1, V - 2, 0, 4096 * 4096, 123456], np.uint32)
    d = np.array([0, V - 1, V - 1, 17, V - 3], np.uint32)
    w = np.array([5, 6, 7, 8, 9], np.uint32)
    assert np.array_equal(g.insert(s, d, w).cpu().numpy(), np.ones(5, np.uint8))
    bm, wt = g.query(s, d)
    assert mk.to_numpy_u32(bm)[0] == 0b11111
    assert np.array_equal(mk.to_numpy_u32(wt), w)
    absent_bm, _ = g.query(s, ((d.astype(np.uint64) + 2) % V).astype(np.uint32))
    assert mk.to_numpy_u32(absent_bm)[0] == 0
    assert g.last_error() == mk.MK_OK
