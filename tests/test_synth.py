"""Input generators: published SplitMix64 outputs, determinism and shapes."""
import numpy as np

import synth


def test_splitmix64_reference_outputs():
    # first outputs of SplitMix64 started from state 0 (Vigna's reference
    # splitmix64.c): 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f
    assert synth.splitmix_at(0, 0) == 0xE220A8397B1DCDAF
    assert synth.splitmix_at(0, 1) == 0x6E789E6AA1B965F4
    assert synth.splitmix_at(0, 2) == 0x06C45D188009454F


def test_generators_are_deterministic_and_in_range():
    a = synth.rmat_pairs(10, 5000, 7)
    b = synth.rmat_pairs(10, 5000, 7)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    assert a[0].max() < 1024 and a[1].max() < 1024
    w = synth.weights(10000, 3, 1, 100)
    assert w.min() >= 1 and w.max() <= 100
    assert len(np.unique(w)) == 100
    p = synth.permutation(1000, 9)
    assert np.array_equal(np.sort(p), np.arange(1000))


def test_rmat_quadrant_skew():
    s, d = synth.rmat_pairs(16, 200000, 11)
    # top bit of (src, dst) follows the first-level quadrant probabilities
    top_s = (s >> 15) & 1
    top_d = (d >> 15) & 1
    q = np.bincount(top_s * 2 + top_d, minlength=4) / len(s)
    assert np.allclose(q, [0.57, 0.19, 0.19, 0.05], atol=0.01)


def test_dedup_keeps_first_occurrence():
    s = np.array([1, 2, 1, 3, 3, 2], np.uint32)
    d = np.array([2, 2, 2, 3, 1, 2], np.uint32)
    ks, kd = synth.dedup_pairs(s, d, 8, drop_self=False)
    assert ks.tolist() == [1, 2, 3, 3] and kd.tolist() == [2, 2, 3, 1]
    ks, kd = synth.dedup_pairs(s, d, 8, drop_self=True)
    assert ks.tolist() == [1, 3] and kd.tolist() == [2, 1]


def test_grid_edge_count():
    s, d = synth.grid_pairs(4, 5)
    assert len(s) == 2 * (4 * 4 + 5 * 3)
    diff = np.abs(s.astype(int) - d.astype(int))
    assert set(diff.tolist()) == {1, 5}


def test_tiny_workload_shape():
    w = synth.tiny_workload()
    assert len(w.g_src) == 8192 and len(w.ins_src) == 1024
    assert len(w.del_src) == 1024 and len(w.q_src) == 4096
    assert w.g_w.min() >= 1 and w.g_w.max() <= 100


def test_powerlaw_stream_draws_live_deletes_and_half_live_queries():
    """Replayed on the oracle, every batch of the power-law stream deletes
    only live edges and has exactly half its queries present, at mixed batch
    sizes and far past the point where the initial edges are used up."""
    import oracle

    G = synth.powerlaw_graph(scale=13, draws=1 << 14)
    S = synth.PowerlawStream(G, max_batch=1 << 12)
    o = oracle.OracleGraph(G.V)
    o.insert(G.src, G.dst, G.w)
    E0 = len(G.src)
    total = 0
    for k, B in enumerate([256, 1 << 12, 1000, 1 << 12, 1 << 12, 7, 1 << 12] * 3):
        b = S.batch(B)
        assert b.k == k and len(b.ins_src) == len(b.del_src) == len(b.q_src) == B
        fi = o.insert(b.ins_src, b.ins_dst, b.ins_w)
        assert int(fi.sum()) == b.n_inserted
        assert o.delete(b.del_src, b.del_dst).all()
        bm, _ = o.query(b.q_src, b.q_dst)
        assert int(oracle.bitmap_to_bool(bm, B).sum()) == B // 2 == b.n_present
        assert o.num_edges == S.n_live == len(S.live)
        total += B
    assert total > 2 * E0


def test_edge_set_matches_a_python_set():
    rng = np.random.default_rng(1)
    es = synth.EdgeSet(4000)
    ref = set()
    for it in range(60):
        s = rng.integers(0, 40, 200).astype(np.uint32)
        d = rng.integers(0, 40, 200).astype(np.uint32)
        op = it % 3
        if op == 0:
            got = es.add(s, d)
        elif op == 1:
            got = es.remove(s, d)
        else:
            got = es.contains(s, d)
        want = []
        for a, b in zip(s.tolist(), d.tolist()):
            present = (a, b) in ref
            want.append(not present if op == 0 else present)
            if op == 0:
                ref.add((a, b))
            elif op == 1:
                ref.discard((a, b))
        assert got.tolist() == want
        assert len(es) == len(ref)


def test_serving_stream_live_window_on_the_oracle():
    """Replayed on the oracle in arrival order, the serving stream's inserts
    add exactly the predicted new edges, its deletes remove the predicted
    live ones, and its live-window queries are all present."""
    import oracle

    G = synth.powerlaw_graph(scale=12, draws=1 << 15)
    ring = synth.new_edge_pool(G, 1 << 17)
    R = synth.request_stream(600, G.V, len(G.src), len(ring.src), hi=1 << 11, n_sources=4, absent_pool=1 << 14)
    perm = synth.permutation(len(G.src), synth.substream(3100, 3))
    tail = min(R.hi, len(ring.src))
    ss = np.concatenate([G.src[perm], ring.src, ring.src[:tail]])
    sd = np.concatenate([G.dst[perm], ring.dst, ring.dst[:tail]])
    sw = np.concatenate([G.w[perm], ring.w, ring.w[:tail]])
    o = oracle.OracleGraph(G.V)
    o.insert(G.src, G.dst, G.w)
    n_present = 0
    for i in range(600):
        k, n, off = int(R.kind[i]), int(R.size[i]), int(R.offset[i])
        if k == 1:
            assert int(o.insert(ss[off:off + n], sd[off:off + n], sw[off:off + n]).sum()) == R.applied[i] == n
        elif k == 2:
            assert int(o.delete(ss[off:off + n], sd[off:off + n]).sum()) == R.applied[i]
        elif k == 0 and not R.qsrc[i] and n:
            bm, _ = o.query(ss[off:off + n], sd[off:off + n])
            assert oracle.bitmap_to_bool(bm, n).all()
            n_present += 1
    assert n_present > 50
    assert R.applied[R.kind == 2].sum() == R.size[R.kind == 2].sum()
