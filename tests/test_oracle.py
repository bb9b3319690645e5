"""Pins for the CPU oracle against facts that do not come from the oracle.

Each test checks the oracle against an independent computation: a brute-force
bit-matrix model, Floyd-Warshall, transitive closure, a library routine, a
closed form or an invariant fixed by the definitions the oracle follows
(edge-set semantics of the store; the shortest-path tree with min-id tight
parents; weakly connected components labelled by their smallest vertex).
"""
import numpy as np
import pytest

import oracle
import synth

NONE = 0xFFFFFFFF


def _rng(seed):
    return np.random.default_rng(seed)


# ----------------------------------------------------------------- edge set

class BitMatrixModel:
    """Brute-force store model for V <= 64: a presence matrix and a weight
    matrix, updated one operation at a time."""

    def __init__(self, V):
        self.present = np.zeros((V, V), bool)
        self.weight = np.zeros((V, V), np.int64)

    def insert(self, s, d, w):
        out = []
        for a, b, c in zip(s, d, w):
            if self.present[a, b]:
                out.append(0)
            else:
                self.present[a, b] = True
                self.weight[a, b] = c
                out.append(1)
        return np.array(out, np.uint8)

    def delete(self, s, d):
        out = []
        for a, b in zip(s, d):
            out.append(int(self.present[a, b]))
            self.present[a, b] = False
        return np.array(out, np.uint8)


@pytest.mark.parametrize("seed", range(6))
def test_store_matches_bit_matrix_model(seed):
    rng = _rng(seed)
    V = int(rng.integers(2, 65))
    g = oracle.OracleGraph(V)
    m = BitMatrixModel(V)
    for step in range(12):
        n = int(rng.integers(0, 200))
        s = rng.integers(0, V, n).astype(np.uint32)
        d = rng.integers(0, V, n).astype(np.uint32)
        op = step % 3
        if op == 0:
            w = rng.integers(1, 100, n).astype(np.uint32)
            assert np.array_equal(g.insert(s, d, w), m.insert(s, d, w))
        elif op == 1:
            assert np.array_equal(g.delete(s, d), m.delete(s, d))
        else:
            bm, w = g.query(s, d)
            hit = oracle.bitmap_to_bool(bm, n)
            assert np.array_equal(hit, m.present[s, d])
            assert np.array_equal(w, np.where(m.present[s, d], m.weight[s, d], 0))
        es, ed, ew = g.export()
        ref_s, ref_d = np.nonzero(m.present)  # row-major = sorted by (src, dst)
        assert np.array_equal(es, ref_s) and np.array_equal(ed, ref_d)
        assert np.array_equal(ew, m.weight[ref_s, ref_d])
        assert g.num_edges == int(m.present.sum())
        assert int(g.out_degree().sum()) == g.num_edges
        # out-degree = row sums of the adjacency bit matrix (column sums
        # would be the in-degree)
        assert np.array_equal(g.out_degree(), m.present.sum(axis=1))


def test_out_degree_of_an_out_star_and_an_in_star():
    """Vertex 0 points at 1..5 and vertices 2..4 point at 6: out-degree
    counts edges by their source only."""
    g = oracle.OracleGraph(8)
    g.insert([0, 0, 0, 0, 0, 2, 3, 4], [1, 2, 3, 4, 5, 6, 6, 6])
    assert g.out_degree().tolist() == [5, 0, 1, 1, 1, 0, 0, 0]


def test_first_occurrence_wins_within_a_batch():
    g = oracle.OracleGraph(4)
    f = g.insert([1, 1, 1], [2, 2, 2], [7, 3, 9])
    assert f.tolist() == [1, 0, 0]
    assert g.query([1], [2])[1].tolist() == [7]
    # an insert of a present edge keeps the stored weight
    assert g.insert([1], [2], [1]).tolist() == [0]
    assert g.query([1], [2])[1].tolist() == [7]
    # repeated deletes: only the first one removes the edge
    assert g.delete([1, 1], [2, 2]).tolist() == [1, 0]


def test_deleting_every_present_edge_empties_the_graph():
    w = synth.tiny_workload()
    g = oracle.OracleGraph(w.V)
    g.insert(w.g_src, w.g_dst, w.g_w)
    s, d, _ = g.export()
    perm = np.random.default_rng(0).permutation(len(s))
    assert g.delete(s[perm], d[perm]).all()
    assert g.num_edges == 0
    assert g.export()[0].size == 0


def test_flags_agree_with_prior_membership():
    w = synth.tiny_workload()
    g = oracle.OracleGraph(w.V)
    g.insert(w.g_src, w.g_dst, w.g_w)
    before = oracle.bitmap_to_bool(g.query(w.ins_src, w.ins_dst)[0], len(w.ins_src))
    f = g.insert(w.ins_src, w.ins_dst, w.ins_w)
    # a pair absent before the batch is stored by its first occurrence only
    key = w.ins_src.astype(np.uint64) << np.uint64(32) | w.ins_dst
    _, first = np.unique(key, return_index=True)
    expect = np.zeros(len(key), np.uint8)
    expect[first] = 1
    expect &= ~before
    assert np.array_equal(f, expect)


# ------------------------------------------------------- BFS / SSSP pins

def floyd_warshall(V, s, d, w):
    inf = np.iinfo(np.int64).max // 4
    D = np.full((V, V), inf, np.int64)
    np.fill_diagonal(D, 0)
    for a, b, c in zip(s, d, w):
        if a != b:
            D[a, b] = min(D[a, b], c)
    for k in range(V):
        D = np.minimum(D, D[:, [k]] + D[[k], :])
    return D, inf


def min_tight_parent(V, src, s, d, w, dist, inf):
    par = np.full(V, NONE, np.int64)
    for a, b, c in zip(s, d, w):
        if b == src or dist[a] >= inf or dist[b] >= inf:
            continue
        if dist[a] + c == dist[b]:
            par[b] = min(par[b], a)
    par[src] = src
    return par


@pytest.mark.parametrize("seed", range(8))
def test_sssp_and_bfs_match_floyd_warshall(seed):
    rng = _rng(100 + seed)
    V = int(rng.integers(2, 48))
    n = int(rng.integers(0, 4 * V))
    s = rng.integers(0, V, n).astype(np.uint32)
    d = rng.integers(0, V, n).astype(np.uint32)
    w = rng.integers(1, 20, n).astype(np.uint32)
    g = oracle.OracleGraph(V)
    g.insert(s, d, w)
    es, ed, ew = g.export()
    src = int(rng.integers(0, V))
    for unit in (False, True):
        ww = np.ones_like(ew) if unit else ew
        D, inf = floyd_warshall(V, es, ed, ww)
        dist_ref = D[src]
        dist, par = g.bfs(src) if unit else g.sssp(src)
        expect_dist = np.where(dist_ref >= inf, NONE, dist_ref)
        assert np.array_equal(dist.astype(np.int64), expect_dist)
        expect_par = min_tight_parent(V, src, es, ed, ww, dist_ref, inf)
        assert np.array_equal(par.astype(np.int64), expect_par)


def test_grid_unit_weights_closed_form():
    rows, cols = 37, 53
    s, d = synth.grid_pairs(rows, cols)
    g = oracle.OracleGraph(rows * cols)
    g.insert(s, d, np.ones(len(s), np.uint32))
    r, c = np.divmod(np.arange(rows * cols), cols)
    for dist, par in (g.bfs(0), g.sssp(0)):
        assert np.array_equal(dist, r + c)
        # min-id tight predecessor: the upper neighbour (v - cols) when r > 0,
        # else the left neighbour
        expect = np.where(r > 0, np.arange(rows * cols) - cols, np.arange(rows * cols) - 1)
        expect[0] = 0
        assert np.array_equal(par.astype(np.int64), expect)
    assert np.all(g.wcc() == 0)


def test_path_graph_prefix_sums_and_star():
    V = 200
    w = synth.weights(V - 1, 5, 1, 1000)
    g = oracle.OracleGraph(V)
    g.insert(np.arange(V - 1), np.arange(1, V), w)
    dist, par = g.sssp(0)
    assert np.array_equal(dist[1:], np.cumsum(w.astype(np.int64)))
    assert dist[0] == 0 and par[0] == 0
    assert np.array_equal(par[1:], np.arange(V - 1))
    # from the middle: vertices before it are unreachable
    dist, par = g.sssp(100)
    assert np.all(dist[:100] == NONE) and np.all(par[:100] == NONE)
    star = oracle.OracleGraph(V)
    star.insert(np.zeros(V - 1), np.arange(1, V), w)
    dist, par = star.sssp(0)
    assert np.array_equal(dist[1:], w) and np.all(par[1:] == 0)
    dist, _ = star.bfs(0)
    assert np.all(dist[1:] == 1)


def test_tree_invariants_on_power_law_graph():
    g_in = synth.powerlaw_graph(scale=12, draws=1 << 16)
    g = oracle.OracleGraph(g_in.V)
    g.insert(g_in.src, g_in.dst, g_in.w)
    s, d, w = g.export()
    src = int(np.argmax(g.out_degree()))
    for unit in (False, True):
        dist, par = g.bfs(src) if unit else g.sssp(src)
        ww = np.ones_like(w, dtype=np.int64) if unit else w.astype(np.int64)
        du = dist[s].astype(np.int64)
        dv = dist[d].astype(np.int64)
        reach_u = dist[s] != NONE
        # triangle inequality on every live edge out of a reachable vertex
        assert np.all(dv[reach_u] <= du[reach_u] + ww[reach_u])
        # no live edge leaves the reachable set
        assert np.all(dist[d][reach_u] != NONE)
        # every reachable non-source vertex's parent edge is live and tight
        key = s.astype(np.uint64) << np.uint64(32) | d
        wmap = dict(zip(key.tolist(), ww.tolist()))
        for v in np.nonzero((dist != NONE))[0][:2000]:
            if v == src:
                assert par[v] == src and dist[v] == 0
                continue
            p = int(par[v])
            k = (p << 32) | int(v)
            assert k in wmap and int(dist[p]) + wmap[k] == int(dist[v])
        assert np.all(par[dist == NONE] == NONE)


# ------------------------------------------------------------------- WCC

@pytest.mark.parametrize("seed", range(6))
def test_wcc_matches_transitive_closure(seed):
    rng = _rng(200 + seed)
    V = int(rng.integers(1, 64))
    n = int(rng.integers(0, V + 5))
    s = rng.integers(0, V, n).astype(np.uint32)
    d = rng.integers(0, V, n).astype(np.uint32)
    g = oracle.OracleGraph(V)
    g.insert(s, d)
    R = np.eye(V, dtype=bool)
    R[s, d] = True
    R[d, s] = True
    for _ in range(V):
        R = R | ((R.astype(np.int32) @ R.astype(np.int32)) > 0)
    expect = np.array([int(np.nonzero(R[v])[0].min()) for v in range(V)])
    assert np.array_equal(g.wcc(), expect)


def test_wcc_partition_matches_library_components():
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components

    g_in = synth.powerlaw_graph(scale=13, draws=1 << 14)
    g = oracle.OracleGraph(g_in.V)
    g.insert(g_in.src, g_in.dst, g_in.w)
    lab = g.wcc()
    A = coo_matrix((np.ones(len(g_in.src)), (g_in.src, g_in.dst)), shape=(g_in.V, g_in.V))
    nc, comp = connected_components(A, directed=True, connection="weak")
    assert len(np.unique(lab)) == nc
    # same partition: the map component -> label is a bijection
    pairs = np.unique(np.stack([comp, lab]), axis=1)
    assert pairs.shape[1] == nc
    # each label is the smallest member of its class
    first = np.full(nc, g_in.V)
    np.minimum.at(first, comp, np.arange(g_in.V))
    assert np.array_equal(lab, first[comp])


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_sharded_cpu_baseline_matches_the_oracle(threads):
    """The all-cores CPU baseline (edge set sharded by source, one thread per
    shard) gives the oracle's flags, hits and weights on mixed batches with
    repeated pairs."""
    from oracle.sharded import ShardedGraph

    rng = _rng(40 + threads)
    V = 300
    o, p = oracle.OracleGraph(V), ShardedGraph(V, threads)
    for step in range(9):
        n = 5000
        s = rng.integers(0, V, n).astype(np.uint32)
        d = rng.integers(0, V // 10, n).astype(np.uint32)
        if step % 3 == 0:
            w = rng.integers(1, 100, n).astype(np.uint32)
            assert np.array_equal(p.insert(s, d, w), o.insert(s, d, w))
        elif step % 3 == 1:
            assert np.array_equal(p.delete(s, d), o.delete(s, d))
        else:
            hit, w = p.query(s, d)
            obm, ow = o.query(s, d)
            assert np.array_equal(hit.astype(bool), oracle.bitmap_to_bool(obm, n))
            assert np.array_equal(w, ow)
        assert p.num_edges == o.num_edges


def _dense_pagerank(V, s, d, damping):
    """Closed form of the PageRank fixpoint: (I - d M) x = (1 - d) / V * 1,
    M[v, u] = 1 / out(u) per edge u -> v, and 1 / V in every row for a
    column u without out-edges (the teleport term)."""
    M = np.zeros((V, V))
    out = np.bincount(s, minlength=V)
    for u, v in zip(s, d):
        M[v, u] += 1.0 / out[u]
    M[:, out == 0] = 1.0 / V
    return np.linalg.solve(np.eye(V) - damping * M, np.full(V, (1 - damping) / V))


@pytest.mark.parametrize("seed", range(4))
def test_pagerank_matches_the_closed_form(seed):
    rng = _rng(70 + seed)
    V = int(rng.integers(3, 41))
    n = int(rng.integers(1, 4 * V))
    s = rng.integers(0, V, n).astype(np.uint32)
    d = rng.integers(0, V, n).astype(np.uint32)
    g = oracle.OracleGraph(V)
    g.insert(s, d)
    es, ed, _ = g.export()
    for damping in (0.85, 0.5):
        pr, it = g.pagerank(damping=damping, eps=1e-15, max_iter=5000)
        assert np.allclose(pr, _dense_pagerank(V, es, ed, damping), rtol=0, atol=1e-12)
        assert abs(pr.sum() - 1.0) < 1e-12
    # a warm start at the fixpoint stops after one step
    pr, _ = g.pagerank(eps=1e-14, max_iter=5000)
    _, it = g.pagerank(eps=1e-12, init=pr)
    assert it == 1


def test_pagerank_of_a_cycle_is_uniform_and_a_sink_takes_the_teleport():
    g = oracle.OracleGraph(5)
    g.insert([0, 1, 2, 3, 4], [1, 2, 3, 4, 0])
    pr, _ = g.pagerank()
    assert np.allclose(pr, 0.2, atol=1e-13)
    # 0 -> 1 and a sink 1: PR1 = (1-d)/2 + d (PR0 + PR1/2), PR0 = (1-d)/2 + d PR1/2
    g = oracle.OracleGraph(2)
    g.insert([0], [1])
    pr, _ = g.pagerank(damping=0.85)
    p1 = (1 - 0.85) / 2 + 0.85 * (pr[0] + pr[1] / 2)
    assert np.isclose(pr[1], p1, atol=1e-13) and np.isclose(pr.sum(), 1.0, atol=1e-13)
    assert np.isclose(pr[0], 0.15 / 2 + 0.85 * pr[1] / 2, atol=1e-13)


def test_triangles_closed_forms_and_brute_force():
    # complete graph K_n (one direction only: the count ignores direction)
    for n in (3, 4, 7):
        g = oracle.OracleGraph(n)
        s, d = np.triu_indices(n, 1)
        g.insert(s.astype(np.uint32), d.astype(np.uint32))
        assert g.triangles() == n * (n - 1) * (n - 2) // 6
    # wheel: hub 0 joined to a cycle of n rim vertices has n triangles
    n = 9
    rim = np.arange(1, n + 1)
    g = oracle.OracleGraph(n + 1)
    g.insert(np.zeros(n, np.uint32), rim.astype(np.uint32))
    g.insert(rim.astype(np.uint32), (rim % n + 1).astype(np.uint32))
    g.insert([3], [3])  # a self-loop adds nothing
    assert g.triangles() == n
    # a grid and a bipartite graph have none
    g = oracle.OracleGraph(64)
    gs, gd = synth.grid_pairs(8, 8)
    g.insert(gs, gd)
    assert g.triangles() == 0
    # brute force over all triples on random small graphs, both directions
    for seed in range(5):
        rng = _rng(90 + seed)
        V = int(rng.integers(4, 30))
        n = int(rng.integers(0, 3 * V))
        s = rng.integers(0, V, n).astype(np.uint32)
        d = rng.integers(0, V, n).astype(np.uint32)
        g = oracle.OracleGraph(V)
        g.insert(s, d)
        A = np.zeros((V, V), bool)
        A[s, d] = True
        A |= A.T
        np.fill_diagonal(A, False)
        brute = sum(1 for a in range(V) for b in range(a + 1, V) for c in range(b + 1, V)
                    if A[a, b] and A[b, c] and A[a, c])
        assert g.triangles() == brute
