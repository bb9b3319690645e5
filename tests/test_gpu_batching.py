"""Batched execution: the multi-request query launch, the CUDA-graph
batcher and every kernel shape the autotuner can pick give results
identical to one plain query launch per request (and to the oracle)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _setup():
    import torch

    import paper_2305_17813_gb300 as mk

    mk.load()
    G = synth.powerlaw_graph(scale=13, draws=1 << 17)
    b = mk.bucket_rule(G.V, G.src, 0.7)
    g = mk.Graph(G.V, edge_capacity_hint=len(G.src) * 2, buckets=b)
    g.insert(G.src, G.dst, G.w)
    g.commit()
    o = oracle.OracleGraph(G.V)
    o.insert(G.src, G.dst, G.w)
    return torch, mk, G, g, o


def requests(G, sizes, seed):
    rng = np.random.default_rng(seed)
    out = []
    for n in sizes:
        pick = rng.integers(0, len(G.src), n)
        s = np.where(rng.random(n) < 0.5, G.src[pick], rng.integers(0, G.V, n)).astype(np.uint32)
        d = np.where(rng.random(n) < 0.5, G.dst[pick], rng.integers(0, G.V, n)).astype(np.uint32)
        out.append((s, d))
    return out


def test_multi_request_launch_matches_plain_queries(cuda_lib):
    torch, mk, G, g, o = _setup()
    reqs = requests(G, [1, 31, 32, 33, 1000, 5000, 0, 77, 4096], 1)
    multi = g.query_multi(reqs)
    for (s, d), (bm, w) in zip(reqs, multi):
        if len(s) == 0:
            continue
        pbm, pw = g.query(s, d)
        obm, ow = o.query(s, d)
        assert np.array_equal(mk.to_numpy_u32(bm), obm) and np.array_equal(mk.to_numpy_u32(w), ow)
        assert torch.equal(bm, pbm) and torch.equal(w, pw)
    assert g.last_error() == mk.MK_OK


def test_graph_batcher_ticks_match_oracle(cuda_lib):
    torch, mk, G, g, o = _setup()
    b = mk.Batcher(g, max_requests=64)
    for tick in range(4):
        reqs = requests(G, [3 + tick, 1000 * (tick + 1), 64, 129], 10 + tick)
        bufs = []
        for s, d in reqs:
            ts, td = mk.to_device_u32(s), mk.to_device_u32(d)
            bm = torch.full(((len(s) + 31) // 32,), -1, dtype=torch.int32, device="cuda")
            w = torch.full((len(s),), -1, dtype=torch.int32, device="cuda")
            b.add_query(ts, td, bm, w)
            bufs.append((ts, td, bm, w))
        b.launch()
        torch.cuda.synchronize()
        for (s, d), (_, _, bm, w) in zip(reqs, bufs):
            obm, ow = o.query(s, d)
            assert np.array_equal(mk.to_numpy_u32(bm), obm) and np.array_equal(mk.to_numpy_u32(w), ow)
    b.close()
    assert g.last_error() == mk.MK_OK


def test_every_tuned_shape_gives_identical_results(cuda_lib):
    torch, mk, G, g, o = _setup()
    (s, d), = requests(G, [20000], 5)
    obm, ow = o.query(s, d)
    src = int(np.argmax(o.out_degree()))
    od, op = o.bfs(src)
    for grp in (4, 8, 16, 32):
        for blk in (128, 256, 512):
            g.set_tuning(grp, blk, 0)
            bm, w = g.query(s, d)
            assert np.array_equal(mk.to_numpy_u32(bm), obm) and np.array_equal(mk.to_numpy_u32(w), ow), (grp, blk)
    deg = o.out_degree()
    for bps, v in zip((1, 2, 3), np.argsort(deg)[::-1][1:4]):
        g.set_tuning(8, 256, bps)
        dist, par = g.bfs(int(v))  # a new source: a static run through the round kernel
        vd, vp = o.bfs(int(v))
        assert np.array_equal(mk.to_numpy_u32(dist), vd) and np.array_equal(mk.to_numpy_u32(par), vp), bps
    t = g.autotune(s, d, src)
    assert t["query_group"] in (4, 8, 16, 32) and t["query_block"] in (128, 256, 512)
    assert t["rounds_blocks_per_sm"] >= 1
    assert g.tuning()["query_group"] == t["query_group"]
    bm, w = g.query(s, d)
    assert np.array_equal(mk.to_numpy_u32(bm), obm)
    dist, par = g.bfs(src)
    assert np.array_equal(mk.to_numpy_u32(dist), od) and np.array_equal(mk.to_numpy_u32(par), op)
    assert g.last_error() == mk.MK_OK
