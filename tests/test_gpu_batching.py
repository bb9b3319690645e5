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


def update_requests(G, seed, count=40):
    """Mixed insert/delete requests with runs of one kind, empty requests,
    pairs repeated inside and across requests, and deletes of pairs that an
    earlier request of the same run inserted."""
    rng = np.random.default_rng(seed)
    out = []
    recent = []
    kinds = []
    while len(kinds) < count:
        kinds += [rng.choice(["insert", "delete"])] * int(rng.integers(1, 6))
    for kind in kinds[:count]:
        n = int(rng.choice([0, 1, 7, 64, 300, 2000]))
        pick = rng.integers(0, len(G.src), n)
        s = np.where(rng.random(n) < 0.5, G.src[pick], rng.integers(0, G.V, n)).astype(np.uint32)
        d = np.where(rng.random(n) < 0.5, G.dst[pick], rng.integers(0, G.V, n)).astype(np.uint32)
        if recent and n:
            k = min(n // 3, len(recent[-1][0]))
            s[:k], d[:k] = recent[-1][0][:k], recent[-1][1][:k]
        if kind == "insert":
            w = rng.integers(1, 100, n).astype(np.uint32)
            out.append(("insert", s, d, w))
        else:
            out.append(("delete", s, d))
        recent.append((s, d))
    return out


def test_update_multi_matches_one_call_per_request(cuda_lib):
    """mk_update_multi (runs merged into one staged batch each) against one
    mk_insert_batch / mk_delete_batch per request and the oracle: every
    request's flags, the final edge set, and incremental SSSP/BFS/WCC after
    the merged updates (the change log and the UpdateIterator markers)."""
    torch, mk, G, g, o = _setup()
    b = mk.bucket_rule(G.V, G.src, 0.7)
    ref = mk.Graph(G.V, edge_capacity_hint=len(G.src) * 2, buckets=b)
    ref.insert(G.src, G.dst, G.w)
    ref.commit()
    src = int(np.argmax(np.bincount(G.src, minlength=G.V)))
    for x in (g, ref):
        x.sssp(src)
        x.bfs(src)
        x.wcc()
        x.commit()
    for part in range(3):
        reqs = update_requests(G, 20 + part)
        flags = g.update_multi(reqs)
        for req, f in zip(reqs, flags):
            if req[0] == "insert":
                rf = ref.insert(req[1], req[2], req[3])
                of = o.insert(req[1], req[2], req[3])
            else:
                rf = ref.delete(req[1], req[2])
                of = o.delete(req[1], req[2])
            assert np.array_equal(f.cpu().numpy(), of) and torch.equal(f, rf)
        for x in (g, ref):
            d, p = x.sssp(src)
            assert np.array_equal(mk.to_numpy_u32(d), o.sssp(src)[0])
            assert np.array_equal(mk.to_numpy_u32(p), o.sssp(src)[1])
            d, p = x.bfs(src)
            assert np.array_equal(mk.to_numpy_u32(d), o.bfs(src)[0])
            assert np.array_equal(mk.to_numpy_u32(x.wcc()), o.wcc())
            x.commit()
    es, ed, ew = g.export()
    os_, od, ow = o.export()
    assert np.array_equal(mk.to_numpy_u32(es), os_) and np.array_equal(mk.to_numpy_u32(ed), od)
    assert np.array_equal(mk.to_numpy_u32(ew), ow)
    assert g.last_error() == mk.MK_OK and ref.last_error() == mk.MK_OK
    # no request flags asked for, and an empty list
    g.update_multi(update_requests(G, 30), flags=False)
    g.update_multi([])
    assert g.last_error() == mk.MK_OK
