"""L2 persistence windows (mk_l2_window) change where lines live, never a
result: with a window over each part of the store on the stream, updates,
queries and SSSP match the oracle, and removing the window succeeds."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_l2_windows_keep_results_exact(cuda_lib):
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
    src = int(np.argmax(o.out_degree()))
    S = synth.PowerlawStream(G, max_batch=1 << 11)
    stream = torch.cuda.Stream()
    for region in (mk.MK_L2_VINFO, mk.MK_L2_HEADS, mk.MK_L2_POOL):
        info = g.l2_window(region, stream=stream)
        assert info["window_bytes"] > 0 and 0.0 < info["hit_ratio"] <= 1.0
        bt = S.batch(1 << 11)
        with torch.cuda.stream(stream):
            f = g.insert(bt.ins_src, bt.ins_dst, bt.ins_w, stream=stream)
            d, p = g.sssp(src, stream=stream)
            fd = g.delete(bt.del_src, bt.del_dst, stream=stream)
            d2, p2 = g.sssp(src, stream=stream)
            bm, w = g.query(bt.q_src, bt.q_dst, stream=stream)
            g.commit(stream=stream)
        stream.synchronize()
        assert np.array_equal(f.cpu().numpy(), o.insert(bt.ins_src, bt.ins_dst, bt.ins_w))
        od, op = o.sssp(src)
        assert np.array_equal(mk.to_numpy_u32(d), od) and np.array_equal(mk.to_numpy_u32(p), op)
        assert np.array_equal(fd.cpu().numpy(), o.delete(bt.del_src, bt.del_dst))
        od, op = o.sssp(src)
        assert np.array_equal(mk.to_numpy_u32(d2), od) and np.array_equal(mk.to_numpy_u32(p2), op)
        obm, ow = o.query(bt.q_src, bt.q_dst)
        assert np.array_equal(mk.to_numpy_u32(bm), obm) and np.array_equal(mk.to_numpy_u32(w), ow)
    info = g.l2_window(mk.MK_L2_NONE, stream=stream)
    assert info["window_bytes"] == 0
    assert g.last_error() == mk.MK_OK
    g.close()
