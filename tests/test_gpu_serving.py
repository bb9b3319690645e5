"""Serving engine: each request's result is the same alone (plain, one
launch per request in arrival order) and in the mix (continuous batching:
merged query groups in CUDA graphs, SSSP on a second stream, updates as
barriers), and both equal a sequential replay on the CPU oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_served_mix_equals_requests_alone_and_oracle(cuda_lib):
    import bench
    import paper_2305_17813_gb300 as mk

    G = synth.powerlaw_graph(scale=12, draws=1 << 15)
    R = synth.request_stream(400, G.V, len(G.src), hi=1 << 12, n_sources=4, query_pool=1 << 14,
                             insert_pool=1 << 14)
    res = bench.serve_experiment(G, R, rate_fracs=(0.5,), max_inflight=16, commit_every=3, retain_every=1,
                                 retain_sssp_every=1, keep_outputs=True, query_pool=1 << 14, insert_pool=1 << 14)
    store_p, store_s = res["outputs"]
    inputs = res["inputs"]
    assert res["compared_requests"] == 400 and res["mismatches"] == 0
    # sequential oracle replay
    o = oracle.OracleGraph(G.V)
    o.insert(G.src, G.dst, G.w)
    for i in range(400):
        k = int(R.kind[i])
        a, b, w = inputs(i)
        got = store_s[i]
        if k == 0:
            obm, _ = o.query(mk.to_numpy_u32(a), mk.to_numpy_u32(b))
            assert np.array_equal(mk.to_numpy_u32(got[0]), obm), i
        elif k == 1:
            f = o.insert(mk.to_numpy_u32(a), mk.to_numpy_u32(b), mk.to_numpy_u32(w))
            assert np.array_equal(got[0].cpu().numpy(), f), i
        elif k == 2:
            f = o.delete(mk.to_numpy_u32(a), mk.to_numpy_u32(b))
            assert np.array_equal(got[0].cpu().numpy(), f), i
        else:
            od, op = o.sssp(int(R.source[i]))
            assert np.array_equal(mk.to_numpy_u32(got[0]), od) and np.array_equal(mk.to_numpy_u32(got[1]), op), i
    assert res["capacity"]["served"]["requests_per_s"] > 0
