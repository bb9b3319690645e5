"""Serving engine: each request's result is the same alone (plain, one
launch per request in arrival order) and in the mix (continuous batching:
merged query groups in CUDA graphs, SSSP on a second stream, updates as
barriers), and both equal a sequential replay on the CPU oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _served_against_oracle(scale, draws, ring_draws, n_req, hi, n_sources, absent_pool, max_inflight, commit_every):
    import bench
    import paper_2305_17813_gb300 as mk

    G = synth.powerlaw_graph(scale=scale, draws=draws)
    ring = synth.new_edge_pool(G, ring_draws)
    R = synth.request_stream(n_req, G.V, len(G.src), len(ring.src), hi=hi, n_sources=n_sources,
                             absent_pool=absent_pool)
    res = bench.serve_experiment(G, R, ring, rate_fracs=(0.5,), max_inflight=max_inflight, commit_every=commit_every,
                                 retain_every=1, retain_sssp_every=1, keep_outputs=True)
    store_p, store_s = res["outputs"]
    inputs = res["inputs"]
    assert res["compared_requests"] == n_req and res["mismatches"] == 0
    # sequential oracle replay
    o = oracle.OracleGraph(G.V)
    o.insert(G.src, G.dst, G.w)
    for i in range(n_req):
        k = int(R.kind[i])
        a, b, w = inputs(i)
        got = store_s[i]
        if k == 0:
            obm, _ = o.query(mk.to_numpy_u32(a), mk.to_numpy_u32(b))
            assert np.array_equal(mk.to_numpy_u32(got[0]), obm), i
            if not R.qsrc[i] and int(R.size[i]):
                # live-window queries are all present
                assert oracle.bitmap_to_bool(obm, int(R.size[i])).all(), i
        elif k == 1:
            f = o.insert(mk.to_numpy_u32(a), mk.to_numpy_u32(b), mk.to_numpy_u32(w))
            assert np.array_equal(got[0].cpu().numpy(), f), i
            assert int(f.sum()) == int(R.applied[i]), i  # the stream's live window predicts the new edges
        elif k == 2:
            f = o.delete(mk.to_numpy_u32(a), mk.to_numpy_u32(b))
            assert np.array_equal(got[0].cpu().numpy(), f), i
            assert int(f.sum()) == int(R.applied[i]), i
        else:
            od, op = o.sssp(int(R.source[i]))
            assert np.array_equal(mk.to_numpy_u32(got[0]), od) and np.array_equal(mk.to_numpy_u32(got[1]), op), i
    assert res["capacity"]["served"]["requests_per_s"] > 0
    return res


def test_served_mix_equals_requests_alone_and_oracle(cuda_lib):
    _served_against_oracle(scale=12, draws=1 << 15, ring_draws=1 << 17, n_req=400, hi=1 << 12, n_sources=4,
                           absent_pool=1 << 14, max_inflight=16, commit_every=3)


def test_served_mix_mid_scale(cuda_lib):
    """The served workload's shape at R-MAT scale 16 (0.9 M edges): 2,000
    requests of up to 2^14 edges, every result against the oracle."""
    _served_against_oracle(scale=16, draws=1 << 20, ring_draws=1 << 21, n_req=2000, hi=1 << 14, n_sources=8,
                           absent_pool=1 << 16, max_inflight=64, commit_every=8)
