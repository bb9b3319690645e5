"""Learned slab sizing on the GPU: the network's forward pass, gradient,
features and targets against the float64 oracle (same bf16-rounded
weights, same inputs drawn on the host), training lowers the loss, and on a
growth stream the learned bucket counts shorten the chains a query walks
while every result stays identical to the oracle."""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


def _mods():
    import torch

    import paper_2305_17813_gb300 as mk
    from paper_2305_17813_gb300 import sizing

    mk.load()
    return torch, mk, sizing


def test_forward_and_gradient_match_oracle(cuda_lib):
    torch, mk, sizing = _mods()
    m = sizing.SizingModel(seed=3)
    rng = np.random.default_rng(0)
    P = (rng.normal(0, 0.2, omlp.NPARAMS)).astype(np.float32)
    m.set_params(P)
    assert np.array_equal(m.params(), P)
    for n in (1, 127, 128, 1000, 5000):
        X = rng.normal(0, 1, (n, 8)).astype(np.float32)
        T = rng.normal(0, 1, n).astype(np.float32)
        Xd = torch.from_numpy(X).cuda()
        Td = torch.from_numpy(T).cuda()
        y = m.forward(Xd).cpu().numpy().astype(np.float64)
        y_ref = omlp.forward(P, X)
        # fp32 accumulation of <= 64-term dot products of O(1) values
        assert np.allclose(y, y_ref, rtol=1e-5, atol=1e-5 * (1 + np.abs(y_ref).max()))
        G, sse = m.gradient(Xd, Td)
        g = G.cpu().numpy().astype(np.float64)
        g_ref, sse_ref = omlp.gradient(P, X, T)
        scale = np.abs(g_ref).max()
        assert np.allclose(g, g_ref, rtol=1e-4, atol=1e-5 * scale), (n, np.abs(g - g_ref).max(), scale)
        assert np.isclose(float(sse.item()), sse_ref, rtol=1e-5)


def test_features_and_targets_match_oracle(cuda_lib):
    torch, mk, sizing = _mods()
    rng = np.random.default_rng(1)
    V = 10007
    hist = np.sort(rng.integers(0, 500, (5, V)), axis=0)[::-1].astype(np.uint32).copy()
    hist[:, :100] = 0
    ind = rng.integers(0, 800, V).astype(np.uint32)
    bk = rng.integers(1, 50, V).astype(np.uint32)
    tr = sizing.DegreeTrace(V)
    tr.hist.copy_(torch.from_numpy(hist.view(np.int32)))
    tr.in_deg.copy_(torch.from_numpy(ind.view(np.int32)))
    X = tr.features(mk.to_device_u32(bk)).cpu().numpy()
    X_ref = omlp.features(hist, ind, bk)
    assert np.allclose(X, X_ref, rtol=2e-6, atol=2e-6)
    T = sizing.growth_targets(mk.to_device_u32(hist[4]), mk.to_device_u32(hist[0]), 4.0).cpu().numpy()
    assert np.allclose(T, omlp.growth_targets(hist[4], hist[0], 4.0), rtol=2e-6, atol=2e-6)


def test_degree_trace_counts_flagged_edges(cuda_lib):
    torch, mk, sizing = _mods()
    V = 64
    tr = sizing.DegreeTrace(V)
    s = mk.to_device_u32([1, 1, 2, 3, 1])
    d = mk.to_device_u32([2, 3, 3, 1, 2])
    f = torch.tensor([1, 1, 0, 1, 1], dtype=torch.uint8, device="cuda")
    tr.apply(s, d, f, +1)
    tr.apply(s[:1], d[:1], None, -1)
    out = tr.out_deg.cpu().numpy()
    inn = tr.in_deg.cpu().numpy()
    assert out[1] == 2 and out[2] == 0 and out[3] == 1
    assert inn[2] == 1 and inn[3] == 1 and inn[1] == 1


def test_training_lowers_the_loss(cuda_lib):
    torch, mk, sizing = _mods()
    rng = np.random.default_rng(2)
    X = rng.normal(0, 1, (20000, 8)).astype(np.float32)
    T = (np.log1p(np.abs(X[:, 0] * 2 + X[:, 1])) + 0.1 * X[:, 2]).astype(np.float32)
    m = sizing.SizingModel(seed=1)
    losses = m.train(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), epochs=15, batch=2048, lr=3e-3)
    assert losses[-1] < 0.2 * losses[0], losses


def test_learned_sizing_shortens_chains_with_identical_results(cuda_lib):
    import bench
    import synth

    torch, mk, sizing = _mods()
    S = synth.growth_stream(scale=15, draws=1 << 19, n_batches=16)
    res = bench.growth_experiment(S, split=8, horizon=2, epochs=12, keep_graphs=True)
    gl, gr = res.pop("graphs")
    # identical results on both layouts, and identical to the oracle
    o = oracle.OracleGraph(S.V)
    o.insert(S.init.src, S.init.dst, S.init.w)
    for b in S.batches:
        o.insert(b.ins_src, b.ins_dst, b.ins_w)
        o.delete(b.del_src, b.del_dst)
    os_, od, ow = o.export()
    for g in (gl, gr):
        s, d, w = g.export()
        assert np.array_equal(mk.to_numpy_u32(s), os_) and np.array_equal(mk.to_numpy_u32(d), od)
        assert np.array_equal(mk.to_numpy_u32(w), ow)
        dist, par = g.sssp(res["source"])
        od_, op_ = o.sssp(res["source"])
        assert np.array_equal(mk.to_numpy_u32(dist), od_) and np.array_equal(mk.to_numpy_u32(par), op_)
        assert g.last_error() == mk.MK_OK
    # what the network gains over the load-factor rule
    assert res["learned"]["query_slabs_per_query"] < res["rule"]["query_slabs_per_query"], res
    assert res["learned"]["chain_max"] <= res["rule"]["chain_max"], res
    assert res["train_losses"][-1] < res["train_losses"][0]
