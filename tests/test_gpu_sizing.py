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


def test_adam_steps_match_oracle(cuda_lib):
    """Two Adam steps of the device (mk_mlp_adam_step: gradient kernel, then
    the update kernel with bias corrections for steps 1 and 2) against the
    float64 Adam of the oracle applied to the oracle's gradients.  The
    device works in fp32, so where a gradient is tiny against the largest
    one its sign can differ; there the step is only bounded by lr."""
    torch, mk, sizing = _mods()
    rng = np.random.default_rng(4)
    P = rng.normal(0, 0.2, omlp.NPARAMS).astype(np.float32)
    m = sizing.SizingModel(seed=5)
    m.set_params(P)  # also clears the moments
    lr = 1e-2
    Pr, Mr, Vr = P.astype(np.float64), np.zeros(omlp.NPARAMS), np.zeros(omlp.NPARAMS)
    sse = torch.zeros(1, dtype=torch.float64, device="cuda")
    for t in (1, 2):
        X = rng.normal(0, 1, (3000, 8)).astype(np.float32)
        T = rng.normal(0, 1, 3000).astype(np.float32)
        # the oracle's gradient at the device's current masters
        g_ref, _ = omlp.gradient(m.params(), X, T)
        Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
        mk.check(m.lib.mk_mlp_adam_step(m._h, sizing._p(Xd), sizing._p(Td), 3000, lr, sizing._p(sse), sizing._s()),
                 "mk_mlp_adam_step")
        torch.cuda.synchronize()
        Pd = m.params().astype(np.float64)
        before = Pr.copy()
        Pr, Mr, Vr = omlp.adam_step(Pr, Mr, Vr, g_ref, t, lr)
        big = np.abs(g_ref) > 1e-3 * np.abs(g_ref).max()
        assert big.sum() > omlp.NPARAMS // 4
        step_d, step_r = Pd - before, Pr - before
        assert np.allclose(step_d[big], step_r[big], rtol=2e-3, atol=1e-3 * lr), np.abs(step_d - step_r)[big].max()
        # Kingma and Ba, Sec. 2.1: with 1 - b1 > sqrt(1 - b2) a step is at
        # most lr (1 - b1) / sqrt(1 - b2) = 3.16 lr in size
        assert np.all(np.abs(step_d) <= 3.2 * lr)
        Pr = Pd.copy()  # continue both from the device's masters


def test_sizing_buckets_match_oracle(cuda_lib):
    """mk_sizing_buckets: the network's prediction y against the oracle's
    forward pass, and the bucket counts against the oracle's bucket rule
    applied to the device's own y (a ceiling decided in fp32 on the device
    may differ only where the float64 quotient is within rounding of an
    integer)."""
    torch, mk, sizing = _mods()
    rng = np.random.default_rng(6)
    V = 20011
    P = rng.normal(0, 0.3, omlp.NPARAMS).astype(np.float32)
    m = sizing.SizingModel(seed=7)
    m.set_params(P)
    X = rng.normal(0, 1, (V, 8)).astype(np.float32)
    deg = rng.integers(0, 3000, V).astype(np.uint32)
    deg[:50] = 0
    for horizon, lf, cap in ((8.0, 0.7, 1 << 16), (32.0, 0.5, 40)):
        B, Y = m.buckets(torch.from_numpy(X).cuda(), mk.to_device_u32(deg), horizon, lf, cap)
        y = Y.cpu().numpy().astype(np.float64)
        y_ref = omlp.forward(P, X)
        assert np.allclose(y, y_ref, rtol=1e-5, atol=1e-5 * (1 + np.abs(y_ref).max()))
        b = mk.to_numpy_u32(B)
        b_ref = omlp.learned_buckets(y, deg, horizon, lf, cap)
        q = (deg + horizon * np.expm1(np.maximum(y, 0.0))) / (lf * 15.0)
        edge = np.abs(q - np.round(q)) <= 1e-5 * np.maximum(1.0, q)
        assert np.array_equal(b[~edge], b_ref[~edge]), np.nonzero(b != b_ref)[0][:10]
        assert np.all(np.abs(b[edge].astype(np.int64) - b_ref[edge]) <= 1)
        assert b.min() >= 1 and b.max() <= cap


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
    S = synth.growth_stream(scale=18, draws=1 << 22, n_batches=16)
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
