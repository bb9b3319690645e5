"""mk_incr_multi: several BFS/SSSP states advanced by one call (one pass
over the change log and the slab array for all of them, shared rounds) give
exactly the results of one call per state and of the oracle, through
static, incremental, decremental and mixed (stale + current) calls."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _setup():
    import paper_2305_17813_gb300 as mk

    mk.load()
    G = synth.powerlaw_graph(scale=14, draws=1 << 18)
    b = mk.bucket_rule(G.V, G.src, 0.7)
    graphs = []
    for _ in range(2):
        g = mk.Graph(G.V, edge_capacity_hint=len(G.src) * 2, buckets=b)
        g.insert(G.src, G.dst, G.w)
        g.commit()
        graphs.append(g)
    o = oracle.OracleGraph(G.V)
    o.insert(G.src, G.dst, G.w)
    return mk, G, graphs, o


def _check(mk, got, want, what):
    d, p = got
    assert np.array_equal(mk.to_numpy_u32(d), want[0]), "distances, " + what
    assert np.array_equal(mk.to_numpy_u32(p), want[1]), "parents, " + what


def test_multi_matches_single_calls_and_oracle(cuda_lib):
    mk, G, (gm, gs), o = _setup()
    deg = np.bincount(G.src, minlength=G.V)
    hub, s2, s3 = int(np.argmax(deg)), int(np.argsort(deg)[-2]), 7
    reqs = [("bfs", hub), ("sssp", hub), ("sssp", s2), ("bfs", s3)]

    def run_and_check(what, subset=None):
        rq = reqs if subset is None else [reqs[i] for i in subset]
        multi = gm.incr_multi(rq)
        for (kind, src), got in zip(rq, multi):
            single = getattr(gs, kind)(src)
            want = o.bfs(src) if kind == "bfs" else o.sssp(src)
            _check(mk, got, want, "%s %s(%d)" % (what, kind, src))
            _check(mk, single, want, "single %s %s(%d)" % (what, kind, src))

    run_and_check("static")
    for g in (gm, gs):
        g.commit()
    S = synth.PowerlawStream(G, max_batch=1 << 12)
    for k in range(3):
        bt = S.batch(1 << 12)
        for g in (gm, gs):
            g.insert(bt.ins_src, bt.ins_dst, bt.ins_w)
        o.insert(bt.ins_src, bt.ins_dst, bt.ins_w)
        # after batch 1 the last state skips an epoch and recomputes
        # statically beside the incremental ones
        run_and_check("after insert %d" % k, subset=[0, 1, 2] if k == 1 else None)
        for g in (gm, gs):
            g.commit()
        for g in (gm, gs):
            g.delete(bt.del_src, bt.del_dst)
        o.delete(bt.del_src, bt.del_dst)
        run_and_check("after delete %d" % k, subset=[0, 1, 2] if k == 1 else None)
        for g in (gm, gs):
            g.commit()
    # a mixed epoch (deletes then inserts) in one call, two states
    bt = S.batch(1 << 12)
    for g in (gm, gs):
        g.delete(bt.del_src, bt.del_dst)
        g.insert(bt.ins_src, bt.ins_dst, bt.ins_w)
    o.delete(bt.del_src, bt.del_dst)
    o.insert(bt.ins_src, bt.ins_dst, bt.ins_w)
    run_and_check("mixed epoch", subset=[1, 2])
    assert gm.last_error() == mk.MK_OK and gs.last_error() == mk.MK_OK


def test_multi_host_rounds_and_bad_requests(cuda_lib):
    import ctypes

    from paper_2305_17813_gb300._native import MK_DEBUG_HOST_ROUNDS, MK_REQ_SSSP, mk_algo_req

    mk, G, (g, _), o = _setup()
    lib = mk.load()
    mk.check(lib.mk_debug_set(g.handle, MK_DEBUG_HOST_ROUNDS, 1), "mk_debug_set")
    out = g.incr_multi([("sssp", 3), ("bfs", 3)])
    _check(mk, out[0], o.sssp(3), "host rounds sssp")
    _check(mk, out[1], o.bfs(3), "host rounds bfs")
    mk.check(lib.mk_debug_set(g.handle, MK_DEBUG_HOST_ROUNDS, 0), "mk_debug_set")
    arr = (mk_algo_req * 5)()
    for i in range(5):
        arr[i].kind, arr[i].source = MK_REQ_SSSP, i
    assert lib.mk_incr_multi(g.handle, arr, 5, None) == mk.MK_ERR_INVALID_ARG  # too many
    arr[1].source = 0
    assert lib.mk_incr_multi(g.handle, arr, 2, None) == mk.MK_ERR_INVALID_ARG  # the same state twice
    arr[1].source = G.V
    assert lib.mk_incr_multi(g.handle, arr, 2, None) == mk.MK_ERR_INVALID_ARG  # source out of range
    assert g.last_error() == mk.MK_OK
