"""Failure paths on the GPU without a GPU fault: a bounded wait made to run
out (the round kernel's grid barrier with a poll limit of zero) reports
MK_ERR_TIMEOUT through mk_last_error and leaves the context usable, after
which the next call recomputes statically and matches the oracle again; and
the host-driven round loop (the fallback for a refused cooperative launch)
gives the oracle's results on static, incremental and decremental calls."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _setup(scale=14):
    import paper_2305_17813_gb300 as mk
    from paper_2305_17813_gb300._native import MK_DEBUG_BARRIER_SPINS, MK_DEBUG_HOST_ROUNDS

    mk.load()
    G = synth.powerlaw_graph(scale=scale, draws=1 << (scale + 4))
    b = mk.bucket_rule(G.V, G.src, 0.7)
    g = mk.Graph(G.V, edge_capacity_hint=len(G.src) * 2, buckets=b)
    g.insert(G.src, G.dst, G.w)
    g.commit()
    o = oracle.OracleGraph(G.V)
    o.insert(G.src, G.dst, G.w)
    src = int(np.argmax(o.out_degree()))
    return mk, G, g, o, src, MK_DEBUG_BARRIER_SPINS, MK_DEBUG_HOST_ROUNDS


def _same(mk, got, want):
    return all(np.array_equal(mk.to_numpy_u32(a), b) for a, b in zip(got, want))


def test_barrier_timeout_is_reported_and_the_next_call_recovers(cuda_lib):
    mk, G, g, o, src, SPINS, _ = _setup()
    lib = mk.load()
    assert _same(mk, g.sssp(src), o.sssp(src))
    g.commit()
    S = synth.PowerlawStream(G, max_batch=1 << 12)
    b = S.batch(1 << 12)
    g.insert(b.ins_src, b.ins_dst, b.ins_w)
    o.insert(b.ins_src, b.ins_dst, b.ins_w)
    # every grid-barrier wait gives up at its first poll
    mk.check(lib.mk_debug_set(g.handle, SPINS, 1), "mk_debug_set")
    g.sssp(src)
    assert g.last_error() == mk.MK_ERR_TIMEOUT
    # the context is usable and the status was cleared
    assert g.last_error() == mk.MK_OK
    mk.check(lib.mk_debug_set(g.handle, SPINS, 0), "mk_debug_set")
    # the half-updated state recomputes statically: exact again
    assert _same(mk, g.sssp(src), o.sssp(src))
    assert g.last_error() == mk.MK_OK
    g.commit()
    g.delete(b.del_src, b.del_dst)
    o.delete(b.del_src, b.del_dst)
    assert _same(mk, g.sssp(src), o.sssp(src))
    assert g.last_error() == mk.MK_OK
    g.close()


def test_host_driven_round_loop_matches_oracle(cuda_lib):
    mk, G, g, o, src, _, HOST = _setup(scale=13)
    lib = mk.load()
    mk.check(lib.mk_debug_set(g.handle, HOST, 1), "mk_debug_set")
    assert _same(mk, g.sssp(src), o.sssp(src))
    assert _same(mk, g.bfs(src), o.bfs(src))
    g.commit()
    S = synth.PowerlawStream(G, max_batch=1 << 11)
    for _ in range(2):
        b = S.batch(1 << 11)
        g.insert(b.ins_src, b.ins_dst, b.ins_w)
        o.insert(b.ins_src, b.ins_dst, b.ins_w)
        assert _same(mk, g.sssp(src), o.sssp(src))
        assert _same(mk, g.bfs(src), o.bfs(src))
        g.commit()
        g.delete(b.del_src, b.del_dst)
        o.delete(b.del_src, b.del_dst)
        assert _same(mk, g.sssp(src), o.sssp(src))
        assert _same(mk, g.bfs(src), o.bfs(src))
        g.commit()
    assert g.last_error() == mk.MK_OK
    # and back on the cooperative kernel, incrementally
    mk.check(lib.mk_debug_set(g.handle, HOST, 0), "mk_debug_set")
    b = S.batch(1 << 11)
    g.insert(b.ins_src, b.ins_dst, b.ins_w)
    o.insert(b.ins_src, b.ins_dst, b.ins_w)
    assert _same(mk, g.sssp(src), o.sssp(src))
    assert g.last_error() == mk.MK_OK
    g.close()
