"""mk_insert_batch_noalloc against mk_insert_batch.

Some callers cannot let the library allocate device memory while they run
(a serving loop that must not synchronise the device between requests, or a
process whose device memory belongs to another allocator or is fixed at
start-up).  For them the library offers an insert that stages its batch in a
fixed device array instead of growing buffers with cudaMalloc.  This test
calls it through the C ABI and checks, on two calls in a row, that its flags
and the resulting edge set are identical to those of the ordinary insert on a
twin graph; it also checks that an oversized batch is refused.  It lives in a
file of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_no_alloc_insert_matches_insert_batch(cuda_lib):
    import torch

    import paper_2305_17813_gb300 as mk
    from paper_2305_17813_gb300._native import MK_NOALLOC_MAX_BATCH

    lib = mk.load()
    w = synth.tiny_workload()
    a = mk.Graph(w.V, edge_capacity_hint=1 << 18, buckets=3)
    b = mk.Graph(w.V, edge_capacity_hint=1 << 18, buckets=3)
    for g in (a, b):
        g.insert(w.g_src, w.g_dst, w.g_w)
        g.commit()
    rng = np.random.default_rng(7)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for n in (5003, MK_NOALLOC_MAX_BATCH):  # two calls in a row, the second at the limit
        s = rng.integers(0, w.V, n).astype(np.uint32)
        d = rng.integers(0, w.V, n).astype(np.uint32)
        ww = rng.integers(1, 100, n).astype(np.uint32)
        fa = a.insert(s, d, ww).cpu().numpy()
        ts, td, tw = (mk.to_device_u32(x) for x in (s, d, ww))
        fb = torch.empty(n, dtype=torch.uint8, device="cuda")
        rc = lib.mk_insert_batch_noalloc(b.handle, ctypes.c_void_p(ts.data_ptr()), ctypes.c_void_p(td.data_ptr()),
                                         ctypes.c_void_p(tw.data_ptr()), n, ctypes.c_void_p(fb.data_ptr()), stream)
        assert rc == mk.MK_OK
        assert b.last_error() == mk.MK_OK and a.last_error() == mk.MK_OK
        assert np.array_equal(fa, fb.cpu().numpy())
        ea, eb = a.export(), b.export()
        for x, y in zip(ea, eb):
            assert torch.equal(x, y)
    big = torch.zeros(MK_NOALLOC_MAX_BATCH + 1, dtype=torch.int32, device="cuda")
    rc = lib.mk_insert_batch_noalloc(b.handle, ctypes.c_void_p(big.data_ptr()), ctypes.c_void_p(big.data_ptr()),
                                     None, MK_NOALLOC_MAX_BATCH + 1, None, stream)
    assert rc == mk.MK_ERR_INVALID_ARG
    a.close()
    b.close()
