"""mk_insert_batch_noalloc against mk_insert_batch.

Some callers cannot let the library allocate device memory while they run
(a serving loop that must not synchronise the device between requests, or a
process whose device memory belongs to another allocator or is fixed at
start-up).  For them the library offers an insert that stages its batch in a
fixed device array instead of growing buffers with cudaMalloc.  This test
calls it through the C ABI and checks, on two calls in a row, that its flags
and the resulting edge set are identical to those of the ordinary insert on a
twin graph, that the device's free memory and the graph's own device bytes
are unchanged across the two calls, and that an oversized batch is refused.
It lives in a file of its own that pytest collects last.
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
    P = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    # two calls in a row, the second at the limit: inputs, outputs and the
    # ordinary insert's results on the twin graph are made first, so that
    # nothing else allocates while the allocation-free calls run
    calls = []
    for n in (5003, MK_NOALLOC_MAX_BATCH):
        s = rng.integers(0, w.V, n).astype(np.uint32)
        d = rng.integers(0, w.V, n).astype(np.uint32)
        ww = rng.integers(1, 100, n).astype(np.uint32)
        fa = a.insert(s, d, ww).cpu().numpy()
        calls.append((n, fa, [mk.to_device_u32(x) for x in (s, d, ww)], torch.empty(n, dtype=torch.uint8,
                                                                                   device="cuda")))
    ea = a.export()
    # set-up call (the first on this device), then the two compared calls
    one = mk.to_device_u32([0])
    assert lib.mk_insert_batch_noalloc(b.handle, P(one), P(one), None, 0, None, stream) == mk.MK_OK
    bytes0 = b.stats()["device_bytes"]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for n, fa, (ts, td, tw), fb in calls:
        rc = lib.mk_insert_batch_noalloc(b.handle, P(ts), P(td), P(tw), n, P(fb), stream)
        assert rc == mk.MK_OK
        assert b.last_error() == mk.MK_OK
        assert np.array_equal(fa, fb.cpu().numpy())
    torch.cuda.synchronize()
    # no device memory came or went, and the graph holds what it held
    assert torch.cuda.mem_get_info()[0] == free0
    assert b.stats()["device_bytes"] == bytes0
    assert a.last_error() == mk.MK_OK
    eb = b.export()
    for x, y in zip(ea, eb):
        assert torch.equal(x, y)
    big = torch.zeros(MK_NOALLOC_MAX_BATCH + 1, dtype=torch.int32, device="cuda")
    rc = lib.mk_insert_batch_noalloc(b.handle, P(big), P(big), None, MK_NOALLOC_MAX_BATCH + 1, None, stream)
    assert rc == mk.MK_ERR_INVALID_ARG
    a.close()
    b.close()
