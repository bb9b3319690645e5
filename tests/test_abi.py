"""The C-ABI library builds, loads without a GPU and exports every function
that include/meerkat.h declares; the Python binding declares the same set.
Also checks host-side facts of the boundary that need no device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "meerkat.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mk_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2305_17813_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ["mk_graph_create", "mk_graph_destroy", "mk_insert_batch", "mk_delete_batch", "mk_query_batch",
                     "mk_incr_bfs", "mk_incr_sssp", "mk_incr_wcc", "mk_graph_export", "mk_graph_stats",
                     "mk_last_error", "mk_commit_batch"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib):
    from paper_2305_17813_gb300 import _native

    assert set(_native.SIGNATURES) == set(declared_functions())


def test_host_side_argument_errors_need_no_device(lib):
    import paper_2305_17813_gb300 as mk

    L = mk.load()
    out = ctypes.c_void_p()
    # V = 0 and reserved ids are refused before any CUDA call
    assert L.mk_graph_create(0, 0, 1, None, None, ctypes.byref(out)) == mk.MK_ERR_INVALID_ARG
    assert L.mk_graph_create(0xFFFFFFFE, 0, 1, None, None, ctypes.byref(out)) == mk.MK_ERR_INVALID_ARG
    assert L.mk_insert_batch(None, None, None, None, 0, None, None) == mk.MK_ERR_INVALID_ARG
    assert L.mk_last_error(None) == mk.MK_ERR_INVALID_ARG
    # the later entry points refuse a null graph the same way
    assert L.mk_update_multi(None, None, 0, None) == mk.MK_ERR_INVALID_ARG
    assert L.mk_incr_multi(None, None, 1, None) == mk.MK_ERR_INVALID_ARG
    assert L.mk_pagerank(None, None, 0, 0.85, 1e-7, 10, None, None, None) == mk.MK_ERR_INVALID_ARG
    assert L.mk_tc_count(None, None, None, None, 0, None, None) == mk.MK_ERR_INVALID_ARG
    assert L.mk_tc_static(None, None, None) == mk.MK_ERR_INVALID_ARG
    assert L.mk_tc_update(None, None, None, None, 0, 0, None, None) == mk.MK_ERR_INVALID_ARG
    assert L.mk_l2_window(None, mk.MK_L2_VINFO, None, None) == mk.MK_ERR_INVALID_ARG
    assert L.mk_debug_set(None, 1, 0) == mk.MK_ERR_INVALID_ARG
    assert L.mk_set_sssp_delta(None, 0, 0) == mk.MK_ERR_INVALID_ARG
    # the set layout's entry points
    assert L.mk_set_create(0, 0, 1, None, None, ctypes.byref(out)) == mk.MK_ERR_INVALID_ARG
    assert L.mk_set_create(0xFFFFFFFE, 0, 1, None, None, ctypes.byref(out)) == mk.MK_ERR_INVALID_ARG
    assert L.mk_set_create(4, 0, 1, None, None, None) == mk.MK_ERR_INVALID_ARG
    assert L.mk_set_bucket_rule(0, None, 0, 0.7, None, None) == mk.MK_ERR_INVALID_ARG
    assert L.mk_set_destroy(None) == mk.MK_ERR_INVALID_ARG
    assert L.mk_set_insert_batch(None, None, None, 0, None, None) == mk.MK_ERR_INVALID_ARG
    assert L.mk_set_delete_batch(None, None, None, 0, None, None) == mk.MK_ERR_INVALID_ARG
    assert L.mk_set_query_batch(None, None, None, 0, None, None) == mk.MK_ERR_INVALID_ARG
    assert L.mk_set_bfs(None, 0, None, None, None) == mk.MK_ERR_INVALID_ARG
    assert L.mk_set_wcc(None, None, None) == mk.MK_ERR_INVALID_ARG
    assert L.mk_set_stats(None, None, None, None, None) == mk.MK_ERR_INVALID_ARG
    assert L.mk_set_last_error(None) == mk.MK_ERR_INVALID_ARG
    assert L.mk_version().decode().startswith("meerkat-gb300")


def test_warp_enqueue_offset_formula():
    """The paper's frontier enqueue (Algorithm 'Warp device APIs: broadcast,
    and frontier enqueue') places lane l at popc(brev(mask) & (~0 << (32 - l))),
    the number of participating lanes below l; the kernels compute the same
    count as popc(mask & ((1 << l) - 1)).  Exhaustive over lanes, random masks
    (a shift by 32 is taken as 0, as the hardware shift does)."""
    import numpy as np

    def brev(x):
        return int("{:032b}".format(x)[::-1], 2)

    rng = np.random.default_rng(0)
    masks = [0, 0xFFFFFFFF, 1, 0x80000000] + [int(m) for m in rng.integers(0, 2**32, 200, dtype=np.uint64)]
    for m in masks:
        for lane in range(32):
            shifted = (0xFFFFFFFF << (32 - lane)) & 0xFFFFFFFF if lane > 0 else 0
            paper = bin(brev(m) & shifted).count("1")
            ours = bin(m & ((1 << lane) - 1)).count("1")
            assert paper == ours
