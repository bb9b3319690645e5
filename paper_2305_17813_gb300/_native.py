"""ctypes declarations of the C ABI in ``include/meerkat.h``.

Argument marshalling only: every call goes straight to ``libmeerkat.so``.
The functions keep the C names (``mk_insert_batch`` and so on).
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmeerkat.so")

MK_OK = 0
MK_ERR_INVALID_ARG = -1
MK_ERR_POOL_EXHAUSTED = -2
MK_ERR_TIMEOUT = -3
MK_ERR_CUDA = -4
MK_ERR_NO_MEMORY = -5
MK_ERR_INTERNAL = -6
MK_NONE = 0xFFFFFFFF
MK_INVALID_LANE = 0xFF
MK_NOALLOC_MAX_BATCH = 65536
MK_MLP_NPARAMS = 4801

COUNTER_NAMES = ["query_slabs", "insert_slabs", "insert_new_slabs", "delete_slabs", "relax_lists", "relax_slabs",
                 "relax_edges", "relax_improved", "invalidated", "wcc_slabs", "wcc_edges", "commit_slabs",
                 "seed_lists", "seed_slabs", "seed_edges", "seed_improved", "wcc_upd_slabs", "wcc_upd_edges",
                 "rounds", "grid_barriers", "scan_owners", "scan_slabs", "scan_edges", "scan_targets", "scan_improved",
                 "walk_vertices", "unpacked", "seed_log", "wcc_log"]

STATUS_NAMES = {
    MK_OK: "MK_OK",
    MK_ERR_INVALID_ARG: "MK_ERR_INVALID_ARG",
    MK_ERR_POOL_EXHAUSTED: "MK_ERR_POOL_EXHAUSTED",
    MK_ERR_TIMEOUT: "MK_ERR_TIMEOUT",
    MK_ERR_CUDA: "MK_ERR_CUDA",
    MK_ERR_NO_MEMORY: "MK_ERR_NO_MEMORY",
    MK_ERR_INTERNAL: "MK_ERR_INTERNAL",
}


class MkError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__("%s failed: %s" % (what, STATUS_NAMES.get(status, status)))
        self.status = status


class mk_config(ctypes.Structure):
    _fields_ = [
        ("V", ctypes.c_uint32),
        ("edge_capacity_hint", ctypes.c_uint64),
        ("buckets", ctypes.c_uint32),
        ("d_bucket_per_vertex", ctypes.c_void_p),
        ("pool_slabs", ctypes.c_uint64),
    ]


class mk_stats(ctypes.Structure):
    _fields_ = [
        ("V", ctypes.c_uint32),
        ("lists", ctypes.c_uint64),
        ("pool_slabs", ctypes.c_uint64),
        ("pool_used", ctypes.c_uint64),
        ("chain_slabs", ctypes.c_uint64),
        ("live_edges", ctypes.c_uint64),
        ("tombstones", ctypes.c_uint64),
        ("chain_max", ctypes.c_uint32),
        ("chain_mean", ctypes.c_double),
        ("device_bytes", ctypes.c_uint64),
        ("epoch", ctypes.c_uint64),
    ]


class mk_query_req(ctypes.Structure):
    _fields_ = [("d_src", ctypes.c_void_p), ("d_dst", ctypes.c_void_p), ("n", ctypes.c_uint64),
                ("d_bitmap", ctypes.c_void_p), ("d_w", ctypes.c_void_p)]


class mk_update_req(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("d_src", ctypes.c_void_p), ("d_dst", ctypes.c_void_p),
                ("d_w", ctypes.c_void_p), ("n", ctypes.c_uint64), ("d_flags", ctypes.c_void_p)]


class mk_algo_req(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("source", ctypes.c_uint32), ("d_dist", ctypes.c_void_p),
                ("d_parent", ctypes.c_void_p)]


class mk_l2_info(ctypes.Structure):
    _fields_ = [("window_bytes", ctypes.c_uint64), ("max_bytes", ctypes.c_uint64), ("hit_ratio", ctypes.c_float)]


class mk_tuning(ctypes.Structure):
    _fields_ = [("query_group", ctypes.c_int), ("query_block", ctypes.c_int), ("rounds_blocks_per_sm", ctypes.c_int),
                ("query_best_ms", ctypes.c_float), ("rounds_best_ms", ctypes.c_float),
                ("query_ms", ctypes.c_float * 16), ("rounds_ms", ctypes.c_float * 8)]


class mk_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("d_src", ctypes.c_void_p), ("d_dst", ctypes.c_void_p),
                ("d_w", ctypes.c_void_p), ("n", ctypes.c_uint64), ("source", ctypes.c_uint32),
                ("d_out0", ctypes.c_void_p), ("d_out1", ctypes.c_void_p), ("tag", ctypes.c_uint64)]


MK_REQ_QUERY, MK_REQ_INSERT, MK_REQ_DELETE, MK_REQ_SSSP, MK_REQ_BFS = 0, 1, 2, 3, 4
MK_DEBUG_BARRIER_SPINS, MK_DEBUG_HOST_ROUNDS = 1, 2
MK_L2_NONE, MK_L2_VINFO, MK_L2_HEADS, MK_L2_POOL = 0, 1, 2, 3


class mk_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double)]


_P = ctypes.c_void_p
_U32 = ctypes.c_uint32
_U64 = ctypes.c_uint64
_INT = ctypes.c_int

# name -> (restype, argtypes)
SIGNATURES = {
    "mk_bucket_rule": (_INT, [_U32, _P, _U64, ctypes.c_float, _P, _P]),
    "mk_graph_create_ex": (_INT, [ctypes.POINTER(mk_config), _P, ctypes.POINTER(_P)]),
    "mk_graph_create": (_INT, [_U32, _U64, _U32, _P, _P, ctypes.POINTER(_P)]),
    "mk_graph_destroy": (_INT, [_P]),
    "mk_insert_batch": (_INT, [_P, _P, _P, _P, _U64, _P, _P]),
    "mk_insert_batch_noalloc": (_INT, [_P, _P, _P, _P, _U64, _P, _P]),
    "mk_delete_batch": (_INT, [_P, _P, _P, _U64, _P, _P]),
    "mk_query_batch": (_INT, [_P, _P, _P, _U64, _P, _P, _P]),
    "mk_commit_batch": (_INT, [_P, _P]),
    "mk_incr_sssp": (_INT, [_P, _U32, _P, _P, _P]),
    "mk_incr_bfs": (_INT, [_P, _U32, _P, _P, _P]),
    "mk_incr_wcc": (_INT, [_P, _P, _P]),
    "mk_incr_multi": (_INT, [_P, ctypes.POINTER(mk_algo_req), _U32, _P]),
    "mk_graph_export": (_INT, [_P, _U64, _P, _P, _P, _P, _P]),
    "mk_graph_stats": (_INT, [_P, ctypes.POINTER(mk_stats), _P]),
    "mk_last_error": (_INT, [_P]),
    "mk_pool_free": (_INT, [_P, ctypes.POINTER(_U64), _P]),
    "mk_list_marker": (_INT, [_P, _U32, _U32, ctypes.POINTER(_U32), ctypes.POINTER(_U32), ctypes.POINTER(_U32), _P]),
    "mk_counters": (_INT, [_P, ctypes.POINTER(_U64), _INT, _INT, _P]),
    "mk_profile_enable": (_INT, [_P, _INT]),
    "mk_profile_read": (_INT, [_P, ctypes.POINTER(mk_kernel_time), _INT, ctypes.POINTER(_INT)]),
    "mk_launch_count": (_U64, [_P]),
    "mk_version": (ctypes.c_char_p, []),
    "mk_debug_set": (_INT, [_P, _INT, _U64]),
    "mk_l2_window": (_INT, [_P, _INT, _P, ctypes.POINTER(mk_l2_info)]),
    "mk_set_bucket_rule": (_INT, [_U32, _P, _U64, ctypes.c_float, _P, _P]),
    "mk_set_create": (_INT, [_U32, _U64, _U32, _P, _P, ctypes.POINTER(_P)]),
    "mk_set_destroy": (_INT, [_P]),
    "mk_set_insert_batch": (_INT, [_P, _P, _P, _U64, _P, _P]),
    "mk_set_delete_batch": (_INT, [_P, _P, _P, _U64, _P, _P]),
    "mk_set_query_batch": (_INT, [_P, _P, _P, _U64, _P, _P]),
    "mk_set_bfs": (_INT, [_P, _U32, _P, _P, _P]),
    "mk_set_wcc": (_INT, [_P, _P, _P]),
    "mk_set_stats": (_INT, [_P, ctypes.POINTER(_U64), ctypes.POINTER(_U64), ctypes.POINTER(_U64), _P]),
    "mk_set_last_error": (_INT, [_P]),
    "mk_set_sssp_delta": (_INT, [_P, _U32, _U32]),
    "mk_pagerank": (_INT, [_P, _P, _INT, ctypes.c_float, ctypes.c_float, _U32, ctypes.POINTER(_U32),
                           ctypes.POINTER(ctypes.c_float), _P]),
    "mk_tc_count": (_INT, [_P, _P, _P, _P, _U64, _P, _P]),
    "mk_tc_static": (_INT, [_P, ctypes.POINTER(_U64), _P]),
    "mk_tc_update": (_INT, [_P, _P, _P, _P, _U64, _INT, ctypes.POINTER(ctypes.c_int64), _P]),
    "mk_server_create": (_INT, [_P, _U32, _U32, ctypes.POINTER(_P)]),
    "mk_server_destroy": (_INT, [_P]),
    "mk_server_submit": (_INT, [_P, ctypes.POINTER(mk_request)]),
    "mk_server_progress": (_INT, [_P, _P, _P, _U32, ctypes.POINTER(_U32)]),
    "mk_server_pending": (_INT, [_P, ctypes.POINTER(_U64), ctypes.POINTER(_U64)]),
    "mk_query_multi": (_INT, [_P, ctypes.POINTER(mk_query_req), _U32, _P]),
    "mk_update_multi": (_INT, [_P, ctypes.POINTER(mk_update_req), _U32, _P]),
    "mk_batcher_create": (_INT, [_P, _U32, ctypes.POINTER(_P)]),
    "mk_batcher_destroy": (_INT, [_P]),
    "mk_batcher_add_query": (_INT, [_P, _P, _P, _U64, _P, _P]),
    "mk_batcher_launch": (_INT, [_P, _P]),
    "mk_autotune": (_INT, [_P, _P, _P, _U64, _U32, _P, ctypes.POINTER(mk_tuning)]),
    "mk_get_tuning": (_INT, [_P, ctypes.POINTER(mk_tuning)]),
    "mk_set_tuning": (_INT, [_P, ctypes.POINTER(mk_tuning)]),
    "mk_mlp_create": (_INT, [_U64, ctypes.POINTER(_P)]),
    "mk_mlp_destroy": (_INT, [_P]),
    "mk_mlp_num_params": (_INT, []),
    "mk_mlp_get_params": (_INT, [_P, _P]),
    "mk_mlp_set_params": (_INT, [_P, _P]),
    "mk_mlp_forward": (_INT, [_P, _P, _U64, _P, _P]),
    "mk_mlp_gradient": (_INT, [_P, _P, _P, _U64, _P, _P, _P]),
    "mk_mlp_adam_step": (_INT, [_P, _P, _P, _U64, ctypes.c_float, _P, _P]),
    "mk_degree_update": (_INT, [_U32, _P, _P, _P, _U64, _INT, _P, _P, _P]),
    "mk_sizing_features": (_INT, [_U32, _P, _P, _P, _P, _P]),
    "mk_sizing_targets": (_INT, [_U32, _P, _P, ctypes.c_float, _P, _P]),
    "mk_sizing_buckets": (_INT, [_P, _P, _P, _U32, ctypes.c_float, ctypes.c_float, _U32, _P, _P, _P]),
}

_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Loads ``libmeerkat.so``.  Raises if it has not been built: there is no
    fallback implementation."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(
                    "libmeerkat.so is missing at %s; build it with paper_2305_17813_gb300.build.build()" % p)
            lib = ctypes.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def check(status: int, what: str) -> None:
    if status != MK_OK:
        raise MkError(status, what)
