"""Multi-core CPU baseline of the batched edge operations (TEST AND
BENCHMARK INFRASTRUCTURE ONLY).

``ShardedGraph`` wraps ``sharded.cpp``: the oracle's edge-set semantics with
the set partitioned by source vertex over one host thread per shard.  It is
timed beside the GPU path as the all-cores CPU figure for insert, delete and
query; the single-thread oracle (``OracleGraph``) stays the reference for
results.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sharded.cpp")
_LIB = os.path.join(_HERE, "libsharded.so")
_lock = threading.Lock()
_lib = None
_u8p = ctypes.POINTER(ctypes.c_uint8)
_u32p = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> str:
    """Compile ``sharded.cpp`` (C++17, std::thread) into ``libsharded.so``."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-Wall", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.shd_create.restype = ctypes.c_void_p
            lib.shd_create.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
            lib.shd_destroy.argtypes = [ctypes.c_void_p]
            lib.shd_num_edges.restype = ctypes.c_uint64
            lib.shd_num_edges.argtypes = [ctypes.c_void_p]
            lib.shd_insert.argtypes = [ctypes.c_void_p, _u32p, _u32p, _u32p, ctypes.c_uint64, _u8p]
            lib.shd_delete.argtypes = [ctypes.c_void_p, _u32p, _u32p, ctypes.c_uint64, _u8p]
            lib.shd_query.argtypes = [ctypes.c_void_p, _u32p, _u32p, ctypes.c_uint64, _u8p, _u32p]
            _lib = lib
    return _lib


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


def _p(a, t=_u32p):
    return a.ctypes.data_as(t)


class ShardedGraph:
    """Edge set partitioned by source over `threads` host threads."""

    def __init__(self, V: int, threads: int = 0):
        self._lib = _load()
        self.threads = int(threads or os.cpu_count() or 1)
        self._h = self._lib.shd_create(int(V), self.threads)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.shd_destroy(h)
            self._h = None

    @property
    def num_edges(self) -> int:
        return int(self._lib.shd_num_edges(self._h))

    def insert(self, src, dst, w=None):
        s, d = _u32(src), _u32(dst)
        ww = None if w is None else _u32(w)
        f = np.zeros(len(s), np.uint8)
        self._lib.shd_insert(self._h, _p(s), _p(d), None if ww is None else _p(ww), len(s), _p(f, _u8p))
        return f

    def delete(self, src, dst):
        s, d = _u32(src), _u32(dst)
        f = np.zeros(len(s), np.uint8)
        self._lib.shd_delete(self._h, _p(s), _p(d), len(s), _p(f, _u8p))
        return f

    def query(self, src, dst):
        s, d = _u32(src), _u32(dst)
        hit = np.zeros(len(s), np.uint8)
        w = np.zeros(len(s), np.uint32)
        self._lib.shd_query(self._h, _p(s), _p(d), len(s), _p(hit, _u8p), _p(w))
        return hit, w
