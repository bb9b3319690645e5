"""CPU oracle for the dynamic graph store (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline arm of
``bench.py`` may import this package.  The library path never does, and the
two share no code: the oracle is the plain definition of what the store and
the algorithms compute (see ``oracle.cpp`` for the passages it follows),
recomputed from scratch after every batch.

``OracleGraph`` wraps the C++ functions with numpy arrays:

* ``insert(src, dst, w) -> flags``, ``delete(src, dst) -> flags`` in batch order;
* ``query(src, dst) -> (bitmap, weights)``;
* ``export() -> (src, dst, w)`` sorted by (src, dst);
* ``bfs(source)`` / ``sssp(source) -> (dist, parent)`` with the min-id tight
  parent; ``wcc() -> labels`` (smallest vertex id per component);
* ``pagerank() -> (ranks, iterations)``, ``triangles() -> count``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_u8p = ctypes.POINTER(ctypes.c_uint8)
_u32p = ctypes.POINTER(ctypes.c_uint32)
NONE32 = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile ``oracle.cpp`` (plain C++17, single thread) into ``liboracle.so``."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-Wall", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_create.restype = ctypes.c_void_p
            lib.orc_create.argtypes = [ctypes.c_uint32]
            lib.orc_destroy.argtypes = [ctypes.c_void_p]
            lib.orc_num_edges.restype = ctypes.c_uint64
            lib.orc_num_edges.argtypes = [ctypes.c_void_p]
            lib.orc_insert.argtypes = [ctypes.c_void_p, _u32p, _u32p, _u32p, ctypes.c_uint64, _u8p]
            lib.orc_delete.argtypes = [ctypes.c_void_p, _u32p, _u32p, ctypes.c_uint64, _u8p]
            lib.orc_query.argtypes = [ctypes.c_void_p, _u32p, _u32p, ctypes.c_uint64, _u32p, _u32p]
            lib.orc_export.argtypes = [ctypes.c_void_p, _u32p, _u32p, _u32p]
            lib.orc_out_degree.argtypes = [ctypes.c_void_p, _u32p]
            lib.orc_bfs.restype = ctypes.c_int
            lib.orc_bfs.argtypes = [ctypes.c_void_p, ctypes.c_uint32, _u32p, _u32p]
            lib.orc_sssp.restype = ctypes.c_int
            lib.orc_sssp.argtypes = [ctypes.c_void_p, ctypes.c_uint32, _u32p, _u32p]
            lib.orc_wcc.argtypes = [ctypes.c_void_p, _u32p]
            lib.orc_pagerank.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_uint32,
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                         _u32p]
            lib.orc_triangles.restype = ctypes.c_uint64
            lib.orc_triangles.argtypes = [ctypes.c_void_p]
            _lib = lib
    return _lib


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


def _p(a: np.ndarray, t=_u32p):
    return a.ctypes.data_as(t)


class OracleGraph:
    """Edge set of a directed weighted graph on vertices [0, V)."""

    def __init__(self, V: int):
        self._lib = _load()
        self.V = int(V)
        self._h = self._lib.orc_create(self.V)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    @property
    def num_edges(self) -> int:
        return int(self._lib.orc_num_edges(self._h))

    def insert(self, src, dst, w=None) -> np.ndarray:
        s, d = _u32(src), _u32(dst)
        ww = None if w is None else _u32(w)
        f = np.zeros(len(s), np.uint8)
        self._lib.orc_insert(self._h, _p(s), _p(d), None if ww is None else _p(ww), len(s), _p(f, _u8p))
        return f

    def delete(self, src, dst) -> np.ndarray:
        s, d = _u32(src), _u32(dst)
        f = np.zeros(len(s), np.uint8)
        self._lib.orc_delete(self._h, _p(s), _p(d), len(s), _p(f, _u8p))
        return f

    def query(self, src, dst):
        s, d = _u32(src), _u32(dst)
        bm = np.zeros((len(s) + 31) // 32, np.uint32)
        w = np.zeros(len(s), np.uint32)
        self._lib.orc_query(self._h, _p(s), _p(d), len(s), _p(bm), _p(w))
        return bm, w

    def export(self):
        m = self.num_edges
        s, d, w = (np.empty(m, np.uint32) for _ in range(3))
        self._lib.orc_export(self._h, _p(s), _p(d), _p(w))
        return s, d, w

    def out_degree(self) -> np.ndarray:
        deg = np.empty(self.V, np.uint32)
        self._lib.orc_out_degree(self._h, _p(deg))
        return deg

    def bfs(self, source: int):
        dist = np.empty(self.V, np.uint32)
        par = np.empty(self.V, np.uint32)
        self._lib.orc_bfs(self._h, int(source), _p(dist), _p(par))
        return dist, par

    def sssp(self, source: int):
        dist = np.empty(self.V, np.uint32)
        par = np.empty(self.V, np.uint32)
        rc = self._lib.orc_sssp(self._h, int(source), _p(dist), _p(par))
        if rc != 0:
            raise OverflowError("a shortest-path length does not fit in 32 bits")
        return dist, par

    def wcc(self) -> np.ndarray:
        lab = np.empty(self.V, np.uint32)
        self._lib.orc_wcc(self._h, _p(lab))
        return lab

    def pagerank(self, damping=0.85, eps=1e-12, max_iter=1000, init=None):
        """(ranks as float64, iterations run)."""
        dp = ctypes.POINTER(ctypes.c_double)
        out = np.empty(self.V, np.float64)
        it = np.zeros(1, np.uint32)
        ini = None if init is None else np.ascontiguousarray(init, dtype=np.float64)
        self._lib.orc_pagerank(self._h, damping, eps, max_iter, None if ini is None else ini.ctypes.data_as(dp),
                               out.ctypes.data_as(dp), _p(it))
        return out, int(it[0])

    def triangles(self) -> int:
        return int(self._lib.orc_triangles(self._h))


def bitmap_to_bool(bitmap: np.ndarray, n: int) -> np.ndarray:
    """Unpack a query bitmap (bit i % 32 of word i // 32) into n booleans."""
    bits = np.unpackbits(np.ascontiguousarray(bitmap, dtype="<u4").view(np.uint8), bitorder="little")
    return bits[:n].astype(bool)
