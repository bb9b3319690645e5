"""Learned slab sizing (Python binding of the learned-sizing kernels).

The paper sizes every vertex's hash table once, from the load factor and the
degree it has at that moment (Sec. "Motivation"), so vertices that keep
growing end up with long slab chains.  This module trains a small MLP on the
degree traces of the running graph to predict how many edges each vertex will
gain, and turns the prediction into bucket counts for a rebuilt graph.  The
load-factor rule stays the fallback and the yardstick; bucket counts change the
layout (chain lengths, memory) but never a result.

Every computation runs in ``libmeerkat.so`` (``mk_degree_update``,
``mk_sizing_features``, ``mk_sizing_targets``, ``mk_mlp_*``,
``mk_sizing_buckets``); torch only allocates and moves tensors.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native
from ._native import MK_MLP_NPARAMS, check, load


def _torch():
    import torch

    return torch


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _s(stream=None):
    torch = _torch()
    return ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)


class DegreeTrace:
    """Out/in degree counters of a graph maintained from batch flags, plus
    the last five out-degree snapshots (one per batch)."""

    def __init__(self, V: int, device="cuda"):
        torch = _torch()
        self.V = V
        self.lib = load()
        self.out_deg = torch.zeros(V, dtype=torch.int32, device=device)
        self.in_deg = torch.zeros(V, dtype=torch.int32, device=device)
        self.hist = torch.zeros((5, V), dtype=torch.int32, device=device)

    def apply(self, src, dst, flags=None, sign: int = 1, stream=None):
        n = src.numel()
        check(self.lib.mk_degree_update(self.V, _p(src), _p(dst), _p(flags), n, sign, _p(self.out_deg),
                                        _p(self.in_deg), _s(stream)), "mk_degree_update")

    def snapshot(self):
        self.hist[1:] = self.hist[:-1].clone()
        self.hist[0].copy_(self.out_deg)

    def features(self, buckets, stream=None):
        torch = _torch()
        X = torch.empty((self.V, 8), dtype=torch.float32, device=self.out_deg.device)
        check(self.lib.mk_sizing_features(self.V, _p(self.hist), _p(self.in_deg), _p(buckets), _p(X), _s(stream)),
              "mk_sizing_features")
        return X


def growth_targets(deg_then, deg_later, horizon: float, stream=None):
    torch = _torch()
    V = deg_then.numel()
    T = torch.empty(V, dtype=torch.float32, device=deg_then.device)
    check(load().mk_sizing_targets(V, _p(deg_then), _p(deg_later), float(horizon), _p(T), _s(stream)),
          "mk_sizing_targets")
    return T


class SizingModel:
    """The 8 -> 64 -> 64 -> 1 network (bf16 weights, fp32 accumulation)."""

    def __init__(self, seed: int = 0):
        self.lib = load()
        h = ctypes.c_void_p()
        check(self.lib.mk_mlp_create(seed, ctypes.byref(h)), "mk_mlp_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self.lib.mk_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.empty(MK_MLP_NPARAMS, np.float32)
        check(self.lib.mk_mlp_get_params(self._h, out.ctypes.data_as(ctypes.c_void_p)), "mk_mlp_get_params")
        return out

    def set_params(self, P):
        a = np.ascontiguousarray(P, dtype=np.float32)
        assert a.shape == (MK_MLP_NPARAMS,)
        check(self.lib.mk_mlp_set_params(self._h, a.ctypes.data_as(ctypes.c_void_p)), "mk_mlp_set_params")

    def forward(self, X, stream=None):
        torch = _torch()
        Y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
        check(self.lib.mk_mlp_forward(self._h, _p(X), X.shape[0], _p(Y), _s(stream)), "mk_mlp_forward")
        return Y

    def gradient(self, X, T, stream=None):
        torch = _torch()
        G = torch.empty(MK_MLP_NPARAMS, dtype=torch.float32, device=X.device)
        sse = torch.zeros(1, dtype=torch.float64, device=X.device)
        check(self.lib.mk_mlp_gradient(self._h, _p(X), _p(T), X.shape[0], _p(G), _p(sse), _s(stream)),
              "mk_mlp_gradient")
        return G, sse

    def train(self, X, T, epochs: int = 20, batch: int = 1 << 18, lr: float = 3e-3, seed: int = 0, stream=None):
        """Adam over shuffled minibatches; returns the mean squared error of
        each epoch (as measured during that epoch)."""
        torch = _torch()
        n = X.shape[0]
        gen = torch.Generator(device="cpu")
        gen.manual_seed(seed)
        sse = torch.zeros(1, dtype=torch.float64, device=X.device)
        losses = []
        for _ in range(epochs):
            perm = torch.randperm(n, generator=gen).to(X.device)
            Xs, Ts = X[perm].contiguous(), T[perm].contiguous()
            total = 0.0
            for i in range(0, n, batch):
                xb, tb = Xs[i:i + batch], Ts[i:i + batch]
                check(self.lib.mk_mlp_adam_step(self._h, _p(xb), _p(tb), xb.shape[0], lr, _p(sse), _s(stream)),
                      "mk_mlp_adam_step")
                total += float(sse.item())
            losses.append(total / n)
        return losses

    def buckets(self, X, deg, horizon: float, load_factor: float = 0.7, max_buckets: int = 1 << 16, stream=None):
        torch = _torch()
        V = X.shape[0]
        Y = torch.empty(V, dtype=torch.float32, device=X.device)
        B = torch.empty(V, dtype=torch.int32, device=X.device)
        check(self.lib.mk_sizing_buckets(self._h, _p(X), _p(deg), V, float(horizon), float(load_factor),
                                         int(max_buckets), _p(Y), _p(B), _s(stream)), "mk_sizing_buckets")
        return B, Y


__all__ = ["DegreeTrace", "SizingModel", "growth_targets", "_native"]
