"""B300-native per-edge AML pattern counting (multi-stage graph mining).

Thin Python layer over the C ABI of ``libaml_b300.so`` (include/aml.h):
argument marshalling only, every step of the computation runs in the
library's CUDA kernels.  PyTorch provides device memory and streams.

    import paper_2604_12241_b300 as aml
    g = aml.Graph(src, dst, ts, n_nodes)                 # numpy (host) or torch CUDA tensors
    ps = aml.PatternSet(aml.patterns.standard(86400))    # stage programs -> columns
    counts = aml.mine(g, ps)                             # torch int32 [E, P] (uint32 bits)
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np

from . import patterns  # noqa: F401
from ._lib import (ASSUME_SORTED, MINE_FUSED, MINE_GRAPH, MINE_HOST_ASYNC,  # noqa: F401
                   MINE_HOST_OUTPUT, MINE_LEARNED, MINE_PERSISTENT, PTR_DEVICE, PTR_HOST, AmlError, aml_column_info,
                   aml_cost_report, aml_graph_info, aml_stream_batch, aml_stream_info,
                   aml_tuning, check, lib, make_patterns)

__all__ = ["Graph", "PatternSet", "Stream", "mine", "autotune", "cost_train", "AmlError",
           "patterns"]


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(x):
    """(pointer, is_device) of a numpy array or torch tensor (contiguous)."""
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("arrays must be contiguous")
        return x.ctypes.data, False
    import torch
    if isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr(), x.is_cuda
    raise TypeError(type(x))


class Graph:
    """Device-resident transaction graph (aml_graph_create)."""

    def __init__(self, src, dst, ts, n_nodes: int, amount=None, assume_sorted: bool = False,
                 stream=None):
        L = lib()
        if isinstance(src, np.ndarray):
            src = np.ascontiguousarray(src, dtype=np.int32)
            dst = np.ascontiguousarray(dst, dtype=np.int32)
            ts = np.ascontiguousarray(ts, dtype=np.int32)
            if amount is not None:
                amount = np.ascontiguousarray(amount, dtype=np.float32)
        ps, dev = _ptr(src)
        pd, _ = _ptr(dst)
        pt, _ = _ptr(ts)
        pa = _ptr(amount)[0] if amount is not None else None
        flags = (PTR_DEVICE if dev else PTR_HOST) | (ASSUME_SORTED if assume_sorted else 0)
        n_edges = int(src.shape[0])
        h = ctypes.c_void_p()
        s = _stream_handle(stream)
        check(L.aml_graph_create(ps, pd, pt, pa, n_edges, int(n_nodes), flags, s,
                                 ctypes.byref(h)))
        self._h = h
        self.n_edges = n_edges
        self.n_nodes = int(n_nodes)

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = aml_graph_info()
        check(lib().aml_graph_get_info(self._h, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in inf._fields_ if f != "reserved"}

    def window_stats(self, delta: int) -> dict:
        """Work sizes earlier mines measured for one window
        (aml_graph_window_stats): legs and cycle-search frontier per level."""
        n_legs = ctypes.c_int64()
        front = (ctypes.c_int64 * 9)()
        check(lib().aml_graph_window_stats(self._h, int(delta), ctypes.byref(n_legs), front))
        return {"n_legs": n_legs.value,
                "n_front": {j: front[j] for j in range(2, 9) if front[j] >= 0}}

    def sync(self) -> None:
        check(lib().aml_sync(self._h))

    def tuning(self) -> dict:
        t = aml_tuning()
        check(lib().aml_graph_get_tuning(self._h, ctypes.byref(t)))
        return {f: getattr(t, f) for f, _ in t._fields_}

    def set_tuning(self, **kw) -> None:
        cur = self.tuning()
        cur.update(kw)
        t = aml_tuning(**cur)
        check(lib().aml_graph_set_tuning(self._h, ctypes.byref(t)))

    def set_count_limit(self, limit: int) -> None:
        """Saturation bound of this graph's counts (aml_graph_set_count_limit)."""
        check(lib().aml_graph_set_count_limit(self._h, int(limit)))

    def set_wait_limit(self, cycles: int) -> None:
        """Bound on device-side waits in SM cycles (aml_graph_set_wait_limit)."""
        check(lib().aml_graph_set_wait_limit(self._h, int(cycles)))

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().aml_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PatternSet:
    """Validated, planned set of stage programs (aml_pattern_set_create)."""

    def __init__(self, pats: Sequence["patterns.Pattern"]):
        arr, keep = make_patterns(pats)
        h = ctypes.c_void_p()
        check(lib().aml_pattern_set_create(arr, len(pats), ctypes.byref(h)))
        self._h = h
        self.patterns = list(pats)
        n = ctypes.c_int32()
        check(lib().aml_pattern_set_num_columns(h, ctypes.byref(n)))
        self.n_cols = n.value
        self.columns = []
        for j in range(self.n_cols):
            ci = aml_column_info()
            check(lib().aml_pattern_set_column(h, j, ctypes.byref(ci)))
            self.columns.append(dict(family=ci.family, k=ci.k, delta=ci.delta,
                                     name=ci.name.decode()))

    @property
    def handle(self):
        return self._h

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().aml_pattern_set_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(graph: Graph, pset: PatternSet, repeats: int = 3, stream=None):
    """Pick the fastest tunables for this graph and pattern set (aml_autotune);
    returns (tuning dict, median ms of the best setting)."""
    t = aml_tuning()
    ms = ctypes.c_float()
    check(lib().aml_autotune(graph.handle, pset.handle, repeats, _stream_handle(stream),
                             ctypes.byref(t), ctypes.byref(ms)))
    return {f: getattr(t, f) for f, _ in t._fields_}, ms.value


def cost_train(graph: Graph, pset: PatternSet, max_samples: int = 1_000_000, epochs: int = 20,
               seed: int = 1, stream=None) -> dict:
    """Train the cycle-search cost model on the GPU (aml_cost_train)."""
    r = aml_cost_report()
    check(lib().aml_cost_train(graph.handle, pset.handle, int(max_samples), int(epochs), int(seed),
                               _stream_handle(stream), ctypes.byref(r)))
    return {f: getattr(r, f) for f, _ in r._fields_}


MODES = {"plain": 0, "persistent": MINE_PERSISTENT, "learned": MINE_LEARNED,
         "fused": MINE_FUSED}


def mine(graph: Graph, pset: PatternSet, out=None, stream=None, host_output: bool = False,
         use_graph: bool = False, mode: str = "plain", host_async: bool = False):
    """Per-edge counts, [E, P] (aml_mine).

    Device mode (default) returns / fills a torch int32 CUDA tensor holding
    the uint32 counts bit-for-bit (``.view(torch.uint32)`` or numpy
    ``.view(np.uint32)`` to read them unsigned).  ``host_output=True``
    returns a numpy uint32 array copied back by the library; with
    ``host_async=True`` the copy is only enqueued on ``stream`` (``out`` must
    be page-locked, e.g. a pinned torch tensor's ``.numpy()``) and the caller
    synchronizes ``stream`` before reading it.  ``use_graph``
    replays the whole mine as one captured CUDA graph (AML_MINE_GRAPH).
    ``mode``: "plain" (level-by-level cycle search), "fused" (a window's
    leg pass and cycle search in one cooperative persistent launch with
    work queues), "persistent" (one
    persistent launch, degree-binned queues) or "learned" (queues from the
    trained cost model).  All modes give identical counts.
    """
    flags = MODES[mode]
    P = pset.n_cols
    E = graph.n_edges
    s = _stream_handle(stream)
    if host_output:
        arr = out if out is not None else np.empty((E, P), dtype=np.uint32)
        ptr, dev = _ptr(arr)
        if dev:
            raise ValueError("host_output needs a host array")
        check(lib().aml_mine(graph.handle, pset.handle, ptr, arr.shape[1],
                             MINE_HOST_OUTPUT | (MINE_HOST_ASYNC if host_async else 0) | flags,
                             s))
        return arr
    import torch
    if out is None:
        out = torch.empty((E, P), dtype=torch.int32, device="cuda")
    ptr, dev = _ptr(out)
    if not dev:
        raise ValueError("device mode needs a CUDA tensor")
    check(lib().aml_mine(graph.handle, pset.handle, ptr, out.shape[1],
                         (MINE_GRAPH if use_graph else 0) | flags, s))
    return out


class Stream:
    """Streaming recount (aml_stream_*): append time-ordered batches, read
    full-history counts of the resident rows."""

    def __init__(self, pset: PatternSet, n_nodes: int, resident_window: int,
                 mem_budget: int = 8 << 30):
        h = ctypes.c_void_p()
        check(lib().aml_stream_open(pset.handle, int(n_nodes), int(resident_window),
                                    int(mem_budget), ctypes.byref(h)))
        self._h = h
        self.n_cols = pset.n_cols

    def append(self, src, dst, ts, amount=None, stream=None) -> dict:
        if isinstance(src, np.ndarray):
            src = np.ascontiguousarray(src, dtype=np.int32)
            dst = np.ascontiguousarray(dst, dtype=np.int32)
            ts = np.ascontiguousarray(ts, dtype=np.int32)
            if amount is not None:
                amount = np.ascontiguousarray(amount, dtype=np.float32)
        ps, dev = _ptr(src)
        info = aml_stream_batch()
        check(lib().aml_stream_append(self._h, ps, _ptr(dst)[0], _ptr(ts)[0],
                                      _ptr(amount)[0] if amount is not None else None,
                                      int(src.shape[0]), PTR_DEVICE if dev else PTR_HOST,
                                      _stream_handle(stream), ctypes.byref(info)))
        return {f: getattr(info, f) for f, _ in info._fields_}

    def read(self, row0: int, n: int) -> np.ndarray:
        out = np.empty((n, self.n_cols), dtype=np.uint32)
        if n:
            check(lib().aml_stream_read(self._h, int(row0), int(n), out.ctypes.data,
                                        self.n_cols, MINE_HOST_OUTPUT, _stream_handle(None)))
        return out

    def info(self) -> dict:
        inf = aml_stream_info()
        check(lib().aml_stream_get_info(self._h, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in inf._fields_}

    def check_graph(self) -> int:
        """Elements in which the kept window graph differs from a fresh build
        of the same window (0 when they agree)."""
        n = ctypes.c_int64(0)
        check(lib().aml_stream_check_graph(self._h, ctypes.byref(n)))
        return int(n.value)

    def set_count_limit(self, limit: int) -> None:
        """Saturation bound of the stored counts (aml_stream_set_count_limit)."""
        check(lib().aml_stream_set_count_limit(self._h, int(limit)))

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().aml_stream_close(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
