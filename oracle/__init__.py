"""CPU oracle for per-edge AML pattern counts -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It wraps ``aml_oracle.c`` (plain C + OpenMP) via
ctypes and shares no code with the CUDA library.

Columns are ``(kind, delta)`` or ``("cyc", k, delta)`` tuples with kind one of
``deg_out, deg_in, fan_out, fan_in, gs, sg, cyc``; the definitions are the
ones in ``aml_oracle.h`` (the paper's stage semantics, Sec. 5 and Alg. 1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Iterable, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aml_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

KINDS = {"deg_out": 0, "deg_in": 1, "fan_out": 2, "fan_in": 3, "gs": 4, "sg": 5, "cyc": 6,
         "cycw": 7}


class _Col(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("k", ctypes.c_int32), ("delta", ctypes.c_int64)]


class _Stage(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int32) for f in
                ("op", "a_var", "a_dir", "b_var", "b_dir", "out_var", "order", "window")] + \
               [("skip_eq", ctypes.c_uint32), ("amount_flags", ctypes.c_uint32)] + \
               [(f, ctypes.c_float) for f in ("amount_min", "amount_max", "ratio_min",
                                              "ratio_max")]


STAGE_FIELDS = ("op", "a_var", "a_dir", "b_var", "b_dir", "out_var", "order", "window",
                "skip_eq", "amount_flags", "amount_min", "amount_max", "ratio_min", "ratio_max")


# stage-program vocabulary (the values of the library's ABI, restated)
OP_TRIGGER, OP_FOR_ALL, OP_INTERSECT = 0, 1, 2
DIR_OUT, DIR_IN = 0, 1
ORD_NONE, ORD_AFTER, ORD_BEFORE, ORD_LEG, ORD_AFTER_TRIGGER = 0, 1, 2, 3, 4
WIN_TRAILING, WIN_SPAN = 0, 1
AGG_EDGES, AGG_DISTINCT, AGG_INSTANCES, AGG_SETS = 0, 1, 2, 3
AMT_RANGE, AMT_RATIO = 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -fopenmp) if the .so is stale."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)
            and os.path.getmtime(_LIB) >= os.path.getmtime(os.path.join(_HERE, "aml_oracle.h"))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-Wall", "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def load_library(path: str) -> ctypes.CDLL:
    """Load an oracle shared library and declare its signatures."""
    lib = ctypes.CDLL(path)
    lib.og_graph_new.restype = ctypes.c_void_p
    lib.og_graph_new.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int64, ctypes.c_int32]
    lib.og_graph_free.argtypes = [ctypes.c_void_p]
    lib.og_count_all.restype = ctypes.c_int
    lib.og_count_all.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                 ctypes.c_void_p, ctypes.c_int32]
    lib.og_graph_set_amounts.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.og_program_count.restype = ctypes.c_int
    lib.og_program_count.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                     ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p,
                                     ctypes.c_int32]
    lib.og_count_edges.restype = ctypes.c_int
    lib.og_count_edges.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                   ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                   ctypes.c_int32]
    lib.og_count_all_limit.restype = ctypes.c_int
    lib.og_count_all_limit.argtypes = lib.og_count_all.argtypes + [ctypes.c_uint32]
    lib.og_count_edges_limit.restype = ctypes.c_int
    lib.og_count_edges_limit.argtypes = lib.og_count_edges.argtypes + [ctypes.c_uint32]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = load_library(build())
    return _lib


def _cols(cols: Sequence[Tuple]) -> ctypes.Array:
    arr = (_Col * len(cols))()
    for i, c in enumerate(cols):
        if c[0] in ("cyc", "cycw"):
            arr[i].kind, arr[i].k, arr[i].delta = KINDS[c[0]], int(c[1]), int(c[2])
        else:
            arr[i].kind, arr[i].k, arr[i].delta = KINDS[c[0]], 0, int(c[1])
    return arr


def columns_from_names(names: Sequence[str]) -> list:
    """Column tuples for column names of the form FAMILY@delta (DEG_OUT@86400,
    CYC3@86400, CYCW4@604800, ...), the names the library gives its columns."""
    out = []
    for name in names:
        fam, _, rest = name.partition("@")
        d = int(rest)
        if fam.startswith("CYCW"):
            out.append(("cycw", int(fam[4:]), d))
        elif fam.startswith("CYC"):
            out.append(("cyc", int(fam[3:]), d))
        else:
            kind = fam.lower()
            if kind not in KINDS:
                raise ValueError(f"no oracle column for {name}")
            out.append((kind, d))
    return out


class OracleGraph:
    """Host copy of the graph with (t,id)-sorted out/in rows."""

    def __init__(self, src, dst, ts, n_nodes: int, lib: ctypes.CDLL = None, amount=None):
        self._lib = lib = lib if lib is not None else _load()
        self._src = np.ascontiguousarray(src, dtype=np.int32)
        self._dst = np.ascontiguousarray(dst, dtype=np.int32)
        self._ts = np.ascontiguousarray(ts, dtype=np.int32)
        self.n_edges = int(self._src.shape[0])
        self.n_nodes = int(n_nodes)
        self._h = lib.og_graph_new(self._src.ctypes.data, self._dst.ctypes.data,
                                   self._ts.ctypes.data, self.n_edges, self.n_nodes)
        if not self._h:
            raise ValueError("oracle rejected the graph (ids out of range?)")
        if amount is not None:
            self._amount = np.ascontiguousarray(amount, dtype=np.float32)
            lib.og_graph_set_amounts(self._h, self._amount.ctypes.data)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.og_graph_free(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def count_all(self, cols: Sequence[Tuple], threads: int = 0,
                  limit: int = 0xFFFFFFFF) -> np.ndarray:
        """Canonical enumeration over the whole graph: uint32 [E, len(cols)],
        every count saturated at ``limit`` (2^32-1 unless a test lowers it)."""
        out = np.zeros((self.n_edges, len(cols)), dtype=np.uint32)
        rc = self._lib.og_count_all_limit(self._h, ctypes.byref(_cols(cols)), len(cols),
                                          out.ctypes.data, threads, int(limit))
        if rc:
            raise ValueError(f"og_count_all failed ({rc})")
        return out

    def count_edges(self, cols: Sequence[Tuple], eids: Iterable[int],
                    threads: int = 0, limit: int = 0xFFFFFFFF) -> np.ndarray:
        """Edge-centric query for the listed edges: uint32 [n, len(cols)],
        saturated at ``limit`` like ``count_all``."""
        ids = np.ascontiguousarray(np.asarray(list(eids) if not isinstance(eids, np.ndarray)
                                              else eids, dtype=np.int64))
        out = np.zeros((ids.shape[0], len(cols)), dtype=np.uint32)
        rc = self._lib.og_count_edges_limit(self._h, ctypes.byref(_cols(cols)), len(cols),
                                            ids.ctypes.data, ids.shape[0], out.ctypes.data,
                                            threads, int(limit))
        if rc:
            raise ValueError(f"og_count_edges failed ({rc})")
        return out

    def program_count(self, stages: Sequence[Sequence[int]], aggregate: int, delta: int,
                      threads: int = 0) -> np.ndarray:
        """One stage program interpreted as ``og_program_count`` defines it:
        uint32 [E].  ``stages`` = (op, a_var, a_dir, b_var, b_dir, out_var,
        order, window, skip_eq[, amount_flags, amount_min, amount_max,
        ratio_min, ratio_max]) tuples, stage 0 the trigger."""
        arr = (_Stage * len(stages))()
        for i, st in enumerate(stages):
            for f, v in zip(STAGE_FIELDS, st):
                setattr(arr[i], f, float(v) if f.endswith(("_min", "_max")) else int(v))
        out = np.zeros(self.n_edges, dtype=np.uint32)
        rc = self._lib.og_program_count(self._h, ctypes.byref(arr), len(stages), int(aggregate),
                                        int(delta), out.ctypes.data, threads)
        if rc:
            raise ValueError(f"og_program_count rejected the program ({rc})")
        return out
