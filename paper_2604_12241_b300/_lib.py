"""ctypes binding of libaml_b300.so (argument marshalling only).

Function names match the C ABI in include/aml.h.  Every status other than
AML_OK raises ``AmlError`` carrying aml_last_error().  There is no fallback:
if the shared library is missing or fails to load, importing anything that
needs it raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libaml_b300.so")

STATUS = {0: "AML_OK", 1: "AML_EINVAL", 2: "AML_ENOMEM", 3: "AML_ECUDA", 4: "AML_EUNSUPPORTED",
          5: "AML_EUNSORTED", 6: "AML_ELATE", 7: "AML_EADMIT", 8: "AML_ETIMEOUT",
          9: "AML_EINTERNAL"}

PTR_HOST, PTR_DEVICE, ASSUME_SORTED = 0x0, 0x1, 0x2
MINE_HOST_OUTPUT = 0x1
MINE_GRAPH = 0x2
MINE_PERSISTENT = 0x4
MINE_LEARNED = 0x8
MINE_HOST_ASYNC = 0x10
MINE_FUSED = 0x20


class AmlError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class aml_stage(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("a_var", ctypes.c_int32), ("a_dir", ctypes.c_int32),
                ("b_var", ctypes.c_int32), ("b_dir", ctypes.c_int32), ("out_var", ctypes.c_int32),
                ("order", ctypes.c_int32), ("window", ctypes.c_int32), ("skip_eq", ctypes.c_uint32),
                ("amount_flags", ctypes.c_uint32), ("amount_min", ctypes.c_float),
                ("amount_max", ctypes.c_float), ("ratio_min", ctypes.c_float),
                ("ratio_max", ctypes.c_float)]


class aml_pattern(ctypes.Structure):
    _fields_ = [("stages", ctypes.POINTER(aml_stage)), ("n_stages", ctypes.c_int32),
                ("aggregate", ctypes.c_int32), ("delta", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


PAT_INTERPRET = 0x1


class aml_graph_info(ctypes.Structure):
    _fields_ = [("n_edges", ctypes.c_int64), ("n_list_edges", ctypes.c_int64),
                ("n_nodes", ctypes.c_int32), ("max_out_degree", ctypes.c_int32),
                ("max_in_degree", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64)]


class aml_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double)]


class aml_tuning(ctypes.Structure):
    _fields_ = [("own_max", ctypes.c_int32), ("sg_bucket_mean", ctypes.c_int32),
                ("close_scan_max", ctypes.c_int32), ("block", ctypes.c_int32)]


class aml_stream_batch(ctypes.Structure):
    _fields_ = [("first_row", ctypes.c_int64), ("n_rows", ctypes.c_int64),
                ("rows_recounted", ctypes.c_int64), ("resident_first_row", ctypes.c_int64),
                ("resident_rows", ctypes.c_int64)]


class aml_stream_info(ctypes.Structure):
    _fields_ = [("resident_first_row", ctypes.c_int64), ("resident_rows", ctypes.c_int64),
                ("capacity_rows", ctypes.c_int64), ("final_end_row", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("t_max", ctypes.c_int32),
                ("delta_max", ctypes.c_int32)]


class aml_cost_report(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_int32), ("epochs", ctypes.c_int32), ("n_items", ctypes.c_int64),
                ("n_train", ctypes.c_int64), ("n_test", ctypes.c_int64),
                ("final_train_mse", ctypes.c_float), ("test_log_mae", ctypes.c_float),
                ("test_spearman", ctypes.c_float), ("degree_spearman", ctypes.c_float),
                ("warp_threshold_cycles", ctypes.c_float), ("probe_ms", ctypes.c_float),
                ("total_ms", ctypes.c_float)]


class aml_column_info(ctypes.Structure):
    _fields_ = [("family", ctypes.c_int32), ("k", ctypes.c_int32), ("delta", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("name", ctypes.c_char * 32)]


_VP = ctypes.c_void_p
_SIGS = {
    "aml_status_str": (ctypes.c_char_p, [ctypes.c_int32]),
    "aml_last_error": (ctypes.c_char_p, []),
    "aml_version": (ctypes.c_int32, []),
    "aml_graph_create": (ctypes.c_int32, [_VP, _VP, _VP, _VP, ctypes.c_int64, ctypes.c_int32,
                                          ctypes.c_uint32, _VP, ctypes.POINTER(_VP)]),
    "aml_graph_destroy": (ctypes.c_int32, [_VP]),
    "aml_graph_get_info": (ctypes.c_int32, [_VP, ctypes.POINTER(aml_graph_info)]),
    "aml_graph_window_stats": (ctypes.c_int32, [_VP, ctypes.c_int32,
                                                ctypes.POINTER(ctypes.c_int64),
                                                ctypes.POINTER(ctypes.c_int64)]),
    "aml_pattern_set_create": (ctypes.c_int32, [ctypes.POINTER(aml_pattern), ctypes.c_int32,
                                                ctypes.POINTER(_VP)]),
    "aml_pattern_set_destroy": (ctypes.c_int32, [_VP]),
    "aml_pattern_set_num_columns": (ctypes.c_int32, [_VP, ctypes.POINTER(ctypes.c_int32)]),
    "aml_pattern_set_column": (ctypes.c_int32, [_VP, ctypes.c_int32,
                                                ctypes.POINTER(aml_column_info)]),
    "aml_mine": (ctypes.c_int32, [_VP, _VP, _VP, ctypes.c_int64, ctypes.c_uint32, _VP]),
    "aml_sync": (ctypes.c_int32, [_VP]),
    "aml_graph_get_tuning": (ctypes.c_int32, [_VP, ctypes.POINTER(aml_tuning)]),
    "aml_graph_set_tuning": (ctypes.c_int32, [_VP, ctypes.POINTER(aml_tuning)]),
    "aml_graph_set_count_limit": (ctypes.c_int32, [_VP, ctypes.c_uint32]),
    "aml_graph_set_wait_limit": (ctypes.c_int32, [_VP, ctypes.c_int64]),
    "aml_autotune": (ctypes.c_int32, [_VP, _VP, ctypes.c_int32, _VP, ctypes.POINTER(aml_tuning),
                                      ctypes.POINTER(ctypes.c_float)]),
    "aml_stream_open": (ctypes.c_int32, [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_size_t,
                                         ctypes.POINTER(_VP)]),
    "aml_stream_append": (ctypes.c_int32, [_VP, _VP, _VP, _VP, _VP, ctypes.c_int64,
                                           ctypes.c_uint32, _VP,
                                           ctypes.POINTER(aml_stream_batch)]),
    "aml_stream_read": (ctypes.c_int32, [_VP, ctypes.c_int64, ctypes.c_int64, _VP,
                                         ctypes.c_int64, ctypes.c_uint32, _VP]),
    "aml_stream_get_info": (ctypes.c_int32, [_VP, ctypes.POINTER(aml_stream_info)]),
    "aml_stream_check_graph": (ctypes.c_int32, [_VP, ctypes.POINTER(ctypes.c_int64)]),
    "aml_stream_close": (ctypes.c_int32, [_VP]),
    "aml_stream_set_count_limit": (ctypes.c_int32, [_VP, ctypes.c_uint32]),
    "aml_fan_noalloc": (ctypes.c_int32, [_VP, ctypes.c_int32, ctypes.c_int32, _VP, _VP]),
    "aml_cost_train": (ctypes.c_int32, [_VP, _VP, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                        _VP, ctypes.POINTER(aml_cost_report)]),
    "aml_mlp_loss_grad": (ctypes.c_int32, [_VP, _VP, _VP, ctypes.c_int64, _VP, _VP]),
    "aml_mlp_adam_step": (ctypes.c_int32, [_VP, _VP, _VP, _VP, ctypes.c_int32, ctypes.c_float,
                                           ctypes.c_float, ctypes.c_float, ctypes.c_float]),
    "aml_mlp_predict": (ctypes.c_int32, [_VP, _VP, _VP, ctypes.c_int64, _VP]),
    "aml_launch_count": (ctypes.c_int32, [ctypes.POINTER(ctypes.c_int64)]),
    "aml_profile_enable": (ctypes.c_int32, [ctypes.c_int32]),
    "aml_profile_read": (ctypes.c_int32, [ctypes.POINTER(aml_kernel_stat), ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]),
}

_lib: Optional[ctypes.CDLL] = None


def exported_names() -> Sequence[str]:
    return list(_SIGS)


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it was not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "or `python -m paper_2604_12241_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int) -> None:
    if status != 0:
        raise AmlError(status, lib().aml_last_error().decode(errors="replace"))


def make_patterns(patterns) -> tuple:
    """ctypes aml_pattern array (and the stage arrays it points into)."""
    keep = []
    arr = (aml_pattern * len(patterns))()
    for i, p in enumerate(patterns):
        st = (aml_stage * len(p.stages))()
        for j, s in enumerate(p.stages):
            st[j] = aml_stage(s.op, s.a_var, s.a_dir, s.b_var, s.b_dir, s.out_var, s.order,
                              s.window, s.skip_eq, s.amount_flags, s.amount_min, s.amount_max,
                              s.ratio_min, s.ratio_max)
        keep.append(st)
        arr[i].stages = ctypes.cast(st, ctypes.POINTER(aml_stage))
        arr[i].n_stages = len(p.stages)
        arr[i].aggregate = p.aggregate
        arr[i].delta = p.delta
        arr[i].flags = PAT_INTERPRET if getattr(p, "interpret", False) else 0
    return arr, keep


def launch_count() -> int:
    n = ctypes.c_int64()
    check(lib().aml_launch_count(ctypes.byref(n)))
    return n.value


def profile_enable(on: bool) -> None:
    check(lib().aml_profile_enable(1 if on else 0))


def profile_read(reset: bool = True) -> dict:
    """{kernel name: (launches, total_ms)} of the timed launches so far."""
    n = ctypes.c_int32()
    check(lib().aml_profile_read(None, 0, ctypes.byref(n), 0))
    arr = (aml_kernel_stat * max(1, n.value))()
    check(lib().aml_profile_read(arr, n.value, ctypes.byref(n), 1 if reset else 0))
    return {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms) for i in range(n.value)}
