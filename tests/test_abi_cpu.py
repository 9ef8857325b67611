"""C-ABI checks that need no GPU: the library loads, exports every symbol
include/aml.h declares, and its host-only logic (status strings, stage-program
validation and planning, argument checks) behaves as documented."""
import ctypes
import dataclasses
import os
import re

import numpy as np
import pytest

import paper_2604_12241_b300 as aml
from paper_2604_12241_b300 import _lib, patterns as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if hdr.endswith(".h"):
            text = open(os.path.join(ROOT, "include", hdr)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(aml_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = _lib.lib()
    declared = declared_functions()
    assert len(declared) >= 12
    for name in declared:
        assert hasattr(L, name), name
    assert set(declared) == set(_lib.exported_names())


def test_status_strings_and_version():
    L = _lib.lib()
    for code, name in _lib.STATUS.items():
        assert L.aml_status_str(code).decode() == name
    assert L.aml_status_str(12345).decode() == "AML_UNKNOWN_STATUS"
    assert L.aml_version() >= 100


def _ps(pats):
    return aml.PatternSet(pats)


def test_planner_maps_builtin_programs():
    pats = (P.standard(P.DAY, 5)
            + [P.gather_scatter(5, mirrored=True), P.scatter_gather(7, trigger="gather")]
            + [P.cycle(k, 9, closing="intersect") for k in range(3, 8)])
    ps = _ps(pats)
    names = [c["name"] for c in ps.columns]
    assert names[:10] == ["DEG_OUT@86400", "DEG_IN@86400", "FAN_OUT@86400", "FAN_IN@86400",
                          "GS@86400", "SG@86400", "CYC2@86400", "CYC3@86400", "CYC4@86400",
                          "CYC5@86400"]
    assert names[10:] == ["GS@5", "SG@7", "CYC3@9", "CYC4@9", "CYC5@9", "CYC6@9", "CYC7@9"]


def _raw(stages, agg=P.AGG_INSTANCES, delta=10):
    return P.Pattern(tuple(stages), agg, delta)


def _err(pats):
    with pytest.raises(aml.AmlError) as ei:
        _ps(pats)
    return ei.value.name


def test_planner_rejects_invalid_programs():
    T = P.TRIGGER
    # the first stage must be the trigger
    assert _err([_raw([P.Stage(P.OP_FOR_ALL, 0, P.DIR_OUT, out_var=2)])]) == "AML_EINVAL"
    # operand not bound yet
    assert _err([_raw([T, P.Stage(P.OP_FOR_ALL, 3, P.DIR_OUT, out_var=2)])]) == "AML_EINVAL"
    # skip mask names an unbound variable
    assert _err([_raw([T, P.Stage(P.OP_FOR_ALL, 1, P.DIR_OUT, out_var=2, skip_eq=1 << 5)])]) \
        == "AML_EINVAL"
    # closing onto a bound variable before the last stage
    assert _err([_raw([T, P.Stage(P.OP_FOR_ALL, 1, P.DIR_OUT, out_var=0),
                       P.Stage(P.OP_FOR_ALL, 1, P.DIR_OUT, out_var=2)])]) == "AML_EINVAL"
    # bad window, negative delta, bad aggregate
    assert _err([_raw([T, P.Stage(P.OP_FOR_ALL, 1, P.DIR_OUT, out_var=2, window=9)])]) == "AML_EINVAL"
    assert _err([_raw([T, P.Stage(P.OP_FOR_ALL, 0, P.DIR_OUT, out_var=2)], delta=-1)]) == "AML_EINVAL"
    assert _err([_raw([T, P.Stage(P.OP_FOR_ALL, 0, P.DIR_OUT, out_var=2)], agg=7)]) == "AML_EINVAL"


def test_planner_interprets_programs_no_family_matches():
    T = P.TRIGGER
    # valid, but an in-neighbour chain is no implemented family: interpreted
    prog = _raw([T, P.Stage(P.OP_FOR_ALL, 1, P.DIR_IN, out_var=2, order=P.ORDER_AFTER,
                            window=P.WIN_SPAN)])
    # a cycle whose middle stage forgets to skip N0 is not the simple-cycle family
    st = list(P.cycle(4, 10).stages)
    st[1] = P.Stage(P.OP_FOR_ALL, 1, P.DIR_OUT, out_var=2, order=P.ORDER_AFTER,
                    window=P.WIN_SPAN, skip_eq=0b10)
    ps = _ps([prog, _raw(st), P.interpreted(P.gather_scatter(10)), P.gather_scatter(10)])
    fams = [c["family"] for c in ps.columns]
    assert fams == [8, 8, 8, 4]
    assert [c["name"] for c in ps.columns[:3]] == ["PROGRAM0@10", "PROGRAM1@10", "PROGRAM2@10"]


def test_planner_reports_programs_beyond_the_interpreter():
    T = P.TRIGGER
    # LEG order is defined for INTERSECT stages only
    leg = _raw([T, P.Stage(P.OP_FOR_ALL, 1, P.DIR_OUT, out_var=2, order=P.ORDER_LEG,
                           window=P.WIN_SPAN)])
    assert _err([leg]) == "AML_EUNSUPPORTED"
    assert "LEG order" in _lib.lib().aml_last_error().decode()
    # nine stages that are no cycle: beyond the interpreter's eight
    chain = [T] + [P.Stage(P.OP_FOR_ALL, v, P.DIR_OUT, out_var=v + 1, window=P.WIN_SPAN)
                   for v in range(1, 9)]
    assert _err([_raw(chain)]) == "AML_EUNSUPPORTED"
    assert "at most 8 stages" in _lib.lib().aml_last_error().decode()
    # unknown pattern flag bits
    bad = _raw([T, P.Stage(P.OP_FOR_ALL, 0, P.DIR_OUT, out_var=2)])
    arr, keep = _lib.make_patterns([bad])
    arr[0].flags = 0x6
    h = ctypes.c_void_p()
    assert _lib.lib().aml_pattern_set_create(arr, 1, ctypes.byref(h)) == 1


def test_planner_counts_sets_for_scatter_gathers_of_n_intermediaries_only():
    T = P.TRIGGER
    ps = _ps([P.scatter_gather_exact(2, 10), P.scatter_gather_exact(2, 10, interpret=True),
              P.scatter_gather_exact(3, 10), P.scatter_gather_exact(7, 10)])
    assert [c["family"] for c in ps.columns] == [5, 8, 8, 8]   # SG, then interpreted
    # SETS of another program, or of a scatter-gather with amount constraints
    # or a missing skip, has no definition here
    assert _err([P.Pattern(P.gather_scatter(10).stages, P.AGG_SETS, 10)]) == "AML_EUNSUPPORTED"
    assert "AML_AGG_SETS" in _lib.lib().aml_last_error().decode()
    st = list(P.scatter_gather_n(3, 10).stages)
    st[3] = dataclasses.replace(st[3], skip_eq=0b10)
    assert _err([P.Pattern(tuple(st), P.AGG_SETS, 10)]) == "AML_EUNSUPPORTED"
    st = list(P.scatter_gather_n(3, 10).stages)
    st[2] = dataclasses.replace(st[2], amount_flags=1, amount_min=0.0, amount_max=5.0)
    assert _err([P.Pattern(tuple(st), P.AGG_SETS, 10)]) == "AML_EUNSUPPORTED"
    assert _err([P.Pattern((T,), P.AGG_SETS, 10)]) == "AML_EUNSUPPORTED"


def test_argument_errors_need_no_device():
    L = _lib.lib()
    h = ctypes.c_void_p()
    src = np.zeros(4, np.int32)
    # NULL out, negative sizes and unknown flags are rejected before any CUDA call
    assert L.aml_graph_create(src.ctypes.data, src.ctypes.data, src.ctypes.data, None, 4, 3, 0,
                              None, None) == 1
    assert L.aml_graph_create(src.ctypes.data, src.ctypes.data, src.ctypes.data, None, -1, 3, 0,
                              None, ctypes.byref(h)) == 1
    assert L.aml_graph_create(src.ctypes.data, src.ctypes.data, src.ctypes.data, None, 4, 0, 0,
                              None, ctypes.byref(h)) == 1
    assert L.aml_graph_create(src.ctypes.data, src.ctypes.data, src.ctypes.data, None, 4, 3, 0x80,
                              None, ctypes.byref(h)) == 1
    assert L.aml_mine(None, None, None, 0, 0, None) == 1
    assert L.aml_sync(None) == 1
    assert L.aml_graph_set_count_limit(None, 5) == 1
    assert L.aml_stream_set_count_limit(None, 5) == 1
    assert L.aml_graph_destroy(None) == 0
    assert "NULL" in L.aml_last_error().decode() or L.aml_last_error() is not None


def test_no_device_maps_to_ecuda():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    L = _lib.lib()
    h = ctypes.c_void_p()
    src = np.array([0, 1], np.int32)
    dst = np.array([1, 0], np.int32)
    ts = np.array([0, 1], np.int32)
    rc = L.aml_graph_create(src.ctypes.data, dst.ctypes.data, ts.ctypes.data, None, 2, 2, 0, None,
                            ctypes.byref(h))
    assert rc == 3  # AML_ECUDA: no CUDA device here
    assert L.aml_last_error().decode()
