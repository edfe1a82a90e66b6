"""The C ABI library builds, loads and exports every function include/rt.h
declares; host-side argument checks work without a GPU."""
import ctypes
import os
import re

import pytest

from paper_1410_1629_gb300 import rt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+(rt_[a-z0-9_]+)\s*\(", text, re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_calls():
    names = declared_functions()
    for n in ["rt_create_grid", "rt_set_optics", "rt_add_sources", "rt_add_instruments", "rt_launch_packets",
              "rt_read_absorption", "rt_read_images"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    L = rt.lib()
    for name in sorted(declared_functions()):
        assert hasattr(L, name), f"{name} declared but not exported"
    assert set(rt.SIGNATURES) <= declared_functions()


def test_version_and_defaults():
    assert "sm_103a" in rt.rt_version()
    o = rt.rt_default_opts()
    assert o.w_min == 1e-4 and o.max_events == 1000 and o.weight_cut == 1
    assert o.peel_emission == 1 and o.peel_scatter == 1 and o.records is None


def test_null_context_is_rejected():
    L = rt.lib()
    assert L.rt_launch_packets(None, 1, 0, 0, None, None) == rt.RT_ERR_ARG
    assert L.rt_read_stats(None, None) == rt.RT_ERR_ARG
    assert L.rt_context_destroy(None) == rt.RT_OK
    assert L.rt_context_create(0, None) == rt.RT_ERR_ARG


def test_struct_sizes_match_the_header():
    # int32 x4 + 6 doubles + ptr + int64 + ptr + int64 + 2 int32
    assert ctypes.sizeof(rt.rt_grid_desc) == 16 + 48 + 8 + 8 + 8 + 8 + 8
    assert ctypes.sizeof(rt.rt_record) == 40 == rt.RECORD_DTYPE.itemsize
    assert ctypes.sizeof(rt.rt_instrument_desc) == 24 + 8 + 32 + 8
    assert ctypes.sizeof(rt.rt_stats) == 32 + 48 + 8


def test_no_gpu_context_creation_reports_an_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(rt.RTError) as e:
        rt.rt_context_create(0)
    assert e.value.status in (rt.RT_ERR_CUDA, rt.RT_ERR_ARG)
