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
    # int32 x4 + 6 doubles + ptr + int64 + ptr + int64 + 2 int32 + 3 ptr + ptr
    assert ctypes.sizeof(rt.rt_grid_desc) == 16 + 48 + 8 + 8 + 8 + 8 + 8 + 24 + 8 + 16
    assert ctypes.sizeof(rt.rt_record) == 40 == rt.RECORD_DTYPE.itemsize
    assert ctypes.sizeof(rt.rt_instrument_desc) == 24 + 8 + 32 + 8
    assert ctypes.sizeof(rt.rt_stats) == 32 + 72 + 8


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """Every ctypes struct of the binding has the size and field offsets the
    C compiler gives the header's struct."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = {"rt_grid_desc": rt.rt_grid_desc, "rt_source_desc": rt.rt_source_desc,
               "rt_instrument_desc": rt.rt_instrument_desc, "rt_record": rt.rt_record,
               "rt_trace_row": rt.rt_trace_row, "rt_launch_opts": rt.rt_launch_opts, "rt_stats": rt.rt_stats,
               "rt_model_desc": rt.rt_model_desc}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rt.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            # a trailing underscore marks a C member named like a Python keyword
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f.rstrip("_")}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)


def test_no_gpu_context_creation_reports_an_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(rt.RTError) as e:
        rt.rt_context_create(0)
    assert e.value.status in (rt.RT_ERR_CUDA, rt.RT_ERR_ARG)
