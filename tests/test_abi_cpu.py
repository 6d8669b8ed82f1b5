"""CPU-side checks of the C-ABI boundary: the library builds, loads, and exports every
entry point declared in include/*.h; the binding's struct layouts match the header's
stated sizes. No compute call is made (there may be no GPU here)."""
import ctypes
import glob
import os
import re

import numpy as np

from paper_2508_16376_gb300 import build, rtlfs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(rtlfs_[a-z_0-9]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    names = _declared()
    assert "rtlfs_run" in names and "rtlfs_load_design" in names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    # every declared entry point has a binding with the same name
    assert names <= set(rtlfs.EXPORTS) | {n for n in names if n.startswith("rtlfs_x")}


def test_struct_sizes_match_header():
    assert rtlfs.NODE_DTYPE.itemsize == 24
    assert rtlfs.REG_DTYPE.itemsize == 8
    assert rtlfs.FAULT_DTYPE.itemsize == 8
    assert rtlfs.RESULT_DTYPE.itemsize == 12
    assert rtlfs.FAULT_EX_DTYPE.itemsize == 16
    assert ctypes.sizeof(rtlfs.rtlfs_run_opts) == 4 * 6 + 8 + 36 + 4   # + tail padding to 8
    assert ctypes.sizeof(rtlfs.rtlfs_stats) == 6 * 8 + 4 * 8 + 8 + 4 * 8


def test_binding_layouts_match_the_compiled_header(tmp_path):
    """Sizes and field offsets as a C compiler lays out include/rtlfs.h equal the
    binding's ctypes structures and numpy record types."""
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    checks = {
        "rtlfs_node": ("NODE_DTYPE", ["op", "width", "a", "b", "c", "imm"]),
        "rtlfs_reg": ("REG_DTYPE", ["d_net", "width"]),
        "rtlfs_fault": ("FAULT_DTYPE", ["net", "bit", "stuck"]),
        "rtlfs_fault_ex": ("FAULT_EX_DTYPE", ["net", "bit", "kind", "cycle"]),
        "rtlfs_result": ("RESULT_DTYPE", ["cycle", "port", "detected"]),
    }
    ctypes_checks = {"rtlfs_run_opts": rtlfs.rtlfs_run_opts, "rtlfs_stats": rtlfs.rtlfs_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rtlfs.h"', "int main(void) {"]
    for st, (_, fields) in checks.items():
        lines.append(f'printf("{st} size %zu\\n", sizeof({st}));')
        for fl in fields:
            lines.append(f'printf("{st} {fl} %zu\\n", offsetof({st}, {fl}));')
    for st, cls in ctypes_checks.items():
        lines.append(f'printf("{st} size %zu\\n", sizeof({st}));')
        for fl, _ in cls._fields_:
            if fl != "reserved":
                lines.append(f'printf("{st} {fl} %zu\\n", offsetof({st}, {fl}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = str(tmp_path / "layout")
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(root, "include"), "-o", exe, str(src)])
    got = {}
    for line in subprocess.check_output([exe]).decode().splitlines():
        st, fl, v = line.split()
        got[(st, fl)] = int(v)
    for st, (dt, fields) in checks.items():
        d = getattr(rtlfs, dt)
        assert got[(st, "size")] == d.itemsize, st
        for fl in fields:
            assert got[(st, fl)] == d.fields[fl][1], (st, fl)
    for st, cls in ctypes_checks.items():
        assert got[(st, "size")] == ctypes.sizeof(cls), st
        for fl, _ in cls._fields_:
            if fl != "reserved":
                assert got[(st, fl)] == getattr(cls, fl).offset, (st, fl)


def test_create_without_device_fails_cleanly():
    """With no usable GPU, rtlfs_create returns an error status instead of crashing."""
    import torch
    if torch.cuda.is_available():
        return
    lib = rtlfs.load_library()
    h = ctypes.c_void_p()
    rc = lib.rtlfs_create(ctypes.byref(h), 0)
    assert rc != rtlfs.RTLFS_OK and not h.value


def test_binding_raises_without_library(tmp_path):
    try:
        rtlfs.load_library(str(tmp_path / "missing.so"))
    except RuntimeError as e:
        assert "not built" in str(e)
    else:
        raise AssertionError("expected a loud failure")


def test_design_arrays_roundtrip():
    from paper_2508_16376_gb300 import synth
    d = synth.tiny_design(1)
    nodes, regs, iw, outs = rtlfs.design_arrays(d)
    assert np.array_equal(nodes["a"], d.node_a) and np.array_equal(regs["d_net"], d.reg_d)
    assert len(iw) == d.n_in and len(outs) == d.n_out
