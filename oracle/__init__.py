"""CPU oracle for RTL stuck-at fault simulation -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import this
package. It shares no code with the CUDA path: `oracle_sim.c` is its own simulator
(its own topological sort, op evaluator and fault forcing) and `mlp.py` its own
forward/backward pass of the load predictor.

The C library is compiled by `build()` with plain gcc; `ctypes` releases the GIL during
each call, so `fault_sim(..., threads=k)` runs k disjoint slices of the fault list on k
host cores at once.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle_sim.c")
_LIB = os.path.join(_HERE, "_build", "liboracle_sim.so")
_lock = threading.Lock()
_lib = None


class _CDesign(ctypes.Structure):
    _fields_ = [
        ("n_in", ctypes.c_int32), ("n_reg", ctypes.c_int32),
        ("n_node", ctypes.c_int32), ("n_out", ctypes.c_int32),
        ("in_w", ctypes.c_void_p), ("reg_w", ctypes.c_void_p), ("reg_d", ctypes.c_void_p),
        ("op", ctypes.c_void_p), ("w", ctypes.c_void_p),
        ("a", ctypes.c_void_p), ("b", ctypes.c_void_p), ("c", ctypes.c_void_p),
        ("imm", ctypes.c_void_p), ("out", ctypes.c_void_p),
    ]


def build(force: bool = False) -> str:
    """Compile oracle_sim.c into a shared library (no machine-specific flags)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _open(path: str):
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER(_CDesign)
    lib.oracle_topo_order.argtypes = [P, ctypes.c_void_p]
    lib.oracle_good_run.argtypes = [P, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p]
    lib.oracle_fault_sim.argtypes = [P, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p]
    lib.oracle_fault_sim_ex.argtypes = [P, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]
    for f in (lib.oracle_topo_order, lib.oracle_good_run, lib.oracle_fault_sim, lib.oracle_fault_sim_ex):
        f.restype = ctypes.c_int
    return lib


class use_library:
    """Context manager: route every oracle call through another build of oracle_sim.c
    (the mutation tests compile deliberately broken copies to show the pins catch them)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        with _lock:
            self.saved = _lib
            _lib = _open(self.path)
        return self

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self.saved
        return False


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _open(build())
    return _lib


class _Pinned:
    """Keeps contiguous copies of a design's arrays alive while C reads them."""

    def __init__(self, d):
        self.arrs = dict(
            in_w=np.ascontiguousarray(d.input_widths, np.uint8),
            reg_w=np.ascontiguousarray(d.reg_widths, np.uint8),
            reg_d=np.ascontiguousarray(d.reg_d, np.uint32),
            op=np.ascontiguousarray(d.node_op, np.uint8),
            w=np.ascontiguousarray(d.node_w, np.uint8),
            a=np.ascontiguousarray(d.node_a, np.uint32),
            b=np.ascontiguousarray(d.node_b, np.uint32),
            c=np.ascontiguousarray(d.node_c, np.uint32),
            imm=np.ascontiguousarray(d.node_imm, np.uint64),
            out=np.ascontiguousarray(d.outputs, np.uint32),
        )
        # a 1-element dummy keeps every pointer non-null for empty arrays
        for k, v in self.arrs.items():
            if v.size == 0:
                self.arrs[k] = np.zeros(1, v.dtype)
        self.c = _CDesign(d.n_in, d.n_reg, d.n_node, d.n_out,
                          *[self.arrs[k].ctypes.data for k in
                            ("in_w", "reg_w", "reg_d", "op", "w", "a", "b", "c", "imm", "out")])


def topo_order(design) -> Optional[np.ndarray]:
    """Node indices in a topological order, or None on a combinational cycle."""
    lib = _load()
    p = _Pinned(design)
    order = np.zeros(max(1, design.n_node), np.int32)
    rc = lib.oracle_topo_order(ctypes.byref(p.c), order.ctypes.data)
    return None if rc != 0 else order[:design.n_node]


def good_run(design, stim: np.ndarray, with_trace: bool = False):
    """Good machine: [T, n_out] output values and, if with_trace, the [T, n_net] values of
    every net in every cycle (the good trace)."""
    lib = _load()
    p = _Pinned(design)
    stim = np.ascontiguousarray(stim, np.uint64)
    T = int(stim.shape[0])
    gout = np.zeros((max(T, 1), max(design.n_out, 1)), np.uint64)
    trace = np.zeros((max(T, 1), max(design.n_net, 1)), np.uint64) if with_trace else None
    s = stim if stim.size else np.zeros(1, np.uint64)
    rc = lib.oracle_good_run(ctypes.byref(p.c), T, s.ctypes.data, gout.ctypes.data,
                             trace.ctypes.data if with_trace else None)
    if rc != 0:
        raise ValueError("combinational cycle")
    gout = gout[:T, :design.n_out]
    return (gout, trace[:T, :design.n_net]) if with_trace else gout


def good_outputs(design, stim: np.ndarray) -> np.ndarray:
    """[T, n_out] uint64 good-machine output values."""
    return good_run(design, stim)


def fault_sim(design, stim: np.ndarray, faults, threads: int = 1,
              gout: Optional[np.ndarray] = None) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Serial single-fault simulation of every fault; returns (detected u8, cycle i32,
    port i32) per fault. `threads` host threads each take a contiguous slice. Faults with
    a `cycle` array (kinds 2 = SEU, 3 = SET in `val`) or port sites (net ids n_net + o)
    go through the general entry point."""
    if getattr(faults, "cycle", None) is not None or (len(faults) and int(np.max(faults.net)) >= design.n_net):
        return fault_sim_ex(design, stim, faults, threads, gout)[:3]
    lib = _load()
    p = _Pinned(design)
    stim = np.ascontiguousarray(stim, np.uint64)
    T = int(stim.shape[0])
    if gout is None:
        gout = good_outputs(design, stim)
    g = np.ascontiguousarray(gout, np.uint64)
    if g.size == 0:
        g = np.zeros(1, np.uint64)
    s = stim if stim.size else np.zeros(1, np.uint64)
    F = len(faults)
    fnet = np.ascontiguousarray(faults.net, np.uint32)
    fbit = np.ascontiguousarray(faults.bit, np.uint8)
    fval = np.ascontiguousarray(faults.val, np.uint8)
    det = np.zeros(max(F, 1), np.uint8)
    cyc = np.zeros(max(F, 1), np.int32)
    port = np.zeros(max(F, 1), np.int32)
    if F == 0:
        return det[:0], cyc[:0], port[:0]

    def run(lo, hi):
        return lib.oracle_fault_sim(ctypes.byref(p.c), T, s.ctypes.data, g.ctypes.data, hi - lo,
                                    fnet[lo:].ctypes.data, fbit[lo:].ctypes.data,
                                    fval[lo:].ctypes.data, det[lo:].ctypes.data,
                                    cyc[lo:].ctypes.data, port[lo:].ctypes.data)

    _in_slices(run, F, threads)
    return det[:F], cyc[:F], port[:F]


def fault_sim_ex(design, stim: np.ndarray, faults, threads: int = 1,
                 gout: Optional[np.ndarray] = None, no_drop: bool = False):
    """The general form: per-fault kinds in `val` (0 SA0, 1 SA1, 2 SEU, 3 SET with the
    flip cycle in `faults.cycle`), port sites (net ids n_net + o), and the no-drop mode.
    Returns (detected u8, cycle i32, port i32, mismatch cycles u32) per fault."""
    lib = _load()
    p = _Pinned(design)
    stim = np.ascontiguousarray(stim, np.uint64)
    T = int(stim.shape[0])
    if gout is None:
        gout = good_outputs(design, stim)
    g = np.ascontiguousarray(gout, np.uint64)
    if g.size == 0:
        g = np.zeros(1, np.uint64)
    s = stim if stim.size else np.zeros(1, np.uint64)
    F = len(faults)
    fnet = np.ascontiguousarray(faults.net, np.uint32)
    fbit = np.ascontiguousarray(faults.bit, np.uint8)
    fkind = np.ascontiguousarray(faults.val, np.uint8)
    cycle = getattr(faults, "cycle", None)
    fcyc = np.ascontiguousarray(cycle if cycle is not None else np.zeros(F), np.uint32)
    det = np.zeros(max(F, 1), np.uint8)
    cyc = np.zeros(max(F, 1), np.int32)
    port = np.zeros(max(F, 1), np.int32)
    mism = np.zeros(max(F, 1), np.uint32)
    if F == 0:
        return det[:0], cyc[:0], port[:0], mism[:0]

    def run(lo, hi):
        return lib.oracle_fault_sim_ex(ctypes.byref(p.c), T, s.ctypes.data, g.ctypes.data, hi - lo,
                                       fnet[lo:].ctypes.data, fbit[lo:].ctypes.data,
                                       fkind[lo:].ctypes.data, fcyc[lo:].ctypes.data,
                                       1 if no_drop else 0, det[lo:].ctypes.data,
                                       cyc[lo:].ctypes.data, port[lo:].ctypes.data,
                                       mism[lo:].ctypes.data)

    _in_slices(run, F, threads)
    return det[:F], cyc[:F], port[:F], mism[:F]


def _in_slices(run, F: int, threads: int) -> None:
    """run(lo, hi) on `threads` contiguous slices of [0, F) in parallel host threads."""
    threads = max(1, min(int(threads), F))
    bounds = np.linspace(0, F, threads + 1).astype(np.int64)
    spans = [(int(bounds[k]), int(bounds[k + 1])) for k in range(threads) if bounds[k + 1] > bounds[k]]
    if len(spans) == 1:
        rcs = [run(*spans[0])]
    else:
        with ThreadPoolExecutor(len(spans)) as ex:
            rcs = list(ex.map(lambda sp: run(*sp), spans))
    if any(rc != 0 for rc in rcs):
        raise ValueError("combinational cycle")


def fault_cycles(detected: np.ndarray, cycle: np.ndarray, T: int) -> int:
    """Work unit W = sum over faults of (cycle+1 if detected else T)."""
    detected = np.asarray(detected).astype(bool)
    return int(np.where(detected, np.asarray(cycle, np.int64) + 1, T).sum())
