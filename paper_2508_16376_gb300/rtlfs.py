"""Thin ctypes binding of librtlfs (include/rtlfs.h): same entry-point names, argument
marshalling only. Every step of the simulation runs in the library's CUDA kernels; if
the library is missing or cannot be loaded this module raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librtlfs.so")

RTLFS_OK = 0
RTLFS_E_ARG = -1
RTLFS_E_CYCLE = -2
RTLFS_E_WIDTH = -3
RTLFS_E_NOMEM = -4
RTLFS_E_CUDA = -5
RTLFS_E_TIMEOUT = -6
RTLFS_E_STATE = -7
SCHED_PLAIN, SCHED_HEURISTIC, SCHED_MLP = 0, 1, 2

NODE_DTYPE = np.dtype([("op", np.uint8), ("width", np.uint8), ("reserved", np.uint16),
                       ("a", np.uint32), ("b", np.uint32), ("c", np.uint32), ("imm", np.uint64)])
REG_DTYPE = np.dtype([("d_net", np.uint32), ("width", np.uint8), ("reserved", np.uint8, 3)])
FAULT_DTYPE = np.dtype([("net", np.uint32), ("bit", np.uint8), ("stuck", np.uint8),
                        ("reserved", np.uint16)])
RESULT_DTYPE = np.dtype([("cycle", np.int32), ("port", np.int32), ("detected", np.uint8),
                         ("reserved", np.uint8, 3)])
FAULT_EX_DTYPE = np.dtype([("net", np.uint32), ("bit", np.uint8), ("kind", np.uint8),
                           ("reserved", np.uint16), ("cycle", np.uint32), ("reserved2", np.uint32)])
FAULT_SA0, FAULT_SA1, FAULT_SEU, FAULT_SET = 0, 1, 2, 3
assert NODE_DTYPE.itemsize == 24 and REG_DTYPE.itemsize == 8
assert FAULT_DTYPE.itemsize == 8 and RESULT_DTYPE.itemsize == 12 and FAULT_EX_DTYPE.itemsize == 16


class rtlfs_run_opts(ctypes.Structure):
    _fields_ = [("scheduler", ctypes.c_int32), ("light_block", ctypes.c_int32),
                ("heavy_block", ctypes.c_int32), ("heavy_ctas", ctypes.c_int32),
                ("heavy_frac", ctypes.c_float), ("use_graph", ctypes.c_int32),
                ("fault_budget", ctypes.c_uint64), ("light_cap", ctypes.c_int32),
                ("window", ctypes.c_int32), ("no_drop", ctypes.c_int32),
                ("stop_cycle", ctypes.c_int32), ("resume", ctypes.c_int32),
                ("heavy_form", ctypes.c_int32), ("good_cluster", ctypes.c_int32),
                ("good_staging", ctypes.c_int32), ("good_first", ctypes.c_int32),
                ("order_classes", ctypes.c_int32)]


class rtlfs_stats(ctypes.Structure):
    _fields_ = [("total_ms", ctypes.c_double), ("good_ms", ctypes.c_double),
                ("prep_ms", ctypes.c_double), ("faulty_ms", ctypes.c_double),
                ("light_ms", ctypes.c_double), ("heavy_ms", ctypes.c_double),
                ("fault_cycles", ctypes.c_uint64), ("node_evals", ctypes.c_uint64),
                ("promoted", ctypes.c_uint64), ("heavy_initial", ctypes.c_uint64),
                ("n_launches", ctypes.c_uint32), ("heavy_form", ctypes.c_uint32),
                ("light_evals", ctypes.c_uint64), ("light_fault_cycles", ctypes.c_uint64),
                ("heavy_evals", ctypes.c_uint64), ("heavy_fault_cycles", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class RtlfsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rtlfs error {code}: {msg}")
        self.code = code


_lib = None
V = ctypes.c_void_p
EXPORTS = {
    "rtlfs_create": ([V, ctypes.c_int], ctypes.c_int),
    "rtlfs_destroy": ([V], None),
    "rtlfs_last_error": ([V], ctypes.c_char_p),
    "rtlfs_load_design": ([V, V, ctypes.c_uint32, V, ctypes.c_uint32, V, ctypes.c_uint32, V,
                           ctypes.c_uint32, V], ctypes.c_int),
    "rtlfs_set_stimulus": ([V, ctypes.c_uint32, V, ctypes.c_uint32], ctypes.c_int),
    "rtlfs_set_faults": ([V, ctypes.c_uint32, V, ctypes.c_uint32], ctypes.c_int),
    "rtlfs_set_faults_ex": ([V, ctypes.c_uint32, V, ctypes.c_uint32], ctypes.c_int),
    "rtlfs_mismatch_counts": ([V, ctypes.c_uint32, V], ctypes.c_int),
    "rtlfs_run": ([V, V, V, V], ctypes.c_int),
    "rtlfs_run_plain": ([V, V], ctypes.c_int),
    "rtlfs_get_stats": ([V, V], ctypes.c_int),
    "rtlfs_good_outputs": ([V, ctypes.c_uint32, V], ctypes.c_int),
    "rtlfs_good_trace": ([V, ctypes.c_uint32, V], ctypes.c_int),
    "rtlfs_design_info": ([V, ctypes.c_uint32, V, V, V], ctypes.c_int),
    "rtlfs_features": ([V, ctypes.c_uint32, V], ctypes.c_int),
    "rtlfs_mlp_set_weights": ([V, V], ctypes.c_int),
    "rtlfs_mlp_get_weights": ([V, V], ctypes.c_int),
    "rtlfs_mlp_forward": ([V, V, ctypes.c_uint32, V], ctypes.c_int),
    "rtlfs_mlp_grad": ([V, V, V, ctypes.c_uint32, V, V], ctypes.c_int),
    "rtlfs_mlp_train": ([V, V, V, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                         ctypes.c_float, V], ctypes.c_int),
    "rtlfs_fault_sim_static": ([V, ctypes.c_uint32, V, ctypes.c_uint32, V, V], ctypes.c_int),
    "rtlfs_checkpoint_size": ([V, V], ctypes.c_int),
    "rtlfs_checkpoint_save": ([V, V, ctypes.c_uint64], ctypes.c_int),
    "rtlfs_checkpoint_load": ([V, V, ctypes.c_uint64], ctypes.c_int),
}
RTLFS_PENDING = 254
MLP_PARAMS = 4609
MLP_IN = 5


def load_library(path: Optional[str] = None):
    """Load librtlfs.so (built by paper_2508_16376_gb300.build); raises if absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"librtlfs not built: {p} missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(p)
    for name, (args, res) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    if path is None:
        _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data if a.size else None


# ---- entry points with the ABI's names --------------------------------------------------

def rtlfs_create(device: int = 0) -> ctypes.c_void_p:
    lib = load_library()
    h = ctypes.c_void_p()
    rc = lib.rtlfs_create(ctypes.byref(h), device)
    if rc != RTLFS_OK:
        raise RtlfsError(rc, "rtlfs_create failed")
    return h


def rtlfs_destroy(ctx) -> None:
    load_library().rtlfs_destroy(ctx)


def rtlfs_last_error(ctx) -> str:
    return load_library().rtlfs_last_error(ctx).decode()


def _check(ctx, rc: int) -> int:
    if rc != RTLFS_OK:
        raise RtlfsError(rc, rtlfs_last_error(ctx))
    return rc


def design_arrays(design) -> Tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
    """AoS arrays of the ABI from a synth.Design (structure of arrays)."""
    nodes = np.zeros(design.n_node, NODE_DTYPE)
    nodes["op"] = design.node_op
    nodes["width"] = design.node_w
    nodes["a"] = design.node_a
    nodes["b"] = design.node_b
    nodes["c"] = design.node_c
    nodes["imm"] = design.node_imm
    regs = np.zeros(design.n_reg, REG_DTYPE)
    regs["d_net"] = design.reg_d
    regs["width"] = design.reg_widths
    return (nodes, regs, np.ascontiguousarray(design.input_widths, np.uint8),
            np.ascontiguousarray(design.outputs, np.uint32))


def rtlfs_load_design(ctx, nodes: np.ndarray, regs: np.ndarray, input_widths: np.ndarray,
                      output_nets: np.ndarray) -> int:
    lib = load_library()
    did = ctypes.c_uint32()
    nodes = np.ascontiguousarray(nodes, NODE_DTYPE)
    regs = np.ascontiguousarray(regs, REG_DTYPE)
    iw = np.ascontiguousarray(input_widths, np.uint8)
    on = np.ascontiguousarray(output_nets, np.uint32)
    rc = lib.rtlfs_load_design(ctx, _ptr(nodes), len(nodes), _ptr(regs), len(regs), _ptr(iw),
                               len(iw), _ptr(on), len(on), ctypes.byref(did))
    _check(ctx, rc)
    return did.value


def rtlfs_set_stimulus(ctx, design_id: int, inputs: np.ndarray) -> None:
    x = np.ascontiguousarray(inputs, np.uint64)
    _check(ctx, load_library().rtlfs_set_stimulus(ctx, design_id, _ptr(x), int(x.shape[0])))


def fault_array(faults) -> np.ndarray:
    a = np.zeros(len(faults), FAULT_DTYPE)
    a["net"] = faults.net
    a["bit"] = faults.bit
    a["stuck"] = faults.val
    return a


def rtlfs_set_faults(ctx, design_id: int, faults: np.ndarray) -> None:
    x = np.ascontiguousarray(faults, FAULT_DTYPE)
    _check(ctx, load_library().rtlfs_set_faults(ctx, design_id, _ptr(x), len(x)))


def fault_array_ex(faults) -> np.ndarray:
    a = np.zeros(len(faults), FAULT_EX_DTYPE)
    a["net"] = faults.net
    a["bit"] = faults.bit
    a["kind"] = faults.val
    if getattr(faults, "cycle", None) is not None:
        a["cycle"] = faults.cycle
    return a


def rtlfs_set_faults_ex(ctx, design_id: int, faults: np.ndarray) -> None:
    x = np.ascontiguousarray(faults, FAULT_EX_DTYPE)
    _check(ctx, load_library().rtlfs_set_faults_ex(ctx, design_id, _ptr(x), len(x)))


def rtlfs_mismatch_counts(ctx, design_id: int, n_faults: int) -> np.ndarray:
    out = np.zeros(max(n_faults, 0), np.uint32)
    _check(ctx, load_library().rtlfs_mismatch_counts(ctx, design_id, _ptr(out)))
    return out


def rtlfs_checkpoint_size(ctx) -> int:
    n = ctypes.c_uint64()
    _check(ctx, load_library().rtlfs_checkpoint_size(ctx, ctypes.byref(n)))
    return int(n.value)


def rtlfs_checkpoint_save(ctx) -> bytes:
    """The checkpoint held by the context (after a run with stop_cycle) as bytes."""
    buf = np.zeros(rtlfs_checkpoint_size(ctx), np.uint8)
    _check(ctx, load_library().rtlfs_checkpoint_save(ctx, _ptr(buf), buf.size))
    return buf.tobytes()


def rtlfs_checkpoint_load(ctx, data: bytes) -> None:
    buf = np.frombuffer(data, np.uint8)
    _check(ctx, load_library().rtlfs_checkpoint_load(ctx, _ptr(buf), buf.size))


def _set_any_faults(ctx, did: int, faults) -> None:
    """Stuck-at lists through rtlfs_set_faults, lists with transient kinds through the
    extended entry point."""
    if getattr(faults, "cycle", None) is not None:
        rtlfs_set_faults_ex(ctx, did, fault_array_ex(faults))
    else:
        rtlfs_set_faults(ctx, did, fault_array(faults))


def make_opts(**kw) -> rtlfs_run_opts:
    o = rtlfs_run_opts()
    o.scheduler = kw.pop("scheduler", SCHED_HEURISTIC)
    o.heavy_frac = kw.pop("heavy_frac", -1.0)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def rtlfs_run(ctx, n_faults: Sequence[int], opts: Optional[rtlfs_run_opts] = None,
              want_load: bool = False, check: bool = True):
    """Returns (results, loads, rc): per design a RESULT_DTYPE array and optionally a
    uint64 load array."""
    lib = load_library()
    res = [np.zeros(max(n, 0), RESULT_DTYPE) for n in n_faults]
    loads = [np.zeros(max(n, 0), np.uint64) for n in n_faults] if want_load else None
    rp = (ctypes.c_void_p * len(res))(*[_ptr(r) for r in res])
    lp = (ctypes.c_void_p * len(res))(*[_ptr(x) for x in loads]) if want_load else None
    rc = lib.rtlfs_run(ctx, ctypes.byref(opts) if opts is not None else None, rp, lp)
    if check:
        _check(ctx, rc)
    return res, loads, rc


def rtlfs_run_plain(ctx, n_faults: Sequence[int]):
    lib = load_library()
    res = [np.zeros(max(n, 0), RESULT_DTYPE) for n in n_faults]
    rp = (ctypes.c_void_p * len(res))(*[_ptr(r) for r in res])
    _check(ctx, lib.rtlfs_run_plain(ctx, rp))
    return res


def rtlfs_get_stats(ctx) -> dict:
    st = rtlfs_stats()
    _check(ctx, load_library().rtlfs_get_stats(ctx, ctypes.byref(st)))
    return st.as_dict()


def rtlfs_good_outputs(ctx, design_id: int, n_cycles: int, n_outputs: int) -> np.ndarray:
    out = np.zeros((n_cycles, n_outputs), np.uint64)
    if out.size == 0:
        return out
    _check(ctx, load_library().rtlfs_good_outputs(ctx, design_id, _ptr(out)))
    return out


def rtlfs_good_trace(ctx, design_id: int, n_cycles: int, n_nets: int) -> np.ndarray:
    out = np.zeros((n_cycles, n_nets), np.uint64)
    _check(ctx, load_library().rtlfs_good_trace(ctx, design_id, _ptr(out)))
    return out


def rtlfs_design_info(ctx, design_id: int) -> Tuple[int, int, int]:
    a, b, c = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    _check(ctx, load_library().rtlfs_design_info(ctx, design_id, ctypes.byref(a),
                                                 ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def rtlfs_features(ctx, design_id: int, n_faults: int) -> np.ndarray:
    out = np.zeros((n_faults, MLP_IN), np.float32)
    if n_faults:
        _check(ctx, load_library().rtlfs_features(ctx, design_id, _ptr(out)))
    return out


def rtlfs_mlp_set_weights(ctx, w_bf16: np.ndarray) -> None:
    w = np.ascontiguousarray(w_bf16, np.uint16)
    assert w.size == MLP_PARAMS
    _check(ctx, load_library().rtlfs_mlp_set_weights(ctx, _ptr(w)))


def rtlfs_mlp_get_weights(ctx) -> np.ndarray:
    w = np.zeros(MLP_PARAMS, np.uint16)
    _check(ctx, load_library().rtlfs_mlp_get_weights(ctx, _ptr(w)))
    return w


def rtlfs_mlp_forward(ctx, X: np.ndarray) -> np.ndarray:
    X = np.ascontiguousarray(X, np.float32)
    y = np.zeros(X.shape[0], np.float32)
    _check(ctx, load_library().rtlfs_mlp_forward(ctx, _ptr(X), X.shape[0], _ptr(y)))
    return y


def rtlfs_mlp_grad(ctx, X: np.ndarray, t: np.ndarray):
    X = np.ascontiguousarray(X, np.float32)
    t = np.ascontiguousarray(t, np.float32)
    g = np.zeros(MLP_PARAMS, np.float32)
    loss = ctypes.c_float()
    _check(ctx, load_library().rtlfs_mlp_grad(ctx, _ptr(X), _ptr(t), X.shape[0],
                                              ctypes.byref(loss), _ptr(g)))
    return float(loss.value), g


def rtlfs_mlp_train(ctx, X: np.ndarray, t: np.ndarray, epochs: int, batch: int, lr: float) -> float:
    X = np.ascontiguousarray(X, np.float32)
    t = np.ascontiguousarray(t, np.float32)
    loss = ctypes.c_float()
    _check(ctx, load_library().rtlfs_mlp_train(ctx, _ptr(X), _ptr(t), X.shape[0], epochs, batch,
                                               lr, ctypes.byref(loss)))
    return float(loss.value)


def rtlfs_fault_sim_static(ctx, design_id: int, faults_dev_ptr: int, n_faults: int,
                           results_dev_ptr: int, stream_ptr: int = 0) -> int:
    """Allocation-free plain-form simulation on caller-owned device buffers (raw device
    pointers: faults as FAULT_DTYPE records, results as RESULT_DTYPE records). Returns the
    status code; raises nothing so that callers can inspect it."""
    return load_library().rtlfs_fault_sim_static(ctx, design_id, faults_dev_ptr or None, n_faults,
                                                  results_dev_ptr or None, stream_ptr or None)


# ---- convenience wrapper ----------------------------------------------------------------

class Simulator:
    """One context; designs are synth.Design objects, stimuli uint64 [T, I] arrays,
    fault lists synth.Faults."""

    def __init__(self, device: int = 0):
        self.ctx = rtlfs_create(device)
        self.n_faults: List[int] = []
        self.designs = []
        self.T: List[int] = []

    def close(self):
        if self.ctx is not None:
            rtlfs_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def add(self, design, stim: np.ndarray, faults) -> int:
        did = rtlfs_load_design(self.ctx, *design_arrays(design))
        rtlfs_set_stimulus(self.ctx, did, stim)
        _set_any_faults(self.ctx, did, faults)
        self.designs.append(design)
        self.n_faults.append(len(faults))
        self.T.append(int(stim.shape[0]))
        return did

    def set_faults(self, did: int, faults) -> None:
        _set_any_faults(self.ctx, did, faults)
        self.n_faults[did] = len(faults)

    def mismatch_counts(self, did: int) -> np.ndarray:
        """Per fault: cycles with a differing output in the last no-drop run."""
        return rtlfs_mismatch_counts(self.ctx, did, self.n_faults[did])

    def checkpoint(self) -> bytes:
        return rtlfs_checkpoint_save(self.ctx)

    def restore(self, data: bytes) -> None:
        rtlfs_checkpoint_load(self.ctx, data)

    def run(self, want_load: bool = False, **opts):
        o = make_opts(**opts) if opts else None
        res, loads, _ = rtlfs_run(self.ctx, self.n_faults, o, want_load)
        return res, loads

    def run_plain(self):
        return rtlfs_run_plain(self.ctx, self.n_faults)

    def stats(self) -> dict:
        return rtlfs_get_stats(self.ctx)

    def good_outputs(self, did: int) -> np.ndarray:
        return rtlfs_good_outputs(self.ctx, did, self.T[did], self.designs[did].n_out)

    def good_trace(self, did: int) -> np.ndarray:
        return rtlfs_good_trace(self.ctx, did, self.T[did], self.designs[did].n_net)


def split(results: np.ndarray):
    """(detected, cycle, port) arrays from a RESULT_DTYPE array."""
    return results["detected"], results["cycle"], results["port"]
