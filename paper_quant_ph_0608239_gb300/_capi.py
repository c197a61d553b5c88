"""ctypes declarations of the C ABI in include/qsim.h (marshalling only).

Loading fails loudly when ``libqsim.so`` has not been built: there is no
fallback implementation of any kind.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqsim.so")

QSIM_OK, QSIM_EINVAL, QSIM_ENOMEM, QSIM_ECUDA, QSIM_ETIMEOUT, QSIM_EUNSUPPORTED = range(6)
QSIM_C64, QSIM_C128 = 0, 1
MODE_PERGATE, MODE_FUSED, MODE_AUTO = 0, 1, 2

GATE_KIND = {"H": 0, "X": 1, "Y": 2, "XB": 3, "YB": 4, "NOT": 5, "R": 6, "V": 7,
             "SU2": 8, "U": 9, "SWAP": 10}

c_handle = ctypes.c_void_p


class QsimGate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("target", ctypes.c_int32),
                ("target2", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("ctrl_mask", ctypes.c_uint64), ("param", ctypes.c_double * 8)]


class QsimOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("tile_bits", ctypes.c_int32),
                ("fuse_k", ctypes.c_int32), ("max_swap", ctypes.c_int32),
                ("wait_budget_us", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class QsimBatchStats(ctypes.Structure):
    _fields_ = [("circuits", ctypes.c_int64), ("gates", ctypes.c_int64), ("passes", ctypes.c_int64),
                ("items", ctypes.c_int64), ("graph", ctypes.c_int32), ("fused", ctypes.c_int32),
                ("alg_bytes", ctypes.c_double), ("alg_flops", ctypes.c_double), ("blocks", ctypes.c_int64),
                ("kernels", ctypes.c_int64)]


class QsimCircuit(ctypes.Structure):
    _fields_ = [("state", c_handle), ("x0", ctypes.c_uint64),
                ("gates", ctypes.POINTER(QsimGate)), ("ng", ctypes.c_size_t)]


class QsimPlanStats(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_int32), ("sweeps", ctypes.c_int32), ("ops", ctypes.c_int32),
                ("tile_bits", ctypes.c_int32), ("phases", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("gates", ctypes.c_double), ("alg_bytes", ctypes.c_double),
                ("alg_flops", ctypes.c_double), ("mode", ctypes.c_int32), ("fuse_k", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("chosen", ctypes.c_int32),
                ("cand_tile_bits", ctypes.c_int32 * 8), ("cand_fuse_k", ctypes.c_int32 * 8),
                ("cand_ms", ctypes.c_double * 8)]


class QsimKernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double),
                ("alg_bytes", ctypes.c_double), ("alg_flops", ctypes.c_double)]


class QsimCounters(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("h2d_bytes", ctypes.c_uint64), ("d2h_bytes", ctypes.c_uint64)]


class QsimError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("qsim status %d: %s" % (status, msg))
        self.status = status


_lib = None

# name -> (argtypes, restype); restype None means qsim_status checked by _call
_SIGS = {
    "qsim_default_opts": ([ctypes.POINTER(QsimOpts)], "void"),
    "qsim_alloc": ([ctypes.c_int, ctypes.c_int, ctypes.POINTER(c_handle)], None),
    "qsim_attach": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(c_handle)], None),
    "qsim_free": ([c_handle], None),
    "qsim_set_stream": ([c_handle, ctypes.c_void_p], None),
    "qsim_info": ([c_handle, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                   ctypes.POINTER(ctypes.c_void_p)], None),
    "qsim_set_basis": ([c_handle, ctypes.c_uint64], None),
    "qsim_set_shor_state": ([c_handle, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64], None),
    "qsim_set_state": ([c_handle, ctypes.c_void_p, ctypes.c_size_t], None),
    "qsim_apply_1q": ([c_handle, ctypes.c_int, ctypes.POINTER(ctypes.c_double)], None),
    "qsim_apply_ctrl": ([c_handle, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(ctypes.c_double)], None),
    "qsim_apply_gate": ([c_handle, ctypes.POINTER(QsimGate)], None),
    "qsim_apply_fused": ([c_handle, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)],
                         None),
    "qsim_swap_qubits": ([c_handle, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)], None),
    "qsim_permute_bits": ([c_handle, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
                          None),
    "qsim_get_layout": ([c_handle, ctypes.POINTER(ctypes.c_int)], None),
    "qsim_run_circuit": ([c_handle, ctypes.POINTER(QsimGate), ctypes.c_size_t, ctypes.POINTER(QsimOpts)], None),
    "qsim_run_batch": ([ctypes.POINTER(QsimCircuit), ctypes.c_size_t, ctypes.POINTER(QsimOpts)], None),
    "qsim_batch_create": ([ctypes.POINTER(QsimCircuit), ctypes.c_size_t, ctypes.POINTER(QsimOpts),
                           ctypes.POINTER(ctypes.c_void_p)], None),
    "qsim_batch_run": ([ctypes.c_void_p], None),
    "qsim_batch_sync": ([ctypes.c_void_p], None),
    "qsim_batch_get_stats": ([ctypes.c_void_p, ctypes.POINTER(QsimBatchStats)], None),
    "qsim_batch_free": ([ctypes.c_void_p], None),
    "qsim_norm": ([c_handle, ctypes.POINTER(ctypes.c_double)], None),
    "qsim_probs": ([c_handle, ctypes.c_void_p, ctypes.c_size_t], None),
    "qsim_qubit_probs": ([c_handle, ctypes.c_void_p], None),
    "qsim_qubit_probs_noalloc": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p],
                                 None),
    "qsim_sample": ([c_handle, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p], None),
    "qsim_get_state": ([c_handle, ctypes.c_void_p, ctypes.c_size_t], None),
    "qsim_sync": ([c_handle], None),
    "qsim_plan_create": ([c_handle, ctypes.POINTER(QsimGate), ctypes.c_size_t, ctypes.POINTER(QsimOpts),
                          ctypes.POINTER(ctypes.c_void_p)], None),
    "qsim_plan_run": ([c_handle, ctypes.c_void_p], None),
    "qsim_plan_get_stats": ([ctypes.c_void_p, ctypes.POINTER(QsimPlanStats)], None),
    "qsim_plan_free": ([ctypes.c_void_p], None),
    "qsim_fuse_blocks": ([ctypes.c_int, ctypes.POINTER(QsimGate), ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p,
                          ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)], None),
    "qsim_profile_enable": ([c_handle, ctypes.c_int], None),
    "qsim_profile_read": ([c_handle, ctypes.POINTER(QsimKernelTime), ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
                          None),
    "qsim_get_counters": ([c_handle, ctypes.POINTER(QsimCounters)], None),
    "qsim_last_error": ([], ctypes.c_char_p),
    "qsim_version": ([], ctypes.c_char_p),
}

EXPORTED = tuple(_SIGS)


def load():
    """Load libqsim.so (raises ImportError if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libqsim.so not built: run __graft_entry__.build() or "
                          "python paper_quant_ph_0608239_gb300/build.py")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = None if res == "void" else (ctypes.c_int if res is None else res)
    _lib = lib
    return lib


def call(name, *args):
    """Call an entry point returning qsim_status; raise QsimError unless OK."""
    lib = load()
    st = getattr(lib, name)(*args)
    if st != QSIM_OK:
        raise QsimError(st, lib.qsim_last_error().decode())
    return st


def gate_record(g, out=None):
    """Marshal one symbolic gate (kind, targets, controls, params) into a QsimGate."""
    r = QsimGate() if out is None else out
    r.kind = GATE_KIND[g.kind]
    r.target = int(g.targets[0])
    r.target2 = int(g.targets[1]) if len(g.targets) > 1 else -1
    r.reserved = 0
    m = 0
    for c in g.controls:
        m |= 1 << int(c)
    r.ctrl_mask = m
    for k in range(8):
        r.param[k] = float(g.params[k]) if k < len(g.params) else 0.0
    return r


def gate_array(gates):
    """Marshal a gate list into a contiguous ctypes array of QsimGate."""
    arr = (QsimGate * max(1, len(gates)))()
    for i, g in enumerate(gates):
        gate_record(g, arr[i])
    return arr
