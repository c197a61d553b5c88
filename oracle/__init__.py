"""CPU oracle: a plain complex128 simulator written from the paper's update rules.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA path (``paper_quant_ph_0608239_gb300``) and the CUDA path never calls
it.  The numerics live in ``oracle.c`` (see its header for the conventions and
citations); this module compiles it with gcc, loads it with ctypes and turns
the symbolic gates of ``inputs`` into the oracle's own gate records.

Parity status of each function (what pins it, in tests/test_oracle_pins.py):

* ``run`` / gate rules: worked examples Eqs. CNOT2, COMM5, COMM4, Toffoli;
  matrix identities against scipy's matrix exponential (Eqs. Hadamard,
  Xoperation, Yoperation, singlephase); dense Kronecker products for n <= 8;
  H^n|0> uniform; QFT closed form; QFT then inverse QFT = I; adder sums
  (Fig. adder 1365 + 682 = 2047 and others); Shor table at L = 24.
* ``apply_dense``: brute force against the Kronecker-product matrix and
  against sequential gates.
* ``permute_bits``: Tables onequbittab and twoqubittab (tests/golden).
* ``norm``, ``probs``, ``qubit_probs``: closed forms and Table Shortab.
* ``sample``: exact inverse-CDF answers on hand-built distributions.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
# A test may point the oracle at a deliberately broken build of oracle.c to
# check that the pins catch the mistake (tests/test_oracle_mutants.py).
_LIB_OVERRIDE = os.environ.get("QSIM_ORACLE_LIB")
_lock = threading.Lock()
_lib = None

KINDS = {"H": 0, "X": 1, "Y": 2, "XB": 3, "YB": 4, "NOT": 5, "R": 6, "V": 7,
         "SU2": 8, "U": 9, "SWAP": 10}


class _OrGate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("t0", ctypes.c_int32),
                ("t1", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("cmask", ctypes.c_uint64), ("p", ctypes.c_double * 8)]


def build(force=False):
    """Compile oracle.c into liboracle.so (gcc, -O2, OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if _LIB_OVERRIDE:
            lib = ctypes.CDLL(_LIB_OVERRIDE)
        else:
            build()
            lib = ctypes.CDLL(_LIB)
        cp = ctypes.c_void_p
        lib.or_num_threads.restype = ctypes.c_int
        lib.or_set_threads.argtypes = [ctypes.c_int]
        lib.or_set_basis.argtypes = [cp, ctypes.c_int, ctypes.c_uint64]
        lib.or_gate_matrix.argtypes = [ctypes.c_int, cp, cp]
        lib.or_gate_matrix.restype = ctypes.c_int
        lib.or_apply_2x2.argtypes = [cp, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, cp]
        lib.or_run.argtypes = [cp, ctypes.c_int, cp, ctypes.c_int64]
        lib.or_run.restype = ctypes.c_int64
        lib.or_apply_dense.argtypes = [cp, ctypes.c_int, ctypes.c_int, cp, cp]
        lib.or_apply_dense.restype = ctypes.c_int
        lib.or_permute_bits.argtypes = [cp, cp, ctypes.c_int, ctypes.c_int, cp, cp]
        lib.or_norm.argtypes = [cp, ctypes.c_int]
        lib.or_norm.restype = ctypes.c_double
        lib.or_probs.argtypes = [cp, ctypes.c_int, cp]
        lib.or_qubit_probs.argtypes = [cp, ctypes.c_int, cp]
        lib.or_sample.argtypes = [cp, ctypes.c_int, cp, ctypes.c_int64, cp]
        _lib = lib
        return lib


def _ptr(arr):
    return arr.ctypes.data_as(ctypes.c_void_p)


def num_threads():
    """Host threads the oracle's sweeps use (OpenMP max threads)."""
    return int(_load().or_num_threads())


def set_threads(n):
    _load().or_set_threads(int(n))


def _records(gates):
    recs = (_OrGate * max(1, len(gates)))()
    for i, g in enumerate(gates):
        r = recs[i]
        r.kind = KINDS[g.kind]
        r.t0 = int(g.targets[0])
        r.t1 = int(g.targets[1]) if len(g.targets) > 1 else -1
        m = 0
        for c in g.controls:
            m |= 1 << int(c)
        r.cmask = m
        for k, v in enumerate(g.params[:8]):
            r.p[k] = float(v)
    return recs


def basis(n, x=0):
    """State |x> of n qubits (INITIAL STATE x, App. A)."""
    a = np.empty(1 << n, dtype=np.complex128)
    _load().or_set_basis(_ptr(a), n, int(x))
    return a


def gate_matrix(g):
    """2x2 complex matrix the oracle uses for a single-target gate."""
    U = np.zeros(4, dtype=np.complex128)
    p = np.zeros(8, dtype=np.float64)
    p[:len(g.params)] = g.params
    if _load().or_gate_matrix(KINDS[g.kind], _ptr(p), _ptr(U)) != 0:
        raise ValueError("no 2x2 matrix for gate kind %s" % g.kind)
    return U.reshape(2, 2)


def run(n, gates, state=None, x0=0):
    """Apply ``gates`` in order.  ``state`` (complex128, length 2^n) is updated
    in place if given, else the run starts from |x0>.  Returns the state."""
    a = basis(n, x0) if state is None else state
    assert a.dtype == np.complex128 and a.size == (1 << n) and a.flags.c_contiguous
    if gates:
        recs = _records(gates)
        bad = _load().or_run(_ptr(a), n, ctypes.cast(recs, ctypes.c_void_p), len(gates))
        if bad:
            raise ValueError("oracle: bad gate at position %d" % (bad - 1))
    return a


def apply_dense(state, n, qubits, U):
    """Dense 2^k x 2^k unitary on ``qubits`` (qubits[j] = bit j of U's index)."""
    k = len(qubits)
    U = np.ascontiguousarray(U, dtype=np.complex128).reshape(1 << k, 1 << k)
    q = np.ascontiguousarray(qubits, dtype=np.int32)
    if _load().or_apply_dense(_ptr(state), n, k, _ptr(q), _ptr(U)) != 0:
        raise ValueError("bad dense gate")
    return state


def permute_bits(state, n, pairs):
    """Physical layout after exchanging bit positions (l, h) for each pair."""
    l = np.ascontiguousarray([p[0] for p in pairs], dtype=np.int32)
    h = np.ascontiguousarray([p[1] for p in pairs], dtype=np.int32)
    out = np.empty_like(state)
    _load().or_permute_bits(_ptr(state), _ptr(out), n, len(pairs), _ptr(l), _ptr(h))
    return out


def norm(state, n):
    return float(_load().or_norm(_ptr(state), n))


def probs(state, n):
    out = np.empty(1 << n, dtype=np.float64)
    _load().or_probs(_ptr(state), n, _ptr(out))
    return out


def qubit_probs(state, n):
    out = np.empty(n, dtype=np.float64)
    _load().or_qubit_probs(_ptr(state), n, _ptr(out))
    return out


def sample(state, n, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty(u.size, dtype=np.uint64)
    _load().or_sample(_ptr(state), n, _ptr(u), u.size, _ptr(out))
    return out
