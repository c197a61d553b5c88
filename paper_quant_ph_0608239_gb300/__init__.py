"""GB300 state-vector simulator: Python binding of the C ABI (include/qsim.h).

Everything that touches amplitudes runs in the CUDA kernels of ``libqsim.so``;
this module only marshals arguments.  PyTorch provides the device memory and
the stream (``State(..., use_torch=True)``, the default) -- it never computes.

    st = State(10, "c128")
    st.set_basis(x)
    st.run(gates)                 # list of Gate records, planner path
    p = st.qubit_probs()          # <Q_q>, Eq. Shor7
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _capi
from .gate import Gate  # noqa: F401
from ._capi import (QsimError, QsimGate, QsimOpts, QsimCircuit, QsimPlanStats, QsimKernelTime,  # noqa: F401
                    QsimCounters, gate_array, gate_record,
                    MODE_PERGATE, MODE_FUSED, MODE_AUTO, QSIM_C64, QSIM_C128, QSIM_ETIMEOUT, QSIM_EINVAL)

_DT = {"c64": QSIM_C64, "complex64": QSIM_C64, "c128": QSIM_C128, "complex128": QSIM_C128}
_NP = {QSIM_C64: np.complex64, QSIM_C128: np.complex128}


def version():
    return _capi.load().qsim_version().decode()


def opts(mode=MODE_FUSED, tile_bits=0, fuse_k=0, max_swap=0):
    o = QsimOpts()
    _capi.load().qsim_default_opts(ctypes.byref(o))
    o.mode, o.tile_bits, o.fuse_k, o.max_swap = int(mode), int(tile_bits), int(fuse_k), int(max_swap)
    return o


def _dbl(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    if a.size != n:
        raise ValueError("expected %d doubles" % n)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _mat8(U):
    U = np.asarray(U, dtype=np.complex128).reshape(2, 2)
    return _dbl(np.stack([U.real, U.imag], axis=-1).reshape(-1), 8)


class State:
    """An n-qubit register on the current CUDA device.

    With ``use_torch=True`` the amplitudes live in a torch tensor (complex64 or
    complex128) attached through ``qsim_attach`` and the work runs on torch's
    current stream; otherwise ``qsim_alloc`` owns the memory.
    """

    def __init__(self, n, dtype="c64", use_torch=True, stream=None):
        self.n = int(n)
        self.dt = _DT[dtype] if isinstance(dtype, str) else int(dtype)
        self.np_dtype = _NP[self.dt]
        self.tensor = None
        h = _capi.c_handle()
        if use_torch:
            import torch
            tdt = torch.complex64 if self.dt == QSIM_C64 else torch.complex128
            self.tensor = torch.empty(1 << self.n, dtype=tdt, device="cuda")
            s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
            _capi.call("qsim_attach", ctypes.c_void_p(self.tensor.data_ptr()), self.n, self.dt,
                       ctypes.c_void_p(s), ctypes.byref(h))
            self.handle = h
            self.set_basis(0)
        else:
            _capi.call("qsim_alloc", self.n, self.dt, ctypes.byref(h))
            self.handle = h
            if stream is not None:
                self.set_stream(stream)

    # -- lifetime ---------------------------------------------------------
    def free(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _capi.call("qsim_free", self.handle)
            self.handle = None
        self.tensor = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    @property
    def nbytes(self):
        return (8 if self.dt == QSIM_C64 else 16) << self.n

    def set_stream(self, stream):
        _capi.call("qsim_set_stream", self.handle, ctypes.c_void_p(stream))

    def sync(self):
        _capi.call("qsim_sync", self.handle)

    # -- state ------------------------------------------------------------
    def set_basis(self, x=0):
        _capi.call("qsim_set_basis", self.handle, ctypes.c_uint64(int(x)))

    def set_shor_state(self, X, y, G):
        """Eq. Shor2: x-register on qubits 0..X-1, f-register above it."""
        _capi.call("qsim_set_shor_state", self.handle, int(X), ctypes.c_uint64(int(y)), ctypes.c_uint64(int(G)))

    def set_state(self, psi):
        psi = np.ascontiguousarray(psi, dtype=self.np_dtype)
        _capi.call("qsim_set_state", self.handle, psi.ctypes.data_as(ctypes.c_void_p), psi.nbytes)

    def get_state(self):
        out = np.empty(1 << self.n, dtype=self.np_dtype)
        _capi.call("qsim_get_state", self.handle, out.ctypes.data_as(ctypes.c_void_p), out.nbytes)
        return out

    def layout(self):
        out = (ctypes.c_int * self.n)()
        _capi.call("qsim_get_layout", self.handle, out)
        return list(out)

    # -- gates ------------------------------------------------------------
    def apply_1q(self, t, U):
        keep, p = _mat8(U)
        _capi.call("qsim_apply_1q", self.handle, int(t), p)

    def apply_ctrl(self, ctrl_mask, t, U):
        keep, p = _mat8(U)
        _capi.call("qsim_apply_ctrl", self.handle, ctypes.c_uint64(int(ctrl_mask)), int(t), p)

    def apply_gate(self, g):
        r = gate_record(g)
        _capi.call("qsim_apply_gate", self.handle, ctypes.byref(r))

    def apply_fused(self, qubits, U):
        k = len(qubits)
        q = (ctypes.c_int * k)(*[int(x) for x in qubits])
        U = np.asarray(U, dtype=np.complex128).reshape(1 << k, 1 << k)
        keep, p = _dbl(np.stack([U.real, U.imag], axis=-1).reshape(-1), 2 << (2 * k))
        _capi.call("qsim_apply_fused", self.handle, k, q, p)

    def swap_qubits(self, a, b):
        K = len(a)
        _capi.call("qsim_swap_qubits", self.handle, K, (ctypes.c_int * K)(*a), (ctypes.c_int * K)(*b))

    def permute_bits(self, l, h):
        K = len(l)
        _capi.call("qsim_permute_bits", self.handle, K, (ctypes.c_int * K)(*l), (ctypes.c_int * K)(*h))

    def run(self, gates, mode=MODE_FUSED, tile_bits=0, fuse_k=0, gate_arr=None):
        """Apply a gate list (Gate records, or a pre-marshalled array)."""
        arr = gate_arr if gate_arr is not None else gate_array(gates)
        ng = len(gates) if gates is not None else len(arr)
        o = opts(mode, tile_bits, fuse_k)
        _capi.call("qsim_run_circuit", self.handle, arr, ng, ctypes.byref(o))

    def plan(self, gates, mode=MODE_FUSED, tile_bits=0, fuse_k=0):
        """Plan and upload a circuit once (qsim_plan_create); returns a Plan."""
        return Plan(self, gates, mode, tile_bits, fuse_k)

    # -- instrumentation --------------------------------------------------
    def profile(self, on=True):
        _capi.call("qsim_profile_enable", self.handle, 1 if on else 0)

    def profile_read(self):
        """{kernel family: (launches, total_ms, alg_bytes, alg_flops)} since the last read."""
        out = (QsimKernelTime * 16)()
        cnt = ctypes.c_int()
        _capi.call("qsim_profile_read", self.handle, out, 16, ctypes.byref(cnt))
        return {out[i].name.decode(): (out[i].launches, out[i].total_ms, out[i].alg_bytes, out[i].alg_flops)
                for i in range(cnt.value)}

    def counters(self):
        c = QsimCounters()
        _capi.call("qsim_get_counters", self.handle, ctypes.byref(c))
        return {"launches": c.launches, "h2d_bytes": c.h2d_bytes, "d2h_bytes": c.d2h_bytes}

    # -- measurement ------------------------------------------------------
    def norm(self):
        out = ctypes.c_double()
        _capi.call("qsim_norm", self.handle, ctypes.byref(out))
        return out.value

    def probs(self):
        out = np.empty(1 << self.n, dtype=np.float64)
        _capi.call("qsim_probs", self.handle, out.ctypes.data_as(ctypes.c_void_p), out.size)
        return out

    def qubit_probs(self):
        out = np.empty(self.n, dtype=np.float64)
        _capi.call("qsim_qubit_probs", self.handle, out.ctypes.data_as(ctypes.c_void_p))
        return out

    def sample(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.empty(u.size, dtype=np.uint64)
        _capi.call("qsim_sample", self.handle, u.ctypes.data_as(ctypes.c_void_p), u.size,
                   out.ctypes.data_as(ctypes.c_void_p))
        return out


class Plan:
    """A circuit planned and uploaded once; ``run()`` only enqueues kernels."""

    def __init__(self, state, gates, mode=MODE_FUSED, tile_bits=0, fuse_k=0):
        self.state = state
        arr = gate_array(gates)
        o = opts(mode, tile_bits, fuse_k)
        p = ctypes.c_void_p()
        _capi.call("qsim_plan_create", state.handle, arr, len(gates), ctypes.byref(o), ctypes.byref(p))
        self.ptr = p

    def run(self, state=None):
        _capi.call("qsim_plan_run", (state or self.state).handle, self.ptr)

    def stats(self):
        s = QsimPlanStats()
        _capi.call("qsim_plan_get_stats", self.ptr, ctypes.byref(s))
        out = {"passes": s.passes, "sweeps": s.sweeps, "ops": s.ops, "tile_bits": s.tile_bits, "phases": s.phases,
               "gates": s.gates, "alg_bytes": s.alg_bytes, "alg_flops": s.alg_flops, "mode": s.mode,
               "fuse_k": s.fuse_k, "candidates": s.candidates, "chosen": s.chosen}
        out["autotune"] = [{"tile_bits": s.cand_tile_bits[i], "fuse_k": s.cand_fuse_k[i], "ms": s.cand_ms[i]}
                           for i in range(min(s.candidates, 8))]
        return out

    def free(self):
        if self.ptr is not None and self.ptr.value:
            _capi.call("qsim_plan_free", self.ptr)
        self.ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def fuse_blocks(n, gates, k):
    """The dense blocks a plan with ``fuse_k=k`` applies, planned on the host
    (no device): a list of (qubits, U), U the 2^k x 2^k complex128 product of
    the block's gates (bit j of U's index = qubits[j]).  Applied in order the
    blocks equal the circuit."""
    arr = gate_array(gates)
    nb = ctypes.c_size_t()
    _capi.call("qsim_fuse_blocks", int(n), arr, len(gates), int(k), None, None, 0, ctypes.byref(nb))
    m = nb.value
    pos = np.zeros((max(m, 1), k), dtype=np.int32)
    D = 1 << k
    U = np.zeros((max(m, 1), D, D, 2), dtype=np.float64)
    _capi.call("qsim_fuse_blocks", int(n), arr, len(gates), int(k), pos.ctypes.data_as(ctypes.c_void_p),
               U.ctypes.data_as(ctypes.c_void_p), m, ctypes.byref(nb))
    Uc = U[..., 0] + 1j * U[..., 1]
    return [(tuple(int(q) for q in pos[b]), Uc[b]) for b in range(m)]


def _circuit_array(states, x0s, gate_lists):
    nc = len(states)
    arr = (QsimCircuit * nc)()
    keep = []
    for i, (st, x0, gl) in enumerate(zip(states, x0s, gate_lists)):
        ga = gl if isinstance(gl, ctypes.Array) else gate_array(gl)
        keep.append(ga)
        arr[i].state = st.handle
        arr[i].x0 = int(x0)
        arr[i].gates = ctypes.cast(ga, ctypes.POINTER(QsimGate))
        arr[i].ng = len(ga) if isinstance(gl, ctypes.Array) else len(gl)
    return arr, keep


def run_batch(states, x0s, gate_lists, wait_budget_us=0, fuse_k=0):
    """Run independent circuits (complex64 states): one persistent launch,
    and circuits of 20 qubits or more as dense blocks on the tensor cores
    (6-qubit blocks, or fuse_k; fuse_k=-1 keeps them in the persistent
    launch)."""
    arr, keep = _circuit_array(states, x0s, gate_lists)
    o = opts(fuse_k=fuse_k)
    o.wait_budget_us = int(wait_budget_us)
    _capi.call("qsim_run_batch", arr, len(states), ctypes.byref(o))


class Batch:
    """A planned batch (qsim_batch_create): every run() is one graph launch."""

    def __init__(self, states, x0s, gate_lists, wait_budget_us=0, fuse_k=0):
        arr, keep = _circuit_array(states, x0s, gate_lists)
        o = opts(fuse_k=fuse_k)
        o.wait_budget_us = int(wait_budget_us)
        p = ctypes.c_void_p()
        _capi.call("qsim_batch_create", arr, len(states), ctypes.byref(o), ctypes.byref(p))
        self.ptr = p
        self.states = states

    def run(self):
        _capi.call("qsim_batch_run", self.ptr)

    def sync(self):
        _capi.call("qsim_batch_sync", self.ptr)

    def stats(self):
        s = _capi.QsimBatchStats()
        _capi.call("qsim_batch_get_stats", self.ptr, ctypes.byref(s))
        return {"circuits": s.circuits, "gates": s.gates, "passes": s.passes, "items": s.items,
                "graph": bool(s.graph), "fused": s.fused, "blocks": s.blocks, "kernels": s.kernels,
                "alg_bytes": s.alg_bytes, "alg_flops": s.alg_flops}

    def free(self):
        if self.ptr is not None and self.ptr.value:
            _capi.call("qsim_batch_free", self.ptr)
        self.ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
