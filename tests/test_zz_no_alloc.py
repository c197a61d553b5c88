"""Allocation-free per-qubit marginals (qsim_qubit_probs_noalloc).

Callers that must not allocate device memory -- a framework that owns the
device through its own pool, a latency-bound loop that cannot take the
implicit synchronisation of cudaMalloc/cudaFree, an embedder that forbids
allocation after start-up -- get the marginals on a static scratch array
inside the library.  This file runs last (pytest collects it after the other
test files) and also passes on its own in a fresh process.

Two calls in a row, on different states, go through the C ABI and must agree
with the allocating entry point qsim_qubit_probs; the second call (smaller
register) also shows that partial sums the first call left in the shared
array do not leak into its result.
"""
import ctypes

import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-13, "c64": 1e-6}


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_noalloc_marginals_match_allocating_entry_point(dt):
    import torch
    torch.cuda.set_device(0)
    import paper_quant_ph_0608239_gb300 as q
    from paper_quant_ph_0608239_gb300 import _capi
    lib = _capi.load()
    dcode = q.QSIM_C64 if dt == "c64" else q.QSIM_C128
    # calls in a row: the second on a smaller register, the third on one small
    # enough to be reduced by a single block without the scratch array
    for n, seed in ((20, 5), (13, 6), (5, 7)):
        st = q.State(n, dt)
        st.set_basis(inputs.random_basis(n, seed))
        st.run(inputs.random_circuit(n, 4, seed))
        ref = st.qubit_probs()            # allocating entry point (handle scratch)
        out = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        rc = lib.qsim_qubit_probs_noalloc(ctypes.c_void_p(st.tensor.data_ptr()), n, dcode,
                                          ctypes.c_void_p(stream), ctypes.c_void_p(out.data_ptr()))
        assert rc == q._capi.QSIM_OK, lib.qsim_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.max(np.abs(got - ref)) < TOL[dt], (n, got, ref)
        st.free()


def test_noalloc_rejects_sizes_beyond_the_scratch_array():
    import torch
    torch.cuda.set_device(0)
    from paper_quant_ph_0608239_gb300 import _capi
    lib = _capi.load()
    buf = torch.zeros(64, dtype=torch.complex64, device="cuda")
    out = torch.zeros(64, dtype=torch.float64, device="cuda")
    for n in (0, 35):
        rc = lib.qsim_qubit_probs_noalloc(ctypes.c_void_p(buf.data_ptr()), n, 0, None, ctypes.c_void_p(out.data_ptr()))
        assert rc == _capi.QSIM_EINVAL
        assert b"static scratch array" in lib.qsim_last_error()
